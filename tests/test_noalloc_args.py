"""Argument checks of the no-allocation step's binding (cbl.lbm_step_noalloc), on the CPU.

The C entry point receives bare device pointers and cannot check sizes, element types or where the
memory lives, so the binding checks them before the call: a wrong buffer must be a ValueError on the
host, never a memory fault on the GPU. No GPU is needed: every case is refused before the library
is called.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_1902_10432_gb300 import cbl  # noqa: E402

NX, NY, NZ = 8, 6, 5
N19 = 19 * NX * NY * NZ


def _call(f_in, f_out, mass_out=None):
    cbl.lbm_step_noalloc(f_in, f_out, NX, NY, NZ, mass_out=mass_out)


def test_wrong_dtype_refused():
    with pytest.raises(ValueError, match="float32"):
        _call(torch.zeros(N19, dtype=torch.float64), torch.zeros(N19))
    with pytest.raises(ValueError, match="float32"):
        _call(torch.zeros(N19), torch.zeros(N19, dtype=torch.float16))


def test_non_contiguous_refused():
    with pytest.raises(ValueError, match="contiguous"):
        _call(torch.zeros(2 * N19)[::2], torch.zeros(N19))


def test_too_small_refused():
    with pytest.raises(ValueError, match="19\\*nx\\*ny\\*nz"):
        _call(torch.zeros(N19 - 1), torch.zeros(N19))
    with pytest.raises(ValueError, match="19\\*nx\\*ny\\*nz"):
        _call(torch.zeros(N19), torch.zeros(10))


def test_overlap_refused():
    buf = torch.zeros(2 * N19)
    with pytest.raises(ValueError, match="overlap"):
        _call(buf[:N19], buf[N19 // 2:N19 // 2 + N19])
    with pytest.raises(ValueError, match="overlap"):
        _call(buf[:N19], buf[:N19])


def test_mass_out_type_refused():
    with pytest.raises(ValueError, match="mass_out"):
        _call(torch.zeros(N19), torch.zeros(N19), mass_out=torch.zeros(1, dtype=torch.float32))
    with pytest.raises(ValueError, match="mass_out"):
        _call(torch.zeros(N19), torch.zeros(N19), mass_out=torch.zeros(0, dtype=torch.float64))


def test_host_memory_refused():
    # well-formed buffers in host memory: a device kernel given them would fault
    with pytest.raises(ValueError, match="CUDA tensor"):
        _call(torch.zeros(N19), torch.zeros(N19))
    with pytest.raises(ValueError, match="CUDA tensor"):
        _call(torch.zeros(N19), torch.zeros(N19), mass_out=torch.zeros(1, dtype=torch.float64))
