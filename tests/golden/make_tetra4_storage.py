"""Write tests/golden/tetra4_half_storage.json: what storing the populations in FP32, or as binary16
deviations from the lattice weights, does to the four-sphere cluster, with FP64 arithmetic
everywhere else.

The CUDA library can store the populations in FP64, FP32 or binary16 deviations h_i = f_i - w_i
(FP32 arithmetic for the last two). The oracle's storage model (store_prec 1 and 2, an analysis
option: the stored populations are rounded the same way after every store, the method is otherwise
the FP64 oracle's) separates what the storage costs from what FP32 arithmetic costs. The cluster at
half scale (128^3, four spheres R = 12, surface gap 4, jitter U{-2..2}^3 from seed 0, liquid 0.05 of
the solid volume, 60 degrees, D3Q19, tau = 1, MPF kinetics on) is run three times in lockstep (FP64,
FP32 storage, binary16-deviation storage); the relative L-infinity differences of density and
velocity over the fluid cells of the central 64^3 crop and of the whole lattice, of the per-body
force, and the number of differing flags, at steps 150, 300 and 500, are recorded.

Run: python tests/golden/make_tetra4_storage.py [threads]   (calls only oracle/; ~15 minutes on 8 cores)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

STEPS = (150, 300, 500)
N, R, GAP = 128, 12.0, 4.0


def rel(a, b, m):
    a, b = a[m], b[m]
    return float(np.abs(a - b).max() / np.abs(b).max())


def main():
    import oracle
    from paper_1902_10432_gb300 import workloads

    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    w = workloads.tetra4(seed=0, prec="fp64", n=N, R=R, surface_gap=GAP)
    kw = {k: v for k, v in w.params.items() if k != "prec"}
    runs = {sp: oracle.Oracle(w.nx, w.ny, w.nz, nthreads=threads, store_prec=sp, **kw) for sp in (0, 1, 2)}
    for o in runs.values():
        workloads.build(o, w)
    h = N // 4
    crop = (slice(N // 2 - h, N // 2 + h),) * 3
    out, done = {}, 0
    for s in STEPS:
        for o in runs.values():
            o.step(s - done)
        done = s
        r0, v0, _ = runs[0].fields()
        s0, _ = runs[0].flags()
        F0, _, _ = runs[0].body_forces()
        out[str(s)] = {}
        for sp, name in ((1, "fp32"), (2, "fp16dev")):
            r, v, _ = runs[sp].fields()
            sl, _ = runs[sp].flags()
            F, _, _ = runs[sp].body_forces()
            fl = (s0 == 0) & (sl == 0)
            cf = fl[crop]
            out[str(s)][name] = dict(
                rho_crop=rel(r[crop], r0[crop], cf), vel_crop=max(rel(v[crop][..., a], v0[crop][..., a], cf) for a in range(3)),
                rho=rel(r, r0, fl), vel=max(rel(v[..., a], v0[..., a], fl) for a in range(3)),
                force=float(np.abs(F - F0).max() / np.abs(F0).max()), flag_mismatch=int((s0 != sl).sum()))
        print(s, json.dumps(out[str(s)]), flush=True)
    d = {"description": __doc__.split("\n\n")[0].strip(),
         "workload": "tetra4 128^3, R = 12, surface gap 4, seed 0, FP64 oracle with its storage model",
         "errors_vs_fp64": out}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tetra4_half_storage.json"), "w") as f:
        json.dump(d, f, indent=1)


if __name__ == "__main__":
    main()
