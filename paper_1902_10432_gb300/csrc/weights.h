// FP32 lattice weights of the collision, shared by the device code and host-side checks.
//
// The BGK equilibria sum to rho because the weights sum to 1 (Sec. 3.2.1). The FP32 values nearest
// to 1/3, 1/18, 1/36 sum to 1 + 1.49e-8 (and those nearest to 8/27, 2/27, 1/54, 1/216 to
// 1 + 7.5e-9), so an FP32 collision that used them would scale the mass of every cell by that factor
// at every step. The values below are the FP32 numbers within 2 ulp of each weight whose sum is
// exactly 1 (as real numbers: w_0 + 6 w_1 + 12 w_2 for D3Q19, w_0 + 6 w_1 + 12 w_2 + 8 w_3 for
// D3Q27), chosen to keep the largest relative change smallest (1.2e-7 and 1.1e-7).
//
// This header needs no CUDA header, so host-side tests compile it as plain C++.
#pragma once

#if defined(__CUDACC__)
#define CBL_WHD __host__ __device__
#else
#define CBL_WHD
#endif

namespace cbl {
namespace q19 {
CBL_WHD constexpr float wf_of(int i) {
  return i == 0 ? 0x1.555558p-2f : (i <= 6 ? 0x1.c71c7p-5f : 0x1.c71c7p-6f);
}
}  // namespace q19
namespace q27 {
CBL_WHD constexpr float wf_of(int i) {
  return i == 0 ? 0x1.2f684ap-2f : (i <= 6 ? 0x1.2f684cp-4f : (i <= 18 ? 0x1.2f684ep-6f : 0x1.2f684cp-8f));
}
}  // namespace q27
}  // namespace cbl
