// Force surrogate network: 4 -> 64 -> 64 -> 64 -> 6 multilayer perceptron with tanh hidden units and
// a linear output, bfloat16 weights, FP32 accumulation, FP32 master weights for Adam.
//
// The network is small (9,030 parameters) and the batches are at most a few ten thousand samples, so
// the kernels are latency-shaped rather than throughput-shaped: one thread per sample for the
// forward pass with the weights in shared memory, and for training one block per 64 samples that
// keeps the samples' activations and back-propagated deltas in shared memory and forms the weight
// gradients there (dW = sum_s delta_s h_s^T), adding one partial per block to the FP32 gradient.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cbl.h"

namespace {

constexpr int IN = 4, H = 64, OUT = 6, NL = 4;  // NL weight layers
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + OUT * H,
              NPARAM = OFF_B4 + OUT;
constexpr int BS = 64;  // samples per training block

__device__ __forceinline__ float wv(const __nv_bfloat16* w, int k) { return __bfloat162float(w[k]); }

__device__ __forceinline__ void load_weights(const __nv_bfloat16* __restrict__ g, __nv_bfloat16* s) {
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) s[k] = g[k];
  __syncthreads();
}

// forward of one sample with the weights in shared memory; keeps the hidden activations if asked
template <bool KEEP>
__device__ __forceinline__ void fwd_one(const __nv_bfloat16* w, const float x[IN], float y[OUT], float* h1o,
                                        float* h2o, float* h3o) {
  float h1[H], h2[H];
#pragma unroll 4
  for (int o = 0; o < H; ++o) {
    float z = wv(w, OFF_B1 + o);
#pragma unroll
    for (int i = 0; i < IN; ++i) z = fmaf(wv(w, OFF_W1 + o * IN + i), x[i], z);
    h1[o] = tanhf(z);
    if (KEEP) h1o[o] = h1[o];
  }
#pragma unroll 4
  for (int o = 0; o < H; ++o) {
    float z = wv(w, OFF_B2 + o);
#pragma unroll 16
    for (int i = 0; i < H; ++i) z = fmaf(wv(w, OFF_W2 + o * H + i), h1[i], z);
    h2[o] = tanhf(z);
    if (KEEP) h2o[o] = h2[o];
  }
  // layer 3 overwrites h1 (no longer needed)
#pragma unroll 4
  for (int o = 0; o < H; ++o) {
    float z = wv(w, OFF_B3 + o);
#pragma unroll 16
    for (int i = 0; i < H; ++i) z = fmaf(wv(w, OFF_W3 + o * H + i), h2[i], z);
    h1[o] = tanhf(z);
    if (KEEP) h3o[o] = h1[o];
  }
#pragma unroll
  for (int o = 0; o < OUT; ++o) {
    float z = wv(w, OFF_B4 + o);
#pragma unroll 16
    for (int i = 0; i < H; ++i) z = fmaf(wv(w, OFF_W4 + o * H + i), h1[i], z);
    y[o] = z;
  }
}

__global__ void __launch_bounds__(128) k_mlp_fwd(const __nv_bfloat16* __restrict__ wg, const float* __restrict__ x,
                                                 float* __restrict__ y, int n) {
  __shared__ __nv_bfloat16 w[NPARAM];
  load_weights(wg, w);
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float xi[IN], yo[OUT];
#pragma unroll
  for (int i = 0; i < IN; ++i) xi[i] = x[(size_t)s * IN + i];
  fwd_one<false>(w, xi, yo, nullptr, nullptr, nullptr);
#pragma unroll
  for (int o = 0; o < OUT; ++o) y[(size_t)s * OUT + o] = yo[o];
}

struct TrainSmem {
  __nv_bfloat16 w[NPARAM];
  float x[BS][IN];
  float h1[BS][H], h2[BS][H], h3[BS][H];
  float d4[BS][OUT];
  float da[BS][H], db[BS][H];
  float loss[BS];
};

// dW[o][i] += sum_s d[s][o] a[s][i] and db[o] += sum_s d[s][o] for the block's samples
template <int NO, int NI>
__device__ __forceinline__ void add_outer(float* __restrict__ gW, float* __restrict__ gb, const float (*d)[NO == OUT ? OUT : H],
                                          const float (*a)[NI == IN ? IN : H]) {
  for (int e = threadIdx.x; e < NO * NI; e += blockDim.x) {
    const int o = e / NI, i = e % NI;
    float acc = 0.f;
    for (int s = 0; s < BS; ++s) acc = fmaf(d[s][o], a[s][i], acc);
    if (acc != 0.f) atomicAdd(gW + e, acc);
  }
  for (int o = threadIdx.x; o < NO; o += blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < BS; ++s) acc += d[s][o];
    if (acc != 0.f) atomicAdd(gb + o, acc);
  }
}

// Mean-squared-error gradient of a batch (added to grad) and the loss (added to *loss).
__global__ void __launch_bounds__(256) k_mlp_grad(const __nv_bfloat16* __restrict__ wg, const float* __restrict__ x,
                                                  const float* __restrict__ t, int n, float* __restrict__ grad,
                                                  float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(raw);
  load_weights(wg, S.w);
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * BS;
  const float inv = 1.0f / ((float)n * OUT);
  if (tid < BS) {
    const int s = s0 + tid;
    float xi[IN], yo[OUT];
    const bool ok = s < n;
#pragma unroll
    for (int i = 0; i < IN; ++i) xi[i] = ok ? x[(size_t)s * IN + i] : 0.f;
#pragma unroll
    for (int i = 0; i < IN; ++i) S.x[tid][i] = xi[i];
    fwd_one<true>(S.w, xi, yo, S.h1[tid], S.h2[tid], S.h3[tid]);
    float l = 0.f;
#pragma unroll
    for (int o = 0; o < OUT; ++o) {
      const float r = ok ? yo[o] - t[(size_t)s * OUT + o] : 0.f;
      S.d4[tid][o] = 2.f * r * inv;
      l += r * r;
    }
    S.loss[tid] = l * inv;
  }
  __syncthreads();
  // output layer
  add_outer<OUT, H>(grad + OFF_W4, grad + OFF_B4, S.d4, S.h3);
  // delta of layer 3: (W4^T d4) * (1 - h3^2)
  for (int e = tid; e < BS * H; e += blockDim.x) {
    const int s = e / H, k = e % H;
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < OUT; ++j) a = fmaf(wv(S.w, OFF_W4 + j * H + k), S.d4[s][j], a);
    S.da[s][k] = a * (1.f - S.h3[s][k] * S.h3[s][k]);
  }
  __syncthreads();
  add_outer<H, H>(grad + OFF_W3, grad + OFF_B3, S.da, S.h2);
  for (int e = tid; e < BS * H; e += blockDim.x) {
    const int s = e / H, k = e % H;
    float a = 0.f;
    for (int j = 0; j < H; ++j) a = fmaf(wv(S.w, OFF_W3 + j * H + k), S.da[s][j], a);
    S.db[s][k] = a * (1.f - S.h2[s][k] * S.h2[s][k]);
  }
  __syncthreads();
  add_outer<H, H>(grad + OFF_W2, grad + OFF_B2, S.db, S.h1);
  for (int e = tid; e < BS * H; e += blockDim.x) {
    const int s = e / H, k = e % H;
    float a = 0.f;
    for (int j = 0; j < H; ++j) a = fmaf(wv(S.w, OFF_W2 + j * H + k), S.db[s][j], a);
    S.da[s][k] = a * (1.f - S.h1[s][k] * S.h1[s][k]);
  }
  __syncthreads();
  add_outer<H, IN>(grad + OFF_W1, grad + OFF_B1, S.da, S.x);
  if (tid == 0) {
    float l = 0.f;
    for (int s = 0; s < BS; ++s) l += S.loss[s];
    atomicAdd(loss, l);
  }
}

__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  w[k] = wk;
  wb[k] = __float2bfloat16_rn(wk);
  g[k] = 0.f;
}

__global__ void k_round_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NPARAM) wb[k] = __float2bfloat16_rn(w[k]);
}

}  // namespace

// ---- bodies advanced by the network's pair forces (the surrogate window, on the device) ----------
// One block runs `steps` semi-implicit Euler steps of nb rigid spheres under the network's forces and
// torques of the bridged pairs plus a fixed per-body bias force, with the fluid frozen. Per step,
// one thread per (pair, side) forms the pair's features in its frame (e_z from the body to its
// partner, minimum image), standardises them (clipped to the training range), runs the network with
// the weights in shared memory, and adds the de-standardised force and torque, turned back to the
// lattice frame, to its body; then one thread per free body updates V, X (periodic) and omega.
// Features and targets are those of the host-side surrogate: gap s sqrt(R*/V_L), cos(theta),
// R_i/R_j, V_L/R*^3; force over 2 pi R* sigma and torque over 2 pi R*^2 sigma, R* = 2 R_i R_j/(R_i+R_j).
struct AdvNorm {
  float xm[IN], xs[IN], xlo[IN], xhi[IN], ym[OUT], ys[OUT];
};

__device__ __forceinline__ double mimg_adv(double d, double n) { return d - n * rint(d / n); }

__global__ void __launch_bounds__(256) k_mlp_advance(const __nv_bfloat16* __restrict__ wg, double* __restrict__ X,
                                                     double* __restrict__ V, double* __restrict__ Wang,
                                                     const double* __restrict__ M, const double* __restrict__ Iinv,
                                                     const double* __restrict__ R, const int* __restrict__ fixed,
                                                     const double* __restrict__ bias, const int* __restrict__ pairs,
                                                     const double* __restrict__ VL, int nb, int npairs, int steps,
                                                     int nx, int ny, int nz, double cth, AdvNorm nm, double sigma) {
  extern __shared__ __align__(16) unsigned char raw[];
  __nv_bfloat16* w = reinterpret_cast<__nv_bfloat16*>(raw);
  double* F = reinterpret_cast<double*>(raw + ((NPARAM * sizeof(__nv_bfloat16) + 15) / 16) * 16);
  double* T = F + 3 * nb;
  load_weights(wg, w);
  const double dims[3] = {(double)nx, (double)ny, (double)nz};
  for (int it = 0; it < steps; ++it) {
    for (int k = threadIdx.x; k < 3 * nb; k += blockDim.x) F[k] = T[k] = 0.0;
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * npairs; k += blockDim.x) {
      const int p = k >> 1, a = pairs[2 * p + (k & 1)], b = pairs[2 * p + 1 - (k & 1)];
      double d[3], r = 0.0;
      for (int c = 0; c < 3; ++c) {
        d[c] = mimg_adv(X[3 * b + c] - X[3 * a + c], dims[c]);
        r += d[c] * d[c];
      }
      r = sqrt(r);
      double ez[3] = {d[0] / r, d[1] / r, d[2] / r};
      const double ref[3] = {fabs(ez[0]) < 0.9 ? 1.0 : 0.0, fabs(ez[0]) < 0.9 ? 0.0 : 1.0, 0.0};
      double ex[3] = {ref[1] * ez[2] - ref[2] * ez[1], ref[2] * ez[0] - ref[0] * ez[2], ref[0] * ez[1] - ref[1] * ez[0]};
      const double en = sqrt(ex[0] * ex[0] + ex[1] * ex[1] + ex[2] * ex[2]);
      for (int c = 0; c < 3; ++c) ex[c] /= en;
      const double ey[3] = {ez[1] * ex[2] - ez[2] * ex[1], ez[2] * ex[0] - ez[0] * ex[2], ez[0] * ex[1] - ez[1] * ex[0]};
      const double Ra = R[a], Rb = R[b], Rs = 2.0 * Ra * Rb / (Ra + Rb), vl = VL[p];
      const double feat[IN] = {(r - Ra - Rb) * sqrt(Rs / vl), cth, Ra / Rb, vl / (Rs * Rs * Rs)};
      float xi[IN], yo[OUT];
      for (int i = 0; i < IN; ++i) {
        const float v = fminf(fmaxf((float)feat[i], nm.xlo[i]), nm.xhi[i]);
        xi[i] = (v - nm.xm[i]) / nm.xs[i];
      }
      fwd_one<false>(w, xi, yo, nullptr, nullptr, nullptr);
      const double sc = 2.0 * 3.14159265358979323846 * Rs * sigma;
      double fl[3], tl[3];
      for (int c = 0; c < 3; ++c) {
        fl[c] = (double)(yo[c] * nm.ys[c] + nm.ym[c]) * sc;
        tl[c] = (double)(yo[3 + c] * nm.ys[3 + c] + nm.ym[3 + c]) * sc * Rs;
      }
      for (int c = 0; c < 3; ++c) {  // frame rows ex, ey, ez: world = frame^T local
        atomicAdd(&F[3 * a + c], ex[c] * fl[0] + ey[c] * fl[1] + ez[c] * fl[2]);
        atomicAdd(&T[3 * a + c], ex[c] * tl[0] + ey[c] * tl[1] + ez[c] * tl[2]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      if (fixed[i]) continue;
      for (int c = 0; c < 3; ++c) {
        V[3 * i + c] += (F[3 * i + c] + bias[3 * i + c]) / M[i];
        double x = X[3 * i + c] + V[3 * i + c];
        x -= dims[c] * floor(x / dims[c]);
        X[3 * i + c] = x;
        Wang[3 * i + c] += T[3 * i + c] * Iinv[i];
      }
    }
    __syncthreads();
  }
}

struct cbl_mlp {
  cudaStream_t s = nullptr;
  bool own = false;
  float* w = nullptr;  // FP32 master
  __nv_bfloat16* wb = nullptr;
  float *g = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
  int t = 0;
};

extern "C" {

cbl_status cbl_mlp_create(int n_in, int hidden, int n_hidden_layers, int n_out, void* stream, cbl_mlp** out) {
  if (!out) return CBL_ERR_ARG;
  if (n_in != IN || hidden != H || n_hidden_layers != NL - 1 || n_out != OUT) return CBL_ERR_UNSUPPORTED;
  cbl_mlp* m = new cbl_mlp();
  if (stream) {
    m->s = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&m->s, cudaStreamNonBlocking) != cudaSuccess) {
      delete m;
      return CBL_ERR_CUDA;
    }
    m->own = true;
  }
  bool ok = cudaMalloc(&m->w, NPARAM * 4) == cudaSuccess && cudaMalloc(&m->wb, NPARAM * 2) == cudaSuccess &&
            cudaMalloc(&m->g, NPARAM * 4) == cudaSuccess && cudaMalloc(&m->m, NPARAM * 4) == cudaSuccess &&
            cudaMalloc(&m->v, NPARAM * 4) == cudaSuccess && cudaMalloc(&m->loss, 4) == cudaSuccess;
  if (!ok) {
    cbl_mlp_destroy(m);
    return CBL_ERR_OOM;
  }
  cudaMemsetAsync(m->w, 0, NPARAM * 4, m->s);
  cudaMemsetAsync(m->g, 0, NPARAM * 4, m->s);
  cudaMemsetAsync(m->m, 0, NPARAM * 4, m->s);
  cudaMemsetAsync(m->v, 0, NPARAM * 4, m->s);
  cudaMemsetAsync(m->wb, 0, NPARAM * 2, m->s);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
    attr = true;
  }
  *out = m;
  return cudaGetLastError() == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

int64_t cbl_mlp_num_params(const cbl_mlp* m) { return m ? NPARAM : 0; }

cbl_status cbl_mlp_set_params(cbl_mlp* m, const float* host) {
  if (!m || !host) return CBL_ERR_ARG;
  if (cudaMemcpyAsync(m->w, host, NPARAM * 4, cudaMemcpyHostToDevice, m->s) != cudaSuccess) return CBL_ERR_CUDA;
  k_round_bf16<<<(NPARAM + 255) / 256, 256, 0, m->s>>>(m->w, m->wb);
  cudaMemsetAsync(m->m, 0, NPARAM * 4, m->s);
  cudaMemsetAsync(m->v, 0, NPARAM * 4, m->s);
  m->t = 0;
  return cudaStreamSynchronize(m->s) == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

cbl_status cbl_mlp_get_params(cbl_mlp* m, float* host) {
  if (!m || !host) return CBL_ERR_ARG;
  if (cudaMemcpyAsync(host, m->w, NPARAM * 4, cudaMemcpyDeviceToHost, m->s) != cudaSuccess) return CBL_ERR_CUDA;
  return cudaStreamSynchronize(m->s) == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

cbl_status cbl_mlp_forward(cbl_mlp* m, const float* x, float* y, int n) {
  if (!m || !x || !y || n < 0) return CBL_ERR_ARG;
  if (n == 0) return CBL_OK;
  k_mlp_fwd<<<(n + 127) / 128, 128, 0, m->s>>>(m->wb, x, y, n);
  return cudaGetLastError() == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

cbl_status cbl_mlp_advance(cbl_mlp* m, double* X, double* V, double* Wang, const double* M, const double* Iinv,
                           const double* R, const int* fixed, const double* bias, const int* pairs, const double* VL,
                           int nb, int npairs, int steps, const int* dims, double cos_theta, const float* norm,
                           double sigma) {
  if (!m || !X || !V || !Wang || !M || !Iinv || !R || !fixed || !bias || !dims || !norm) return CBL_ERR_ARG;
  if (nb <= 0 || nb > 2048 || npairs < 0 || (npairs && (!pairs || !VL)) || steps < 0) return CBL_ERR_ARG;
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || !(sigma > 0)) return CBL_ERR_ARG;
  for (int k = 0; k < 4 * IN + 2 * OUT; ++k)
    if (!std::isfinite(norm[k])) return CBL_ERR_ARG;
  for (int k = 0; k < IN; ++k)
    if (!(norm[IN + k] > 0) || norm[2 * IN + k] > norm[3 * IN + k]) return CBL_ERR_ARG;
  if (steps == 0) return CBL_OK;
  AdvNorm nm;
  std::memcpy(&nm, norm, sizeof(nm));
  const size_t smem = ((NPARAM * sizeof(__nv_bfloat16) + 15) / 16) * 16 + sizeof(double) * 6 * (size_t)nb;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_advance, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_mlp_advance<<<1, 256, smem, m->s>>>(m->wb, X, V, Wang, M, Iinv, R, fixed, bias, pairs, VL, nb, npairs, steps,
                                        dims[0], dims[1], dims[2], cos_theta, nm, sigma);
  return cudaGetLastError() == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

cbl_status cbl_mlp_grad(cbl_mlp* m, const float* x, const float* t, int n, float* loss_host) {
  if (!m || !x || !t || n <= 0) return CBL_ERR_ARG;
  cudaMemsetAsync(m->loss, 0, 4, m->s);
  k_mlp_grad<<<(n + BS - 1) / BS, 256, sizeof(TrainSmem), m->s>>>(m->wb, x, t, n, m->g, m->loss);
  if (cudaGetLastError() != cudaSuccess) return CBL_ERR_CUDA;
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, m->loss, 4, cudaMemcpyDeviceToHost, m->s) != cudaSuccess) return CBL_ERR_CUDA;
    if (cudaStreamSynchronize(m->s) != cudaSuccess) return CBL_ERR_CUDA;
  }
  return CBL_OK;
}

cbl_status cbl_mlp_read_grad(cbl_mlp* m, float* host) {
  if (!m || !host) return CBL_ERR_ARG;
  if (cudaMemcpyAsync(host, m->g, NPARAM * 4, cudaMemcpyDeviceToHost, m->s) != cudaSuccess) return CBL_ERR_CUDA;
  return cudaStreamSynchronize(m->s) == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

cbl_status cbl_mlp_zero_grad(cbl_mlp* m) {
  if (!m) return CBL_ERR_ARG;
  return cudaMemsetAsync(m->g, 0, NPARAM * 4, m->s) == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

cbl_status cbl_mlp_adam_step(cbl_mlp* m, float lr, float beta1, float beta2, float eps) {
  if (!m || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1)) return CBL_ERR_ARG;
  m->t += 1;
  const float c1 = 1.f - powf(beta1, (float)m->t), c2 = 1.f - powf(beta2, (float)m->t);
  k_adam<<<(NPARAM + 255) / 256, 256, 0, m->s>>>(m->w, m->wb, m->g, m->m, m->v, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

cbl_status cbl_mlp_sync(cbl_mlp* m) {
  if (!m) return CBL_ERR_ARG;
  return cudaStreamSynchronize(m->s) == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}

cbl_status cbl_mlp_destroy(cbl_mlp* m) {
  if (!m) return CBL_OK;
  if (m->s) cudaStreamSynchronize(m->s);
  cudaFree(m->w);
  cudaFree(m->wb);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->loss);
  if (m->own) cudaStreamDestroy(m->s);
  delete m;
  return CBL_OK;
}

}  // extern "C"
