// Access-pattern probe for the roofline of the collision pass (run by `bench.py --pattern-probe`,
// not part of the library): the bandwidth of the D3Q19 pull-stream pattern on a 128x128x256 FP32
// lattice without any collision arithmetic, against the same 38 streams without the pull offsets
// and a plain copy. pull19: each cell loads its 19 populations from x - c_i (periodic) and stores
// them at x; pullrow: the same with every load aligned (one block per x-row, the x shift done with
// warp shuffles and shared memory at the warp edges); local38: 19 loads and 19 stores at x; copy:
// one contiguous copy of the same bytes. Prints one line per kernel and round, then a check that
// pull19 and pullrow store the same values, then the FP32 and FP64 FMA throughput (independent
// chains, all SMs).
#include <cstdio>
#include <cuda_runtime.h>
#include <cstdlib>
__constant__ int cx[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int cy[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ int cz[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
__global__ void __launch_bounds__(128) pull(const float* __restrict__ a, float* __restrict__ b, int nx, int ny, int nz, long long st) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 4 + (threadIdx.x >> 5);
  const int z = blockIdx.z;
  if (x >= nx || y >= ny) return;
  const long long n = x + (long long)nx * (y + (long long)ny * z);
  float f[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    int xs = x - cx[i], ys = y - cy[i], zs = z - cz[i];
    xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
    f[i] = a[i * st + xs + (long long)nx * (ys + (long long)ny * zs)];
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) s += f[i];
#pragma unroll
  for (int i = 0; i < 19; ++i) b[i * st + n] = f[i] + 1e-30f * s;
}

// one block per x-row (nx == blockDim.x, a multiple of 32): every population is loaded aligned from
// row (y - cy, z - cz); the x shift by cx = +-1 is done on chip (warp shuffle, shared memory at warp
// edges, periodic wrap inside the row)
__global__ void __launch_bounds__(128) pullrow(const float* __restrict__ a, float* __restrict__ b, int nx, int ny, int nz, long long st) {
  __shared__ float edge[19][2][4];  // [population][0: lane 31 value, 1: lane 0 value][warp]
  const int x = threadIdx.x, y = blockIdx.x, z = blockIdx.y;
  const int lane = x & 31, wid = x >> 5, nw = blockDim.x >> 5;
  const long long n = x + (long long)nx * (y + (long long)ny * z);
  float raw[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    int ys = y - cy[i], zs = z - cz[i];
    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
    raw[i] = a[i * st + x + (long long)nx * (ys + (long long)ny * zs)];
  }
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    if (lane == 31) edge[i][0][wid] = raw[i];
    if (lane == 0) edge[i][1][wid] = raw[i];
  }
  __syncthreads();
  float f[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    if (cx[i] == 0) { f[i] = raw[i]; continue; }
    if (cx[i] == 1) {  // value at x - 1
      float v = __shfl_up_sync(0xffffffffu, raw[i], 1);
      if (lane == 0) v = edge[i][0][(wid + nw - 1) % nw];
      f[i] = v;
    } else {           // value at x + 1
      float v = __shfl_down_sync(0xffffffffu, raw[i], 1);
      if (lane == 31) v = edge[i][1][(wid + 1) % nw];
      f[i] = v;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) s += f[i];
#pragma unroll
  for (int i = 0; i < 19; ++i) b[i * st + n] = f[i] + 1e-30f * s;
}


// FMA throughput: 8 independent chains per thread, ITER iterations; one store per thread keeps the
// chains live
template <typename T>
__global__ void __launch_bounds__(256) fma_rate(T* out, int iter, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iter; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(128) local38(const float* __restrict__ a, float* __restrict__ b, int nx, int ny, int nz, long long st) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 4 + (threadIdx.x >> 5);
  const int z = blockIdx.z;
  if (x >= nx || y >= ny) return;
  const long long n = x + (long long)nx * (y + (long long)ny * z);
  float f[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = a[i * st + n];
#pragma unroll
  for (int i = 0; i < 19; ++i) b[i * st + n] = f[i];
}
__global__ void copy1(const float4* __restrict__ a, float4* __restrict__ b, long long n4) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) b[i] = a[i];
}
int main() {
  const int nx = 128, ny = 128, nz = 256;
  const long long N = (long long)nx * ny * nz, st = N + 4096;
  float *a, *b;
  cudaMalloc(&a, 19 * st * 4); cudaMalloc(&b, 19 * st * 4);
  cudaMemset(a, 0, 19 * st * 4); cudaMemset(b, 0, 19 * st * 4);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  dim3 g(nx / 32, ny / 4, nz);
  const double bytes = 2.0 * 19 * 4 * N;
  for (int k = 0; k < 3; ++k) {
    float ms;
    for (int w = 0; w < 5; ++w) pull<<<g, 128>>>(a, b, nx, ny, nz, st);
    cudaEventRecord(e0); for (int r = 0; r < 50; ++r) { pull<<<g, 128>>>(k & 1 ? b : a, k & 1 ? a : b, nx, ny, nz, st); } cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1); printf("pull19   %.1f us  %.1f GB/s\n", ms * 1000 / 50, bytes / (ms / 50 * 1e-3) / 1e9);
    cudaEventRecord(e0); for (int r = 0; r < 50; ++r) pullrow<<<dim3(ny, nz), nx>>>(a, b, nx, ny, nz, st); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1); printf("pullrow  %.1f us  %.1f GB/s\n", ms * 1000 / 50, bytes / (ms / 50 * 1e-3) / 1e9);
    cudaEventRecord(e0); for (int r = 0; r < 50; ++r) local38<<<g, 128>>>(a, b, nx, ny, nz, st); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1); printf("local38  %.1f us  %.1f GB/s\n", ms * 1000 / 50, bytes / (ms / 50 * 1e-3) / 1e9);
    long long n4 = 19 * st / 4;
    cudaEventRecord(e0); for (int r = 0; r < 50; ++r) copy1<<<152 * 8, 256>>>((const float4*)a, (float4*)b, n4); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1); printf("copy     %.1f us  %.1f GB/s\n", ms * 1000 / 50, 2.0 * 19 * st * 4 / (ms / 50 * 1e-3) / 1e9);
  }
  {
    float* h = (float*)malloc(19 * st * 4);
    for (long long k = 0; k < 19 * st; ++k) h[k] = (float)((k * 2654435761u) % 1000) * 1e-3f;
    cudaMemcpy(a, h, 19 * st * 4, cudaMemcpyHostToDevice);
    float *c; cudaMalloc(&c, 19 * st * 4);
    pull<<<g, 128>>>(a, b, nx, ny, nz, st);
    pullrow<<<dim3(ny, nz), nx>>>(a, c, nx, ny, nz, st);
    float* h2 = (float*)malloc(19 * st * 4);
    cudaMemcpy(h, b, 19 * st * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(h2, c, 19 * st * 4, cudaMemcpyDeviceToHost);
    long long bad = 0;
    for (int i = 0; i < 19; ++i) for (long long k = 0; k < N; ++k) bad += h[i * st + k] != h2[i * st + k];
    printf("pullrow mismatches vs pull: %lld\n", bad);
  }
  {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = nsm * 8, threads = 256;
    float* o32; double* o64;
    cudaMalloc(&o32, (size_t)blocks * threads * sizeof(float));
    cudaMalloc(&o64, (size_t)blocks * threads * sizeof(double));
    float ms;
    const int it32 = 4096, it64 = 64;
    fma_rate<float><<<blocks, threads>>>(o32, it32, 0.999f, 0.001f);
    cudaEventRecord(e0); fma_rate<float><<<blocks, threads>>>(o32, it32, 0.999f, 0.001f); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fma32    %.1f us  %.1f TFLOP/s\n", ms * 1000, 2.0 * 8 * it32 * (double)blocks * threads / (ms * 1e-3) / 1e12);
    fma_rate<double><<<blocks, threads>>>(o64, it64, 0.999, 0.001);
    cudaEventRecord(e0); fma_rate<double><<<blocks, threads>>>(o64, it64, 0.999, 0.001); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fma64    %.1f us  %.3f TFLOP/s\n", ms * 1000, 2.0 * 8 * it64 * (double)blocks * threads / (ms * 1e-3) / 1e12);
    cudaFree(o32); cudaFree(o64);
  }
  printf("err %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
