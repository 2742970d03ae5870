// FMA throughput microbenchmark (see include/nrmg_peak.h): 8 independent FMA chains per
// thread so that the FMA pipe, not the dependent-issue latency, limits the rate.
#include "nrmg_peak.h"

#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T *out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-7, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
int run(int iters, cudaStream_t st, double *res) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  const int threads = 256, blocks = nsm * 8;
  T *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(T) * threads * blocks) != cudaSuccess) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // warm-up, then the timed launch
  fma_chains<T><<<blocks, threads, 0, st>>>(buf, iters / 10 + 1, (T)0.999999, (T)1e-6);
  cudaEventRecord(e0, st);
  fma_chains<T><<<blocks, threads, 0, st>>>(buf, iters, (T)0.999999, (T)1e-6);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess || ms <= 0.f) return 2;
  double flops = 2.0 * 8.0 * 16.0 * (double)iters * threads * blocks;
  *res = flops / (ms * 1e-3);
  return 0;
}

}  // namespace

extern "C" int nrmg_peak_fma(int precision, int iters, void *cuda_stream, double *flops_per_s) {
  if (!flops_per_s || iters < 1 || (precision != 0 && precision != 1)) return 1;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  return precision == 0 ? run<double>(iters, st, flops_per_s) : run<float>(iters, st, flops_per_s);
}
