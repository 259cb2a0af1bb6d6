// bench_fma_probe.cu -- measurement aid of bench.py, not part of the library:
// throughput of the plain FP64 / FP32 fused multiply-add pipes, the roofline
// denominators of the element kernels (which do their arithmetic on these
// pipes).  bench.py compiles it into bench_fma_probe.so on first use.
//
//   int fma_probe_tflops(int fp64, double* tflops)
//     one timed launch of independent FMA chains on every SM of the current
//     device (legacy default stream, synchronous); 0 on success.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == (T)-12345.0) out[threadIdx.x] = s;   // keeps the chains live
}

template <typename T>
int probe(double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 2048 : 65536;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  k_fma_probe<T><<<blocks, threads>>>(nullptr, 16, (T)0.999999, (T)1e-7);   // warm-up
  cudaEventRecord(e0);
  k_fma_probe<T><<<blocks, threads>>>(nullptr, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1;
  *tflops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return 0;
}

}  // namespace

extern "C" int fma_probe_tflops(int fp64, double* tflops) {
  if (!tflops) return 1;
  return fp64 ? probe<double>(tflops) : probe<float>(tflops);
}
