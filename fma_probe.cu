// FMA throughput probe used by bench.py for the denominators of the ALU-bound
// rooflines (the FP64 pipe bounds the TT arithmetic of the solver).  It is a
// measurement helper of the benchmark, not part of the solver library: built
// into its own shared library with one C entry point.
//
// Every thread runs eight independent FMA chains so the pipe, not the chain
// latency, limits the rate; four CTAs of 256 threads per SM, timed with CUDA
// events on a stream of its own after one warm-up launch.
#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)12345.678) out[0] = s;  // keeps the chains alive; practically never taken
}

template <typename T> int probe(cudaStream_t st, int sms, int iters, double *tflops) {
  const int grid = 4 * sms, threads = 256;
  T *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return -2;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = -3;
  if (!rc) {
    k_fma_probe<T><<<grid, threads, 0, st>>>(out, iters / 8, (T)0.999, (T)1e-3);  // warm-up
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<grid, threads, 0, st>>>(out, iters, (T)0.999, (T)1e-3);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
      rc = -3;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (!rc) *tflops = 2.0 * 8.0 * (double)iters * grid * threads / (ms * 1e-3) / 1e12;
  return rc;
}

}  // namespace

// Measured FP64 and FP32 FMA throughput (TFLOP/s, one FMA = 2 FLOP) of `device`.
// Returns 0, or -1 (bad argument), -2 (allocation failed), -3 (CUDA error).
extern "C" int fma_probe_tflops(int device, double *fp64_tflops, double *fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return -1;
  if (cudaSetDevice(device) != cudaSuccess) return -3;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) return -3;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -3;
  int rc = probe<double>(st, sms, 1 << 12, fp64_tflops);
  if (!rc) rc = probe<float>(st, sms, 1 << 16, fp32_tflops);
  cudaStreamDestroy(st);
  return rc;
}
