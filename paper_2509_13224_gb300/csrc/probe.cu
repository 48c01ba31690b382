// Measured arithmetic throughput of this GPU, for roofline denominators of the
// ALU-bound kernels (the FP64 pipe bounds the TT arithmetic of the solver).
// Every thread runs eight independent FMA chains so the pipe, not the chain
// latency, limits the rate; four CTAs of 256 threads per SM.
#include "common.cuh"

namespace ttiga {

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

template <typename T> double probe(Ctx *c, int iters) {
  const int grid = 4 * c->num_sms, threads = 256;
  DBuf out(c, sizeof(T));
  cudaEvent_t e0, e1;
  TTI_CUDA(cudaEventCreate(&e0));
  TTI_CUDA(cudaEventCreate(&e1));
  k_fma_probe<T><<<grid, threads, 0, c->stream>>>(out.as<T>(), iters / 8, (T)0.999, (T)1e-3);  // warm-up
  TTI_LAUNCH();
  TTI_CUDA(cudaEventRecord(e0, c->stream));
  k_fma_probe<T><<<grid, threads, 0, c->stream>>>(out.as<T>(), iters, (T)0.999, (T)1e-3);
  TTI_LAUNCH();
  TTI_CUDA(cudaEventRecord(e1, c->stream));
  TTI_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  TTI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8.0 * (double)iters * grid * threads;
  return flops / (ms * 1e-3) / 1e12;
}

}  // namespace

void fma_peaks(Ctx *c, double *fp64_tflops, double *fp32_tflops) {
  if (fp64_tflops) *fp64_tflops = probe<double>(c, 1 << 12);
  if (fp32_tflops) *fp32_tflops = probe<float>(c, 1 << 16);
}

}  // namespace ttiga
