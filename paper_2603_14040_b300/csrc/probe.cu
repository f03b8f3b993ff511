// Diagnostic: the FP64 fused multiply-add rate of the current GPU, measured with CUDA events on
// a kernel of independent FMA chains. The FP64 stencils of this library (the operator, the FP64
// smoother, the Krylov passes) are bound by this rate rather than by HBM on B300, so their roofline
// is reported against this measured number.
#include <cuda_runtime.h>

#include "../../include/pyro.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

// kChains independent chains x <- x * m + c per thread, `iters` times; the chains' sum is stored
// (only by a thread whose sum is exactly 12345, which never happens for these inputs) so that the
// compiler keeps the arithmetic
__global__ void k_fp64_fma_chains(int iters, double m, double c, double* __restrict__ sink) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == 12345.0) sink[0] = s;
}

}  // namespace

extern "C" int pyro_fp64_fma_rate(int iters, double* tflops, void* cuda_stream) {
  if (iters < 1 || !tflops) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PYRO_E_CUDA;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int status = PYRO_OK;
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) { cudaGetLastError(); return PYRO_E_NOMEM; }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) status = PYRO_E_CUDA;
  const int blocks = sms * 8;
  if (status == PYRO_OK) {
    k_fp64_fma_chains<<<blocks, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-7, sink);   // warm-up
    cudaEventRecord(e0, s);
    k_fp64_fma_chains<<<blocks, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-7, sink);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
      status = PYRO_E_CUDA;
    else
      *tflops = 2.0 * kChains * (double)iters * blocks * kProbeThreads / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (status != PYRO_OK) cudaGetLastError();
  return status;
}
