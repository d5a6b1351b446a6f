// FP32 FFMA throughput microbenchmark: the roofline of the plain FP32 form, whose
// convolutions run on the SIMT pipes.
#include <cuda_runtime.h>

#include "ideq_internal.h"

namespace ideq {

constexpr int kFmaChains = 8;     // independent accumulators per thread
constexpr int kFmaIters = 8192;   // FMAs per chain

// Each thread advances kFmaChains independent FMA chains (latency hidden by the
// chains and by 2 resident blocks of 512 threads per SM) and writes one value so
// that nothing is eliminated.
__global__ void __launch_bounds__(512) fma_peak_kernel(float a, float b, float* out) {
  float acc[kFmaChains];
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) acc[c] = (float)(threadIdx.x + c);
#pragma unroll 4
  for (int i = 0; i < kFmaIters; ++i) {
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) acc[c] = fmaf(acc[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) s += acc[c];
  if (s == 12345.678f) out[0] = s;  // practically never true; keeps the chains live
}

}  // namespace ideq

extern "C" ideq_status ideq_fp32_fma_peak(void* stream, double* tflops) {
  using namespace ideq;
  (void)cudaGetLastError();
  if (!tflops) return IDEQ_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IDEQ_ERR_CUDA;
  float* out = nullptr;
  if (cudaMallocAsync((void**)&out, 16, st) != cudaSuccess) return IDEQ_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = 2 * sms, threads = 512;
  fma_peak_kernel<<<blocks, threads, 0, st>>>(0.999f, 1e-3f, out);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, st);
    fma_peak_kernel<<<blocks, threads, 0, st>>>(0.999f, 1e-3f, out);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t > 0.f && t < best) best = t;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  if (e != cudaSuccess) return IDEQ_ERR_CUDA;
  const double flop = 2.0 * blocks * threads * (double)kFmaChains * kFmaIters;
  *tflops = flop / (best * 1e-3) / 1e12;
  return IDEQ_OK;
}
