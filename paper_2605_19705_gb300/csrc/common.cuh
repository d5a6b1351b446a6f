// Shared device/host helpers of the i-DEQ CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstdio>

#define IDEQ_DEV __device__ __forceinline__

namespace ideq {


template <typename T> IDEQ_DEV float ld_f(const T* p);
template <> IDEQ_DEV float ld_f<float>(const float* p) { return *p; }
template <> IDEQ_DEV float ld_f<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <> IDEQ_DEV float ld_f<__half>(const __half* p) { return __half2float(*p); }

template <typename T> IDEQ_DEV T from_f(float v);
template <> IDEQ_DEV float from_f<float>(float v) { return v; }
template <> IDEQ_DEV __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> IDEQ_DEV __half from_f<__half>(float v) { return __float2half_rn(v); }

IDEQ_DEV double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
IDEQ_DEV float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of a double over all threads of a (1-, 2- or 3-D)
// block whose size is a multiple of 32 (<= 1024).  Every thread must call it;
// the result is valid in linear thread 0.
IDEQ_DEV double block_sum(double v, double* red /* >= 32 doubles of shared */) {
  v = warp_sum(v);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, wid = tid >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    const int nw = (nthr + 31) >> 5;
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// softplus(h) = log(1 + e^h) = max(h, 0) + log(1 + e^-|h|), its derivative the
// logistic 1 / (1 + e^-h); fast-path intrinsics (a few ulp, far below the
// 16-bit storage of the tensor-core forms and the 1e-5 FP32 tolerance).
IDEQ_DEV float softplus_f(float h) { return fmaxf(h, 0.f) + __logf(1.f + __expf(-fabsf(h))); }
IDEQ_DEV float sigmoid_f(float h) { return __fdividef(1.f, 1.f + __expf(-h)); }

}  // namespace ideq

namespace ideq {

// Fused conv epilogue on one accumulator value v (see Epi in ideq_internal.h).
// a0..a2 are the auxiliary inputs at the output element; o2 is written only by
// the epilogues that have a second output.
IDEQ_DEV float epi_math(int epi, int act, float v, float a0, float a1, float a2, float* o2) {
  switch (epi) {
    case 1: {  // EP_ACT
      if (act == 0) { *o2 = sigmoid_f(v); return softplus_f(v); }
      *o2 = v > 0.f ? 1.f : 0.f;
      return fmaxf(v, 0.f);
    }
    case 2: return v + a0;                              // EP_ADD
    case 3: return v * a0;                              // EP_MUL
    case 4: *o2 = v; return v * a0;                     // EP_MUL_KEEP
    case 5: return a0 * v + a0 * (1.f - a0) * a1 * a2;  // EP_DUAL
    default: return v;                                  // EP_STORE
  }
}

IDEQ_DEV bool epi_reads_aux0(int epi) { return epi >= 2; }
IDEQ_DEV bool epi_has_out2(int epi) { return epi == 1 || epi == 4; }

}  // namespace ideq
