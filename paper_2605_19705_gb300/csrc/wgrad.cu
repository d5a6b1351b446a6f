// Weight gradients of the implicit-GEMM convolutions (SIMT, FP32 arithmetic).
//
// For a conv with forward GEMM out[m][n] = sum_k A[m][k] B[n][k] (ConvArgs), the
// gradient of <cot, out> in B is dB[n][k] = sum_m cot[m][n] A[m][k].  A is
// gathered exactly as in the forward pass (3x3 taps, stride-2 2x2, pixelwise,
// NHWC or NCHW input); cot is read through the forward's output map (NHWC,
// 2x2 depth-to-space or f32 NCHW).  The pixel sum is split over blockIdx.z;
// each split writes its partial tile and wgrad_reduce sums the splits in a fixed
// order (deterministic), scales and adds into a [N][K] f32 accumulator.
#include "common.cuh"
#include "ideq_internal.h"
#include "net_train.h"

namespace ideq {

constexpr int WB = 64;   // n and k tile
constexpr int WM = 16;   // pixels per chunk

template <typename T>
__device__ __forceinline__ float wg_load_a(const ConvArgs& a, const T* in, long long m, int k,
                                           int K) {
  if (k >= K) return 0.f;
  const int HW = a.H * a.W;
  const int img = (int)(m / HW);
  const int rem = (int)(m - (long long)img * HW);
  const int y = rem / a.W, x = rem - (rem / a.W) * a.W;
  int sy, sx, ci;
  const int SH = a.mode == CM_DOWN ? 2 * a.H : a.H;
  const int SW = a.mode == CM_DOWN ? 2 * a.W : a.W;
  if (a.mode == CM_CONV3) {
    const int t = k / a.Cin;
    ci = k - t * a.Cin;
    sy = y + t / 3 - 1;
    sx = x + t % 3 - 1;
  } else if (a.mode == CM_DOWN) {
    const int q = k / a.Cin;
    ci = k - q * a.Cin;
    sy = 2 * y + (q >> 1);
    sx = 2 * x + (q & 1);
  } else {
    ci = k;
    sy = y;
    sx = x;
  }
  if (sy < 0 || sy >= SH || sx < 0 || sx >= SW) return 0.f;
  if (a.in_nchw) return ((const float*)in)[(((size_t)img * a.Cin + ci) * SH + sy) * SW + sx];
  return ld_f(in + (((size_t)img * SH + sy) * SW + sx) * a.Cin + ci);
}

template <typename T>
__device__ __forceinline__ float wg_load_cot(const ConvArgs& a, const void* cot, long long m,
                                             int n, int N) {
  if (n >= N) return 0.f;
  const int HW = a.H * a.W;
  const int img = (int)(m / HW);
  const int rem = (int)(m - (long long)img * HW);
  const int y = rem / a.W, x = rem - (rem / a.W) * a.W;
  if (a.out_nchw) return ((const float*)cot)[(((size_t)img * a.Cout + n) * a.H + y) * a.W + x];
  size_t o;
  if (a.outmap == OM_D2S) {
    const int q = n / a.Cout, co = n - q * a.Cout;
    o = (((size_t)img * 2 * a.H + 2 * y + (q >> 1)) * 2 * a.W + 2 * x + (q & 1)) * a.Cout + co;
  } else {
    o = (size_t)m * a.Cout + n;
  }
  return ld_f((const T*)cot + o);
}

template <typename T>
__global__ void __launch_bounds__(256) wgrad_kernel(ConvArgs a, const void* cot,
                                                    long long m_per_split, float* part) {
  __shared__ float Cs[WM][WB + 4];
  __shared__ float As[WM][WB + 4];
  const int N = a.N(), K = a.K();
  const long long M = a.M();
  const int n0 = blockIdx.x * WB, k0 = blockIdx.y * WB;
  const long long mb = (long long)blockIdx.z * m_per_split;
  const long long me = mb + m_per_split < M ? mb + m_per_split : M;
  const int tid = threadIdx.x;
  const int tn = tid >> 4, tk = tid & 15;  // 16 x 16 threads, 4 x 4 outputs each
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const T* in = (const T*)a.in;
  for (long long m0 = mb; m0 < me; m0 += WM) {
    for (int e = tid; e < WM * WB; e += 256) {
      const int mm = e / WB, j = e % WB;
      const long long m = m0 + mm;
      const bool ok = m < me;
      Cs[mm][j] = ok ? wg_load_cot<T>(a, cot, m, n0 + j, N) : 0.f;
      As[mm][j] = ok ? wg_load_a<T>(a, in, m, k0 + j, K) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < WM; ++mm) {
      float c[4], v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) c[i] = Cs[mm][tn * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = As[mm][tk * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(c[i], v[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* p = part + (size_t)blockIdx.z * N * K;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = n0 + tn * 4 + i;
    if (n >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + tk * 4 + j;
      if (k < K) p[(size_t)n * K + k] = acc[i][j];
    }
  }
}

__global__ void wgrad_reduce_kernel(long long nk, int splits, const float* __restrict__ part,
                                    float scale, float* __restrict__ dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nk;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * nk + e];
    dst[e] += scale * (float)s;
  }
}

int wgrad_splits(const ConvArgs& a) {
  const long long M = a.M();
  const int tiles = ((a.N() + WB - 1) / WB) * ((a.K() + WB - 1) / WB);
  long long s = (152 * 4 + tiles - 1) / tiles;  // about four waves of blocks
  s = s < 1 ? 1 : s;
  const long long maxs = (M + 255) / 256;      // at least 256 pixels per split
  if (s > maxs) s = maxs;
  if (s > 256) s = 256;
  return (int)s;
}

cudaError_t launch_wgrad(const ConvArgs& a, int in_dt, int cot_dt, const void* cot, float scale,
                         float* part, float* dst, cudaStream_t st) {
  const long long M = a.M();
  if (M == 0) return cudaSuccess;
  if (in_dt != cot_dt && !a.in_nchw && !a.out_nchw) return cudaErrorInvalidValue;
  const int splits = wgrad_splits(a);
  const long long mps = ((M + splits - 1) / splits + WM - 1) / WM * WM;
  dim3 grid((a.N() + WB - 1) / WB, (a.K() + WB - 1) / WB, splits);
  // the feature-side type decides the template; NCHW sides are always f32
  const int dt = a.in_nchw ? cot_dt : in_dt;
  if (dt == DT_BF16)
    wgrad_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(a, cot, mps, part);
  else if (dt == DT_F16)
    wgrad_kernel<__half><<<grid, 256, 0, st>>>(a, cot, mps, part);
  else
    wgrad_kernel<float><<<grid, 256, 0, st>>>(a, cot, mps, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_wgrad_reduce((long long)a.N() * a.K(), splits, part, scale, dst, st);
}

cudaError_t launch_wgrad_reduce(long long nk, int splits, const float* part, float scale,
                                float* dst, cudaStream_t st) {
  const int blocks = (int)std::min<long long>((nk + 255) / 256, 2048);
  wgrad_reduce_kernel<<<blocks, 256, 0, st>>>(nk, splits, part, scale, dst);
  return cudaGetLastError();
}

}  // namespace ideq
