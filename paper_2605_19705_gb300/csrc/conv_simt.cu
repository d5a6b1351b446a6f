// SIMT implicit-GEMM convolution (FP32 arithmetic) for the plain FP32 form,
// for layers whose channel counts are too small for the tensor-core path
// (head 3->64, tail 64->3 and their transposes, the tiny 1->32 nets), and as the
// reference-free baseline of the tensor-core kernel.  See ConvArgs for the
// GEMM view and the epilogues.
#include "common.cuh"
#include "ideq_internal.h"

namespace ideq {

template <typename TIn, typename TOut, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    conv_simt_kernel(ConvArgs a) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int BK = 16;
  constexpr int AR = NT / BK;   // A rows loaded per pass
  constexpr int APT = BM / AR;  // A loads per thread
  static_assert(NT % BK == 0 && BM % AR == 0, "tile");
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  __shared__ double simg[BM];

  const int tid = threadIdx.x;
  const long long M = a.M();
  const int N = a.N(), K = a.K();
  const long long m0 = (long long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int HW = a.H * a.W;
  if (a.skip) {  // every image this block touches is frozen in a solve: nothing needed
    const long long m_last = (m0 + BM < M ? m0 + BM : M) - 1;
    bool any = false;
    for (long long i = m0 / HW; i <= m_last / HW; ++i) any |= a.skip[i] == 0;
    if (!any) return;
  }
  const TIn* __restrict__ in = (const TIn*)a.in;
  const float* __restrict__ inf = (const float*)a.in;
  const float* __restrict__ wf = (const float*)a.wB;

  // rows this thread loads for A
  const int ak = tid % BK;
  int r_img[APT], r_y[APT], r_x[APT];
  bool r_ok[APT];
#pragma unroll
  for (int i = 0; i < APT; ++i) {
    const long long m = m0 + tid / BK + i * AR;
    r_ok[i] = m < M;
    const long long mm = r_ok[i] ? m : 0;
    r_img[i] = (int)(mm / HW);
    const int rem = (int)(mm % HW);
    r_y[i] = rem / a.W;
    r_x[i] = rem % a.W;
  }
  // source image size of the A gather
  const int SH = a.mode == CM_DOWN ? 2 * a.H : a.H;
  const int SW = a.mode == CM_DOWN ? 2 * a.W : a.W;

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  const int tn = tid % (BN / TN), tm = tid / (BN / TN);

  for (int k0 = 0; k0 < K; k0 += BK) {
    const int kg = k0 + ak;
    int dy = 0, dx = 0, ci = kg;
    if (a.mode == CM_CONV3) {
      const int t = kg / a.Cin;
      ci = kg - t * a.Cin;
      dy = t / 3 - 1;
      dx = t % 3 - 1;
    } else if (a.mode == CM_DOWN) {
      const int q = kg / a.Cin;
      ci = kg - q * a.Cin;
      dy = q >> 1;
      dx = q & 1;
    }
#pragma unroll
    for (int i = 0; i < APT; ++i) {
      float v = 0.f;
      if (r_ok[i] && kg < K) {
        int sy, sx;
        if (a.mode == CM_DOWN) {
          sy = 2 * r_y[i] + dy;
          sx = 2 * r_x[i] + dx;
        } else {
          sy = r_y[i] + dy;
          sx = r_x[i] + dx;
        }
        if (sy >= 0 && sy < SH && sx >= 0 && sx < SW) {
          if (a.in_nchw)
            v = inf[(((size_t)r_img[i] * a.Cin + ci) * SH + sy) * SW + sx];
          else
            v = ld_f(in + (((size_t)r_img[i] * SH + sy) * SW + sx) * a.Cin + ci);
        }
      }
      As[ak][tid / BK + i * AR] = v;
    }
    for (int e = tid; e < BK * BN; e += NT) {
      const int kk = e % BK, nn = e / BK;
      const int gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? wf[(size_t)gn * K + gk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float ar[TM], br[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) ar[i] = As[kk][tm * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) br[j] = Bs[kk][tn * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
    }
    __syncthreads();
  }

  // ---------------- epilogue
  const bool sums = a.epi == EP_AXPY_NCHW && a.sumsq != nullptr;
  const int img_first = (int)(m0 / HW);
  if (sums) {
    for (int i = tid; i < BM; i += NT) simg[i] = 0.0;
    __syncthreads();
  }
  TOut* out = (TOut*)a.out;
  TOut* out2 = (TOut*)a.out2;
  const TOut* aux0 = (const TOut*)a.aux0;
  const TOut* aux1 = (const TOut*)a.aux1;
  const TOut* aux2 = (const TOut*)a.aux2;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const long long m = m0 + tm * TM + i;
    if (m >= M) continue;
    const int img = (int)(m / HW);
    const int rem = (int)(m % HW);
    const int y = rem / a.W, x = rem % a.W;
    double ssq = 0.0;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tn * TN + j;
      if (n >= N) continue;
      const float v = acc[i][j];
      if (a.epi == EP_AXPY_NCHW) {
        const size_t o = (((size_t)img * a.Cout + n) * a.H + y) * a.W + x;
        const float r = ((const float*)a.aux0)[o] + a.sign * v;
        ((float*)a.out)[o] = r;
        ssq += 0.5 * (double)r * (double)r;
        continue;
      }
      size_t o;
      if (a.outmap == OM_D2S) {
        const int q = n / a.Cout, co = n - q * a.Cout;
        const int oy = 2 * y + (q >> 1), ox = 2 * x + (q & 1);
        o = (((size_t)img * 2 * a.H + oy) * 2 * a.W + ox) * a.Cout + co;
      } else {
        o = (size_t)m * a.Cout + n;
      }
      const float x0 = aux0 ? ld_f(aux0 + o) : 0.f;
      const float x1 = aux1 ? ld_f(aux1 + o) : 0.f;
      const float x2 = aux2 ? ld_f(aux2 + o) : 0.f;
      float o2 = 0.f;
      const float r = epi_math(a.epi, a.act, v, x0, x1, x2, &o2);
      out[o] = from_f<TOut>(r);
      if (epi_has_out2(a.epi)) out2[o] = from_f<TOut>(o2);
    }
    if (sums && ssq != 0.0) atomicAdd(&simg[img - img_first], ssq);
  }
  if (sums) {
    __syncthreads();
    const long long mlast = (m0 + BM - 1 < M ? m0 + BM - 1 : M - 1);
    const int nimg = (int)(mlast / HW) - img_first + 1;
    for (int i = tid; i < nimg; i += NT)
      if (simg[i] != 0.0) atomicAdd(a.sumsq + img_first + i, simg[i]);
  }
}

// ----------------------------------------------------------------------------
// FP32 fast path (the plain FP32 form's inner layers: NHWC f32, C_in % 16 == 0,
// N % BN == 0).  Tile 128 pixels x BN channels, 256 threads in a 16 x 16 grid,
// each owning 8 x (BN/16) outputs; K chunks of 16 channels of one tap, gathered
// as float4 (4 threads per pixel row of 64 contiguous bytes) and prefetched into
// registers while the previous chunk is multiplied from shared memory.
template <int BN>
__global__ void __launch_bounds__(256) conv_simt_f32_kernel(ConvArgs a) {
  constexpr int BM = 128, BK = 16, TN = BN / 16;
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const long long M = a.M();
  const int N = a.N(), K = a.K();
  const long long m0 = (long long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int HW = a.H * a.W;
  if (a.skip) {  // every image this block touches is frozen in a solve: nothing needed
    const long long m_last = (m0 + BM < M ? m0 + BM : M) - 1;
    bool any = false;
    for (long long i = m0 / HW; i <= m_last / HW; ++i) any |= a.skip[i] == 0;
    if (!any) return;
  }
  const int SH = a.mode == CM_DOWN ? 2 * a.H : a.H;
  const int SW = a.mode == CM_DOWN ? 2 * a.W : a.W;
  const float* __restrict__ in = (const float*)a.in;
  const float* __restrict__ wf = (const float*)a.wB;
  // A loads: 128 rows x 16 k = 512 float4; thread -> rows (tid >> 2) and (tid >> 2) + 64,
  // k quad (tid & 3)
  const int aq = tid & 3;
  int r_img[2], r_y[2], r_x[2];
  bool r_ok[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const long long m = m0 + (tid >> 2) + 64 * i;
    r_ok[i] = m < M;
    const long long mm = r_ok[i] ? m : 0;
    r_img[i] = (int)(mm / HW);
    const int rem = (int)(mm - (long long)r_img[i] * HW);
    r_y[i] = rem / a.W;
    r_x[i] = rem - r_y[i] * a.W;
  }
  // B loads: BN x 16 k = BN*4 float4; thread -> n rows (tid >> 2) + 64 j, k quad (tid & 3)
  float4 ra[2], rb[TN / 4 > 0 ? BN / 64 : 1];
  auto gload = [&](int k0) {
    int dy = 0, dx = 0, c0 = k0;
    if (a.mode == CM_CONV3) {
      const int t = k0 / a.Cin;
      c0 = k0 - t * a.Cin;
      dy = t / 3 - 1;
      dx = t % 3 - 1;
    } else if (a.mode == CM_DOWN) {
      const int q = k0 / a.Cin;
      c0 = k0 - q * a.Cin;
      dy = q >> 1;
      dx = q & 1;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int sy, sx;
      if (a.mode == CM_DOWN) {
        sy = 2 * r_y[i] + dy;
        sx = 2 * r_x[i] + dx;
      } else {
        sy = r_y[i] + dy;
        sx = r_x[i] + dx;
      }
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r_ok[i] && sy >= 0 && sy < SH && sx >= 0 && sx < SW)
        v = *(const float4*)(in + (((size_t)r_img[i] * SH + sy) * SW + sx) * a.Cin + c0 + 4 * aq);
      ra[i] = v;
    }
#pragma unroll
    for (int j = 0; j < BN / 64; ++j) {
      const int nn = n0 + (tid >> 2) + 64 * j;
      rb[j] = *(const float4*)(wf + (size_t)nn * K + k0 + 4 * aq);
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = (tid >> 2) + 64 * i;
      As[buf][4 * aq + 0][r] = ra[i].x;
      As[buf][4 * aq + 1][r] = ra[i].y;
      As[buf][4 * aq + 2][r] = ra[i].z;
      As[buf][4 * aq + 3][r] = ra[i].w;
    }
#pragma unroll
    for (int j = 0; j < BN / 64; ++j) {
      const int nn = (tid >> 2) + 64 * j;
      Bs[buf][4 * aq + 0][nn] = rb[j].x;
      Bs[buf][4 * aq + 1][nn] = rb[j].y;
      Bs[buf][4 * aq + 2][nn] = rb[j].z;
      Bs[buf][4 * aq + 3][nn] = rb[j].w;
    }
  };
  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][TN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  gload(0);
  sstore(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) gload(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float av[8], bv[TN];
      const float4 a0 = *(const float4*)&As[buf][kk][ty * 8];
      const float4 a1 = *(const float4*)&As[buf][kk][ty * 8 + 4];
      av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
      av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
#pragma unroll
      for (int j = 0; j < TN; j += 4) {
        const float4 b4 = *(const float4*)&Bs[buf][kk][tx * TN + j];
        bv[j] = b4.x; bv[j + 1] = b4.y; bv[j + 2] = b4.z; bv[j + 3] = b4.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      sstore(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  float* out = (float*)a.out;
  float* out2 = (float*)a.out2;
  const float* aux0 = (const float*)a.aux0;
  const float* aux1 = (const float*)a.aux1;
  const float* aux2 = (const float*)a.aux2;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long m = m0 + ty * 8 + i;
    if (m >= M) continue;
    const int img = (int)(m / HW);
    const int rem = (int)(m - (long long)img * HW);
    const int y = rem / a.W, x = rem - (rem / a.W) * a.W;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx * TN + j;
      size_t o;
      if (a.outmap == OM_D2S) {
        const int q = n / a.Cout, co = n - q * a.Cout;
        o = (((size_t)img * 2 * a.H + 2 * y + (q >> 1)) * 2 * a.W + 2 * x + (q & 1)) * a.Cout + co;
      } else {
        o = (size_t)m * a.Cout + n;
      }
      const float x0 = aux0 ? aux0[o] : 0.f;
      const float x1 = aux1 ? aux1[o] : 0.f;
      const float x2 = aux2 ? aux2[o] : 0.f;
      float o2 = 0.f;
      out[o] = epi_math(a.epi, a.act, acc[i][j], x0, x1, x2, &o2);
      if (epi_has_out2(a.epi)) out2[o] = o2;
    }
  }
}

static bool f32_fast_ok(const ConvArgs& a) {
  return !a.in_nchw && !a.out_nchw && a.epi != EP_AXPY_NCHW && a.Cin % 16 == 0 &&
         (a.N() % 128 == 0 || a.N() % 64 == 0) && (a.outmap == OM_IDENT || a.Cout % 16 == 0);
}

template <typename TIn, typename TOut>
static cudaError_t launch_typed(const ConvArgs& a, cudaStream_t st) {
  const long long M = a.M();
  const int N = a.N();
  if (N <= 4) {
    constexpr int BM = 128, BN = 4, TM = 2, TN = 1;
    dim3 grid((unsigned)((M + BM - 1) / BM), (N + BN - 1) / BN);
    conv_simt_kernel<TIn, TOut, BM, BN, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(a);
  } else {
    constexpr int BM = 128, BN = 64, TM = 8, TN = 4;
    dim3 grid((unsigned)((M + BM - 1) / BM), (N + BN - 1) / BN);
    conv_simt_kernel<TIn, TOut, BM, BN, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_conv_simt(const ConvArgs& a, int in_dt, int out_dt, cudaStream_t st) {
  if (a.M() == 0) return cudaSuccess;
  if (in_dt == DT_BF16 && out_dt == DT_BF16) return launch_typed<__nv_bfloat16, __nv_bfloat16>(a, st);
  if (in_dt == DT_F16 && out_dt == DT_F16) return launch_typed<__half, __half>(a, st);
  if (in_dt == DT_BF16 && out_dt == DT_F32) return launch_typed<__nv_bfloat16, float>(a, st);
  if (in_dt == DT_F16 && out_dt == DT_F32) return launch_typed<__half, float>(a, st);
  if (in_dt == DT_F32 && out_dt == DT_BF16) return launch_typed<float, __nv_bfloat16>(a, st);
  if (in_dt == DT_F32 && out_dt == DT_F16) return launch_typed<float, __half>(a, st);
  if (in_dt == DT_F32 && out_dt == DT_F32) {
    if (f32_fast_ok(a)) {
      const int N = a.N();
      if (N % 128 == 0) {
        dim3 grid((unsigned)((a.M() + 127) / 128), N / 128);
        conv_simt_f32_kernel<128><<<grid, 256, 0, st>>>(a);
      } else {
        dim3 grid((unsigned)((a.M() + 127) / 128), N / 64);
        conv_simt_f32_kernel<64><<<grid, 256, 0, st>>>(a);
      }
      return cudaGetLastError();
    }
    return launch_typed<float, float>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ideq
