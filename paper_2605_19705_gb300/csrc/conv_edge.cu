// 3x3 convolutions between the image side (f32 planar NCHW, c <= 4 channels)
// and the feature side (NHWC, C channels, f32 / bf16 / f16): the regulariser's
// head and tail and their transposes, and the first/last layers of the plain
// conv nets.  Both directions stage a pixel tile with a one-pixel halo in
// shared memory, move the feature side with 16-byte vector accesses (so that
// consecutive lanes touch consecutive 16-byte chunks of NHWC memory), and read
// each weight as a warp-wide broadcast that feeds several pixels.
//
//   feat2img: out[b][o][y][x] = aux[b][o][y][x] + sign * sum_{t,ci} B[o][t*C+ci] in[b][y+dy][x+dx][ci]
//             (+ per-image 1/2 sum out^2), o < c          -> EP_AXPY_NCHW
//   img2feat: out[b][y][x][o] = epi(sum_{t,ci} B[o][t*c+ci] in[b][ci][y+dy][x+dx]), o < C
#include "common.cuh"
#include "ideq_internal.h"

namespace ideq {

constexpr int ET = 16;      // output tile edge
constexpr int EH = ET + 2;  // with halo

// 8 consecutive elements of T <-> float[8] (16 bytes for 16-bit T, 32 for f32)
template <typename T> struct Vec8;
template <> struct Vec8<float> {
  static IDEQ_DEV void load(const float* p, float (&v)[8]) {
    const float4 a = ((const float4*)p)[0], b = ((const float4*)p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  static IDEQ_DEV void store(float* p, const float (&v)[8]) {
    ((float4*)p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    ((float4*)p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
};
template <typename H2, typename T>
struct Vec8Half {
  static IDEQ_DEV void load(const T* p, float (&v)[8]) {
    const uint4 u = *(const uint4*)p;
    const H2* h = (const H2*)&u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = cvt2(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
  static IDEQ_DEV void store(T* p, const float (&v)[8]) {
    uint4 u;
    H2* h = (H2*)&u;
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = mk2(v[2 * i], v[2 * i + 1]);
    *(uint4*)p = u;
  }
  static IDEQ_DEV float2 cvt2(__nv_bfloat162 x) { return __bfloat1622float2(x); }
  static IDEQ_DEV float2 cvt2(__half2 x) { return __half22float2(x); }
  static IDEQ_DEV __nv_bfloat162 mk2_(float a, float b, __nv_bfloat162*) {
    return __floats2bfloat162_rn(a, b);
  }
  static IDEQ_DEV __half2 mk2_(float a, float b, __half2*) { return __floats2half2_rn(a, b); }
  static IDEQ_DEV H2 mk2(float a, float b) { return mk2_(a, b, (H2*)nullptr); }
};
template <> struct Vec8<__nv_bfloat16> : Vec8Half<__nv_bfloat162, __nv_bfloat16> {};
template <> struct Vec8<__half> : Vec8Half<__half2, __half> {};

// ------------------------------------------------------------------ feat2img
// 32x32-pixel output tile per block, 4 horizontally adjacent pixels per thread;
// feature channels staged 16 at a time (float, padded pixel stride).  Each
// weight read (the same address in every lane: a broadcast) feeds 4 pixels.
constexpr int F2_T = 32;        // output tile edge
constexpr int F2_E = F2_T + 2;  // with halo
constexpr int F2_CC = 16;       // channels per stage
constexpr int F2_CP = F2_CC + 1;

template <typename TIn>
__global__ void __launch_bounds__(256) feat2img_kernel(ConvArgs a) {
  extern __shared__ float sm[];
  __shared__ double red[32];
  float* tile = sm;                       // F2_E * F2_E * F2_CP
  float* wsm = sm + F2_E * F2_E * F2_CP;  // [c][9][C]
  const int C = a.Cin, c = a.Cout;
  const int b = blockIdx.z;
  if (a.skip && a.skip[b]) return;  // frozen image of a solve: not needed
  const int y0 = blockIdx.y * F2_T, x0 = blockIdx.x * F2_T;
  const TIn* in = (const TIn*)a.in;
  const float* w = (const float*)a.wB;  // [c][9*C], k = t*C + ci
  for (int e = threadIdx.x; e < c * 9 * C; e += 256) wsm[e] = w[e];
  // thread -> row ty (0..31), pixels 4*qx .. 4*qx+3 (qx 0..7)
  const int ty = threadIdx.x >> 3, qx = threadIdx.x & 7;
  float acc[4][4];
#pragma unroll
  for (int o = 0; o < 4; ++o)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[o][p] = 0.f;
  for (int c0 = 0; c0 < C; c0 += F2_CC) {
    __syncthreads();
    const int groups = F2_CC / 8;
    for (int e = threadIdx.x; e < F2_E * F2_E * groups; e += 256) {
      const int g = e % groups, px = e / groups;
      const int yy = y0 - 1 + px / F2_E, xx = x0 - 1 + px % F2_E;
      float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
        Vec8<TIn>::load(in + (((size_t)b * a.H + yy) * a.W + xx) * C + c0 + 8 * g, v);
      float* t = tile + px * F2_CP + 8 * g;
#pragma unroll
      for (int i = 0; i < 8; ++i) t[i] = v[i];
    }
    __syncthreads();
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
      const int dy = t / 3, dx = t % 3;
      const float* tp = tile + ((ty + dy) * F2_E + 4 * qx + dx) * F2_CP;
      const float* wt = wsm + t * C + c0;
#pragma unroll 4
      for (int ci = 0; ci < F2_CC; ++ci) {
        float v[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) v[p] = tp[p * F2_CP + ci];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          if (o < c) {
            const float wv = wt[o * 9 * C + ci];
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[o][p] = fmaf(wv, v[p], acc[o][p]);
          }
        }
      }
    }
  }
  const int y = y0 + ty;
  double ssq = 0.0;
  if (y < a.H) {
    for (int o = 0; o < c; ++o) {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int x = x0 + 4 * qx + p;
        if (x >= a.W) continue;
        const size_t idx = (((size_t)b * c + o) * a.H + y) * a.W + x;
        const float r = ((const float*)a.aux0)[idx] + a.sign * acc[o][p];
        ((float*)a.out)[idx] = r;
        ssq += 0.5 * (double)r * (double)r;
      }
    }
  }
  if (a.sumsq) {
    const double s = block_sum(ssq, red);
    if (threadIdx.x == 0) atomicAdd(a.sumsq + b, s);
  }
}

// ------------------------------------------------------------------ img2feat
// 16x16-pixel tile per block.  Warp w computes output-channel groups of 8 with
// a warp-uniform group (weights read as broadcasts), 4 pixels per lane; the
// results go through a shared-memory tile so that the NHWC stores are
// coalesced 16-byte chunks.
template <typename TOut, int CIN>
__global__ void __launch_bounds__(256) img2feat_kernel(ConvArgs a) {
  __shared__ float tile[CIN * EH * EH];
  extern __shared__ float dsm[];
  const int C = a.Cout;
  float* wsm = dsm;                                // [C][9*CIN]
  TOut* stg = (TOut*)(dsm + C * 9 * CIN);          // [256 px][C + 8]
  const int SP = C + 8;                            // padded pixel stride (elements)
  const int b = blockIdx.z;
  if (a.skip && a.skip[b]) return;  // frozen image of a solve: not needed
  const int y0 = blockIdx.y * ET, x0 = blockIdx.x * ET;
  const float* in = (const float*)a.in;
  for (int e = threadIdx.x; e < CIN * EH * EH; e += 256) {
    const int ci = e / (EH * EH), p = e % (EH * EH);
    const int yy = y0 - 1 + p / EH, xx = x0 - 1 + p % EH;
    float v = 0.f;
    if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
      v = in[(((size_t)b * CIN + ci) * a.H + yy) * a.W + xx];
    tile[ci * EH * EH + p] = v;
  }
  const float* w = (const float*)a.wB;
  for (int e = threadIdx.x; e < C * 9 * CIN; e += 256) wsm[e] = w[e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int groups = C / 8;
  // (group, half) pairs: a warp computes one group of 8 channels for 128 of the
  // tile's 256 pixels (4 per lane)
  for (int pair = warp; pair < groups * 2; pair += 8) {
    const int g = pair >> 1, hpx = (pair & 1) * 128;  // 128 pixels per pair, 4 per lane
    float v[4][9 * CIN];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int px = hpx + lane + 32 * p;
      const int ty = px >> 4, tx = px & 15;
#pragma unroll
      for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci)
          v[p][t * CIN + ci] = tile[ci * EH * EH + (ty + t / 3) * EH + tx + t % 3];
    }
#pragma unroll 1
    for (int j = 0; j < 8; ++j) {
      const float* wr = wsm + (8 * g + j) * 9 * CIN;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 9 * CIN; ++k) {
        const float wv = wr[k];
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[p] = fmaf(wv, v[p][k], acc[p]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p) stg[(hpx + lane + 32 * p) * SP + 8 * g + j] = from_f<TOut>(acc[p]);
    }
  }
  __syncthreads();
  // epilogue + coalesced store: item = (pixel, group of 8), consecutive lanes -> consecutive groups
  TOut* out = (TOut*)a.out;
  TOut* out2 = (TOut*)a.out2;
  const TOut* aux0 = (const TOut*)a.aux0;
  for (int item = threadIdx.x; item < ET * ET * groups; item += 256) {
    const int g = item % groups, px = item / groups;
    const int y = y0 + (px >> 4), x = x0 + (px & 15);
    if (y >= a.H || x >= a.W) continue;
    float acc[8], x0v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, r[8], r2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = ld_f(stg + px * SP + 8 * g + j);
    const size_t o = (((size_t)b * a.H + y) * a.W + x) * C + 8 * g;
    if (aux0) Vec8<TOut>::load(aux0 + o, x0v);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      r2[j] = 0.f;
      r[j] = epi_math(a.epi, a.act, acc[j], x0v[j], 0.f, 0.f, &r2[j]);
    }
    Vec8<TOut>::store(out + o, r);
    if (epi_has_out2(a.epi)) Vec8<TOut>::store(out2 + o, r2);
  }
}

bool edge_supported(const ConvArgs& a) {
  if (a.mode != CM_CONV3 || a.outmap != OM_IDENT) return false;
  if (a.in_nchw && !a.out_nchw)
    return a.Cin >= 1 && a.Cin <= 4 && a.Cout % 8 == 0 && a.Cout <= 128 &&
           a.epi != EP_AXPY_NCHW && a.epi != EP_DUAL;
  if (a.out_nchw && !a.in_nchw)
    return a.Cout <= 4 && a.Cin % F2_CC == 0 && a.epi == EP_AXPY_NCHW && a.Cin <= 512;
  return false;
}

template <typename T, int CIN>
static cudaError_t launch_i2f(const ConvArgs& a, cudaStream_t st) {
  dim3 grid((a.W + ET - 1) / ET, (a.H + ET - 1) / ET, a.n);
  const size_t smem =
      (size_t)a.Cout * 9 * CIN * sizeof(float) + (size_t)ET * ET * (a.Cout + 8) * sizeof(T);
  static bool attr = false;  // per instantiation
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(img2feat_kernel<T, CIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  img2feat_kernel<T, CIN><<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_edge_t(const ConvArgs& a, cudaStream_t st) {
  if (a.out_nchw) {
    dim3 grid((a.W + F2_T - 1) / F2_T, (a.H + F2_T - 1) / F2_T, a.n);
    const size_t smem = (size_t)(F2_E * F2_E * F2_CP + a.Cout * 9 * a.Cin) * sizeof(float);
    static bool attr = false;  // per instantiation
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(feat2img_kernel<T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    feat2img_kernel<T><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
  }
  switch (a.Cin) {
    case 1: return launch_i2f<T, 1>(a, st);
    case 2: return launch_i2f<T, 2>(a, st);
    case 3: return launch_i2f<T, 3>(a, st);
    default: return launch_i2f<T, 4>(a, st);
  }
}

cudaError_t launch_conv_edge(const ConvArgs& a, int feat_dt, cudaStream_t st) {
  if (a.M() == 0) return cudaSuccess;
  if (edge_rb_supported(a)) return launch_conv_edge_rb(a, feat_dt, st);
  if (feat_dt == DT_BF16) return launch_edge_t<__nv_bfloat16>(a, st);
  if (feat_dt == DT_F16) return launch_edge_t<__half>(a, st);
  return launch_edge_t<float>(a, st);
}

}  // namespace ideq
