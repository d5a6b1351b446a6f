// 3x3 convolutions between the image side (f32 planar NCHW, c <= 4 channels)
// and the feature side (NHWC, C channels, f32 / bf16 / f16): the regulariser's
// head and tail and their transposes, and the first/last layers of the plain
// conv nets.  Both directions stage a 16x16-pixel tile with a one-pixel halo in
// shared memory and move the feature side with 16-byte vector accesses, so
// that consecutive lanes touch consecutive 16-byte chunks of NHWC memory.
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
// Tile of (EH x EH pixels) x C channels staged as float with a padded pixel
// stride; each thread owns one output pixel and all (<= 4) output channels.
template <typename TIn>
__global__ void __launch_bounds__(256) feat2img_kernel(ConvArgs a) {
  extern __shared__ float sm[];
  __shared__ double red[32];
  const int C = a.Cin, c = a.Cout;
  const int CP = C + 1;  // padded pixel stride (floats)
  float* tile = sm;                  // EH*EH*CP
  float* wsm = sm + EH * EH * CP;    // [c][9*C]
  const int b = blockIdx.z;
  const int y0 = blockIdx.y * ET, x0 = blockIdx.x * ET;
  const TIn* in = (const TIn*)a.in;
  const int groups = C / 8;  // C % 8 == 0
  for (int e = threadIdx.x; e < EH * EH * groups; e += 256) {
    const int g = e % groups, p = e / groups;
    const int yy = y0 - 1 + p / EH, xx = x0 - 1 + p % EH;
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
      Vec8<TIn>::load(in + (((size_t)b * a.H + yy) * a.W + xx) * C + 8 * g, v);
    float* t = tile + p * CP + 8 * g;
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = v[i];
  }
  const float* w = (const float*)a.wB;  // [c][9*C]
  for (int e = threadIdx.x; e < c * 9 * C; e += 256) wsm[e] = w[e];
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int t = 0; t < 9; ++t) {
    const float* tp = tile + ((ty + t / 3) * EH + tx + t % 3) * CP;
    const float* w0 = wsm + t * C;
    for (int ci = 0; ci < C; ++ci) {
      const float v = tp[ci];
      acc[0] = fmaf(w0[ci], v, acc[0]);
      if (c > 1) acc[1] = fmaf(w0[9 * C + ci], v, acc[1]);
      if (c > 2) acc[2] = fmaf(w0[18 * C + ci], v, acc[2]);
      if (c > 3) acc[3] = fmaf(w0[27 * C + ci], v, acc[3]);
    }
  }
  const int y = y0 + ty, x = x0 + tx;
  double ssq = 0.0;
  if (y < a.H && x < a.W) {
    for (int o = 0; o < c; ++o) {
      const size_t idx = (((size_t)b * c + o) * a.H + y) * a.W + x;
      const float r = ((const float*)a.aux0)[idx] + a.sign * acc[o];
      ((float*)a.out)[idx] = r;
      ssq += 0.5 * (double)r * (double)r;
    }
  }
  if (a.sumsq) {
    const double s = block_sum(ssq, red);
    if (threadIdx.x == 0) atomicAdd(a.sumsq + b, s);
  }
}

// ------------------------------------------------------------------ img2feat
// Work item = (pixel, group of 8 output channels); consecutive threads take
// consecutive groups of one pixel, so the 16-byte stores of a warp are contiguous.
template <typename TOut, int CIN>
__global__ void __launch_bounds__(256) img2feat_kernel(ConvArgs a) {
  __shared__ float tile[CIN * EH * EH];
  extern __shared__ float wsm[];  // [C][9*CIN], k = t*CIN + ci
  const int C = a.Cout;
  const int b = blockIdx.z;
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
  const int groups = C / 8;
  TOut* out = (TOut*)a.out;
  TOut* out2 = (TOut*)a.out2;
  const TOut* aux0 = (const TOut*)a.aux0;
  for (int item = threadIdx.x; item < ET * ET * groups; item += 256) {
    const int g = item % groups, p = item / groups;
    const int ty = p / ET, tx = p % ET;
    const int y = y0 + ty, x = x0 + tx;
    if (y >= a.H || x >= a.W) continue;
    float v[9 * CIN];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci)
        v[t * CIN + ci] = tile[ci * EH * EH + (ty + t / 3) * EH + tx + t % 3];
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float* wr = wsm + (8 * g + j) * 9 * CIN;
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 9 * CIN; ++k) s = fmaf(wr[k], v[k], s);
      acc[j] = s;
    }
    const size_t o = (((size_t)b * a.H + y) * a.W + x) * C + 8 * g;
    float x0v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, r[8], r2[8];
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
    return a.Cin >= 1 && a.Cin <= 4 && a.Cout % 8 == 0 && a.Cout * 9 * a.Cin * 4 <= 48 * 1024 &&
           a.epi != EP_AXPY_NCHW && a.epi != EP_DUAL;
  if (a.out_nchw && !a.in_nchw)
    return a.Cout <= 4 && a.Cin % 8 == 0 && a.epi == EP_AXPY_NCHW &&
           (size_t)(EH * EH * (a.Cin + 1) + a.Cout * 9 * a.Cin) * 4 <= 200 * 1024;
  return false;
}

template <typename T, int CIN>
static cudaError_t launch_i2f(const ConvArgs& a, cudaStream_t st) {
  dim3 grid((a.W + ET - 1) / ET, (a.H + ET - 1) / ET, a.n);
  const size_t smem = (size_t)a.Cout * 9 * CIN * sizeof(float);
  img2feat_kernel<T, CIN><<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_edge_t(const ConvArgs& a, cudaStream_t st) {
  dim3 grid((a.W + ET - 1) / ET, (a.H + ET - 1) / ET, a.n);
  if (a.out_nchw) {
    const size_t smem = (size_t)(EH * EH * (a.Cin + 1) + a.Cout * 9 * a.Cin) * sizeof(float);
    static bool attr = false;  // per instantiation
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(feat2img_kernel<T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
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
  if (feat_dt == DT_BF16) return launch_edge_t<__nv_bfloat16>(a, st);
  if (feat_dt == DT_F16) return launch_edge_t<__half>(a, st);
  return launch_edge_t<float>(a, st);
}

}  // namespace ideq
