// Register-blocked 3x3 convolutions between the image side (f32 planar NCHW,
// c = 1, 2 or 3 channels) and the feature side (NHWC, C = 32 or 64 channels, f32 /
// bf16 / f16): the regulariser's head and tail and their transposes.  Every
// weight or input value a thread loads from shared memory feeds 8 to 24 FMAs,
// so the FP32 pipes, not the shared-memory port, set the pace.
//
//   img2feat: out[b][y][x][o] = epi(sum_{t,ci} B[o][t*c+ci] in[b][ci][y+dy][x+dx]), o < C
//   feat2img: out[b][o][y][x] = aux[b][o][y][x] + sign * sum_{t,ci} B[o][t*C+ci] in[b][y+dy][x+dx][ci]
//             (+ per-image 1/2 sum out^2), o < c
// Zero "same" padding, t = 3 * (dy + 1) + (dx + 1).
#include "common.cuh"
#include "ideq_internal.h"

namespace ideq {

template <typename T> struct Chunk16;  // 16 bytes of T <-> floats
template <> struct Chunk16<float> {
  static constexpr int n = 4;
  static IDEQ_DEV void get(const uint4& u, float* v) {
    v[0] = __uint_as_float(u.x); v[1] = __uint_as_float(u.y);
    v[2] = __uint_as_float(u.z); v[3] = __uint_as_float(u.w);
  }
  static IDEQ_DEV uint4 put(const float* v) {
    return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]),
                      __float_as_uint(v[3]));
  }
};
template <typename H2, typename T>
struct Chunk16Half {
  static constexpr int n = 8;
  static IDEQ_DEV void get(const uint4& u, float* v) {
    const H2* h = (const H2*)&u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = cvt(h[i]);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
  static IDEQ_DEV uint4 put(const float* v) {
    uint4 u;
    H2* h = (H2*)&u;
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = mk(v[2 * i], v[2 * i + 1], (H2*)nullptr);
    return u;
  }
  static IDEQ_DEV float2 cvt(__nv_bfloat162 x) { return __bfloat1622float2(x); }
  static IDEQ_DEV float2 cvt(__half2 x) { return __half22float2(x); }
  static IDEQ_DEV __nv_bfloat162 mk(float a, float b, __nv_bfloat162*) {
    return __floats2bfloat162_rn(a, b);
  }
  static IDEQ_DEV __half2 mk(float a, float b, __half2*) { return __floats2half2_rn(a, b); }
};
template <> struct Chunk16<__nv_bfloat16> : Chunk16Half<__nv_bfloat162, __nv_bfloat16> {};
template <> struct Chunk16<__half> : Chunk16Half<__half2, __half> {};

// ------------------------------------------------------------------ img2feat
// Register-blocked: warp w owns output channels 8w .. 8w+7 (its weights are
// warp-wide broadcasts from shared memory), lane (r, q) = (lane / 4, lane % 4)
// owns the 8 pixels x0 + 8q .. 8q+7 of tile row r, so each input value loaded
// feeds 8 channels x (up to) 3 horizontal taps.  A block is C / 8 warps over a
// 32 x 8 pixel tile.  The results are staged per pixel in shared memory with
// the 16-byte chunk index XOR-swizzled by (pixel / 8), conflict-free for both
// the blocked writes and the row-major reads of the coalesced NHWC store.
constexpr int I2_TX = 32, I2_TY = 8, I2_EX = I2_TX + 2, I2_EY = I2_TY + 2;
constexpr int I2_RS = 35;  // tile row stride: (35 r + 8 q) mod 32 distinct over r < 8, q < 4
constexpr int I2_WP = 4;   // weight row padding: transposed writes hit <= 4 lanes per bank

template <typename TOut, int CIN, int C>
__global__ void __launch_bounds__(C * 4) img2feat_rb_kernel(ConvArgs a) {
  constexpr int NT = C * 4;                        // threads: C / 8 warps
  constexpr int CH = C * (int)sizeof(TOut) / 16;  // 16-byte chunks per pixel
  constexpr int EPC = Chunk16<TOut>::n;            // channels per chunk
  static_assert((CH & (CH - 1)) == 0, "chunks per pixel must be a power of two");
  __shared__ float tile[CIN][I2_EY][I2_RS];
  __shared__ __align__(16) float wsm[9 * CIN][C + I2_WP];  // k-major
  extern __shared__ uint4 stg[];                   // [nout][256 px][CH]
  const int b = blockIdx.z, y0 = blockIdx.y * I2_TY, x0 = blockIdx.x * I2_TX;
  if (a.skip && a.skip[b]) return;  // frozen image of a solve: not needed
  const float* in = (const float*)a.in;
  for (int e = threadIdx.x; e < CIN * I2_EY * I2_EX; e += NT) {
    const int ci = e / (I2_EY * I2_EX), p = e % (I2_EY * I2_EX);
    const int yy = y0 - 1 + p / I2_EX, xx = x0 - 1 + p % I2_EX;
    float v = 0.f;
    if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
      v = in[(((size_t)b * CIN + ci) * a.H + yy) * a.W + xx];
    tile[ci][p / I2_EX][p % I2_EX] = v;
  }
  const float* w = (const float*)a.wB;  // [C][9 * CIN], k = t * CIN + ci
  for (int e = threadIdx.x; e < C * 9 * CIN; e += NT) {
    const int o = e / (9 * CIN), k = e % (9 * CIN);
    wsm[k][o] = w[e];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = lane >> 2, q = lane & 3;
  float acc[8][8];
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[p][j] = 0.f;
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      float x[10];
#pragma unroll
      for (int i = 0; i < 10; ++i) x[i] = tile[ci][r + dy][8 * q + i];
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const float4* wp = (const float4*)&wsm[(3 * dy + dx) * CIN + ci][8 * warp];
        const float4 wa = wp[0], wb = wp[1];
        const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[p][j] = fmaf(wv[j], x[p + dx], acc[p][j]);
      }
    }
  const bool two = a.epi == EP_ACT;
  // this warp's 8 channels are elements [8 warp, 8 warp + 8) of the pixel:
  // 16-bit types -> one chunk, f32 -> two chunks
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int px = 32 * r + 8 * q + p;
    float v1[8], v2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v2[j] = 0.f;
      v1[j] = two ? epi_math(EP_ACT, a.act, acc[p][j], 0.f, 0.f, 0.f, &v2[j]) : acc[p][j];
    }
#pragma unroll
    for (int h = 0; h < 8 / EPC; ++h) {
      const int g = (8 * warp) / EPC + h;
      const int gs = g ^ ((px >> 3) & (CH - 1));
      stg[px * CH + gs] = Chunk16<TOut>::put(v1 + h * EPC);
      if (two) stg[(256 + px) * CH + gs] = Chunk16<TOut>::put(v2 + h * EPC);
    }
  }
  __syncthreads();
  uint4* out = (uint4*)a.out;
  uint4* out2 = (uint4*)a.out2;
  for (int item = threadIdx.x; item < 256 * CH; item += NT) {
    const int g = item % CH, px = item / CH;
    const int y = y0 + px / I2_TX, x = x0 + px % I2_TX;
    if (y >= a.H || x >= a.W) continue;
    const int gs = g ^ ((px >> 3) & (CH - 1));
    const size_t o = (((size_t)b * a.H + y) * a.W + x) * CH + g;
    out[o] = stg[px * CH + gs];
    if (two) out2[o] = stg[(256 + px) * CH + gs];
  }
}

// ------------------------------------------------------------------ feat2img
// Lane (pg, g) of warp w: channel chunk g (16 bytes: EPC channels) of the 8
// pixels x0 + 8 pg .. 8 pg + 7 of tile row w; the G = C / EPC lanes of a pixel
// group split the channel sum and combine it with xor-shuffles, after which
// lane g writes pixels p = g (mod G) (consecutive lanes, consecutive pixels).
// Block: 8 warps = 8 rows of (32 / G) x 8 pixels.
template <typename TIn, int C, int CO>
__global__ void __launch_bounds__(256) feat2img_rb_kernel(ConvArgs a) {
  constexpr int EPC = Chunk16<TIn>::n;
  constexpr int G = C / EPC;         // chunks (lanes) per pixel group
  constexpr int TX = (32 / G) * 8;   // tile width
  constexpr int EX = TX + 2, EY = 10;
  constexpr int PS = G + 1;          // staged pixel stride in chunks
  static_assert(G == 4 || G == 8 || G == 16, "channel chunks per pixel");
  extern __shared__ uint4 tile[];  // [EY * EX][PS], then weights
  float* wsm = (float*)(tile + EY * EX * PS);  // [dy][e][g][12]: (o, dx) at 3 o + dx
  __shared__ double red[32];
  const int b = blockIdx.z, y0 = blockIdx.y * 8, x0 = blockIdx.x * TX;
  if (a.skip && a.skip[b]) return;  // frozen image of a solve: not needed
  const uint4* in = (const uint4*)a.in;
  for (int e = threadIdx.x; e < EY * EX * G; e += 256) {
    const int g = e % G, p = e / G;
    const int yy = y0 - 1 + p / EX, xx = x0 - 1 + p % EX;
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
      u = in[(((size_t)b * a.H + yy) * a.W + xx) * G + g];
    tile[p * PS + g] = u;
  }
  const float* w = (const float*)a.wB;  // [CO][9 * C], k = t * C + ci
  for (int i = threadIdx.x; i < 3 * C; i += 256) {  // one (dy, ci) pair: 12 floats
    const int dy = i / C, ci = i % C;
    float v[12];
#pragma unroll
    for (int j = 0; j < 12; ++j)
      v[j] = (j < 3 * CO) ? w[(j / 3) * 9 * C + (3 * dy + j % 3) * C + ci] : 0.f;
    float4* d = (float4*)(wsm + ((dy * EPC + ci % EPC) * G + ci / EPC) * 12);
    d[0] = make_float4(v[0], v[1], v[2], v[3]);
    d[1] = make_float4(v[4], v[5], v[6], v[7]);
    d[2] = make_float4(v[8], v[9], v[10], v[11]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pg = lane / G, g = lane % G;
  float acc[8][CO];
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[p][o] = 0.f;
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    float x[10][EPC];  // this lane's channel chunk of the 10 input pixels, converted once
#pragma unroll
    for (int i = 0; i < 10; ++i)
      Chunk16<TIn>::get(tile[((warp + dy) * EX + 8 * pg + i) * PS + g], x[i]);
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
      const float4* wp = (const float4*)(wsm + ((dy * EPC + e) * G + g) * 12);
      const float4 w0 = wp[0], w1 = wp[1], w2 = wp[2];
      const float wv[12] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w2.x, w2.y, w2.z, w2.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
          for (int o = 0; o < CO; ++o)
            acc[p][o] = fmaf(wv[3 * o + dx], x[p + dx][e], acc[p][o]);
    }
  }
#pragma unroll
  for (int off = 1; off < G; off <<= 1)
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
      for (int o = 0; o < CO; ++o) acc[p][o] += __shfl_xor_sync(0xffffffffu, acc[p][o], off);
  const int y = y0 + warp;
  double ssq = 0.0;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    if (p % G != g) continue;
    const int x = x0 + 8 * pg + p;
    if (y >= a.H || x >= a.W) continue;
#pragma unroll
    for (int o = 0; o < CO; ++o) {
      const size_t idx = (((size_t)b * CO + o) * a.H + y) * a.W + x;
      const float r = ((const float*)a.aux0)[idx] + a.sign * acc[p][o];
      ((float*)a.out)[idx] = r;
      ssq += 0.5 * (double)r * (double)r;
    }
  }
  if (a.sumsq) {
    const double s = block_sum(ssq, red);
    if (threadIdx.x == 0) atomicAdd(a.sumsq + b, s);
  }
}

// ------------------------------------------------------------------ host

static bool rb_width(int C) { return C == 32 || C == 64; }

bool edge_rb_supported(const ConvArgs& a) {
  if (a.mode != CM_CONV3 || a.outmap != OM_IDENT) return false;
  if (a.in_nchw && !a.out_nchw)
    return a.Cin >= 1 && a.Cin <= 3 && rb_width(a.Cout) &&
           (a.epi == EP_STORE || a.epi == EP_ACT);
  if (a.out_nchw && !a.in_nchw)
    return a.Cout >= 1 && a.Cout <= 3 && rb_width(a.Cin) && a.epi == EP_AXPY_NCHW;
  return false;
}

template <typename T, int CIN, int C>
static cudaError_t i2f(const ConvArgs& a, cudaStream_t st) {
  constexpr int CH = C * (int)sizeof(T) / 16;
  const size_t smem = (size_t)(a.epi == EP_ACT ? 2 : 1) * 256 * CH * 16;
  static bool attr = false;  // per instantiation
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(img2feat_rb_kernel<T, CIN, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((a.W + I2_TX - 1) / I2_TX, (a.H + I2_TY - 1) / I2_TY, a.n);
  img2feat_rb_kernel<T, CIN, C><<<grid, C * 4, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int C, int CO>
static cudaError_t f2i(const ConvArgs& a, cudaStream_t st) {
  constexpr int G = C * (int)sizeof(T) / 16, TX = (32 / G) * 8;
  const size_t smem = (size_t)10 * (TX + 2) * (G + 1) * 16 + (size_t)3 * C * 12 * 4;
  static bool attr = false;  // per instantiation
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(feat2img_rb_kernel<T, C, CO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((a.W + TX - 1) / TX, (a.H + 7) / 8, a.n);
  feat2img_rb_kernel<T, C, CO><<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int CIN>
static cudaError_t i2f_c(const ConvArgs& a, cudaStream_t st) {
  return a.Cout == 32 ? i2f<T, CIN, 32>(a, st) : i2f<T, CIN, 64>(a, st);
}

template <typename T, int C>
static cudaError_t f2i_c(const ConvArgs& a, cudaStream_t st) {
  if (a.Cout == 1) return f2i<T, C, 1>(a, st);
  return a.Cout == 2 ? f2i<T, C, 2>(a, st) : f2i<T, C, 3>(a, st);
}

template <typename T>
static cudaError_t launch_rb_t(const ConvArgs& a, cudaStream_t st) {
  if (a.out_nchw) return a.Cin == 32 ? f2i_c<T, 32>(a, st) : f2i_c<T, 64>(a, st);
  if (a.Cin == 1) return i2f_c<T, 1>(a, st);
  return a.Cin == 2 ? i2f_c<T, 2>(a, st) : i2f_c<T, 3>(a, st);
}

cudaError_t launch_conv_edge_rb(const ConvArgs& a, int feat_dt, cudaStream_t st) {
  if (a.M() == 0) return cudaSuccess;
  if (!edge_rb_supported(a)) return cudaErrorInvalidValue;
  if (feat_dt == DT_BF16) return launch_rb_t<__nv_bfloat16>(a, st);
  if (feat_dt == DT_F16) return launch_rb_t<__half>(a, st);
  return launch_rb_t<float>(a, st);
}

}  // namespace ideq
