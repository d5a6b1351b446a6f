// 3x3 convolutions between the image side (f32 planar NCHW, c <= 4 channels)
// and the feature side (NHWC, C channels, f32 / bf16 / f16): the regulariser's
// head and tail and their transposes, and the first/last layers of the plain
// conv nets.  Both directions stage a 16x16-pixel tile with a one-pixel halo in
// shared memory; one thread owns one output pixel.
//
//   feat2img: out[b][o][y][x] = aux[b][o][y][x] + sign * sum_{t,ci} B[o][t*C+ci] in[b][y+dy][x+dx][ci]
//             (+ per-image 1/2 sum out^2), o < c          -> EP_AXPY_NCHW
//   img2feat: out[b][y][x][o] = epi(sum_{t,ci} B[o][t*c+ci] in[b][ci][y+dy][x+dx]), o < C
#include "common.cuh"
#include "ideq_internal.h"

namespace ideq {

constexpr int ET = 16;       // output tile edge
constexpr int EH = ET + 2;   // with halo
constexpr int CC = 32;       // feature channels staged per pass (feat2img)

template <typename TIn>
__global__ void __launch_bounds__(256) feat2img_kernel(ConvArgs a) {
  __shared__ float tile[EH * EH * (CC + 1)];
  __shared__ float wsm[4 * 9 * CC];
  __shared__ double red[32];
  __shared__ double simg;
  const int C = a.Cin, c = a.Cout;  // feature channels in, image channels out
  const int b = blockIdx.z;
  const int y0 = blockIdx.y * ET, x0 = blockIdx.x * ET;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const TIn* in = (const TIn*)a.in;
  const float* w = (const float*)a.wB;  // [c][9*C]
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int c0 = 0; c0 < C; c0 += CC) {
    const int cc = min(CC, C - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < EH * EH * cc; e += 256) {
      const int ci = e % cc, p = e / cc;
      const int yy = y0 - 1 + p / EH, xx = x0 - 1 + p % EH;
      float v = 0.f;
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
        v = ld_f(in + (((size_t)b * a.H + yy) * a.W + xx) * C + c0 + ci);
      tile[p * (CC + 1) + ci] = v;
    }
    for (int e = threadIdx.x; e < c * 9 * cc; e += 256) {
      const int ci = e % cc, t = (e / cc) % 9, o = e / (9 * cc);
      wsm[(o * 9 + t) * CC + ci] = w[(size_t)o * 9 * C + t * C + c0 + ci];
    }
    __syncthreads();
    for (int t = 0; t < 9; ++t) {
      const float* tp = tile + ((ty + t / 3) * EH + tx + t % 3) * (CC + 1);
      for (int ci = 0; ci < cc; ++ci) {
        const float v = tp[ci];
#pragma unroll
        for (int o = 0; o < 4; ++o)
          if (o < c) acc[o] = fmaf(wsm[(o * 9 + t) * CC + ci], v, acc[o]);
      }
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
  (void)simg;
}

template <typename TOut>
__global__ void __launch_bounds__(256) img2feat_kernel(ConvArgs a) {
  __shared__ float tile[4 * EH * EH];
  extern __shared__ float wsm[];  // [C][9*c]
  const int c = a.Cin, C = a.Cout;  // image channels in, feature channels out
  const int b = blockIdx.z;
  const int y0 = blockIdx.y * ET, x0 = blockIdx.x * ET;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float* in = (const float*)a.in;
  for (int e = threadIdx.x; e < c * EH * EH; e += 256) {
    const int ci = e / (EH * EH), p = e % (EH * EH);
    const int yy = y0 - 1 + p / EH, xx = x0 - 1 + p % EH;
    float v = 0.f;
    if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
      v = in[(((size_t)b * c + ci) * a.H + yy) * a.W + xx];
    tile[ci * EH * EH + p] = v;
  }
  const float* w = (const float*)a.wB;  // [C][9*c], k = t*c + ci
  for (int e = threadIdx.x; e < C * 9 * c; e += 256) wsm[e] = w[e];
  __syncthreads();
  const int y = y0 + ty, x = x0 + tx;
  if (y >= a.H || x >= a.W) return;
  float v[36];
#pragma unroll
  for (int t = 0; t < 9; ++t)
#pragma unroll
    for (int ci = 0; ci < 4; ++ci)
      v[t * 4 + ci] = ci < c ? tile[ci * EH * EH + (ty + t / 3) * EH + tx + t % 3] : 0.f;
  const size_t obase = (((size_t)b * a.H + y) * a.W + x) * C;
  TOut* out = (TOut*)a.out;
  TOut* out2 = (TOut*)a.out2;
  const TOut* aux0 = (const TOut*)a.aux0;
  for (int o0 = 0; o0 < C; o0 += 8) {
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (o0 + j >= C) break;
      const float* wr = wsm + (o0 + j) * 9 * c;
      float s = 0.f;
      for (int t = 0; t < 9; ++t)
        for (int ci = 0; ci < c; ++ci) s = fmaf(wr[t * c + ci], v[t * 4 + ci], s);
      acc[j] = s;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int o = o0 + j;
      if (o >= C) break;
      float o2 = 0.f;
      const float x0v = aux0 ? ld_f(aux0 + obase + o) : 0.f;
      const float r = epi_math(a.epi, a.act, acc[j], x0v, 0.f, 0.f, &o2);
      out[obase + o] = from_f<TOut>(r);
      if (epi_has_out2(a.epi)) out2[obase + o] = from_f<TOut>(o2);
    }
  }
}

bool edge_supported(const ConvArgs& a) {
  if (a.mode != CM_CONV3 || a.outmap != OM_IDENT) return false;
  if (a.in_nchw && !a.out_nchw) return a.Cin <= 4 && a.epi != EP_AXPY_NCHW && a.epi != EP_DUAL;
  if (a.out_nchw && !a.in_nchw) return a.Cout <= 4 && a.epi == EP_AXPY_NCHW;
  return false;
}

template <typename T>
static cudaError_t launch_edge_t(const ConvArgs& a, cudaStream_t st) {
  dim3 grid((a.W + ET - 1) / ET, (a.H + ET - 1) / ET, a.n);
  if (a.out_nchw) {
    feat2img_kernel<T><<<grid, 256, 0, st>>>(a);
  } else {
    const size_t smem = (size_t)a.Cout * 9 * a.Cin * sizeof(float);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    img2feat_kernel<T><<<grid, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_conv_edge(const ConvArgs& a, int feat_dt, cudaStream_t st) {
  if (a.M() == 0) return cudaSuccess;
  if (feat_dt == DT_BF16) return launch_edge_t<__nv_bfloat16>(a, st);
  if (feat_dt == DT_F16) return launch_edge_t<__half>(a, st);
  return launch_edge_t<float>(a, st);
}

}  // namespace ideq
