// Orthonormal 2-D DFT of complex images stored as two f32 planes (re, im) per
// image, and the k-space steps of the MRI data term (App. E):
//   A x = M . F x,   A^T r = F^{-1}(M . r),   grad f = F^{-1}(M . F z - y),
//   prox_{tau f}(v) = F^{-1}((tau M y + F v) / (tau M + 1)),
// F the unitary DFT, M a 0/1 k-space mask per image, y zero off the mask.
//
// One launch transforms G lines of one image (rows, or G consecutive columns)
// held in shared memory: the lines are read in bit-reversed order (coalesced in
// both directions), then log2 N radix-2 butterfly stages with a per-block table
// of the N/2 twiddles exp(-+2 pi i k / N), and the 1/sqrt(N) scale on the way
// out; a row pass and a column pass make the 2-D transform.  N is a power of two,
// 8 <= N <= 1024.
#include "common.cuh"
#include "ideq_internal.h"

namespace ideq {

constexpr int FFT_THREADS = 256;

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) {
  return __brev(v) >> (32 - bits);
}

// Shared-memory slot of entry i of a line: one pad slot per 32 entries, so that the
// bit-reversed scatter of the load (consecutive e -> strides of N/2, N/4, ...)
// and the butterflies of every stage spread over the banks.
__device__ __forceinline__ int pad_slot(int i) { return i + (i >> 5); }

// lines: G lines of length N; element e of line l of image b sits at
// base_b + (l0 + l) * line_stride + e * elem_stride in both planes.  Lines are
// N + N/32 + 1 float2 slots apart in shared memory (an odd count of 8-byte slots
// modulo the 16 bank pairs, so the column-mode load hits distinct banks).
__global__ void __launch_bounds__(FFT_THREADS) fft_lines_kernel(
    const float* in, float* out, int N, int logN, int G, int logG,  // in and out may alias
    int lines_per_img, int line_stride, int elem_stride, int plane, int inverse) {
  extern __shared__ float2 sm[];  // [G][N + N/32 + 1] data, then N/2 twiddles
  const int LS = N + (N >> 5) + 1;
  float2* tw = sm + (size_t)G * LS;
  const int b = blockIdx.y;
  const int l0 = blockIdx.x * G;
  const size_t ib = (size_t)b * 2 * plane;  // image base (re plane; im at + plane)
  const bool rows = elem_stride == 1;
  for (int k = threadIdx.x; k < N / 2; k += FFT_THREADS) {
    float s, c;
    sincospif(2.f * (float)k / (float)N, &s, &c);  // exp(-+ 2 pi i k / N)
    tw[k] = make_float2(c, inverse ? s : -s);
  }
  const int total = G << logN;
  for (int idx = threadIdx.x; idx < total; idx += FFT_THREADS) {
    // consecutive threads walk consecutive addresses: along a row, or across columns
    const int l = rows ? idx >> logN : idx & (G - 1);
    const int e = rows ? idx & (N - 1) : idx >> logG;
    if (l0 + l >= lines_per_img) continue;
    const size_t o = ib + (size_t)(l0 + l) * line_stride + (size_t)e * elem_stride;
    sm[l * LS + pad_slot((int)bitrev((unsigned)e, logN))] = make_float2(in[o], in[o + plane]);
  }
  __syncthreads();
  const int half = N >> 1, logh = logN - 1;
  for (int s = 0; s < logN; ++s) {
    const int m = 1 << s;  // butterfly half-span
    for (int t = threadIdx.x; t < (G << logh); t += FFT_THREADS) {
      const int l = t >> logh, k = t & (half - 1);
      const int j = k & (m - 1), i0 = ((k >> s) << (s + 1)) + j;
      float2* L = sm + l * LS;
      const float2 w = tw[j << (logh - s)];
      const int p0 = pad_slot(i0), p1 = pad_slot(i0 + m);
      const float2 a = L[p0], bb = L[p1];
      const float2 wb = make_float2(w.x * bb.x - w.y * bb.y, w.x * bb.y + w.y * bb.x);
      L[p0] = make_float2(a.x + wb.x, a.y + wb.y);
      L[p1] = make_float2(a.x - wb.x, a.y - wb.y);
    }
    __syncthreads();
  }
  const float scale = rsqrtf((float)N);
  for (int idx = threadIdx.x; idx < total; idx += FFT_THREADS) {
    const int l = rows ? idx >> logN : idx & (G - 1);
    const int e = rows ? idx & (N - 1) : idx >> logG;
    if (l0 + l >= lines_per_img) continue;
    const size_t o = ib + (size_t)(l0 + l) * line_stride + (size_t)e * elem_stride;
    const float2 v = sm[l * LS + pad_slot(e)];
    out[o] = v.x * scale;
    out[o + plane] = v.y * scale;
  }
}

// N = 256 lines as 16 x 16 (four-step): a 16-point DFT over n1 of x[16 n1 + n2]
// in registers, the twiddle W_256^(n2 k1), then a 16-point DFT over n2, giving
// X[k1 + 16 k2].  Sixteen threads per line, sixteen lines per block; shared-memory
// slot of entry i is i + i/16 (groups of 16 sit one slot apart, conflict-free for
// both the strided and the contiguous 16-point gathers).
__device__ __forceinline__ int slot16(int i) { return i + (i >> 4); }

__device__ __forceinline__ void dft16(float2 (&v)[16], const float2 (&tw16)[8]) {
  float2 a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = v[(int)(__brev((unsigned)j) >> 28)];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int m = 1 << s;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int j = k & (m - 1), i0 = ((k >> s) << (s + 1)) + j;
      const float2 w = tw16[j << (3 - s)];
      const float2 x = a[i0], y = a[i0 + m];
      const float2 wy = make_float2(w.x * y.x - w.y * y.y, w.x * y.y + w.y * y.x);
      a[i0] = make_float2(x.x + wy.x, x.y + wy.y);
      a[i0 + m] = make_float2(x.x - wy.x, x.y - wy.y);
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = a[j];
}

__global__ void __launch_bounds__(256) fft256_kernel(const float* in, float* out,
                                                     int lines_per_img, int line_stride,
                                                     int elem_stride, int plane, int inverse) {
  constexpr int N = 256, G = 16, LS = N + N / 16 + 1;  // odd slot stride across lines
  __shared__ float2 sm[G * LS];
  __shared__ float2 tw256[N];
  const int b = blockIdx.y;
  const int l0 = blockIdx.x * G;
  const size_t ib = (size_t)b * 2 * plane;
  const bool rows = elem_stride == 1;
  {
    float sn, cs;
    sincospif(2.f * (float)threadIdx.x / (float)N, &sn, &cs);
    tw256[threadIdx.x] = make_float2(cs, inverse ? sn : -sn);
  }
  for (int idx = threadIdx.x; idx < G * N; idx += 256) {
    const int l = rows ? idx >> 8 : idx & (G - 1);
    const int e = rows ? idx & (N - 1) : idx >> 4;
    if (l0 + l >= lines_per_img) continue;
    const size_t o = ib + (size_t)(l0 + l) * line_stride + (size_t)e * elem_stride;
    sm[l * LS + slot16(e)] = make_float2(in[o], in[o + plane]);
  }
  __syncthreads();
  float2 t16[8];  // W_16^j = W_256^(16 j)
#pragma unroll
  for (int j = 0; j < 8; ++j) t16[j] = tw256[16 * j];
  const int l = threadIdx.x >> 4, q = threadIdx.x & 15;
  float2* L = sm + l * LS;
  float2 v[16];
  // step A: thread q = n2 takes x[16 n1 + n2], n1 = 0..15
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) v[n1] = L[slot16(16 * n1 + q)];
  dft16(v, t16);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    const float2 w = tw256[(q * k1) & (N - 1)];
    v[k1] = make_float2(w.x * v[k1].x - w.y * v[k1].y, w.x * v[k1].y + w.y * v[k1].x);
  }
  __syncthreads();
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) L[slot16(16 * k1 + q)] = v[k1];
  __syncthreads();
  // step B: thread q = k1 takes the 16 values of its k1 over n2
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) v[n2] = L[slot16(16 * q + n2)];
  dft16(v, t16);
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) L[slot16(q + 16 * k2)] = v[k2];
  __syncthreads();
  const float scale = 1.f / 16.f;  // 1 / sqrt(256)
  for (int idx = threadIdx.x; idx < G * N; idx += 256) {
    const int ll = rows ? idx >> 8 : idx & (G - 1);
    const int e = rows ? idx & (N - 1) : idx >> 4;
    if (l0 + ll >= lines_per_img) continue;
    const size_t o = ib + (size_t)(l0 + ll) * line_stride + (size_t)e * elem_stride;
    const float2 r = sm[ll * LS + slot16(e)];
    out[o] = r.x * scale;
    out[o + plane] = r.y * scale;
  }
}

static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

bool fft_size_ok(int n) { return n >= 8 && n <= 1024 && (n & (n - 1)) == 0; }

// out = F x (inverse = 0) or F^{-1} x (inverse = 1) for n complex images (2 planes
// each) of H x W; in and out may alias.
cudaError_t launch_fft2(const float* in, float* out, int n, int H, int W, int inverse,
                        cudaStream_t st) {
  if (!fft_size_ok(H) || !fft_size_ok(W)) return cudaErrorInvalidValue;
  const int plane = H * W;
  if (W == 256 && H == 256) {  // the benchmark size: four-step kernel for both passes
    dim3 grid(256 / 16, n);
    fft256_kernel<<<grid, 256, 0, st>>>(in, out, 256, 256, 1, plane, inverse);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fft256_kernel<<<grid, 256, 0, st>>>(out, out, 256, 1, 256, plane, inverse);
    return cudaGetLastError();
  }
  // rows: G rows per block (G a power of two)
  {
    const int G = std::max(1, 4096 / W);
    const int LS = W + W / 32 + 1;
    const size_t smem = (size_t)G * LS * 8 + (size_t)(W / 2) * 8;
    dim3 grid((H + G - 1) / G, n);
    fft_lines_kernel<<<grid, FFT_THREADS, smem, st>>>(in, out, W, ilog2(W), G, ilog2(G), H, W, 1,
                                                      plane, inverse);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // columns: G consecutive columns per block (G a power of two)
  {
    const int G = std::min(W, std::max(1, 4096 / H));
    const int LS = H + H / 32 + 1;
    const size_t smem = (size_t)G * LS * 8 + (size_t)(H / 2) * 8;
    dim3 grid((W + G - 1) / G, n);
    fft_lines_kernel<<<grid, FFT_THREADS, smem, st>>>(out, out, H, ilog2(H), G, ilog2(G), W, 1, W,
                                                      plane, inverse);
  }
  return cudaGetLastError();
}

// k-space residual of the MRI data term: e = M . K - y (both planes; y = null
// reads as 0, giving M . K for the Hessian product A^T A u), written over K, and
// 1/2 |e|^2 summed per image into fsum.
__global__ void __launch_bounds__(256) kspace_residual_kernel(
    int hw, float* __restrict__ K, const float* __restrict__ y, const uint8_t* __restrict__ mask,
    double* __restrict__ fsum) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  double part = 0.0;
  for (int p = blockIdx.x * 256 + threadIdx.x; p < hw; p += gridDim.x * 256) {
    const float m = (float)mask[(size_t)b * hw + p];
    const size_t r = (size_t)b * 2 * hw + p, i = r + hw;
    const float er = m * K[r] - (y ? y[r] : 0.f), ei = m * K[i] - (y ? y[i] : 0.f);
    K[r] = er;
    K[i] = ei;
    part += 0.5 * ((double)er * er + (double)ei * ei);
  }
  if (fsum) {
    const double s = block_sum(part, red);
    if (threadIdx.x == 0) atomicAdd(fsum + b, s);
  }
}

// K <- M . K (plain masking, both planes)
__global__ void kspace_mask_kernel(int hw, float* __restrict__ K, const uint8_t* __restrict__ mask) {
  const int b = blockIdx.y;
  for (int p = blockIdx.x * 256 + threadIdx.x; p < hw; p += gridDim.x * 256) {
    const float m = (float)mask[(size_t)b * hw + p];
    const size_t r = (size_t)b * 2 * hw + p;
    K[r] *= m;
    K[r + hw] *= m;
  }
}

// K <- (tau M y + K) / (tau M + 1): the k-space form of prox_{tau f} (App. E)
__global__ void kspace_prox_kernel(int hw, float* __restrict__ K, const float* __restrict__ y,
                                   const uint8_t* __restrict__ mask, float tau) {
  const int b = blockIdx.y;
  for (int p = blockIdx.x * 256 + threadIdx.x; p < hw; p += gridDim.x * 256) {
    const float tm = tau * (float)mask[(size_t)b * hw + p];
    const size_t r = (size_t)b * 2 * hw + p, i = r + hw;
    K[r] = (tm * y[r] + K[r]) / (tm + 1.f);
    K[i] = (tm * y[i] + K[i]) / (tm + 1.f);
  }
}

static dim3 kgrid(int n, int hw) {
  return dim3((unsigned)std::min((hw + 255) / 256, 64), (unsigned)n);
}

cudaError_t launch_mri_grad(int n, int H, int W, const float* z, const float* y,
                            const uint8_t* mask, float* kbuf, float* gf, double* fsum,
                            cudaStream_t st) {
  cudaError_t e = launch_fft2(z, kbuf, n, H, W, 0, st);
  if (e != cudaSuccess) return e;
  kspace_residual_kernel<<<kgrid(n, H * W), 256, 0, st>>>(H * W, kbuf, y, mask, fsum);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_fft2(kbuf, gf, n, H, W, 1, st);
}

cudaError_t launch_mri_apply(int n, int H, int W, const float* x, const uint8_t* mask,
                             int adjoint, float* out, cudaStream_t st) {
  cudaError_t e;
  if (!adjoint) {  // M . F x
    if ((e = launch_fft2(x, out, n, H, W, 0, st)) != cudaSuccess) return e;
    kspace_mask_kernel<<<kgrid(n, H * W), 256, 0, st>>>(H * W, out, mask);
    return cudaGetLastError();
  }
  // F^{-1}(M . r): mask a copy, then transform it in place
  if ((e = cudaMemcpyAsync(out, x, (size_t)n * 2 * H * W * 4, cudaMemcpyDeviceToDevice, st)) !=
      cudaSuccess)
    return e;
  kspace_mask_kernel<<<kgrid(n, H * W), 256, 0, st>>>(H * W, out, mask);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_fft2(out, out, n, H, W, 1, st);
}

cudaError_t launch_mri_prox(int n, int H, int W, const float* v, const float* y,
                            const uint8_t* mask, float tau, float* out, cudaStream_t st) {
  cudaError_t e = launch_fft2(v, out, n, H, W, 0, st);
  if (e != cudaSuccess) return e;
  kspace_prox_kernel<<<kgrid(n, H * W), 256, 0, st>>>(H * W, out, y, mask, tau);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_fft2(out, out, n, H, W, 1, st);
}

}  // namespace ideq

// ===================================================================== spectral blur
//
// The circular blur A x = k * x is diagonal in the DFT basis: with the unitary F,
// F(k * x) = sqrt(hw) F(k~) F(x), k~ the kernel placed on the h x w torus with its
// centre at the origin.  For power-of-two images the data step runs there:
//   E = K Z - Y  (K = sqrt(hw) F k~, Z = F z, Y = F y),  f = 1/2 ||E||^2 (Parseval),
//   grad f = F^{-1}(conj(K) E).
// Real images are packed two channels per complex image (re = channel 2p,
// im = channel 2p+1, zero when c is odd); the kernel is real, so each part of the
// packed product is the blur of its own channel.

namespace ideq {

// khat[b] (complex plane pair) <- kernel b embedded on the torus, centre at (0, 0)
__global__ void blur_embed_kernel(int H, int W, int kh, int kw, const float* __restrict__ ker,
                                  float* __restrict__ khat) {
  const int b = blockIdx.y;
  const int hw = H * W;
  for (int p = blockIdx.x * 256 + threadIdx.x; p < hw; p += gridDim.x * 256) {
    const int i = p / W, j = p % W;
    // tap (u, v) lands at ((u - cy) mod H, (v - cx) mod W)
    int u = i + kh / 2, v = j + kw / 2;
    u -= (u >= H) ? H : 0;
    v -= (v >= W) ? W : 0;
    float val = 0.f;
    if (u < kh && v < kw) val = ker[(size_t)b * kh * kw + u * kw + v];
    khat[(size_t)b * 2 * hw + p] = val;
    khat[(size_t)b * 2 * hw + hw + p] = 0.f;
  }
}

// pk[b][p] (re, im) <- x[b][2p], x[b][2p+1]
__global__ void pack_pairs_kernel(int c, int hw, const float* __restrict__ x,
                                  float* __restrict__ pk) {
  const int b = blockIdx.y, cc = (c + 1) / 2;
  for (int q = blockIdx.x * 256 + threadIdx.x; q < cc * hw; q += gridDim.x * 256) {
    const int p = q / hw, e = q % hw;
    const size_t o = ((size_t)b * cc + p) * 2 * hw + e;
    pk[o] = x[((size_t)b * c + 2 * p) * hw + e];
    pk[o + hw] = (2 * p + 1 < c) ? x[((size_t)b * c + 2 * p + 1) * hw + e] : 0.f;
  }
}

__global__ void unpack_pairs_kernel(int c, int hw, const float* __restrict__ pk,
                                    float* __restrict__ x) {
  const int b = blockIdx.y, cc = (c + 1) / 2;
  for (int q = blockIdx.x * 256 + threadIdx.x; q < cc * hw; q += gridDim.x * 256) {
    const int p = q / hw, e = q % hw;
    const size_t o = ((size_t)b * cc + p) * 2 * hw + e;
    x[((size_t)b * c + 2 * p) * hw + e] = pk[o];
    if (2 * p + 1 < c) x[((size_t)b * c + 2 * p + 1) * hw + e] = pk[o + hw];
  }
}

// Z <- conj(K) (K Z - Y) per entry (Y = null: conj(K) K Z), with 1/2 |K Z - Y|^2
// summed per image into fsum.  K is scaled by sqrt(hw) here.
__global__ void __launch_bounds__(256) spectral_grad_kernel(int cc, int hw, float kscale,
                                                            const float* __restrict__ khat,
                                                            const float* __restrict__ Y,
                                                            float* __restrict__ Z,
                                                            double* __restrict__ fsum) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  double part = 0.0;
  for (int q = blockIdx.x * 256 + threadIdx.x; q < cc * hw; q += gridDim.x * 256) {
    const int p = q / hw, e = q % hw;
    const float kr = kscale * khat[(size_t)b * 2 * hw + e];
    const float ki = kscale * khat[(size_t)b * 2 * hw + hw + e];
    const size_t o = ((size_t)b * cc + p) * 2 * hw + e;
    const float zr = Z[o], zi = Z[o + hw];
    float er = kr * zr - ki * zi, ei = kr * zi + ki * zr;
    if (Y) {
      er -= Y[o];
      ei -= Y[o + hw];
    }
    part += 0.5 * ((double)er * er + (double)ei * ei);
    Z[o] = kr * er + ki * ei;  // conj(K) E
    Z[o + hw] = kr * ei - ki * er;
  }
  if (fsum) {
    const double s = block_sum(part, red);
    if (threadIdx.x == 0) atomicAdd(fsum + b, s);
  }
}

static dim3 sgrid(int n, long long per) {
  return dim3((unsigned)std::min<long long>((per + 255) / 256, 128), (unsigned)n);
}

cudaError_t launch_blur_spectrum(int n, int H, int W, int kh, int kw, const float* ker,
                                 float* khat, cudaStream_t st) {
  blur_embed_kernel<<<sgrid(n, (long long)H * W), 256, 0, st>>>(H, W, kh, kw, ker, khat);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_fft2(khat, khat, n, H, W, 0, st);
}

cudaError_t launch_pack_fft(int n, int c, int H, int W, const float* x, float* pk,
                            cudaStream_t st) {
  const int cc = (c + 1) / 2;
  pack_pairs_kernel<<<sgrid(n, (long long)cc * H * W), 256, 0, st>>>(c, H * W, x, pk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_fft2(pk, pk, n * cc, H, W, 0, st);
}

cudaError_t launch_blur_grad_spectral(int n, int c, int H, int W, const float* z,
                                      const float* khat, const float* yhat, float* pk, float* gf,
                                      double* fsum, cudaStream_t st) {
  const int cc = (c + 1) / 2;
  cudaError_t e = launch_pack_fft(n, c, H, W, z, pk, st);
  if (e != cudaSuccess) return e;
  spectral_grad_kernel<<<sgrid(n, (long long)cc * H * W), 256, 0, st>>>(
      cc, H * W, sqrtf((float)(H * W)), khat, yhat, pk, fsum);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_fft2(pk, pk, n * cc, H, W, 1, st)) != cudaSuccess) return e;
  unpack_pairs_kernel<<<sgrid(n, (long long)cc * H * W), 256, 0, st>>>(c, H * W, pk, gf);
  return cudaGetLastError();
}

}  // namespace ideq
