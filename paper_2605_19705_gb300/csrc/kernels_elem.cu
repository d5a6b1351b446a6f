// Data-step stencils, the fused RED update with its FP64 reductions, the
// per-image restart/stopping logic of Algorithm 1, and weight re-layouts.
#include "common.cuh"
#include "ideq_internal.h"

#include <cmath>
#include <cstdlib>

namespace ideq {

// ===================================================================== data step
//
// Circular 2-D stencils of the blur forward models (one per-image kernel shared
// by the channels).  A block computes a 32x32 output tile from a shared-memory
// tile with a (kh-1, kw-1) halo that wraps around the image borders; each
// thread owns outputs (ty + 16a, tx + 16b), a, b in {0,1}, so that shared
// reads of neighbouring threads hit consecutive words.
//
//   forward  (k * x)[i,j]   = sum_{u,v} k[u,v] x[i-u+cy, j-v+cx]
//   adjoint  (k^T r)[i,j]   = sum_{u,v} k[u,v] r[i+u-cy, j+v-cx]
// Both reduce to a correlation over the halo tile with the kernel flipped for
// the forward direction.

enum DataEpi { DE_PLAIN = 0, DE_LIN_RES = 1, DE_SAT_RES = 2, DE_SAT_PLAIN = 3, DE_SAT_JW = 4 };

constexpr int BT = 32;       // output tile edge
constexpr int MAXK = 31;     // largest supported kernel edge
constexpr int TILE_E = BT + MAXK - 1;

__global__ void __launch_bounds__(256) blur_tile_kernel(
    int c, int H, int W, int kh, int kw, const float* __restrict__ ker, int flip,
    const float* __restrict__ in, const float* __restrict__ y, float* __restrict__ out,
    double* __restrict__ fsum, int epi, float gain) {
  __shared__ float sk[MAXK * MAXK];
  __shared__ float st[TILE_E * TILE_E];
  __shared__ double red[32];
  const int plane = blockIdx.z;  // b * c + ch
  const int b = plane / c;
  const int i0 = blockIdx.y * BT, j0 = blockIdx.x * BT;
  const int cy = kh / 2, cx = kw / 2;
  const int tw = BT + kw - 1, th = BT + kh - 1;
  const int tid = threadIdx.y * 16 + threadIdx.x;
  const float* kb = ker + (size_t)b * kh * kw;
  for (int e = tid; e < kh * kw; e += 256) {
    const int u = e / kw, v = e % kw;
    sk[e] = flip ? kb[(kh - 1 - u) * kw + (kw - 1 - v)] : kb[e];
  }
  const float* pin = in + (size_t)plane * H * W;
  // forward: rows i - u + cy over u in [0,kh) -> tile starts at i0 - cy (symmetric halo)
  for (int e = tid; e < th * tw; e += 256) {
    const int ti = e / tw, tj = e % tw;
    int gi = (i0 - cy + ti) % H;
    if (gi < 0) gi += H;
    int gj = (j0 - cx + tj) % W;
    if (gj < 0) gj += W;
    st[ti * TILE_E + tj] = pin[(size_t)gi * W + gj];
  }
  __syncthreads();
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  const int ty = threadIdx.y, tx = threadIdx.x;
  for (int u = 0; u < kh; ++u) {
    const float* r0 = st + (ty + u) * TILE_E + tx;
    const float* r1 = r0 + 16 * TILE_E;
    const float* kr = sk + u * kw;
    for (int v = 0; v < kw; ++v) {
      const float kv = kr[v];
      acc[0][0] = fmaf(kv, r0[v], acc[0][0]);
      acc[0][1] = fmaf(kv, r0[v + 16], acc[0][1]);
      acc[1][0] = fmaf(kv, r1[v], acc[1][0]);
      acc[1][1] = fmaf(kv, r1[v + 16], acc[1][1]);
    }
  }
  const float tg = (epi >= DE_SAT_RES) ? tanhf(gain) : 1.f;
  double part = 0.0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * bb;
      if (i >= H || j >= W) continue;
      const size_t idx = (size_t)plane * H * W + (size_t)i * W + j;
      const float q = acc[a][bb];
      float o;
      if (epi == DE_PLAIN) {
        o = q;
      } else if (epi == DE_LIN_RES) {
        const float e = q - (y ? y[idx] : 0.f);
        part += 0.5 * (double)e * (double)e;
        o = e;
      } else if (epi == DE_SAT_PLAIN) {
        o = tanhf(gain * q) / tg;
      } else if (epi == DE_SAT_RES) {
        const float t = tanhf(gain * q);
        const float e = t / tg - y[idx];
        part += 0.5 * (double)e * (double)e;
        o = (gain / tg) * (1.f - t * t) * e;
      } else {  // DE_SAT_JW: Jacobian weight applied to r (passed as y)
        const float t = tanhf(gain * q);
        o = (gain / tg) * (1.f - t * t) * y[idx];
      }
      out[idx] = o;
    }
  if (fsum != nullptr && (epi == DE_LIN_RES || epi == DE_SAT_RES)) {
    const double s = block_sum(part, red);
    if (tid == 0) atomicAdd(fsum + b, s);
  }
}

__global__ void mask_res_kernel(int c, int hw, const uint8_t* __restrict__ m,
                                const float* __restrict__ in, const float* __restrict__ y,
                                float* __restrict__ out, double* __restrict__ fsum, int plain) {
  __shared__ double red[32];
  const int plane = blockIdx.y;  // b * c + ch
  const int b = plane / c;
  double part = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < hw; p += gridDim.x * blockDim.x) {
    const size_t idx = (size_t)plane * hw + p;
    const float mv = (float)m[(size_t)b * hw + p];
    if (plain) {
      out[idx] = mv * in[idx];
    } else {
      const float e = mv * in[idx] - (y ? y[idx] : 0.f);
      part += 0.5 * (double)e * (double)e;
      out[idx] = mv * e;
    }
  }
  if (fsum != nullptr && !plain) {
    const double s = block_sum(part, red);
    if (threadIdx.x == 0) atomicAdd(fsum + b, s);
  }
}

// Strip form for the common square kernel sizes: a block computes 64 rows x 32
// columns; each thread owns a column strip of 8 outputs and, for every kernel
// column v, slides down the KH + 7 input rows it needs, adding each loaded value
// to every output of the strip whose kernel row it meets.  The kernel column
// sits in registers: ~(KH + 7) shared loads per 8 * KH FMAs.
constexpr int SR = 64, SC = 32, SS = 8;  // rows, columns, strip height

template <int KH>
__global__ void __launch_bounds__(256) blur_strip_kernel(
    int c, int H, int W, const float* __restrict__ ker, int flip, const float* __restrict__ in,
    const float* __restrict__ y, float* __restrict__ out, double* __restrict__ fsum, int epi,
    float gain) {
  constexpr int KW = KH;
  constexpr int TR = SR + KH - 1, TC = SC + KW - 1;
  __shared__ float sk[KH * KW];
  __shared__ float st[TR * TC];
  __shared__ double red[32];
  const int plane = blockIdx.z;
  const int b = plane / c;
  const int i0 = blockIdx.y * SR, j0 = blockIdx.x * SC;
  const int cy = KH / 2, cx = KW / 2;
  const int tid = threadIdx.x;
  const float* kb = ker + (size_t)b * KH * KW;
  for (int e = tid; e < KH * KW; e += 256) {
    const int u = e / KW, v = e % KW;
    sk[e] = flip ? kb[(KH - 1 - u) * KW + (KW - 1 - v)] : kb[e];
  }
  const float* pin = in + (size_t)plane * H * W;
  for (int e = tid; e < TR * TC; e += 256) {
    const int ti = e / TC, tj = e % TC;
    int gi = (i0 - cy + ti) % H;
    if (gi < 0) gi += H;
    int gj = (j0 - cx + tj) % W;
    if (gj < 0) gj += W;
    st[e] = pin[(size_t)gi * W + gj];
  }
  __syncthreads();
  const int col = tid & 31, r0 = (tid >> 5) * SS;
  float acc[SS];
#pragma unroll
  for (int i = 0; i < SS; ++i) acc[i] = 0.f;
#pragma unroll 1
  for (int v = 0; v < KW; ++v) {
    float kv[KH];
#pragma unroll
    for (int u = 0; u < KH; ++u) kv[u] = sk[u * KW + v];
    const float* sp = st + r0 * TC + col + v;
#pragma unroll
    for (int R = 0; R < SS + KH - 1; ++R) {
      const float val = sp[R * TC];
#pragma unroll
      for (int i = 0; i < SS; ++i) {
        const int u = R - i;
        if (u >= 0 && u < KH) acc[i] = fmaf(kv[u], val, acc[i]);
      }
    }
  }
  const float tg = (epi >= DE_SAT_RES) ? tanhf(gain) : 1.f;
  double part = 0.0;
  const int j = j0 + col;
#pragma unroll
  for (int i = 0; i < SS; ++i) {
    const int r = i0 + r0 + i;
    if (r >= H || j >= W) continue;
    const size_t idx = (size_t)plane * H * W + (size_t)r * W + j;
    const float q = acc[i];
    float o;
    if (epi == DE_PLAIN) {
      o = q;
    } else if (epi == DE_LIN_RES) {
      const float e = q - (y ? y[idx] : 0.f);
      part += 0.5 * (double)e * (double)e;
      o = e;
    } else if (epi == DE_SAT_PLAIN) {
      o = tanhf(gain * q) / tg;
    } else if (epi == DE_SAT_RES) {
      const float t = tanhf(gain * q);
      const float e = t / tg - y[idx];
      part += 0.5 * (double)e * (double)e;
      o = (gain / tg) * (1.f - t * t) * e;
    } else {
      const float t = tanhf(gain * q);
      o = (gain / tg) * (1.f - t * t) * y[idx];
    }
    out[idx] = o;
  }
  if (fsum != nullptr && (epi == DE_LIN_RES || epi == DE_SAT_RES)) {
    const double s2 = block_sum(part, red);
    if (tid == 0) atomicAdd(fsum + b, s2);
  }
}

static cudaError_t blur_launch(const OpDev& op, int n, int c, int H, int W, int flip,
                               const float* in, const float* y, float* out, double* fsum,
                               int epi, cudaStream_t st) {
  if (op.kh > MAXK || op.kw > MAXK) return cudaErrorInvalidValue;
  if (op.kh == op.kw && (op.kh == 9 || op.kh == 15 || op.kh == 25)) {
    dim3 grid((W + SC - 1) / SC, (H + SR - 1) / SR, n * c);
    if (op.kh == 9)
      blur_strip_kernel<9><<<grid, 256, 0, st>>>(c, H, W, op.kernel, flip, in, y, out, fsum, epi,
                                                 op.gain);
    else if (op.kh == 15)
      blur_strip_kernel<15><<<grid, 256, 0, st>>>(c, H, W, op.kernel, flip, in, y, out, fsum, epi,
                                                  op.gain);
    else
      blur_strip_kernel<25><<<grid, 256, 0, st>>>(c, H, W, op.kernel, flip, in, y, out, fsum, epi,
                                                  op.gain);
    return cudaGetLastError();
  }
  dim3 grid((W + BT - 1) / BT, (H + BT - 1) / BT, n * c), block(16, 16);
  blur_tile_kernel<<<grid, block, 0, st>>>(c, H, W, op.kh, op.kw, op.kernel, flip, in, y, out,
                                           fsum, epi, op.gain);
  return cudaGetLastError();
}

static cudaError_t mask_launch(const OpDev& op, int n, int c, int H, int W, const float* in,
                               const float* y, float* out, double* fsum, int plain,
                               cudaStream_t st) {
  const int hw = H * W;
  dim3 grid(std::min((hw + 255) / 256, 64), n * c);
  mask_res_kernel<<<grid, 256, 0, st>>>(c, hw, op.mask, in, y, out, fsum, plain);
  return cudaGetLastError();
}

cudaError_t launch_data_fwd(const OpDev& op, int n, int c, int H, int W, const float* in,
                            const float* y, float* out, double* fsum, cudaStream_t st) {
  if (op.kind == IDEQ_OP_MASK) return mask_launch(op, n, c, H, W, in, y, out, fsum, 0, st);
  return blur_launch(op, n, c, H, W, 1, in, y, out, fsum,
                     op.kind == IDEQ_OP_SATBLUR ? DE_SAT_RES : DE_LIN_RES, st);
}

cudaError_t launch_blur_adj(const OpDev& op, int n, int c, int H, int W, const float* in,
                            float* out, cudaStream_t st) {
  return blur_launch(op, n, c, H, W, 0, in, nullptr, out, nullptr, DE_PLAIN, st);
}

cudaError_t launch_apply_A(const OpDev& op, int n, int c, int H, int W, const float* x,
                           float* Ax, cudaStream_t st) {
  if (op.kind == IDEQ_OP_MASK) return mask_launch(op, n, c, H, W, x, nullptr, Ax, nullptr, 1, st);
  return blur_launch(op, n, c, H, W, 1, x, nullptr, Ax, nullptr,
                     op.kind == IDEQ_OP_SATBLUR ? DE_SAT_PLAIN : DE_PLAIN, st);
}

cudaError_t launch_sat_jt_weight(const OpDev& op, int n, int c, int H, int W, const float* lin,
                                 const float* r, float* tmp, cudaStream_t st) {
  return blur_launch(op, n, c, H, W, 1, lin, r, tmp, nullptr, DE_SAT_JW, st);
}

// ===================================================================== iteration

// z = x + beta_b (x - x_prev), beta_b per image (0 after a restart or once frozen).
__global__ void extrapolate_kernel(int per_img, long long total, const float* __restrict__ x,
                                   const float* __restrict__ xp, const float* __restrict__ beta,
                                   float* __restrict__ z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float bb = beta[i / per_img];
    const float xv = x[i];
    z[i] = fmaf(bb, xv - xp[i], xv);
  }
}

__global__ void extrapolate4_kernel(int per4, long long total4, const float4* __restrict__ x,
                                    const float4* __restrict__ xp,
                                    const float* __restrict__ beta, float4* __restrict__ z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total4;
       i += (long long)gridDim.x * blockDim.x) {
    const float bb = beta[i / per4];
    const float4 a = x[i], p = xp[i];
    z[i] = make_float4(fmaf(bb, a.x - p.x, a.x), fmaf(bb, a.y - p.y, a.y),
                       fmaf(bb, a.z - p.z, a.z), fmaf(bb, a.w - p.w, a.w));
  }
}

cudaError_t launch_extrapolate(int n, int per_img, const float* x, const float* xp,
                               const float* beta_eff, float* z, cudaStream_t st) {
  const long long total = (long long)n * per_img;
  if (per_img % 4 == 0 && (((uintptr_t)x | (uintptr_t)xp | (uintptr_t)z) & 15) == 0) {
    const long long t4 = total / 4;
    const int blocks = (int)std::min<long long>((t4 + 255) / 256, 152 * 8);
    extrapolate4_kernel<<<blocks, 256, 0, st>>>(per_img / 4, t4, (const float4*)x,
                                                (const float4*)xp, beta_eff, (float4*)z);
  } else {
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
    extrapolate_kernel<<<blocks, 256, 0, st>>>(per_img, total, x, xp, beta_eff, z);
  }
  return cudaGetLastError();
}

// z = x + beta (x - xp), and the averaging step's bookkeeping: the running sum
// (FP64) of the z's gains this z, after its previous value became the snapshot
// if the last update set a new minimum inside the window.
__global__ void extrapolate_avg_kernel(int per, long long total, const float* __restrict__ x,
                                       const float* __restrict__ xp, SolverDev s,
                                       float* __restrict__ z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per);
    const float a = x[i];
    const float zz = fmaf(s.beta_eff[b], a - xp[i], a);
    z[i] = zz;
    const double s0 = s.zsum[i];
    if (s.snap[b]) s.zsnap[i] = s0;
    s.zsum[i] = s0 + (double)zz;
  }
}

cudaError_t launch_extrapolate_avg(int n, int per_img, const float* x, const float* xp,
                                   const SolverDev& s, float* z, cudaStream_t st) {
  const long long total = (long long)n * per_img;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
  extrapolate_avg_kernel<<<blocks, 256, 0, st>>>(per_img, total, x, xp, s, z);
  return cudaGetLastError();
}

// Averaging step output: x_hat = (sum_{k <= K0} z^k) / (K0 + 1) for the images
// that ran all K updates and have a K0; the others keep their last iterate.
__global__ void average_out_kernel(int per, long long total, SolverDev s, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per);
    if (s.status[b] != IDEQ_IMG_MAXITER || s.k0[b] < 0) continue;
    const double sum = s.snap[b] ? s.zsum[i] : s.zsnap[i];
    out[i] = (float)(sum / (double)(s.k0[b] + 1));
  }
}

cudaError_t launch_average_out(int n, int per_img, const SolverDev& s, float* out,
                               cudaStream_t st) {
  const long long total = (long long)n * per_img;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
  average_out_kernel<<<blocks, 256, 0, st>>>(per_img, total, s, out);
  return cudaGetLastError();
}

// Proximal step of i-DEQ-P for the inpainting mask (Eq. red_prox, App. E):
// v = z - tau lambda grad g, x_new = (tau m y + v) / (tau m + 1) with the image's
// 0/1 mask m shared by the channels; same FP64 step-norm partials as the RED update.
__global__ void __launch_bounds__(256) prox_update_kernel(
    int per_img, int hw, const float* __restrict__ z, const float* __restrict__ gg,
    const float* __restrict__ y, const uint8_t* __restrict__ mask, const float* __restrict__ x,
    float* __restrict__ xn, float lam, float tau, const int* __restrict__ status,
    double* __restrict__ part_s, double* __restrict__ part_x) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const int nblk = gridDim.x;
  const bool run = status[b] == IDEQ_IMG_RUNNING;
  double ss = 0.0, sx = 0.0;
  const size_t base = (size_t)b * per_img;
  if (run) {
    for (int i = blockIdx.x * 256 + threadIdx.x; i < per_img; i += nblk * 256) {
      const float v = z[base + i] - tau * lam * gg[base + i];
      const float m = (float)mask[(size_t)b * hw + i % hw];
      const float o = (tau * m * y[base + i] + v) / (tau * m + 1.f);
      xn[base + i] = o;
      const float d = o - x[base + i], xv = x[base + i];
      ss += (double)(d * d);
      sx += (double)(xv * xv);
    }
  }
  const double ts = block_sum(ss, red);
  const double tx = block_sum(sx, red);
  if (threadIdx.x == 0) {
    part_s[(size_t)b * nblk + blockIdx.x] = ts;
    part_x[(size_t)b * nblk + blockIdx.x] = tx;
  }
}

cudaError_t launch_prox_update(int n, int per_img, int hw, int nblk, const float* z,
                               const float* gg, const float* y, const uint8_t* mask,
                               const float* x, float* xn, float lam, float tau,
                               const int* status, double* part_s, double* part_x,
                               cudaStream_t st) {
  prox_update_kernel<<<dim3(nblk, n), 256, 0, st>>>(per_img, hw, z, gg, y, mask, x, xn, lam, tau,
                                                    status, part_s, part_x);
  return cudaGetLastError();
}

// Accept a candidate update computed elsewhere (the MRI proximal step) for the
// running images, with the same FP64 step-norm partials as the RED update.
__global__ void __launch_bounds__(256) commit_update_kernel(
    int per_img, const float* __restrict__ cand, const float* __restrict__ x,
    float* __restrict__ xn, const int* __restrict__ status, double* __restrict__ part_s,
    double* __restrict__ part_x) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const int nblk = gridDim.x;
  double ss = 0.0, sx = 0.0;
  const size_t base = (size_t)b * per_img;
  if (status[b] == IDEQ_IMG_RUNNING) {
    for (int i = blockIdx.x * 256 + threadIdx.x; i < per_img; i += nblk * 256) {
      const float o = cand[base + i];
      xn[base + i] = o;
      const float d = o - x[base + i], xv = x[base + i];
      ss += (double)(d * d);
      sx += (double)(xv * xv);
    }
  }
  const double ts = block_sum(ss, red);
  const double tx = block_sum(sx, red);
  if (threadIdx.x == 0) {
    part_s[(size_t)b * nblk + blockIdx.x] = ts;
    part_x[(size_t)b * nblk + blockIdx.x] = tx;
  }
}

cudaError_t launch_commit_update(int n, int per_img, int nblk, const float* cand, const float* x,
                                 float* xn, const int* status, double* part_s, double* part_x,
                                 cudaStream_t st) {
  commit_update_kernel<<<dim3(nblk, n), 256, 0, st>>>(per_img, cand, x, xn, status, part_s,
                                                      part_x);
  return cudaGetLastError();
}

// ===================================================================== Rician

// B(t) = I1(t)/I0(t) and log I0(t) for t >= 0, from the power series of I0 and I1
// (t < 15) and from their Hankel asymptotic expansions (t >= 15, 14 terms):
//   I0(t) = sum_k (t^2/4)^k / (k!)^2,   I1(t) = (t/2) sum_k (t^2/4)^k / (k! (k+1)!),
//   I_nu(t) ~ e^t / sqrt(2 pi t) sum_k c_k(nu) / (8t)^k,
//   c_k(nu) = prod_{j<=k} ((2j-1)^2 - 4 nu^2) / k!   (nu = 0: 1, 1, 9/2, ...;
//   nu = 1: 1, -3, -15/2, ...); the common factor cancels in the ratio.
// Max relative error of B against SciPy's i1e/i0e over [1e-6, 1e6]: 5.4e-7 (FP32).
struct BesselRatio {
  float B, logI0;
};

IDEQ_DEV BesselRatio bessel_i1_i0(float t) {
  BesselRatio r;
  if (t < 15.f) {
    const float q = 0.25f * t * t;
    float s0 = 0.f, s1 = 0.f, a = 1.f, b = 1.f;
    for (int k = 0; k < 48; ++k) {
      s0 += a;
      s1 += b;
      a = a * q / (float)((k + 1) * (k + 1));
      b = b * q / (float)((k + 1) * (k + 2));
      if (a < s0 * 1e-9f) break;
    }
    r.B = 0.5f * t * s1 / s0;
    r.logI0 = logf(s0);
    return r;
  }
  // I0: terms (1 * 9 * 25 ...)/(k! (8t)^k), all positive; I1: 1 - 3/(8t) - 15/(2!(8t)^2) ...
  const float inv8t = 1.f / (8.f * t);
  float s0 = 0.f, s1 = 0.f, a0 = 1.f, a1 = 1.f;
  for (int k = 0; k < 14; ++k) {
    s0 += a0;
    s1 += a1;
    const int j = k + 1;
    const float odd2 = (float)((2 * j - 1) * (2 * j - 1));
    a0 = a0 * odd2 / (float)j * inv8t;
    a1 = a1 * (odd2 - 4.f) / (float)j * inv8t;
  }
  r.B = s1 / s0;
  r.logI0 = t - 0.5f * logf(6.283185307179586f * t) + logf(s0);
  return r;
}

__global__ void __launch_bounds__(256) rician_grad_kernel(int per_img, const float* __restrict__ x,
                                                          const float* __restrict__ y, float sigma,
                                                          float* __restrict__ gf,
                                                          double* __restrict__ fsum) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const float is2 = 1.f / (sigma * sigma);
  double part = 0.0;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < per_img; i += gridDim.x * 256) {
    const size_t o = (size_t)b * per_img + i;
    const float xv = x[o], yv = y[o];
    const float t = xv * yv * is2;
    const BesselRatio br = bessel_i1_i0(fabsf(t));  // B odd, log I0 even
    const float B = t < 0.f ? -br.B : br.B;
    gf[o] = xv * is2 - yv * is2 * B;
    part += 0.5 * (double)xv * xv * is2 - (double)br.logI0;
  }
  if (fsum) {
    const double s = block_sum(part, red);
    if (threadIdx.x == 0) atomicAdd(fsum + b, s);
  }
}

cudaError_t launch_rician_grad(int n, int per_img, const float* x, const float* y, float sigma,
                               float* gf, double* fsum, cudaStream_t st) {
  dim3 grid((unsigned)std::min((per_img + 255) / 256, 64), (unsigned)n);
  rician_grad_kernel<<<grid, 256, 0, st>>>(per_img, x, y, sigma, gf, fsum);
  return cudaGetLastError();
}

// Blocks per image of the update kernels: one per kUpdateElems values, at most
// kUpdateMaxBlocks (IDEQ_UPDATE_ELEMS / IDEQ_UPDATE_MAXBLK override them, read once).
static int update_cfg(const char* name, int dflt) {
  const char* v = std::getenv(name);
  const int x = (v && *v) ? std::atoi(v) : dflt;
  return x > 0 ? x : dflt;
}

int update_blocks_per_image(int per_img) {
  // 8192: measured on 8 x 3 x 256^2 (CUDA-graph timed, two kernels per call) 10.8 us
  // per call against 12.4-13.4 us at 1024-4096 (more blocks, more FP64 block sums)
  static const int elems = update_cfg("IDEQ_UPDATE_ELEMS", 8192);
  static const int maxb = update_cfg("IDEQ_UPDATE_MAXBLK", 64);
  const int b = (per_img + elems - 1) / elems;
  return std::max(1, std::min(b, maxb));
}

// x_new = z - tau (grad f + lambda grad g) for running images (RED step at z,
// Eq. ideq), with per-block FP64 partial sums of ||x_new - x||^2 and ||x||^2
// (squares summed in FP32 over at most 16 elements, every sum above that in FP64).
// Frozen images are left untouched.
__global__ void __launch_bounds__(256) red_update_kernel(
    int per_img, const float* __restrict__ z, const float* __restrict__ gf,
    const float* __restrict__ gg, const float* __restrict__ x, float* __restrict__ xn,
    float lam, float tau, const int* __restrict__ status, double* __restrict__ part_s,
    double* __restrict__ part_x, const float* __restrict__ addv, int vec4) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const int nblk = gridDim.x;
  const bool run = status == nullptr || status[b] == IDEQ_IMG_RUNNING;
  double ss = 0.0, sx = 0.0;
  const size_t base = (size_t)b * per_img;
  if (run) {
    if (vec4) {
      const int n4 = per_img >> 2;
      const float4* z4 = (const float4*)(z + base);
      const float4* f4 = (const float4*)(gf + base);
      const float4* g4 = (const float4*)(gg + base);
      const float4* x4 = (const float4*)(x + base);
      float4* o4 = (float4*)(xn + base);
      // squares summed in FP32 over at most 16 elements (four float4 iterations;
      // o - x is exact when the two are within a factor of two, as near a fixed
      // point), every sum above that in FP64: FP64 arithmetic per element would
      // bound this pass on this GPU
      // four grid-strided float4 positions per round, all sixteen loads issued
      // before any arithmetic: a round costs one memory latency, not four
      constexpr int U = 4;
      const int stride = nblk * 256;
      for (int i0 = blockIdx.x * 256 + threadIdx.x; i0 < n4; i0 += U * stride) {
        float4 zv[U], fv[U], gv[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = i0 + u * stride;
          if (i < n4) {
            zv[u] = z4[i];
            fv[u] = f4[i];
            gv[u] = g4[i];
            xv[u] = x4[i];
          }
        }
        float s32 = 0.f, x32 = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = i0 + u * stride;
          if (i < n4) {
            float4 o;
            o.x = zv[u].x - tau * (fv[u].x + lam * gv[u].x);
            o.y = zv[u].y - tau * (fv[u].y + lam * gv[u].y);
            o.z = zv[u].z - tau * (fv[u].z + lam * gv[u].z);
            o.w = zv[u].w - tau * (fv[u].w + lam * gv[u].w);
            o4[i] = o;
            const float d0 = o.x - xv[u].x, d1 = o.y - xv[u].y, d2 = o.z - xv[u].z,
                        d3 = o.w - xv[u].w;
            s32 += d0 * d0 + d1 * d1 + (d2 * d2 + d3 * d3);
            x32 += xv[u].x * xv[u].x + xv[u].y * xv[u].y + (xv[u].z * xv[u].z + xv[u].w * xv[u].w);
          }
        }
        ss += (double)s32;
        sx += (double)x32;
      }
    } else {
      for (int i = blockIdx.x * 256 + threadIdx.x; i < per_img; i += nblk * 256) {
        float o = z[base + i] - tau * (gf[base + i] + lam * gg[base + i]);
        if (addv) o += addv[base + i];
        xn[base + i] = o;
        const float d = o - x[base + i], xv = x[base + i];
        ss += (double)(d * d);
        sx += (double)(xv * xv);
      }
    }
  }
  const double ts = block_sum(ss, red);
  const double tx = block_sum(sx, red);
  if (threadIdx.x == 0) {
    part_s[(size_t)b * nblk + blockIdx.x] = ts;
    part_x[(size_t)b * nblk + blockIdx.x] = tx;
  }
}

cudaError_t launch_red_update(int n, int per_img, int nblk, const float* z, const float* gf,
                              const float* gg, const float* x, float* xn, float lam, float tau,
                              const int* status, double* part_s, double* part_x,
                              cudaStream_t st, const float* addv) {
  dim3 grid(nblk, n);
  // float4 path only where every image starts on a 16-byte boundary: a caller's
  // sub-allocation or offset view may be only 4-byte aligned
  const uintptr_t align = (uintptr_t)z | (uintptr_t)gf | (uintptr_t)gg | (uintptr_t)x |
                          (uintptr_t)xn;
  const int vec4 = (per_img & 3) == 0 && addv == nullptr && (align & 15) == 0;
  red_update_kernel<<<grid, 256, 0, st>>>(per_img, z, gf, gg, x, xn, lam, tau, status, part_s,
                                          part_x, addv, vec4);
  return cudaGetLastError();
}

// Per-image bookkeeping after each update (Algorithm 1 and the stopping rule of
// App. D.1.3), one warp per image: sum the partials in a fixed order, then
//   k += 1, total += 1, S += ||dx||^2;
//   non-finite step            -> DIVERGED (frozen)
//   ||dx|| < tol ||x^k||       -> CONVERGED (frozen)
//   total == max_iter          -> MAXITER (frozen)
//   k S > B^2                  -> restart: k = 0, S = 0, next beta 0.
// avg_K > 0: track the averaging step of Algorithm 1 for a run of avg_K
// updates -- the update with index k (x^{k+1} from z^k) competes for K0 when
// floor(K/2) < k < K-1, the first strict minimum of ||x^{k+1} - x^k|| wins, and
// snap marks that the running sum of z up to z^k must be kept.
__global__ void finalize_kernel(int n, int nblk, SolverDev s, int parity_new, float beta,
                                float B, double tol, int max_iter, float lam, int logic,
                                int avg_K) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ int run_cnt[32];
  int my_run = 0;
  for (int b = wid; b < n; b += nw) {
    double ss = 0.0, sx = 0.0;
    for (int i = lane; i < nblk; i += 32) {
      ss += s.part_s[(size_t)b * nblk + i];
      sx += s.part_x[(size_t)b * nblk + i];
    }
    ss = warp_sum(ss);
    sx = warp_sum(sx);
    if (lane == 0) {
      const bool running = s.status[b] == IDEQ_IMG_RUNNING;
      if (avg_K > 0) s.snap[b] = 0;
      if (running) {
        const int kk = s.total[b];  // index k of this update
        if (avg_K > 0 && isfinite(ss) && kk > avg_K / 2 && kk < avg_K - 1 &&
            sqrt(ss) < s.best[b]) {
          s.best[b] = sqrt(ss);
          s.k0[b] = kk;
          s.snap[b] = 1;
        }
        const double rel = sx > 0.0 ? sqrt(ss / sx) : INFINITY;
        s.rel[b] = rel;
        s.energy[b] = s.fsum[b] + (double)lam * s.gsum[b];
        s.parity[b] = parity_new;
        s.total[b] += 1;
        if (logic) {
          s.k[b] += 1;
          s.S[b] += ss;
          int st = IDEQ_IMG_RUNNING;
          float be = beta;
          if (!isfinite(ss)) {
            st = IDEQ_IMG_DIVERGED;
          } else if (tol > 0.0 && sqrt(ss) < tol * sqrt(sx)) {
            st = IDEQ_IMG_CONVERGED;
          } else if (s.total[b] >= max_iter) {
            st = IDEQ_IMG_MAXITER;
          } else if (isfinite(B) && B > 0.f && (double)s.k[b] * s.S[b] > (double)B * B) {
            s.k[b] = 0;
            s.S[b] = 0.0;
            s.restarts[b] += 1;
            be = 0.f;
          }
          s.status[b] = st;
          s.skip[b] = st == IDEQ_IMG_RUNNING ? 0 : 1;  // frozen: later convs skip it
          s.beta_eff[b] = st == IDEQ_IMG_RUNNING ? be : 0.f;
          if (st == IDEQ_IMG_RUNNING) my_run += 1;
        }
      }
      s.fsum[b] = 0.0;
      s.gsum[b] = 0.0;
    }
  }
  if (lane == 0) run_cnt[wid] = my_run;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < nw; ++i) t += run_cnt[i];
    *s.n_running = t;
  }
}

cudaError_t launch_finalize(int n, int nblk, const SolverDev& s, int parity_new, float beta,
                            float B, double tol, int max_iter, float lam, int apply_logic,
                            int avg_K, cudaStream_t st) {
  const int warps = std::min(n, 32);
  finalize_kernel<<<1, 32 * warps, 0, st>>>(n, nblk, s, parity_new, beta, B, tol, max_iter, lam,
                                           apply_logic, avg_K);
  return cudaGetLastError();
}

__global__ void solver_init_kernel(int n, SolverDev s, float beta) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) {
    s.k[b] = 0;
    s.total[b] = 0;
    s.restarts[b] = 0;
    s.status[b] = IDEQ_IMG_RUNNING;
    s.parity[b] = 0;
    s.beta_eff[b] = beta;  // beta of the first extrapolation
    s.S[b] = 0.0;
    s.rel[b] = 0.0;
    s.fsum[b] = 0.0;
    s.gsum[b] = 0.0;
    s.energy[b] = 0.0;
    s.best[b] = INFINITY;
    s.k0[b] = -1;
    s.snap[b] = 0;
    s.skip[b] = 0;
  }
  if (b == 0) *s.n_running = n;
}

// Every image freezes by max_iter updates, so the loop ends by itself; the body
// counter is a guard against a loop that would not (it then stops with an error).
__global__ void loop_cond_kernel(cudaGraphConditionalHandle h, const int* n_running,
                                 int* counter, int first, int max_bodies, int* err) {
  const int c = first ? 0 : *counter + 1;
  *counter = c;
  const bool running = *n_running > 0;
  if (running && c >= max_bodies) atomicCAS(err, 0, 10);
  cudaGraphSetConditional(h, (running && c < max_bodies) ? 1u : 0u);
}

// Condition of the IF node inside the solve loop's body: the body's second
// iteration runs only while an image is running.
__global__ void if_cond_kernel(cudaGraphConditionalHandle h, const int* n_running) {
  cudaGraphSetConditional(h, *n_running > 0 ? 1u : 0u);
}

cudaError_t launch_if_cond(cudaGraphConditionalHandle h, const int* n_running, cudaStream_t st) {
  if_cond_kernel<<<1, 1, 0, st>>>(h, n_running);
  return cudaGetLastError();
}

cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, const int* n_running, int* counter,
                             int first, int max_bodies, int* err, cudaStream_t st) {
  loop_cond_kernel<<<1, 1, 0, st>>>(h, n_running, counter, first, max_bodies, err);
  return cudaGetLastError();
}

cudaError_t launch_solver_init(int n, const SolverDev& s, float beta, cudaStream_t st) {
  solver_init_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, s, beta);
  return cudaGetLastError();
}

__global__ void fill_info_kernel(int n, SolverDev s, ideq_info info) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  if (info.iters) info.iters[b] = s.total[b];
  if (info.restarts) info.restarts[b] = s.restarts[b];
  if (info.status) info.status[b] = s.status[b];
  if (info.rel_res) info.rel_res[b] = s.rel[b];
  if (info.energy) info.energy[b] = s.energy[b];
  if (info.k0) info.k0[b] = s.k0[b];
}

cudaError_t launch_fill_info(int n, const SolverDev& s, ideq_info info, cudaStream_t st) {
  fill_info_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, s, info);
  return cudaGetLastError();
}

__global__ void gather_parity_kernel(int per_img, long long total, const int* __restrict__ par,
                                     const float* __restrict__ b0, const float* __restrict__ b1,
                                     float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    out[i] = par[i / per_img] ? b1[i] : b0[i];
  }
}

cudaError_t launch_gather_parity(int n, int per_img, const int* parity, const float* b0,
                                 const float* b1, float* out, cudaStream_t st) {
  const long long total = (long long)n * per_img;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
  gather_parity_kernel<<<blocks, 256, 0, st>>>(per_img, total, parity, b0, b1, out);
  return cudaGetLastError();
}

// out = x * 2^(sign * e), an exact scaling: e = round(log2(rms)) from the mean
// square *ms (device) when ms is given (0 when ms is zero or not finite), else e_host.
__global__ void ldexp_kernel(long long n, const float* x, const float* ms, int e_host, int sign,
                             float* out) {
  int e = e_host;
  if (ms) {
    const float m = *ms;
    e = (m > 0.f && isfinite(m)) ? (int)rintf(0.5f * log2f(m)) : 0;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = ldexpf(x[i], sign * e);
}

cudaError_t launch_ldexp(long long n, const float* x, const float* ms, int e_host, int sign,
                         float* out, cudaStream_t st) {
  const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
  ldexp_kernel<<<blocks, 256, 0, st>>>(n, x, ms, e_host, sign, out);
  return cudaGetLastError();
}

__global__ void axpby_kernel(long long n, float a, const float* __restrict__ x, float b,
                             const float* __restrict__ y, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i] + (y ? b * y[i] : 0.f);
}

cudaError_t launch_axpby(long long n, float a, const float* x, float b, const float* y,
                         float* out, cudaStream_t st) {
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  axpby_kernel<<<std::max(blocks, 1), 256, 0, st>>>(n, a, x, b, y, out);
  return cudaGetLastError();
}

__global__ void zero_d_kernel(long long n, double* p) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

cudaError_t launch_zero_d(long long n, double* p, cudaStream_t st) {
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 4);
  zero_d_kernel<<<std::max(blocks, 1), 256, 0, st>>>(n, p);
  return cudaGetLastError();
}

// ===================================================================== weights
//
// GEMM B matrices [N][K] from PyTorch-layout weights (see ConvArgs):
//   conv3 fwd    B[co][t*Cin+ci]        = W[co][ci][t]
//   conv3 dgrad  B[ci][t*Cout+co]       = W[co][ci][8-t]        (flipped taps)
//   down fwd     B[co][q*Cin+ci]        = W[co][ci][q]           (q = di*2+dj)
//   down dgrad   B[q*Cin+ci][co]        = W[co][ci][q]           (pixelwise, D2S)
//   up fwd       B[q*Cout+co][ci]       = U[ci][co][q]           (pixelwise, D2S)
//   up dgrad     B[ci][q*Cout+co]       = U[ci][co][q]           (stride-2 gather)
// 3x3 forms may store padded channel counts pcin >= cin, pcout >= cout (zero
// weights on the padded rows and columns); -1 marks a padded entry.
__device__ __forceinline__ long long wform_src(int form, int cin, int cout, int pcin, int pcout,
                                               int nn, int kk) {
  switch (form) {
    case WF_CONV3_FWD: { const int t = kk / pcin, ci = kk % pcin;
      if (nn >= cout || ci >= cin) return -1;
      return ((long long)nn * cin + ci) * 9 + t; }
    case WF_CONV3_DGRAD: { const int t = kk / pcout, co = kk % pcout;
      if (nn >= cin || co >= cout) return -1;
      return ((long long)co * cin + nn) * 9 + (8 - t); }
    case WF_DOWN_FWD: { const int q = kk / cin, ci = kk % cin;
      return ((long long)nn * cin + ci) * 4 + q; }
    case WF_DOWN_DGRAD: { const int q = nn / cin, ci = nn % cin;
      return ((long long)kk * cin + ci) * 4 + q; }
    case WF_UP_FWD: { const int q = nn / cout, co = nn % cout;
      return ((long long)kk * cout + co) * 4 + q; }
    default: { const int q = kk / cout, co = kk % cout;  // WF_UP_DGRAD
      return ((long long)nn * cout + co) * 4 + q; }
  }
}

void weight_form_dims(int form, int cin, int cout, int* N, int* K) {
  weight_form_dims_padded(form, cin, cout, cin, cout, N, K);
}

void weight_form_dims_padded(int form, int cin, int cout, int pcin, int pcout, int* N, int* K) {
  if (form == WF_CONV3_FWD) {
    *N = pcout;
    *K = 9 * pcin;
    return;
  }
  if (form == WF_CONV3_DGRAD) {
    *N = pcin;
    *K = 9 * pcout;
    return;
  }
  switch (form) {
    case WF_CONV3_FWD: *N = cout; *K = 9 * cin; break;
    case WF_CONV3_DGRAD: *N = cin; *K = 9 * cout; break;
    case WF_DOWN_FWD: *N = cout; *K = 4 * cin; break;
    case WF_DOWN_DGRAD: *N = 4 * cin; *K = cout; break;
    case WF_UP_FWD: *N = 4 * cout; *K = cin; break;
    default: *N = cin; *K = 4 * cout; break;
  }
}

__global__ void wform_kernel(int form, int cin, int cout, int pcin, int pcout, int N, int K,
                             const float* __restrict__ src, float* __restrict__ d32,
                             __nv_bfloat16* __restrict__ d16, __half* __restrict__ dh) {
  const long long tot = (long long)N * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int nn = (int)(e / K), kk = (int)(e % K);
    const long long si = wform_src(form, cin, cout, pcin, pcout, nn, kk);
    const float v = si < 0 ? 0.f : src[si];
    if (d32) d32[e] = v;
    if (d16) d16[e] = __float2bfloat16_rn(v);
    if (dh) dh[e] = __float2half_rn(v);
  }
}

__global__ void wunform_kernel(int form, int cin, int cout, int pcin, int pcout, int N, int K,
                               const float* __restrict__ g, float scale, float* __restrict__ dst) {
  const long long tot = (long long)N * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int nn = (int)(e / K), kk = (int)(e % K);
    const long long di = wform_src(form, cin, cout, pcin, pcout, nn, kk);
    if (di >= 0) dst[di] += scale * g[e];
  }
}

cudaError_t launch_weight_form_padded(int form, int cin, int cout, int pcin, int pcout,
                                      const float* src, float* dst_f32, void* dst_bf16,
                                      void* dst_f16, cudaStream_t st) {
  int N, K;
  weight_form_dims_padded(form, cin, cout, pcin, pcout, &N, &K);
  const long long tot = (long long)N * K;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  wform_kernel<<<blocks, 256, 0, st>>>(form, cin, cout, pcin, pcout, N, K, src, dst_f32,
                                       (__nv_bfloat16*)dst_bf16, (__half*)dst_f16);
  return cudaGetLastError();
}

cudaError_t launch_weight_form(int form, int cin, int cout, const float* src, float* dst_f32,
                               void* dst_bf16, void* dst_f16, cudaStream_t st) {
  return launch_weight_form_padded(form, cin, cout, cin, cout, src, dst_f32, dst_bf16, dst_f16,
                                   st);
}

cudaError_t launch_weight_unform_padded(int form, int cin, int cout, int pcin, int pcout,
                                        const float* g, float scale, float* dst,
                                        cudaStream_t st) {
  int N, K;
  weight_form_dims_padded(form, cin, cout, pcin, pcout, &N, &K);
  const long long tot = (long long)N * K;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 4096);
  wunform_kernel<<<blocks, 256, 0, st>>>(form, cin, cout, pcin, pcout, N, K, g, scale, dst);
  return cudaGetLastError();
}

cudaError_t launch_weight_unform_scaled(int form, int cin, int cout, const float* g, float scale,
                                        float* dst, cudaStream_t st) {
  return launch_weight_unform_padded(form, cin, cout, cin, cout, g, scale, dst, st);
}

cudaError_t launch_weight_unform(int form, int cin, int cout, const float* g, float* dst,
                                 cudaStream_t st) {
  return launch_weight_unform_scaled(form, cin, cout, g, 1.f, dst, st);
}

// out = scale * sum_i a[i] b[i] over n elements: FP64 partials of 128 blocks,
// then one block sums them in a fixed order.
__global__ void dot_part_kernel(long long n, const float* __restrict__ a,
                                const float* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void dot_final_kernel(int nb, const double* __restrict__ part, float scale,
                                 float* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) *out = (float)((double)scale * t);
}

cudaError_t launch_dot(long long n, const float* a, const float* b, float scale, double* part,
                       float* out, cudaStream_t st) {
  dot_part_kernel<<<128, 256, 0, st>>>(n, a, b, part);
  dot_final_kernel<<<1, 128, 0, st>>>(128, part, scale, out);
  return cudaGetLastError();
}

// ===================================================================== warm start

// cot = 2 (x - t) / numel; partial sums of (x - t)^2 for the mean squared error.
__global__ void mse_grad_kernel(long long numel, const float* __restrict__ x,
                                const float* __restrict__ t, float* __restrict__ cot,
                                double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  const float sc = (float)(2.0 / (double)numel);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < numel;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = x[i] - t[i];
    cot[i] = sc * d;
    s += (double)d * d;
  }
  const double tt = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tt;
}

__global__ void mean_final_kernel(int nb, const double* __restrict__ part, double inv,
                                  double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0 && out) *out = t * inv;
}

cudaError_t launch_mse_grad(long long numel, const float* x, const float* t, float* cot,
                            double* part, double* loss, cudaStream_t st) {
  mse_grad_kernel<<<128, 256, 0, st>>>(numel, x, t, cot, part);
  mean_final_kernel<<<1, 128, 0, st>>>(128, part, 1.0 / (double)numel, loss);
  return cudaGetLastError();
}

// Adam (Kingma & Ba) with bias correction; the optimiser of the paper's training
// (App. D.1.3), PyTorch's default constants.
__global__ void adam_kernel(long long n, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

cudaError_t launch_adam(long long n, float* p, const float* g, float* m, float* v, int t, float lr,
                        float b1, float b2, float eps, cudaStream_t st) {
  const float c1 = (float)(1.0 - pow((double)b1, (double)t));
  const float c2 = (float)(1.0 - pow((double)b2, (double)t));
  const int blocks = (int)std::min<long long>((n + 255) / 256, 2048);
  adam_kernel<<<blocks, 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- im2col of the
// image-side 3x3 convs: one thread per pixel writes its 32-entry row (9 c taps,
// k = (3 dy + dx) c + ci, then zeros) as four 16-byte stores.
template <typename T> IDEQ_DEV T to16(float v);
template <> IDEQ_DEV __half to16<__half>(float v) { return __float2half_rn(v); }
template <> IDEQ_DEV __nv_bfloat16 to16<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T>
__global__ void __launch_bounds__(256) im2col3_kernel(int c, int H, int W,
                                                      const float* __restrict__ in,
                                                      const int* __restrict__ skip,
                                                      T* __restrict__ out) {
  const int b = blockIdx.y;
  if (skip && skip[b]) return;  // frozen image of a solve: not needed
  const int p = blockIdx.x * 256 + threadIdx.x;
  if (p >= H * W) return;
  const int y = p / W, x = p - y * W;
  const float* img = in + (size_t)b * c * H * W;
  __align__(16) T row[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) row[k] = to16<T>(0.f);
  for (int t = 0; t < 9; ++t) {
    const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
    const bool inside = yy >= 0 && yy < H && xx >= 0 && xx < W;
    for (int ci = 0; ci < c; ++ci) {
      const int k = t * c + ci;
      if (k < 32) row[k] = to16<T>(inside ? __ldg(img + ((size_t)ci * H + yy) * W + xx) : 0.f);
    }
  }
  uint4* o = (uint4*)(out + ((size_t)b * H * W + p) * 32);
  const uint4* r = (const uint4*)row;
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = r[q];
}

cudaError_t launch_im2col3(int n, int c, int H, int W, const float* in, const int* skip,
                           void* out, int out_dt, cudaStream_t st) {
  if (9 * c > 32 || (out_dt != DT_F16 && out_dt != DT_BF16)) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((H * W + 255) / 256), (unsigned)n);
  if (out_dt == DT_F16)
    im2col3_kernel<__half><<<grid, 256, 0, st>>>(c, H, W, in, skip, (__half*)out);
  else
    im2col3_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(c, H, W, in, skip, (__nv_bfloat16*)out);
  return cudaGetLastError();
}

__global__ void i2c_weights_kernel(const float* __restrict__ w32, int N, int K,
                                   __half* __restrict__ h, __nv_bfloat16* __restrict__ bw) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i >= N * 32) return;
  const int nn = i / 32, k = i - nn * 32;
  const float v = k < K ? w32[(size_t)nn * K + k] : 0.f;
  h[i] = __float2half_rn(v);
  bw[i] = __float2bfloat16_rn(v);
}

cudaError_t launch_i2c_weights(const float* w32, int N, int K, __half* h, __nv_bfloat16* b,
                               cudaStream_t st) {
  if (K > 32) return cudaErrorInvalidValue;
  i2c_weights_kernel<<<(N * 32 + 255) / 256, 256, 0, st>>>(w32, N, K, h, b);
  return cudaGetLastError();
}

}  // namespace ideq

// ===================================================================== FP8 forms

#include <cuda_fp8.h>

namespace ideq {

constexpr float kE4M3Max = 448.f;  // largest finite e4m3 value

IDEQ_DEV uint8_t to_e4m3(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// One block per output column n: s[n] = max_k |w[n][k]| / 448 and the row in e4m3
// (round to nearest even, saturating).  An all-zero row gets s = 1.
__global__ void __launch_bounds__(256) weight_fp8_kernel(const float* __restrict__ w, int K,
                                                         uint8_t* __restrict__ w8,
                                                         float* __restrict__ scale) {
  __shared__ float red[32];
  const int n = blockIdx.x;
  const float* row = w + (size_t)n * K;
  float m = 0.f;
  for (int k = threadIdx.x; k < K; k += 256) m = fmaxf(m, fabsf(row[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < 8 ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  const float s = red[0] > 0.f ? red[0] / kE4M3Max : 1.f;
  for (int k = threadIdx.x; k < K; k += 256) w8[(size_t)n * K + k] = to_e4m3(row[k] / s);
  if (threadIdx.x == 0) scale[n] = s;
}

cudaError_t launch_weight_fp8(const float* w32, int N, int K, uint8_t* w8, float* scale,
                              cudaStream_t st) {
  weight_fp8_kernel<<<N, 256, 0, st>>>(w32, K, w8, scale);
  return cudaGetLastError();
}

// 8 consecutive 16-bit values (one 16-byte load) as floats
template <typename T>
IDEQ_DEV void load8(const T* p, float (&v)[8]) {
  const uint4 u = *(const uint4*)p;
  const T* h = (const T*)&u;
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = ld_f(h + i);
}

// n is a multiple of 8 (the channel count of every quantised tensor is)
template <typename T>
__global__ void __launch_bounds__(256) act_amax_kernel(const T* __restrict__ x, long long n,
                                                       float* __restrict__ amax) {
  float m = 0.f;
  for (long long i = (blockIdx.x * 256LL + threadIdx.x) * 8; i < n;
       i += (long long)gridDim.x * 256 * 8) {
    float v[8];
    load8(x + i, v);
#pragma unroll
    for (int j = 0; j < 8; ++j) m = fmaxf(m, fabsf(v[j]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative floats order like their bit patterns read as ints
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax((int*)amax, __float_as_int(m));
}

template <typename T>
__global__ void __launch_bounds__(256) act_fp8_kernel(const T* __restrict__ x, long long n,
                                                      const float* __restrict__ amax,
                                                      uint8_t* __restrict__ x8,
                                                      float* __restrict__ scale) {
  const float a = *amax;
  const float s = a > 0.f ? a / kE4M3Max : 1.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale = s;
  for (long long i = (blockIdx.x * 256LL + threadIdx.x) * 8; i < n;
       i += (long long)gridDim.x * 256 * 8) {
    float v[8];
    load8(x + i, v);
    uint2 q;
    uint8_t* qb = (uint8_t*)&q;
#pragma unroll
    for (int j = 0; j < 8; ++j) qb[j] = to_e4m3(v[j] / s);
    *(uint2*)(x8 + i) = q;
  }
}

static int elem_blocks(long long n) {  // blocks of 256 threads, 8 values per thread
  return (int)std::max<long long>(1, std::min<long long>((n / 8 + 255) / 256, 152 * 8));
}

cudaError_t launch_act_amax(const void* x, int dt, long long n, float* amax, cudaStream_t st) {
  if (n % 8 != 0) return cudaErrorInvalidValue;
  if (dt == DT_BF16)
    act_amax_kernel<<<elem_blocks(n), 256, 0, st>>>((const __nv_bfloat16*)x, n, amax);
  else
    act_amax_kernel<<<elem_blocks(n), 256, 0, st>>>((const __half*)x, n, amax);
  return cudaGetLastError();
}

cudaError_t launch_act_fp8(const void* x, int dt, long long n, const float* amax, uint8_t* x8,
                           float* scale, cudaStream_t st) {
  if (n % 8 != 0) return cudaErrorInvalidValue;
  if (dt == DT_BF16)
    act_fp8_kernel<<<elem_blocks(n), 256, 0, st>>>((const __nv_bfloat16*)x, n, amax, x8, scale);
  else
    act_fp8_kernel<<<elem_blocks(n), 256, 0, st>>>((const __half*)x, n, amax, x8, scale);
  return cudaGetLastError();
}

}  // namespace ideq
