// Internal declarations of the i-DEQ CUDA library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ideq.h"

#ifdef __CUDACC__
#define IDEQ_HD __host__ __device__
#else
#define IDEQ_HD
#endif

namespace ideq {

// element storage of network activations
enum DType { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2, DT_FP8 = 3 };  // DT_FP8: e4m3 operands only

// ------------------------------------------------------------- conv GEMMs
//
// Every network layer is one implicit GEMM  D[M][N] = A[M][K] * B[N][K]^T
// with a fused epilogue.  M runs over the pixels of a "grid" (n, H, W):
//   CM_CONV3  3x3 conv, stride 1, zero padding: grid = output pixels,
//             K = 9 * Cin, k = tap * Cin + ci, tap = ky * 3 + kx.
//   CM_DOWN   2x2 stride-2 conv: grid = output pixels (input is 2H x 2W),
//             K = 4 * Cin, k = (di * 2 + dj) * Cin + ci.
//   CM_PIX    1x1 (pixelwise) product: grid = input pixels, K = Cin.
// Output maps: OM_IDENT writes out[m][n] (NHWC, C = N); OM_D2S scatters column
// n = (di * 2 + dj) * Cout + co to pixel (2y + di, 2x + dj) of a 2H x 2W image.
enum ConvMode { CM_CONV3 = 0, CM_DOWN = 1, CM_PIX = 2 };
enum OutMap { OM_IDENT = 0, OM_D2S = 1 };
enum Epi {
  EP_STORE = 0,    // out = acc
  EP_ACT = 1,      // out = act(acc), out2 = act'(acc)
  EP_ADD = 2,      // out = acc + aux0
  EP_MUL = 3,      // out = acc * aux0
  EP_MUL_KEEP = 4, // out = acc * aux0, out2 = acc
  EP_DUAL = 5,     // out = aux0 * acc + aux0 (1 - aux0) aux1 aux2   (softplus'' = s(1-s))
  EP_AXPY_NCHW = 6 // out (f32 NCHW) = aux0 (f32 NCHW) + sign * acc; optional sum(out^2)
};

struct ConvArgs {
  int mode = CM_CONV3, outmap = OM_IDENT, epi = EP_STORE, act = 0;
  int n = 0, H = 0, W = 0;     // GEMM grid
  int Cin = 0, Cout = 0;       // N = Cout (IDENT) or 4 * Cout (D2S)
  int in_nchw = 0;             // input is f32 planar NCHW
  int out_nchw = 0;            // output is f32 planar NCHW (EP_AXPY_NCHW)
  float sign = -1.f;           // EP_AXPY_NCHW
  const void* in = nullptr;
  const void* wB = nullptr;    // GEMM weights [N][K]
  void* out = nullptr;
  void* out2 = nullptr;
  const void* aux0 = nullptr;
  const void* aux1 = nullptr;
  const void* aux2 = nullptr;
  double* sumsq = nullptr;     // per-image accumulator of 1/2 sum(out^2), or null
  const float* a_scale = nullptr;  // FP8 operands: activation scale (device scalar)
  const float* w_scale = nullptr;  // FP8 operands: weight scale per output column [N]
  // per-image flags (device, n ints; nullable): nonzero = the image is frozen in a
  // solve and its outputs are not needed, so the launch may skip its work
  const int* skip = nullptr;
  // algorithmic K when the GEMM's K is padded (image-side 3x3 convs run as one
  // 32-wide K chunk of im2col taps: 9 c of them carry work), else 0
  int k_algo = 0;
  IDEQ_HD int N() const { return outmap == OM_D2S ? 4 * Cout : Cout; }
  IDEQ_HD int K() const { return mode == CM_CONV3 ? 9 * Cin : (mode == CM_DOWN ? 4 * Cin : Cin); }
  IDEQ_HD long long M() const { return (long long)n * H * W; }
  IDEQ_HD double flops() const { return 2.0 * (double)M() * N() * (k_algo > 0 ? k_algo : K()); }
};

// Element types of NHWC activations: DT_F32, DT_BF16 or DT_F16 (common.cuh);
// NCHW image-side tensors are always f32.  SIMT weights are always f32.
cudaError_t launch_conv_simt(const ConvArgs& a, int in_dt, int out_dt, cudaStream_t st);

// Image-side <-> feature-side 3x3 convs (head, tail, their transposes; see
// conv_edge.cu).  feat_dt is the element type of the NHWC side.
bool edge_supported(const ConvArgs& a);
cudaError_t launch_conv_edge(const ConvArgs& a, int feat_dt, cudaStream_t st);
// register-blocked forms of the common edge shapes (c in {1, 2, 3}, C in {32, 64})
bool edge_rb_supported(const ConvArgs& a);
cudaError_t launch_conv_edge_rb(const ConvArgs& a, int feat_dt, cudaStream_t st);

// tcgen05 path: 16-bit (bf16 or f16) or FP8 e4m3 NHWC input and weights, 16-bit
// NHWC output; Cin a multiple of 64 (16-bit) or 128 (FP8) channels, N % 64 == 0
// (see conv_tc.cu).  op_dt: operand type (DT_BF16, DT_F16, DT_FP8); epi_dt:
// type of the outputs and auxiliary inputs (DT_BF16 or DT_F16).
struct TcPlan;  // tensor maps + launch geometry, built once per (layer, buffers)
bool tc_supported(const ConvArgs& a, int op_dt = DT_F16);
TcPlan* tc_plan_create(const ConvArgs& a, int op_dt, int epi_dt, std::string* err);
void tc_plan_destroy(TcPlan* p);
cudaError_t launch_conv_tc(const TcPlan* p, const ConvArgs& a, int* err_flag, cudaStream_t st);

// Weight forms: GEMM B matrices from the PyTorch-layout weights.
enum WForm { WF_CONV3_FWD = 0, WF_CONV3_DGRAD, WF_DOWN_FWD, WF_DOWN_DGRAD, WF_UP_FWD, WF_UP_DGRAD };

// Image-side 3x3 convs on the tensor cores: im2col of the 9 c taps of an f32
// planar (NCHW) image into one 32-channel 16-bit NHWC row per pixel (k = tap c + ci,
// zero past 9 c and outside the image; frozen images skipped), and the GEMM weights
// [N][9 c] widened to [N][32] with zeros, in both 16-bit types.
cudaError_t launch_im2col3(int n, int c, int H, int W, const float* in, const int* skip,
                           void* out, int out_dt, cudaStream_t st);
cudaError_t launch_i2c_weights(const float* w32, int N, int K, __half* h, __nv_bfloat16* b,
                               cudaStream_t st);
cudaError_t launch_weight_form(int form, int cin, int cout, const float* src, float* dst_f32,
                               void* dst_bf16, void* dst_f16, cudaStream_t st);
void weight_form_dims(int form, int cin, int cout, int* N, int* K);  // the form's [N][K]
// 3x3 forms over padded channel counts (pcin >= cin, pcout >= cout; zero weights on
// the padded rows and columns); the other forms ignore the padding
void weight_form_dims_padded(int form, int cin, int cout, int pcin, int pcout, int* N, int* K);
cudaError_t launch_weight_form_padded(int form, int cin, int cout, int pcin, int pcout,
                                      const float* src, float* dst_f32, void* dst_bf16,
                                      void* dst_f16, cudaStream_t st);
// dst (PyTorch layout) += scale * g, g a padded GEMM-form gradient [N][K]
cudaError_t launch_weight_unform_padded(int form, int cin, int cout, int pcin, int pcout,
                                        const float* g, float scale, float* dst,
                                        cudaStream_t st);
// FP8 e4m3 weight form: w8[n][k] = e4m3(w32[n][k] / s[n]), s[n] = max_k |w32[n][k]| / 448.
cudaError_t launch_weight_fp8(const float* w32, int N, int K, uint8_t* w8, float* scale,
                              cudaStream_t st);
// FP8 e4m3 activation: *amax = max |x| over n 16-bit values (dt; *amax zeroed by the
// caller), then x8 = e4m3(x / s), *scale = s = *amax / 448 (1 when x == 0).
cudaError_t launch_act_amax(const void* x, int dt, long long n, float* amax, cudaStream_t st);
cudaError_t launch_act_fp8(const void* x, int dt, long long n, const float* amax, uint8_t* x8,
                           float* scale, cudaStream_t st);
// Scatter a GEMM-layout weight gradient [N][K] back to PyTorch layout (+=).
cudaError_t launch_weight_unform(int form, int cin, int cout, const float* g, float* dst,
                                 cudaStream_t st);

// ------------------------------------------------------------- data step
struct OpDev {
  int kind, kh, kw;
  const float* kernel;
  const uint8_t* mask;
  float gain;
  float sigma;  // Rician noise level
};
// Rician data term (App. E), A = identity: gf = x/s^2 - (y/s^2) I1/I0(x y/s^2),
// fsum += sum x^2/(2 s^2) - log I0(x y/s^2) per image (n images of per_img values).
cudaError_t launch_rician_grad(int n, int per_img, const float* x, const float* y, float sigma,
                               float* gf, double* fsum, cudaStream_t st);
// e = A(in) - y (y nullable): writes to `out` the vector fed to the adjoint
// pass (e for linear blur; J-weighted e for satblur; M.(M.in - y) directly
// for the mask, which needs no second pass) and accumulates 1/2||e||^2 per
// image into fsum (nullable).
cudaError_t launch_data_fwd(const OpDev& op, int n, int c, int H, int W, const float* in,
                            const float* y, float* out, double* fsum, cudaStream_t st);
// Adjoint pass: out = k^T (in) (blur kinds).
cudaError_t launch_blur_adj(const OpDev& op, int n, int c, int H, int W, const float* in,
                            float* out, cudaStream_t st);
// Ax = A(x) (forward model only).
cudaError_t launch_apply_A(const OpDev& op, int n, int c, int H, int W, const float* x,
                           float* Ax, cudaStream_t st);
// J_A(lin)^T r for satblur: tmp = (s/tanh s) sech^2(s k*lin) . r; out = k^T tmp.
cudaError_t launch_sat_jt_weight(const OpDev& op, int n, int c, int H, int W, const float* lin,
                                 const float* r, float* tmp, cudaStream_t st);

// MRI data term (fft.cu): n complex images of h x w as two f32 planes each.
bool fft_size_ok(int n);
cudaError_t launch_fft2(const float* in, float* out, int n, int H, int W, int inverse,
                        cudaStream_t st);
// gf = F^{-1}(M F z - y), fsum += 1/2 ||M F z - y||^2 per image; kbuf: image-size scratch
cudaError_t launch_mri_grad(int n, int H, int W, const float* z, const float* y,
                            const uint8_t* mask, float* kbuf, float* gf, double* fsum,
                            cudaStream_t st);
// out = M F x (adjoint = 0) or F^{-1}(M x) (adjoint = 1)
cudaError_t launch_mri_apply(int n, int H, int W, const float* x, const uint8_t* mask,
                             int adjoint, float* out, cudaStream_t st);
// out = F^{-1}((tau M y + F v) / (tau M + 1))
cudaError_t launch_mri_prox(int n, int H, int W, const float* v, const float* y,
                            const uint8_t* mask, float tau, float* out, cudaStream_t st);

// Spectral form of the circular blur data step (power-of-two h, w): khat (n
// complex planes) = F of each kernel on the torus; pk, yhat: n * ceil(c/2) complex
// images (channel pairs).  grad f = F^{-1}(conj(K)(K F z - yhat)), fsum as usual;
// yhat = null gives A^T A z.
cudaError_t launch_blur_spectrum(int n, int H, int W, int kh, int kw, const float* ker,
                                 float* khat, cudaStream_t st);
cudaError_t launch_pack_fft(int n, int c, int H, int W, const float* x, float* pk,
                            cudaStream_t st);
cudaError_t launch_blur_grad_spectral(int n, int c, int H, int W, const float* z,
                                      const float* khat, const float* yhat, float* pk, float* gf,
                                      double* fsum, cudaStream_t st);

// ------------------------------------------------------------- solver state
struct SolverDev {
  int* k;          // steps since last restart
  int* total;      // total updates
  int* restarts;
  int* status;     // IDEQ_IMG_*
  int* parity;     // buffer holding the latest iterate
  float* beta_eff; // beta for the next extrapolation (0 after restart / frozen)
  double* S;       // restart accumulator sum ||dx||^2
  double* rel;     // last relative step
  double* fsum;    // 1/2||A z - y||^2 of the current step
  double* gsum;    // 1/2||z - N(z)||^2 of the current step
  double* energy;
  double* part_s;  // [n][nblk] partial sums of ||x_new - x||^2
  double* part_x;  // [n][nblk] partial sums of ||x||^2
  int* skip;       // 1 once the image is frozen (its convolutions are skipped), else 0
  int* n_running;
  int* loop_count;  // bodies run by the device-driven solve loop
  // averaging step of Algorithm 1 (used when the solve asks for it)
  double* best;    // smallest step norm inside the averaging window so far
  int* k0;         // its index K0 (-1: none)
  int* snap;       // 1: the running sum after this update is the new snapshot
  double* zsum;    // [n][per] running sum of the extrapolated points z^k
  double* zsnap;   // [n][per] snapshot sum_{k <= K0} z^k
};

cudaError_t launch_extrapolate(int n, int per_img, const float* x, const float* xp,
                               const float* beta_eff, float* z, cudaStream_t st);
// extrapolation that also keeps the averaging step's running sum of z and its snapshot
cudaError_t launch_extrapolate_avg(int n, int per_img, const float* x, const float* xp,
                                   const SolverDev& s, float* z, cudaStream_t st);
// x_hat = snapshot / (K0 + 1) for the images the averaging step applies to
cudaError_t launch_average_out(int n, int per_img, const SolverDev& s, float* out,
                               cudaStream_t st);
// xn = z - tau (gf + lambda gg) (+ addv when non-null) for running images.
cudaError_t launch_red_update(int n, int per_img, int nblk, const float* z, const float* gf,
                              const float* gg, const float* x, float* xn, float lam, float tau,
                              const int* status, double* part_s, double* part_x,
                              cudaStream_t st, const float* addv = nullptr);
// Proximal step of i-DEQ-P for the inpainting mask: xn = (tau m y + v)/(tau m + 1),
// v = z - tau lambda gg, mask [n][hw] shared by the channels.
cudaError_t launch_prox_update(int n, int per_img, int hw, int nblk, const float* z,
                               const float* gg, const float* y, const uint8_t* mask,
                               const float* x, float* xn, float lam, float tau,
                               const int* status, double* part_s, double* part_x,
                               cudaStream_t st);
// xn = cand for running images, with the FP64 step-norm partials of (xn - x)
cudaError_t launch_commit_update(int n, int per_img, int nblk, const float* cand, const float* x,
                                 float* xn, const int* status, double* part_s, double* part_x,
                                 cudaStream_t st);
cudaError_t launch_finalize(int n, int nblk, const SolverDev& s, int parity_new, float beta,
                            float B, double tol, int max_iter, float lam, int apply_logic,
                            int avg_K, cudaStream_t st);
cudaError_t launch_gather_parity(int n, int per_img, const int* parity, const float* b0,
                                 const float* b1, float* out, cudaStream_t st);
cudaError_t launch_solver_init(int n, const SolverDev& s, float beta, cudaStream_t st);
// Device-driven solve loop: set a graph's while-condition to (*n_running > 0).
// `first` resets the body counter; a body past max_bodies stops the loop and
// raises *err (code 10) instead.
cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, const int* n_running, int* counter,
                             int first, int max_bodies, int* err, cudaStream_t st);
// IF-node condition inside the loop body: (*n_running > 0).
cudaError_t launch_if_cond(cudaGraphConditionalHandle h, const int* n_running, cudaStream_t st);
cudaError_t launch_fill_info(int n, const SolverDev& s, ideq_info info, cudaStream_t st);
int update_blocks_per_image(int per_img);

// small vector helpers
cudaError_t launch_axpby(long long n, float a, const float* x, float b, const float* y,
                         float* out, cudaStream_t st);
cudaError_t launch_zero_d(long long n, double* p, cudaStream_t st);
// out = x * 2^(sign e) (exact; may run in place): e = round(log2 sqrt(*ms)) from a
// device mean square ms (0 when ms is 0 or not finite), or e_host when ms is null
cudaError_t launch_ldexp(long long n, const float* x, const float* ms, int e_host, int sign,
                         float* out, cudaStream_t st);
// *out = scale * <a, b> (n floats), FP64 accumulation; part holds >= 128 doubles.
cudaError_t launch_dot(long long n, const float* a, const float* b, float scale, double* part,
                       float* out, cudaStream_t st);

}  // namespace ideq
