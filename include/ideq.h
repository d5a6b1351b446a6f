/*
 * ideq.h -- C ABI of the GB300 (sm_103a) i-DEQ restoration library.
 *
 * The library computes the inertial deep-equilibrium restoration of the paper
 * "i-DEQ: a stable inertial deep equilibrium model for image restoration":
 * given observations y = A(x) + n, a forward model A with adjoint, and the
 * parameters Theta = {theta, lambda, tau, alpha}, it returns the fixed point
 * x_hat of T = T^RED o T^M (Sec. 3.1, Eq. ideq; Algorithm 1), and for training
 * the gradient of a loss of x_hat with respect to theta and lambda by implicit
 * differentiation (App. D.1.2).
 *
 * Conventions shared by every entry point
 *   - Images are float32, planar NCHW, contiguous: x[((b*c + ch)*h + i)*w + j].
 *   - Every pointer argument is DEVICE memory owned by the caller unless the
 *     comment says "host".  The context owns only its scratch workspace.
 *   - Every call is asynchronous and ordered on the context's CUDA stream.
 *     Argument and shape errors are returned synchronously; per-image
 *     outcomes (converged / iteration cap / diverged) are written to the
 *     ideq_info arrays and are valid after the stream is synchronised.
 *   - No call aborts, exits or traps the device.  Device-side waits are
 *     bounded; an expired wait is reported as IDEQ_ERR_TIMEOUT.
 *   - A context is used by one host thread at a time.
 */
#ifndef IDEQ_H
#define IDEQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ideq_ctx ideq_ctx;

typedef enum {
  IDEQ_OK = 0,
  IDEQ_ERR_ARG = 1,          /* invalid argument or shape                         */
  IDEQ_ERR_CUDA = 2,         /* a CUDA runtime/driver call failed                  */
  IDEQ_ERR_NOMEM = 3,        /* workspace allocation failed                        */
  IDEQ_ERR_UNSUPPORTED = 4,  /* valid request the library does not implement       */
  IDEQ_MAXITER = 5,          /* ideq_solve: some image hit max_iter                 */
  IDEQ_DIVERGED = 6,         /* some image produced a non-finite step              */
  IDEQ_ADJ_MAXITER = 7,      /* ideq_solve_backward: adjoint solve hit its cap      */
  IDEQ_ERR_TIMEOUT = 8       /* a bounded device-side wait expired                 */
} ideq_status;

/* per-image outcome codes written to ideq_info.status */
enum { IDEQ_IMG_RUNNING = 0, IDEQ_IMG_CONVERGED = 1, IDEQ_IMG_MAXITER = 2, IDEQ_IMG_DIVERGED = 3 };

enum { IDEQ_NET_CNN = 0, IDEQ_NET_UNET = 1 };
enum { IDEQ_ACT_SOFTPLUS = 0, IDEQ_ACT_RELU = 1 };
enum { IDEQ_OP_BLUR = 0, IDEQ_OP_MASK = 1, IDEQ_OP_SATBLUR = 2, IDEQ_OP_MRI = 3,
       IDEQ_OP_RICIAN = 4 };
/* Arithmetic of the regulariser network's convolutions: operands in FP32
 * (SIMT), BF16 or FP16 (tensor cores, FP32 accumulation), activations stored in
 * the operand type.  The _FP8 forms run the tensor-core convolutions whose
 * input has >= 256 channels with FP8 e4m3 operands instead (per-output-channel
 * weight scales, a per-tensor activation scale taken from the input's max |x|
 * at every call, FP32 accumulation, 16-bit output); the implicit backward and
 * the warm start use the 16-bit form.  The iterate, the momentum state and the
 * data step are always float32, the step-norm and energy reductions float64. */
enum { IDEQ_FP32 = 0, IDEQ_BF16 = 1, IDEQ_BF16_FP8 = 2, IDEQ_FP16 = 3, IDEQ_FP16_FP8 = 4 };
enum { IDEQ_INIT_ATY = 0, IDEQ_INIT_X0 = 1, IDEQ_INIT_WARM = 2 };
enum { IDEQ_ADJ_JFB = 0, IDEQ_ADJ_IMPLICIT = 1 };

/* Regulariser network N in g(x) = 1/2 ||x - N(x)||^2 (Sec. 2.2, Eq. GS).
 *  IDEQ_NET_UNET: head 3x3 in_ch->widths[0]; per scale l < n_levels-1: n_rb
 *    residual blocks (3x3 conv, activation, 3x3 conv, identity skip), then a
 *    2x2 stride-2 conv widths[l]->widths[l+1]; n_rb blocks at the coarsest
 *    scale; per decoder scale (coarse to fine): 2x2 stride-2 transposed conv
 *    widths[l+1]->widths[l], plus the encoder output of scale l, n_rb blocks;
 *    tail 3x3 widths[0]->in_ch.  No biases, zero "same" padding.
 *  IDEQ_NET_CNN: depth 3x3 convs widths[0]->widths[1]->...->widths[depth],
 *    activation after every conv but the last; widths[0] = widths[depth] = in_ch.
 * Weight vector (float32): tensors in the order above (U-Net: head; per
 * encoder scale rb0.c1, rb0.c2, ..., down; coarsest rbs; per decoder scale up,
 * rbs; tail), each contiguous in PyTorch order: 3x3 and 2x2 convs
 * [C_out][C_in][kh][kw], transposed convs [C_in][C_out][2][2]. */
typedef struct {
  int kind;        /* IDEQ_NET_CNN or IDEQ_NET_UNET                         */
  int act;         /* IDEQ_ACT_SOFTPLUS or IDEQ_ACT_RELU                    */
  int in_ch;       /* image channels c (1 or 3)                             */
  int n_levels;    /* U-Net scales (>= 1, <= 6)                             */
  int n_rb;        /* U-Net residual blocks per scale                       */
  int depth;       /* CNN: number of conv layers (<= 15)                    */
  int widths[16];  /* U-Net: width per scale; CNN: channel list             */
} ideq_net_desc;

typedef struct { int n, c, h, w; } ideq_shape;  /* batch, channels, height, width */

/* Forward model A of one batch (App. E forms; the blur and saturation models
 * are synthetic stand-ins of the same structure):
 *  IDEQ_OP_BLUR    A x = k_b * x, circular convolution with per-image kernel
 *                  k_b (centre (kh/2, kw/2)), shared by the channels.
 *  IDEQ_OP_MASK    A x = M_b . x, per-pixel 0/1 mask shared by the channels.
 *  IDEQ_OP_SATBLUR A x = tanh(s (k_b * x)) / tanh(s), s = sat_gain.
 *  IDEQ_OP_MRI     A x = M_b . F x (App. E, MRI): x a complex image stored as
 *                  c = 2 planes (re, im), F the orthonormal 2-D DFT, M_b a 0/1
 *                  k-space mask (n*h*w, unshifted FFT layout); y is complex
 *                  k-space in the same 2-plane layout, zero off the mask.
 *                  h and w must be powers of two in [8, 1024].
 *  IDEQ_OP_RICIAN  denoising under Rician noise (App. E): y = |x + n_re + i n_im|,
 *                  f(x, y) = sum x^2/(2 s^2) - log I0(x y / s^2), s = sigma,
 *                  grad f = x/s^2 - (y/s^2) I1/I0(x y / s^2) (A = identity).  */
typedef struct {
  int kind;
  int kh, kw;              /* odd kernel sizes (<= 31) for blur kinds        */
  const float *kernel;     /* device, n*kh*kw, row-major per image            */
  const uint8_t *mask;     /* device, n*h*w, values 0/1 (mask kind)           */
  float sat_gain;          /* s for IDEQ_OP_SATBLUR                           */
  float sigma;             /* noise level of IDEQ_OP_RICIAN (> 0)             */
} ideq_operator;

/* Parameters of the inertial iteration (Algorithm 1; beta = 1 - alpha of
 * Eq. Momentum).  restart_B <= 0 or non-finite disables the restart test of
 * Eq. restart.  tol > 0 stops an image once ||x^{k+1}-x^k|| < tol ||x^k||
 * (App. D.1.3); tol = 0 runs exactly max_iter updates.  The output is the
 * last iterate (Remark 1), or, with average = 1, the averaging step of
 * Algorithm 1: x_hat = (1/(K0+1)) sum_{k=0}^{K0} z^k, where K0 is the first
 * minimiser of ||x^{k+1}-x^k|| over floor(K/2) < k < K-1 and K = max_iter.
 * Averaging needs a fixed run -- tol = 0, no restart, max_iter >= 5 -- and is
 * otherwise an argument error; ideq_step ignores it.  An image that diverged
 * returns its last iterate.  prox = 1 replaces the RED step by the proximal step
 * of i-DEQ-P (Algorithm 2, Eq. red_prox): x^{k+1} = prox_{tau f}(z - tau lambda
 * grad g(z)), in closed form for the inpainting mask (App. E:
 * (tau M y + v) / (tau M + 1) per pixel) and for MRI (the same in k-space,
 * F^{-1}((tau M y + F v) / (tau M + 1))); other operators return
 * IDEQ_ERR_UNSUPPORTED.  The restart keeps Algorithm 1's form. */
typedef struct {
  float lambda, tau, beta, restart_B;
  double tol;
  int max_iter;
  int init;               /* IDEQ_INIT_ATY, IDEQ_INIT_X0 (x0 given) or IDEQ_INIT_WARM */
  int average;            /* 0: last iterate; 1: averaging step (ideq_solve)         */
  int prox;               /* 0: RED step (Algorithm 1); 1: proximal step of i-DEQ-P  */
} ideq_params;

/* Per-image results, device arrays of length n; any member may be NULL. */
typedef struct {
  int *iters;       /* updates performed (restarts do not reset it)          */
  int *restarts;    /* number of restarts                                    */
  int *status;      /* IDEQ_IMG_*                                            */
  double *rel_res;  /* last ||x^{k+1}-x^k|| / ||x^k||                          */
  double *energy;   /* F(z) = f(z) + lambda g(z) at the last extrapolated point */
  int *k0;          /* K0 of the averaging step; -1 when no averaging was applied */
} ideq_info;

/* Adjoint (backward) solve parameters (App. D.1.2).  IDEQ_ADJ_JFB uses the
 * Jacobian-free estimate u = v; IDEQ_ADJ_IMPLICIT iterates u <- J_R^T u + v
 * (heavy-ball with beta) until ||u^{k+1}-u^k|| < tol ||u^k|| per image. */
typedef struct {
  int mode;
  double tol;
  int max_iter;
  float beta;
} ideq_adj_params;

/* ---- context ------------------------------------------------------------ */

/* Create a context on the current CUDA device.  `weights` (device, float32)
 * is copied; `precision` selects the convolution arithmetic; `stream` is a
 * cudaStream_t (NULL = legacy default stream). */
ideq_status ideq_create(ideq_ctx **ctx, const ideq_net_desc *net, const float *weights,
                        int precision, void *stream);
ideq_status ideq_destroy(ideq_ctx *ctx);
/* Replace the network weights (device float32, same layout); async. */
ideq_status ideq_set_weights(ideq_ctx *ctx, const float *weights);
ideq_status ideq_set_precision(ideq_ctx *ctx, int precision);
ideq_status ideq_set_stream(ideq_ctx *ctx, void *stream);
/* Number of float32 entries of the network weight vector. */
ideq_status ideq_num_params(const ideq_net_desc *net, int64_t *count);
/* Last error message of the context (host string, valid until the next call). */
const char *ideq_last_error(ideq_ctx *ctx);

/* ---- forward model (Sec. 1 Eq. inv_prob; App. E) ------------------------- */

/* Ax = A(x). */
ideq_status ideq_apply_A(ideq_ctx *ctx, const ideq_operator *op, ideq_shape shape,
                         const float *x, float *Ax);
/* out = A^T r for linear A; out = J_A(lin_point)^T r when lin_point != NULL
 * (required for the saturation model's Jacobian; A^T of its linear part
 * k^T (.) when NULL). */
ideq_status ideq_apply_AT(ideq_ctx *ctx, const ideq_operator *op, ideq_shape shape,
                          const float *r, const float *lin_point, float *out);

/* ---- regulariser (Eq. GS) ------------------------------------------------ */

/* grad = grad g(z) = r - J_N(z)^T r with r = z - N(z); g_val (device, n
 * doubles, nullable) receives g(z) = 1/2 ||r||^2 per image. */
ideq_status ideq_grad_reg(ideq_ctx *ctx, ideq_shape shape, const float *z, float *grad,
                          double *g_val);

/* ---- iteration (Algorithm 1) --------------------------------------------- */

/* One inertial RED update of every image, in place:
 *   z = x_k + beta (x_k - x_km1),  x_{k+1} = z - tau (grad f(z, y) + lambda grad g(z)),
 * then x_km1 <- x_k and x_k <- x_{k+1}.  info.rel_res and info.energy are
 * filled; no restart or stopping logic is applied. */
ideq_status ideq_step(ideq_ctx *ctx, const ideq_operator *op, ideq_shape shape,
                      const float *y, float *x_k, float *x_km1, const ideq_params *p,
                      ideq_info *info);

/* Full solve from x0 = A^T y (IDEQ_INIT_ATY), the given x0 (IDEQ_INIT_X0) or
 * the warm start (IDEQ_INIT_WARM) with restart, per-image stopping and
 * freezing.  Returns IDEQ_MAXITER / IDEQ_DIVERGED if any image ended so
 * (this return synchronises the stream). */
ideq_status ideq_solve(ideq_ctx *ctx, const ideq_operator *op, ideq_shape shape,
                       const float *y, const float *x0, float *x_out, const ideq_params *p,
                       ideq_info *info);

/* ---- implicit backward (App. D.1.2) -------------------------------------- */

/* Given the fixed point x_bar and v = dl/dx_bar, computes
 *   dl_dtheta (device, ideq_num_params floats) = -tau lambda (d grad g(x_bar)/d theta)^T u
 *   dl_dlambda (device, 1 float)              = -tau <u, grad g(x_bar)>
 * summed over the batch, with u from the adjoint solve (or u = v for JFB).
 * info.iters receives the adjoint iterations per image.  Linear operators
 * (blur, mask) only. */
ideq_status ideq_solve_backward(ideq_ctx *ctx, const ideq_operator *op, ideq_shape shape,
                                const float *y, const float *x_bar, const float *dl_dx,
                                const ideq_params *p, const ideq_adj_params *ap,
                                float *dl_dtheta, float *dl_dlambda, ideq_info *info);

/* One training step of the regulariser on a batch with ground truth x_true
 * (App. D.1.2-D.1.3): x_out = x_hat from ideq_solve (x0 = A^T y), the loss
 * l = mean((x_hat - x_true)^2) (device double *loss, nullable), the implicit
 * backward of ideq_solve_backward with `ap`, and one Adam step (beta1 0.9, beta2
 * 0.999, eps 1e-8, learning rate lr; Adam state kept in the context) on theta,
 * after which the context's weights are the updated ones.  dl_dtheta (device,
 * ideq_num_params floats) and dl_dlambda (device, 1 float) receive the gradient
 * of this step (nullable); lambda itself is a parameter of the call and is not
 * updated.  A forward solve that returns IDEQ_MAXITER / IDEQ_DIVERGED, or an
 * adjoint solve that returns IDEQ_ADJ_MAXITER, ends the step with that status
 * before theta changes.  info (nullable) receives the forward solve's results.
 * Linear operators only (as ideq_solve_backward). */
ideq_status ideq_train_step(ideq_ctx *ctx, const ideq_operator *op, ideq_shape shape,
                            const float *y, const float *x_true, const ideq_params *p,
                            const ideq_adj_params *ap, float lr, float *x_out,
                            float *dl_dtheta, float *dl_dlambda, double *loss, ideq_info *info);

/* ---- learned warm start x0 = A^T y + W(A^T y) ----------------------------- */
/* Not in the paper, which leaves x^0 free (Algorithm 1).  W is an
 * IDEQ_NET_CNN network with its own weights and Adam state in the context. */

ideq_status ideq_warm_set(ideq_ctx *ctx, const ideq_net_desc *net, const float *weights);
/* x0 = aty + W(aty). */
ideq_status ideq_warm_forward(ideq_ctx *ctx, ideq_shape shape, const float *aty, float *x0);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error
 * of x0 against target; loss (device, 1 double, nullable) receives the loss
 * before the step. */
ideq_status ideq_warm_train_step(ideq_ctx *ctx, ideq_shape shape, const float *aty,
                                 const float *target, float lr, double *loss);
/* Copy the warm-start weights (device float32). */
ideq_status ideq_warm_get(ideq_ctx *ctx, float *weights);

/* ---- allocation-free RED update ------------------------------------------- */

/* The paper has no counterpart of this call: it exists for callers that cannot
 * allocate device memory -- code embedded in a framework that owns every device
 * allocation, processes with a fixed memory budget, servers that must not
 * allocate while serving.  It performs the RED update of Algorithm 1 on caller
 * buffers, without a context:
 *   x_new = z - tau (grad_f + lambda grad_g)
 *   step_sq[b] = ||x_new_b - x_b||^2,  x_sq[b] = ||x_b||^2   (per image)
 * The squares are summed in FP32 over at most 16 elements and every sum above
 * that in FP64, so the two norms carry a relative error below 16 FP32 ulps
 * (about 1e-6) -- far below any stopping tolerance they are compared with.
 * n images of per_img floats each, contiguous (NCHW), device pointers; step_sq
 * and x_sq are device arrays of n doubles (nullable).  It calls no cudaMalloc or
 * cudaFree: its per-block partial sums live in one static device array of 65536
 * doubles (512 KiB) that every GPU loading the library keeps until the process
 * exits.  It needs 2 * n * min(64, ceil(per_img / 8192)) of them; larger requests
 * (for instance more than 1024 images of 256K floats or more) return
 * IDEQ_ERR_ARG.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current, so make it before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (different streams, no ordering) race; calls on
 * one stream are safe.  Nothing in the array needs clearing between calls.
 * The looked-up address is kept for the life of the process, so a device reset
 * (cudaDeviceReset, or a reset of the primary context) is not supported once the
 * call has been made on that device.  Pointers need only 4-byte alignment; the
 * vectorised path is taken when all five image pointers are 16-byte aligned. */
ideq_status ideq_red_update_noalloc(int n, int per_img, const float *z, const float *grad_f,
                                    const float *grad_g, const float *x, float *x_new,
                                    float lambda, float tau, double *step_sq, double *x_sq,
                                    void *stream);

/* ---- instrumentation ------------------------------------------------------ */

/* When enabled, CUDA events bracket every launch of the tensor-core
 * convolution kernel on the context's stream; ideq_prof_read returns their
 * summed duration (ms), the launch count and the summed algorithmic FLOPs
 * since the last read, and resets them (synchronises the stream). */
ideq_status ideq_prof_enable(ideq_ctx *ctx, int on);
ideq_status ideq_prof_read(ideq_ctx *ctx, double *ms, int64_t *launches, double *flops);
/* Times `reps` back-to-back repetitions of the tensor-core convolution launches
 * of one regulariser evaluation (forward list, then the input-gradient list) on
 * the current plan's buffers, launched exactly as in a solve (programmatic
 * dependent launch kept), with one pair of CUDA events on the context's stream
 * around all of them.  *ms is the elapsed time (host double), *launches and
 * *flops (nullable) the launch count and the summed algorithmic FLOPs (2 M N K
 * per launch).  The plan's buffers hold whatever the last call left; the
 * results written there are meaningless afterwards.  Synchronises the stream.
 * Needs a plan (after a solve, step or ideq_grad_reg), else IDEQ_ERR_ARG. */
ideq_status ideq_time_convs(ideq_ctx *ctx, int reps, double *ms, int64_t *launches,
                            double *flops);
/* Times `reps` repetitions of the weight-gradient pass of the last implicit
 * backward (both products of every conv, the same kernels as in
 * ideq_solve_backward) with one pair of CUDA events on the context's stream.
 * *ms: elapsed time; *flops (nullable): the algorithmic FLOPs of the timed
 * passes (2 x 2 M N K per conv and pass); *tc_convs (nullable): how many convs
 * run on the tensor cores (the others on the SIMT kernel).  Needs a training
 * plan (after ideq_solve_backward), else IDEQ_ERR_ARG.  Synchronises the stream. */
ideq_status ideq_time_wgrad(ideq_ctx *ctx, int reps, double *ms, double *flops,
                            int64_t *tc_convs);
/* Algorithmic FLOPs of every convolution (all kinds, all n images) of one
 * iteration of the current plan: forward pass plus input-gradient pass. */
ideq_status ideq_plan_flops(ideq_ctx *ctx, double *per_iteration);
/* Measured FP32 FFMA throughput of this GPU (host double, TFLOP/s counting 2
 * FLOPs per FMA): a kernel of independent FMA chains on every SM, timed with
 * CUDA events on `stream` (synchronises it); the roofline of the plain FP32 form. */
ideq_status ideq_fp32_fma_peak(void *stream, double *tflops);
/* Number of kernels this context launched since the last call (host count). */
ideq_status ideq_launch_count(ideq_ctx *ctx, int64_t *count);
/* Whether the last ideq_solve on this context ran its iterations after the first
 * two in the device-driven CUDA graph (*graphed = 1) or from the host (0: graphs
 * off, profiler recording, max_iter <= 2, or the runtime refused to build one). */
ideq_status ideq_solve_graphed(ideq_ctx *ctx, int *graphed);

#ifdef __cplusplus
}
#endif
#endif /* IDEQ_H */
