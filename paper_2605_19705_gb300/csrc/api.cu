// C ABI of the i-DEQ library: context, forward model, regulariser gradient,
// single step and full inertial solve (Algorithm 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>

#include "net.h"
#include "net_train.h"

using namespace ideq;

struct ideq_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = IDEQ_FP32;
  std::unique_ptr<NetWeights> w;
  std::unique_ptr<NetPlan> plan;
  std::unique_ptr<TrainPlan> train;
  // learned warm start: weights, its plan for the current shape, Adam state
  std::unique_ptr<NetWeights> warm_w;
  std::unique_ptr<TrainPlan> warm_plan;
  float* warm_m = nullptr;
  float* warm_v = nullptr;
  float* warm_g = nullptr;
  int warm_t = 0;
  // training of the regulariser (ideq_train_step): Adam state of theta, the
  // parameter gradient, the loss cotangent dl/dx_hat and the loss
  float* reg_m = nullptr;
  float* reg_v = nullptr;
  float* reg_g = nullptr;
  float* reg_cot = nullptr;
  size_t reg_cot_bytes = 0;
  double* reg_loss = nullptr;
  float* reg_dlam = nullptr;
  int reg_t = 0;
  // implicit backward: dl/dx_hat scaled by a power of two to unit RMS (so that the
  // 16-bit tangent passes of the adjoint iteration stay in their normal range) and
  // its mean square; the results are scaled back exactly
  float* adj_v = nullptr;
  size_t adj_v_bytes = 0;
  float* adj_ms = nullptr;
  std::string err;
  int* d_err = nullptr;       // device error flag of bounded waits
  int* h_running = nullptr;   // pinned
  Profiler prof;
  long long launches = 0;
  // solver workspace (sized for the current plan)
  int sv_n = 0, sv_per = 0, sv_nblk = 0;
  void* sv_mem = nullptr;
  SolverDev sv{};
  float* xb[2] = {nullptr, nullptr};
  float* gf = nullptr;
  float* tmp = nullptr;
  float* ubuf = nullptr;      // adjoint solution u
  // spectral blur data step (power-of-two images): kernel and observation spectra,
  // packed scratch; `spectral` is set per call by prepare_data_step
  float* khat = nullptr;
  float* yhat = nullptr;
  float* pk = nullptr;
  bool spectral = false;
  double* dot_part = nullptr;
  double* fsum = nullptr;
  double* gsum = nullptr;
  // scratch for the stand-alone operator calls
  float* scratch = nullptr;
  size_t scratch_bytes = 0;
  // Device-driven solve loop: one CUDA graph whose while node repeats a body of
  // two iterations (the second inside an IF node, so the condition is checked
  // after every iteration) for as long as an image is running, so the solve
  // needs no host round trip per iteration.  Rebuilt when the plan, the
  // operator, y or the parameters change; a graph that cannot be built falls back
  // to the host-driven loop.
  struct SolveGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* plan = nullptr;
    OpDev od{};
    const float* y = nullptr;
    ideq_params p{};
    long long body_launches = 0;
  } sg;
  bool graph_ok = true;  // false once building a graph failed in this context
  // private non-blocking stream the solve graph is captured on (the caller's
  // stream may be the legacy default stream, which cannot be captured)
  cudaStream_t cap_stream = nullptr;
  bool last_graphed = false;  // the last solve ran its loop in the device graph
  void drop_graph() {
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    if (sg.g) cudaGraphDestroy(sg.g);
    sg = SolveGraph{};
  }
};

namespace {

// A failed runtime call leaves its (non-sticky) error as the thread's "last
// error"; launchers report cudaGetLastError(), so every entry point clears what
// an earlier, unrelated call may have left behind.
void clear_stale_cuda_error() { (void)cudaGetLastError(); }

ideq_status fail(ideq_ctx* c, ideq_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

ideq_status cuda_fail(ideq_ctx* c, cudaError_t e, const char* where) {
  return fail(c, IDEQ_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

bool shape_ok(const ideq_shape& s) {
  return s.n > 0 && s.c > 0 && s.h > 0 && s.w > 0 && (long long)s.n * s.c * s.h * s.w < (1LL << 40);
}

ideq_status check_op(ideq_ctx* ctx, const ideq_operator* op, const ideq_shape& s, OpDev* od) {
  if (!op) return fail(ctx, IDEQ_ERR_ARG, "operator is NULL");
  od->kind = op->kind;
  od->kh = op->kh;
  od->kw = op->kw;
  od->kernel = op->kernel;
  od->mask = op->mask;
  od->gain = op->sat_gain;
  od->sigma = op->sigma;
  if (op->kind == IDEQ_OP_BLUR || op->kind == IDEQ_OP_SATBLUR) {
    if (!op->kernel) return fail(ctx, IDEQ_ERR_ARG, "blur operator needs a kernel");
    if (op->kh < 1 || op->kw < 1 || op->kh > 31 || op->kw > 31 || !(op->kh & 1) || !(op->kw & 1))
      return fail(ctx, IDEQ_ERR_ARG, "kernel sizes must be odd and <= 31");
    if (op->kh > s.h || op->kw > s.w) return fail(ctx, IDEQ_ERR_ARG, "kernel larger than image");
    if (op->kind == IDEQ_OP_SATBLUR && !(op->sat_gain > 0.f))
      return fail(ctx, IDEQ_ERR_ARG, "sat_gain must be > 0");
  } else if (op->kind == IDEQ_OP_MASK) {
    if (!op->mask) return fail(ctx, IDEQ_ERR_ARG, "mask operator needs a mask");
  } else if (op->kind == IDEQ_OP_RICIAN) {
    if (!(op->sigma > 0.f)) return fail(ctx, IDEQ_ERR_ARG, "Rician operator needs sigma > 0");
  } else if (op->kind == IDEQ_OP_MRI) {
    if (!op->mask) return fail(ctx, IDEQ_ERR_ARG, "MRI operator needs a k-space mask");
    if (s.c != 2) return fail(ctx, IDEQ_ERR_ARG, "MRI images are complex: c = 2 (re, im)");
    if (!fft_size_ok(s.h) || !fft_size_ok(s.w))
      return fail(ctx, IDEQ_ERR_UNSUPPORTED, "MRI needs h, w powers of two in [8, 1024]");
  } else {
    return fail(ctx, IDEQ_ERR_ARG, "unknown operator kind");
  }
  return IDEQ_OK;
}

// IDEQ_SKIP_FROZEN=0 computes frozen images too (for comparisons).
bool skip_frozen_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("IDEQ_SKIP_FROZEN");
    return !(v && v[0] == '0');
  }();
  return on;
}

ideq_status ensure_plan(ideq_ctx* ctx, const ideq_shape& s) {
  if (s.c != ctx->w->desc.in_ch) return fail(ctx, IDEQ_ERR_ARG, "channels differ from the network's in_ch");
  NetPlan* p = ctx->plan.get();
  if (p && p->n == s.n && p->H == s.h && p->W == s.w && p->prec == ctx->precision) return IDEQ_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->drop_graph();
  ctx->plan.reset();
  ctx->train.reset();
  ctx->warm_plan.reset();
  // solver workspace
  if (ctx->sv_mem) {
    cudaFree(ctx->sv_mem);
    ctx->sv_mem = nullptr;
  }
  const int n = s.n, per = s.c * s.h * s.w;
  const int nblk = update_blocks_per_image(per);
  const size_t img = (size_t)n * per * 4;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += (b + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_x0 = take(img), o_x1 = take(img), o_gf = take(img), o_tmp = take(img);
  const size_t o_i = take((size_t)n * 4 * 8), o_f = take((size_t)n * 4), o_d = take((size_t)n * 8 * 6);
  const size_t o_zs = take(2 * img), o_zn = take(2 * img);  // FP64 sums of the averaging step
  const bool pow2 = fft_size_ok(s.h) && fft_size_ok(s.w);
  const size_t pk_bytes = (size_t)n * ((s.c + 1) / 2) * 2 * s.h * s.w * 4;
  const size_t o_kh = pow2 ? take((size_t)n * 2 * s.h * s.w * 4) : 0;
  const size_t o_yh = pow2 ? take(pk_bytes) : 0, o_pk = pow2 ? take(pk_bytes) : 0;
  const size_t o_p = take((size_t)n * nblk * 8 * 2), o_r = take(16), o_dp = take(128 * 8);
  const size_t o_u = take(img);
  char* m = nullptr;
  if (cudaMalloc((void**)&m, off) != cudaSuccess) return fail(ctx, IDEQ_ERR_NOMEM, "cudaMalloc(solver workspace)");
  ctx->sv_mem = m;
  ctx->xb[0] = (float*)(m + o_x0);
  ctx->xb[1] = (float*)(m + o_x1);
  ctx->gf = (float*)(m + o_gf);
  ctx->tmp = (float*)(m + o_tmp);
  int* ip = (int*)(m + o_i);
  SolverDev& v = ctx->sv;
  v.k = ip;
  v.total = ip + n;
  v.restarts = ip + 2 * n;
  v.status = ip + 3 * n;
  v.parity = ip + 4 * n;
  v.beta_eff = (float*)(m + o_f);
  double* dp = (double*)(m + o_d);
  v.S = dp;
  v.rel = dp + n;
  v.fsum = dp + 2 * n;
  v.gsum = dp + 3 * n;
  v.energy = dp + 4 * n;
  v.best = dp + 5 * n;
  v.k0 = ip + 5 * n;
  v.snap = ip + 6 * n;
  v.skip = ip + 7 * n;
  v.zsum = (double*)(m + o_zs);
  v.zsnap = (double*)(m + o_zn);
  v.part_s = (double*)(m + o_p);
  v.part_x = v.part_s + (size_t)n * nblk;
  v.n_running = (int*)(m + o_r);
  v.loop_count = v.n_running + 1;
  ctx->dot_part = (double*)(m + o_dp);
  ctx->khat = pow2 ? (float*)(m + o_kh) : nullptr;
  ctx->yhat = pow2 ? (float*)(m + o_yh) : nullptr;
  ctx->pk = pow2 ? (float*)(m + o_pk) : nullptr;
  ctx->ubuf = (float*)(m + o_u);
  ctx->fsum = v.fsum;
  ctx->gsum = v.gsum;
  ctx->sv_n = n;
  ctx->sv_per = per;
  ctx->sv_nblk = nblk;
  CK(cudaMemsetAsync(m, 0, off, ctx->stream));
  std::unique_ptr<NetPlan> np(new NetPlan());
  std::string e;
  if (!np->build(ctx->w.get(), s.n, s.h, s.w, ctx->precision, v.gsum, &e,
                 skip_frozen_enabled() ? v.skip : nullptr))
    return fail(ctx, IDEQ_ERR_UNSUPPORTED, "plan: " + e);
  ctx->plan = std::move(np);
  return IDEQ_OK;
}

float* ensure_scratch(ideq_ctx* ctx, size_t bytes) {
  if (ctx->scratch_bytes >= bytes) return ctx->scratch;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->scratch) cudaFree(ctx->scratch);
  ctx->scratch = nullptr;
  ctx->scratch_bytes = 0;
  if (cudaMalloc((void**)&ctx->scratch, bytes) != cudaSuccess) return nullptr;
  ctx->scratch_bytes = bytes;
  return ctx->scratch;
}

// IDEQ_SPECTRAL=0 keeps the blur data step on the direct stencils (for comparisons).
bool spectral_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("IDEQ_SPECTRAL");
    return !(v && v[0] == '0');
  }();
  return on;
}

// Before a solve / step / backward: choose the blur's data-step form and, for the
// spectral form, compute the kernel spectra and (when y is given) the spectrum of y.
// The spectral form serves the large kernels (>= 15 x 15 taps, where the stencil's
// kh * kw FMAs per pixel dominate); small kernels keep the exact stencil, whose f is
// not subject to the FFT's cancellation near the fixed point.
cudaError_t prepare_data_step(ideq_ctx* ctx, const OpDev& od, const ideq_shape& s,
                              const float* y) {
  ctx->spectral = od.kind == IDEQ_OP_BLUR && ctx->khat && od.kh * od.kw >= 225 &&
                  spectral_enabled();
  if (!ctx->spectral) return cudaSuccess;
  cudaError_t e = launch_blur_spectrum(s.n, s.h, s.w, od.kh, od.kw, od.kernel, ctx->khat,
                                       ctx->stream);
  if (e == cudaSuccess && y) e = launch_pack_fft(s.n, s.c, s.h, s.w, y, ctx->yhat, ctx->stream);
  ctx->launches += 6;
  return e;
}

// grad f(z) = J_A(z)^T (A(z) - y) into gf, 1/2||A z - y||^2 into fsum.
cudaError_t data_grad(ideq_ctx* ctx, const OpDev& od, const ideq_shape& s, const float* z,
                      const float* y, float* gf, float* tmp, double* fsum) {
  cudaStream_t st = ctx->stream;
  if (ctx->spectral && od.kind == IDEQ_OP_BLUR) {  // y here is the y prepare_data_step saw
    ctx->launches += 7;
    return launch_blur_grad_spectral(s.n, s.c, s.h, s.w, z, ctx->khat, y ? ctx->yhat : nullptr,
                                     ctx->pk, gf, fsum, st);
  }
  if (od.kind == IDEQ_OP_MASK) {
    ctx->launches += 1;
    return launch_data_fwd(od, s.n, s.c, s.h, s.w, z, y, gf, fsum, st);
  }
  if (od.kind == IDEQ_OP_MRI) {
    ctx->launches += 5;
    return launch_mri_grad(s.n, s.h, s.w, z, y, od.mask, tmp, gf, fsum, st);
  }
  if (od.kind == IDEQ_OP_RICIAN) {
    ctx->launches += 1;
    return launch_rician_grad(s.n, s.c * s.h * s.w, z, y, od.sigma, gf, fsum, st);
  }
  cudaError_t e = launch_data_fwd(od, s.n, s.c, s.h, s.w, z, y, tmp, fsum, st);
  if (e != cudaSuccess) return e;
  ctx->launches += 2;
  return launch_blur_adj(od, s.n, s.c, s.h, s.w, tmp, gf, st);
}

// A^T y (adjoint of the linear part; the initial point x0 = A^T y).
cudaError_t back_project(ideq_ctx* ctx, const OpDev& od, const ideq_shape& s, const float* y,
                         float* out) {
  ctx->launches += 1;
  if (od.kind == IDEQ_OP_MASK) return launch_apply_A(od, s.n, s.c, s.h, s.w, y, out, ctx->stream);
  if (od.kind == IDEQ_OP_MRI) {
    ctx->launches += 2;
    return launch_mri_apply(s.n, s.h, s.w, y, od.mask, 1, out, ctx->stream);
  }
  if (od.kind == IDEQ_OP_RICIAN)  // A = identity: x0 = y
    return cudaMemcpyAsync(out, y, (size_t)s.n * s.c * s.h * s.w * 4, cudaMemcpyDeviceToDevice,
                           ctx->stream);
  return launch_blur_adj(od, s.n, s.c, s.h, s.w, y, out, ctx->stream);
}

// One iteration of Algorithm 1 on the plan buffers: x in xb[p], x_prev in
// xb[1-p]; the update is written into xb[1-p].
ideq_status iterate(ideq_ctx* ctx, const OpDev& od, const ideq_shape& s, const float* y,
                    const ideq_params* p, int par, int logic, bool average = false) {
  NetPlan* P = ctx->plan.get();
  cudaStream_t st = ctx->stream;
  const int n = s.n, per = ctx->sv_per;
  float* x = ctx->xb[par];
  float* xp = ctx->xb[1 - par];
  const int avg_K = (logic && average) ? p->max_iter : 0;
  if (avg_K > 0)
    CK(launch_extrapolate_avg(n, per, x, xp, ctx->sv, P->z, st));
  else
    CK(launch_extrapolate(n, per, x, xp, ctx->sv.beta_eff, P->z, st));
  CK(run_steps(P->fwd, ctx->d_err, st, &ctx->prof, &ctx->launches));
  CK(run_steps(P->vjp, ctx->d_err, st, &ctx->prof, &ctx->launches));
  CK(data_grad(ctx, od, s, P->z, y, ctx->gf, ctx->tmp, ctx->sv.fsum));  // also f(z)
  if (p->prox && od.kind == IDEQ_OP_MRI) {
    // v = z - tau lambda grad g into gf (the data gradient is not used by the
    // proximal step), its prox into tmp, accepted for the running images
    CK(launch_axpby((long long)n * per, 1.f, P->z, -p->tau * p->lambda, P->grad, ctx->gf, st));
    CK(launch_mri_prox(n, s.h, s.w, ctx->gf, y, od.mask, p->tau, ctx->tmp, st));
    CK(launch_commit_update(n, per, ctx->sv_nblk, ctx->tmp, x, xp, ctx->sv.status,
                            ctx->sv.part_s, ctx->sv.part_x, st));
    ctx->launches += 7;
  } else if (p->prox)
    CK(launch_prox_update(n, per, s.h * s.w, ctx->sv_nblk, P->z, P->grad, y, od.mask, x, xp,
                          p->lambda, p->tau, ctx->sv.status, ctx->sv.part_s, ctx->sv.part_x, st));
  else
    CK(launch_red_update(n, per, ctx->sv_nblk, P->z, ctx->gf, P->grad, x, xp, p->lambda, p->tau,
                         ctx->sv.status, ctx->sv.part_s, ctx->sv.part_x, st));
  const float B = (std::isfinite(p->restart_B) && p->restart_B > 0.f) ? p->restart_B : INFINITY;
  CK(launch_finalize(n, ctx->sv_nblk, ctx->sv, 1 - par, p->beta, B, p->tol, p->max_iter,
                     p->lambda, logic, avg_K, st));
  ctx->launches += 3;
  return IDEQ_OK;
}

// IDEQ_SOLVE_GRAPH=0 drives every iteration from the host (for comparisons).
bool graph_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("IDEQ_SOLVE_GRAPH");
    return !(v && v[0] == '0');
  }();
  return on;
}

// Everything of the operator that iterate() bakes into the captured graph by
// value: the kind and kernel size pick the kernels, the pointers and the scalars
// (saturation gain, Rician sigma) are launch arguments.  Kernel and mask contents
// are read at run time and may change between solves.
bool same_op(const OpDev& a, const OpDev& b) {
  return a.kind == b.kind && a.kh == b.kh && a.kw == b.kw && a.kernel == b.kernel &&
         a.mask == b.mask && a.gain == b.gain && a.sigma == b.sigma;
}

bool same_params(const ideq_params& a, const ideq_params& b) {
  return a.lambda == b.lambda && a.tau == b.tau && a.beta == b.beta &&
         a.restart_B == b.restart_B && a.tol == b.tol && a.max_iter == b.max_iter &&
         a.average == b.average && a.prox == b.prox;
}

// Build the solve graph for (plan, operator, y, params): a kernel setting the
// while condition from the solver state, then a while node whose body is two
// iterations (parities 0 and 1) and the condition update.  Returns false (and
// leaves no graph and the stream out of capture) when the runtime refuses any
// step; the caller then drives the loop from the host.
bool build_solve_graph(ideq_ctx* ctx, const OpDev& od, const ideq_shape& s, const float* y,
                       const ideq_params* p) {
  ctx->drop_graph();
  ctx->err.clear();
  if (!ctx->cap_stream &&
      cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    ctx->cap_stream = nullptr;
    (void)cudaGetLastError();
    ctx->graph_ok = false;
    return false;
  }
  // iterate() launches on ctx->stream: point it at the capture stream until return
  struct StreamSwap {
    ideq_ctx* c;
    cudaStream_t user;
    ~StreamSwap() { c->stream = user; }
  } swap{ctx, ctx->stream};
  ctx->stream = ctx->cap_stream;
  cudaStream_t st = ctx->stream;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle h;
  bool capturing = false;
  const char* step = "create";
  auto give_up = [&]() {
    const cudaError_t why = cudaGetLastError();
    const std::string before = ctx->err;  // set by a failing launch inside the capture
    ctx->err = std::string("device-driven solve graph not built (") + step + ": " +
               cudaGetErrorString(why) + (before.empty() ? "" : "; " + before) +
               "); the loop runs from the host";
    if (capturing) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(st, &junk);
      if (junk && junk != g) cudaGraphDestroy(junk);
    }
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    ctx->graph_ok = false;
    return false;
  };
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return give_up();
  if (cudaGraphConditionalHandleCreate(&h, g, 0, 0) != cudaSuccess) return give_up();
  step = "capture the condition";
  if (cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
      cudaSuccess)
    return give_up();
  capturing = true;
  // bodies needed: (max_iter - 2) / 2 rounded up, plus one spare
  const int max_bodies = (p->max_iter - 2 + 1) / 2 + 1;
  if (launch_loop_cond(h, ctx->sv.n_running, ctx->sv.loop_count, 1, max_bodies, ctx->d_err, st) !=
      cudaSuccess)
    return give_up();
  capturing = false;
  if (cudaStreamEndCapture(st, &g) != cudaSuccess) return give_up();
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn != 1) return give_up();
  cudaGraphNode_t first;
  if (cudaGraphGetNodes(g, &first, &nn) != cudaSuccess) return give_up();
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if (cudaGraphAddNode(&wnode, g, &first, nullptr, 1, &cp) != cudaSuccess) return give_up();
  // body: iteration (parity 0); an IF node holding iteration (parity 1) that runs
  // only while an image is still running; the while condition.  The loop thus
  // checks after every iteration and never computes an iteration past the last
  // running image.
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaGraphConditionalHandle h_if;
  step = "create the inner condition";
  if (cudaGraphConditionalHandleCreate(&h_if, body, 0, 0) != cudaSuccess) return give_up();
  step = "capture the body";
  if (cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return give_up();
  capturing = true;
  const long long l0 = ctx->launches;
  if (iterate(ctx, od, s, y, p, 0, 1, p->average != 0) != IDEQ_OK) return give_up();
  const long long iter_launches = ctx->launches - l0;
  ctx->launches = l0;
  if (launch_if_cond(h_if, ctx->sv.n_running, st) != cudaSuccess) return give_up();
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if (cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps) != cudaSuccess ||
      ndeps != 1)
    return give_up();
  cudaGraphNode_t cond_node = deps[0];
  capturing = false;
  step = "end the body capture";
  if (cudaStreamEndCapture(st, &body) != cudaSuccess) return give_up();
  cudaGraphNodeParams ip = {};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = h_if;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t if_node;
  step = "add the inner condition";
  if (cudaGraphAddNode(&if_node, body, &cond_node, nullptr, 1, &ip) != cudaSuccess)
    return give_up();
  cudaGraph_t inner = ip.conditional.phGraph_out[0];
  step = "capture the inner iteration";
  if (cudaStreamBeginCaptureToGraph(st, inner, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return give_up();
  capturing = true;
  if (iterate(ctx, od, s, y, p, 1, 1, p->average != 0) != IDEQ_OK) return give_up();
  ctx->launches = l0;
  capturing = false;
  if (cudaStreamEndCapture(st, &inner) != cudaSuccess) return give_up();
  step = "capture the loop condition";
  if (cudaStreamBeginCaptureToGraph(st, body, &if_node, nullptr, 1,
                                    cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return give_up();
  capturing = true;
  if (launch_loop_cond(h, ctx->sv.n_running, ctx->sv.loop_count, 0, max_bodies, ctx->d_err,
                       st) != cudaSuccess)
    return give_up();
  capturing = false;
  if (cudaStreamEndCapture(st, &body) != cudaSuccess) return give_up();
  const long long body_launches = iter_launches;  // per iteration run in the graph
  cudaGraphExec_t exec = nullptr;
  step = "instantiate";
  if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) return give_up();
  ctx->sg.g = g;
  ctx->sg.exec = exec;
  ctx->sg.plan = ctx->plan.get();
  ctx->sg.od = od;
  ctx->sg.y = y;
  ctx->sg.p = *p;
  ctx->sg.body_launches = body_launches;
  return true;
}

ideq_status check_timeout(ideq_ctx* ctx) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h != 0) {
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
    return fail(ctx, IDEQ_ERR_TIMEOUT, "tensor-core kernel wait expired (code " + std::to_string(h) + ")");
  }
  return IDEQ_OK;
}

bool valid_precision(int p) {
  return p == IDEQ_FP32 || p == IDEQ_BF16 || p == IDEQ_FP16 || p == IDEQ_BF16_FP8 ||
         p == IDEQ_FP16_FP8;
}

ideq_status check_params(ideq_ctx* ctx, const ideq_params* p) {
  if (!p) return fail(ctx, IDEQ_ERR_ARG, "params is NULL");
  if (!(p->tau > 0.f) || !(p->lambda >= 0.f) || !(p->beta >= 0.f && p->beta < 1.f))
    return fail(ctx, IDEQ_ERR_ARG, "need tau > 0, lambda >= 0, 0 <= beta < 1");
  if (p->max_iter < 1) return fail(ctx, IDEQ_ERR_ARG, "max_iter must be >= 1");
  if (p->prox != 0 && p->prox != 1) return fail(ctx, IDEQ_ERR_ARG, "prox must be 0 or 1");
  if (!(p->tol >= 0.0)) return fail(ctx, IDEQ_ERR_ARG, "tol must be >= 0");
  return IDEQ_OK;
}

ideq_status ensure_warm_plan(ideq_ctx* ctx, const ideq_shape& s) {
  if (!ctx->warm_w) return fail(ctx, IDEQ_ERR_ARG, "no warm-start network (ideq_warm_set)");
  if (s.c != ctx->warm_w->desc.in_ch) return fail(ctx, IDEQ_ERR_ARG, "warm start channels");
  TrainPlan* T = ctx->warm_plan.get();
  if (T && T->n == s.n && T->H == s.h && T->W == s.w && T->prec == ctx->precision) return IDEQ_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->warm_plan.reset();
  std::unique_ptr<TrainPlan> tp(new TrainPlan());
  std::string e;
  if (!tp->build(ctx->warm_w.get(), s.n, s.h, s.w, ctx->precision, nullptr, &e, true))
    return fail(ctx, IDEQ_ERR_UNSUPPORTED, "warm-start plan: " + e);
  ctx->warm_plan = std::move(tp);
  return IDEQ_OK;
}

// x0 = aty + W(aty) into out (all device, f32 NCHW)
ideq_status warm_forward(ideq_ctx* ctx, const ideq_shape& s, const float* aty, float* out) {
  ideq_status st = ensure_warm_plan(ctx, s);
  if (st != IDEQ_OK) return st;
  TrainPlan* T = ctx->warm_plan.get();
  const size_t bytes = (size_t)s.n * s.c * s.h * s.w * 4;
  CK(cudaMemcpyAsync(T->z, aty, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(run_steps(T->fwd, ctx->d_err, ctx->stream, &ctx->prof, &ctx->launches));
  if (out && out != T->out_img)
    CK(cudaMemcpyAsync(out, T->out_img, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return IDEQ_OK;
}

}  // namespace

// =========================================================================== C ABI

extern "C" {

ideq_status ideq_num_params(const ideq_net_desc* net, int64_t* count) {
  if (!net || !count) return IDEQ_ERR_ARG;
  long long c = 0;
  std::string e;
  if (!net_param_count(*net, &c, nullptr, &e)) return IDEQ_ERR_ARG;
  *count = c;
  return IDEQ_OK;
}

ideq_status ideq_create(ideq_ctx** out, const ideq_net_desc* net, const float* weights,
                        int precision, void* stream) {
  clear_stale_cuda_error();
  if (!out || !net || !weights) return IDEQ_ERR_ARG;
  if (!valid_precision(precision))
    return IDEQ_ERR_UNSUPPORTED;
  std::unique_ptr<ideq_ctx> c(new ideq_ctx());
  ideq_ctx* ctx = c.get();
  CK(cudaGetDevice(&c->device));
  c->stream = (cudaStream_t)stream;
  c->precision = precision;
  c->w.reset(new NetWeights());
  std::string e;
  if (!c->w->build(*net, &e)) return IDEQ_ERR_ARG;
  CK(c->w->upload(weights, c->stream));
  CK(cudaMalloc((void**)&c->d_err, 16));
  CK(cudaMemsetAsync(c->d_err, 0, 16, c->stream));
  CK(cudaMallocHost((void**)&c->h_running, 16));
  CK(cudaStreamSynchronize(c->stream));
  *out = c.release();
  return IDEQ_OK;
}

ideq_status ideq_destroy(ideq_ctx* ctx) {
  clear_stale_cuda_error();
  if (!ctx) return IDEQ_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);
  ctx->drop_graph();
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  ctx->plan.reset();
  ctx->train.reset();
  ctx->warm_plan.reset();
  ctx->warm_w.reset();
  for (float* p : {ctx->warm_m, ctx->warm_v, ctx->warm_g, ctx->reg_m, ctx->reg_v, ctx->reg_g,
                   ctx->reg_cot, ctx->reg_dlam, ctx->adj_v, ctx->adj_ms})
    if (p) cudaFree(p);
  if (ctx->reg_loss) cudaFree(ctx->reg_loss);
  ctx->w.reset();
  if (ctx->sv_mem) cudaFree(ctx->sv_mem);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->h_running) cudaFreeHost(ctx->h_running);
  delete ctx;
  return IDEQ_OK;
}

const char* ideq_last_error(ideq_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

ideq_status ideq_set_weights(ideq_ctx* ctx, const float* weights) {
  clear_stale_cuda_error();
  if (!ctx || !weights) return IDEQ_ERR_ARG;
  CK(ctx->w->upload(weights, ctx->stream));
  return IDEQ_OK;
}

ideq_status ideq_set_precision(ideq_ctx* ctx, int precision) {
  clear_stale_cuda_error();
  if (!ctx) return IDEQ_ERR_ARG;
  if (!valid_precision(precision))
    return fail(ctx, IDEQ_ERR_UNSUPPORTED, "precision");
  ctx->precision = precision;
  return IDEQ_OK;
}

ideq_status ideq_set_stream(ideq_ctx* ctx, void* stream) {
  clear_stale_cuda_error();
  if (!ctx) return IDEQ_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->stream = (cudaStream_t)stream;
  return IDEQ_OK;
}

ideq_status ideq_apply_A(ideq_ctx* ctx, const ideq_operator* op, ideq_shape shape, const float* x,
                         float* Ax) {
  clear_stale_cuda_error();
  if (!ctx || !x || !Ax || !shape_ok(shape)) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  OpDev od;
  ideq_status s = check_op(ctx, op, shape, &od);
  if (s != IDEQ_OK) return s;
  if (od.kind == IDEQ_OP_MRI) {
    CK(launch_mri_apply(shape.n, shape.h, shape.w, x, od.mask, 0, Ax, ctx->stream));
    ctx->launches += 3;
    return IDEQ_OK;
  }
  if (od.kind == IDEQ_OP_RICIAN) {  // A = identity
    CK(cudaMemcpyAsync(Ax, x, (size_t)shape.n * shape.c * shape.h * shape.w * 4,
                       cudaMemcpyDeviceToDevice, ctx->stream));
    return IDEQ_OK;
  }
  CK(launch_apply_A(od, shape.n, shape.c, shape.h, shape.w, x, Ax, ctx->stream));
  ctx->launches += 1;
  return IDEQ_OK;
}

ideq_status ideq_apply_AT(ideq_ctx* ctx, const ideq_operator* op, ideq_shape shape, const float* r,
                          const float* lin_point, float* out) {
  clear_stale_cuda_error();
  if (!ctx || !r || !out || !shape_ok(shape)) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  OpDev od;
  ideq_status s = check_op(ctx, op, shape, &od);
  if (s != IDEQ_OK) return s;
  if (od.kind == IDEQ_OP_SATBLUR && lin_point) {
    float* tmp = ensure_scratch(ctx, (size_t)shape.n * shape.c * shape.h * shape.w * 4);
    if (!tmp) return fail(ctx, IDEQ_ERR_NOMEM, "scratch");
    CK(launch_sat_jt_weight(od, shape.n, shape.c, shape.h, shape.w, lin_point, r, tmp, ctx->stream));
    CK(launch_blur_adj(od, shape.n, shape.c, shape.h, shape.w, tmp, out, ctx->stream));
    ctx->launches += 2;
    return IDEQ_OK;
  }
  CK(back_project(ctx, od, shape, r, out));
  return IDEQ_OK;
}

ideq_status ideq_grad_reg(ideq_ctx* ctx, ideq_shape shape, const float* z, float* grad,
                          double* g_val) {
  clear_stale_cuda_error();
  if (!ctx || !z || !grad || !shape_ok(shape)) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  ideq_status s = ensure_plan(ctx, shape);
  if (s != IDEQ_OK) return s;
  NetPlan* P = ctx->plan.get();
  const size_t bytes = (size_t)shape.n * shape.c * shape.h * shape.w * 4;
  CK(cudaMemcpyAsync(P->z, z, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(launch_zero_d(shape.n, ctx->gsum, ctx->stream));
  CK(cudaMemsetAsync(ctx->sv.skip, 0, shape.n * sizeof(int), ctx->stream));  // every image
  CK(run_steps(P->fwd, ctx->d_err, ctx->stream, &ctx->prof, &ctx->launches));
  CK(run_steps(P->vjp, ctx->d_err, ctx->stream, &ctx->prof, &ctx->launches));
  CK(cudaMemcpyAsync(grad, P->grad, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  if (g_val) CK(cudaMemcpyAsync(g_val, ctx->gsum, shape.n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->launches += 1;
  return IDEQ_OK;
}

ideq_status ideq_step(ideq_ctx* ctx, const ideq_operator* op, ideq_shape shape, const float* y,
                      float* x_k, float* x_km1, const ideq_params* p, ideq_info* info) {
  clear_stale_cuda_error();
  if (!ctx || !y || !x_k || !x_km1 || !shape_ok(shape)) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  ideq_status s = check_params(ctx, p);
  if (s != IDEQ_OK) return s;
  OpDev od;
  if ((s = check_op(ctx, op, shape, &od)) != IDEQ_OK) return s;
  if (p->prox && od.kind != IDEQ_OP_MASK && od.kind != IDEQ_OP_MRI)
    return fail(ctx, IDEQ_ERR_UNSUPPORTED, "the proximal step has a closed form for mask and MRI");
  if ((s = ensure_plan(ctx, shape)) != IDEQ_OK) return s;
  CK(prepare_data_step(ctx, od, shape, y));
  const size_t bytes = (size_t)shape.n * shape.c * shape.h * shape.w * 4;
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->xb[0], x_k, bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(ctx->xb[1], x_km1, bytes, cudaMemcpyDeviceToDevice, st));
  CK(launch_solver_init(shape.n, ctx->sv, p->beta, st));  // every image extrapolates with beta
  if ((s = iterate(ctx, od, shape, y, p, 0, 0)) != IDEQ_OK) return s;
  CK(cudaMemcpyAsync(x_km1, x_k, bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(x_k, ctx->xb[1], bytes, cudaMemcpyDeviceToDevice, st));
  if (info) CK(launch_fill_info(shape.n, ctx->sv, *info, st));
  return check_timeout(ctx);
}

ideq_status ideq_solve(ideq_ctx* ctx, const ideq_operator* op, ideq_shape shape, const float* y,
                       const float* x0, float* x_out, const ideq_params* p, ideq_info* info) {
  clear_stale_cuda_error();
  if (!ctx || !y || !x_out || !shape_ok(shape)) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  ideq_status s = check_params(ctx, p);
  if (s != IDEQ_OK) return s;
  OpDev od;
  if ((s = check_op(ctx, op, shape, &od)) != IDEQ_OK) return s;
  if (p->prox && od.kind != IDEQ_OP_MASK && od.kind != IDEQ_OP_MRI)
    return fail(ctx, IDEQ_ERR_UNSUPPORTED, "the proximal step has a closed form for mask and MRI");
  if (p->init == IDEQ_INIT_X0 && !x0) return fail(ctx, IDEQ_ERR_ARG, "init X0 needs x0");
  if (p->init == IDEQ_INIT_WARM && !ctx->warm_w)
    return fail(ctx, IDEQ_ERR_ARG, "init WARM needs ideq_warm_set");
  const bool restart_on = std::isfinite(p->restart_B) && p->restart_B > 0.f;
  if (p->average && (p->tol > 0.0 || restart_on || p->max_iter < 5))
    return fail(ctx, IDEQ_ERR_ARG, "averaging needs tol = 0, no restart and max_iter >= 5");
  if ((s = ensure_plan(ctx, shape)) != IDEQ_OK) return s;
  CK(prepare_data_step(ctx, od, shape, y));
  const size_t bytes = (size_t)shape.n * shape.c * shape.h * shape.w * 4;
  cudaStream_t st = ctx->stream;
  if (p->init == IDEQ_INIT_X0) {
    CK(cudaMemcpyAsync(ctx->xb[0], x0, bytes, cudaMemcpyDeviceToDevice, st));
  } else if (p->init == IDEQ_INIT_WARM) {
    CK(back_project(ctx, od, shape, y, ctx->tmp));
    if ((s = warm_forward(ctx, shape, ctx->tmp, ctx->xb[0])) != IDEQ_OK) return s;
  } else {
    CK(back_project(ctx, od, shape, y, ctx->xb[0]));
  }
  CK(cudaMemcpyAsync(ctx->xb[1], ctx->xb[0], bytes, cudaMemcpyDeviceToDevice, st));
  CK(launch_solver_init(shape.n, ctx->sv, 0.f, st));  // x^{-1} = x^0
  if (p->average) CK(cudaMemsetAsync(ctx->sv.zsum, 0, 2 * bytes, st));
  // the first two iterations run from the host (they also complete every lazy
  // kernel set-up), the rest in the device-driven graph unless that is off,
  // failed, or the profiler is recording per-launch events
  const bool avg = p->average != 0;
  const bool use_graph = ctx->graph_ok && !ctx->prof.on && graph_enabled();
  const int eager = use_graph ? std::min(2, p->max_iter) : p->max_iter;
  const int poll = p->tol > 0.0 ? 2 : 0;
  bool graphed = false;
  ctx->last_graphed = false;
  for (int it = 0; it < eager; ++it) {
    if ((s = iterate(ctx, od, shape, y, p, it & 1, 1, avg)) != IDEQ_OK) return s;
    if (!use_graph && poll && ((it + 1) % poll == 0) && it + 1 < p->max_iter) {
      CK(cudaMemcpyAsync(ctx->h_running, ctx->sv.n_running, 4, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*ctx->h_running == 0) break;
    }
  }
  if (use_graph && eager < p->max_iter) {
    const bool have = ctx->sg.exec && ctx->sg.plan == ctx->plan.get() && same_op(ctx->sg.od, od) &&
                      ctx->sg.y == y && same_params(ctx->sg.p, *p);
    if (have || build_solve_graph(ctx, od, shape, y, p)) {
      CK(cudaGraphLaunch(ctx->sg.exec, st));
      graphed = true;
    } else {  // no graph: finish from the host
      for (int it = eager; it < p->max_iter; ++it) {
        if ((s = iterate(ctx, od, shape, y, p, it & 1, 1, avg)) != IDEQ_OK) return s;
        if (poll && ((it + 1) % poll == 0) && it + 1 < p->max_iter) {
          CK(cudaMemcpyAsync(ctx->h_running, ctx->sv.n_running, 4, cudaMemcpyDeviceToHost, st));
          CK(cudaStreamSynchronize(st));
          if (*ctx->h_running == 0) break;
        }
      }
    }
  }
  ctx->last_graphed = graphed;
  CK(launch_gather_parity(shape.n, ctx->sv_per, ctx->sv.parity, ctx->xb[0], ctx->xb[1], x_out, st));
  ctx->launches += 1;
  if (p->average) {
    CK(launch_average_out(shape.n, ctx->sv_per, ctx->sv, x_out, st));
    ctx->launches += 1;
  }
  if (info) CK(launch_fill_info(shape.n, ctx->sv, *info, st));
  if ((s = check_timeout(ctx)) != IDEQ_OK) return s;
  // overall status (stream already synchronised by check_timeout)
  std::vector<int> hs(shape.n), ht(shape.n);
  CK(cudaMemcpy(hs.data(), ctx->sv.status, shape.n * 4, cudaMemcpyDeviceToHost));
  if (graphed) {  // launches the graph ran: one condition kernel, then per body up to two
                  // iterations and two condition kernels
    CK(cudaMemcpy(ht.data(), ctx->sv.total, shape.n * 4, cudaMemcpyDeviceToHost));
    const int last = *std::max_element(ht.begin(), ht.end());
    const long long in_graph = std::max(0, last - 2), bodies = (in_graph + 1) / 2;
    ctx->launches += 1 + in_graph * ctx->sg.body_launches + 2 * bodies;
  }
  bool div = false, maxit = false;
  for (int v : hs) {
    div |= v == IDEQ_IMG_DIVERGED;
    maxit |= v == IDEQ_IMG_MAXITER;
  }
  if (div) return fail(ctx, IDEQ_DIVERGED, "an image diverged");
  if (maxit && p->tol > 0.0) return fail(ctx, IDEQ_MAXITER, "an image hit max_iter");
  return IDEQ_OK;
}

ideq_status ideq_solve_backward(ideq_ctx* ctx, const ideq_operator* op, ideq_shape shape,
                                const float* y, const float* x_bar, const float* dl_dx,
                                const ideq_params* p, const ideq_adj_params* ap, float* dl_dtheta,
                                float* dl_dlambda, ideq_info* info) {
  clear_stale_cuda_error();
  if (!ctx || !y || !x_bar || !dl_dx || !dl_dtheta || !dl_dlambda || !ap || !shape_ok(shape))
    return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  ideq_status s = check_params(ctx, p);
  if (s != IDEQ_OK) return s;
  OpDev od;
  if ((s = check_op(ctx, op, shape, &od)) != IDEQ_OK) return s;
  if (p->prox) return fail(ctx, IDEQ_ERR_UNSUPPORTED, "backward of the proximal variant");
  if (od.kind == IDEQ_OP_SATBLUR || od.kind == IDEQ_OP_RICIAN)
    return fail(ctx, IDEQ_ERR_UNSUPPORTED, "backward supports linear operators (blur, mask, MRI)");
  if (ap->mode != IDEQ_ADJ_JFB && ap->mode != IDEQ_ADJ_IMPLICIT)
    return fail(ctx, IDEQ_ERR_ARG, "adjoint mode");
  if (ap->mode == IDEQ_ADJ_IMPLICIT && (ap->max_iter < 1 || !(ap->tol > 0.0) ||
                                        !(ap->beta >= 0.f && ap->beta < 1.f)))
    return fail(ctx, IDEQ_ERR_ARG, "adjoint tol > 0, max_iter >= 1, 0 <= beta < 1");
  if ((s = ensure_plan(ctx, shape)) != IDEQ_OK) return s;
  CK(prepare_data_step(ctx, od, shape, y));
  if (!ctx->train) {
    std::unique_ptr<TrainPlan> tp(new TrainPlan());
    std::string e;
    if (!tp->build(ctx->w.get(), shape.n, shape.h, shape.w, ctx->precision, ctx->gsum, &e))
      return fail(ctx, IDEQ_ERR_UNSUPPORTED, "training plan: " + e);
    ctx->train = std::move(tp);
  }
  TrainPlan* T = ctx->train.get();
  cudaStream_t st = ctx->stream;
  const int n = shape.n, per = ctx->sv_per;
  const size_t bytes = (size_t)n * per * 4;
  if (ctx->adj_v_bytes < bytes) {
    CK(cudaStreamSynchronize(st));
    if (ctx->adj_v) cudaFree(ctx->adj_v);
    ctx->adj_v = nullptr;
    ctx->adj_v_bytes = 0;
    CK(cudaMalloc((void**)&ctx->adj_v, bytes));
    ctx->adj_v_bytes = bytes;
  }
  if (!ctx->adj_ms) CK(cudaMalloc((void**)&ctx->adj_ms, 16));
  // v = dl/dx_hat times 2^-e, e = round(log2 RMS(v)): the adjoint equation and every
  // gradient below are linear in v, so the results are multiplied back by 2^e
  const long long numel = (long long)n * per;
  CK(launch_dot(numel, dl_dx, dl_dx, 1.f / (float)numel, ctx->dot_part, ctx->adj_ms, st));
  CK(launch_ldexp(numel, dl_dx, ctx->adj_ms, 0, -1, ctx->adj_v, st));
  ctx->launches += 3;
  const float* v = ctx->adj_v;
  // fixed point: N(xbar), r and grad g(xbar) with every t-chain cotangent kept
  CK(cudaMemcpyAsync(T->z, x_bar, bytes, cudaMemcpyDeviceToDevice, st));
  CK(launch_zero_d(n, ctx->gsum, st));
  CK(run_steps(T->fwd, ctx->d_err, st, &ctx->prof, &ctx->launches));
  CK(run_steps(T->tchain, ctx->d_err, st, &ctx->prof, &ctx->launches));
  // adjoint: u = J_R^T u + v with J_R = I - tau (H_f + lambda H_g) at xbar
  if (ap->mode == IDEQ_ADJ_IMPLICIT) {
    CK(cudaMemcpyAsync(ctx->xb[0], v, bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->xb[1], v, bytes, cudaMemcpyDeviceToDevice, st));
    CK(launch_solver_init(n, ctx->sv, 0.f, st));
    for (int it = 0; it < ap->max_iter; ++it) {
      const int par = it & 1;
      float* uk = ctx->xb[par];
      float* up = ctx->xb[1 - par];
      CK(launch_extrapolate(n, per, uk, up, ctx->sv.beta_eff, T->zd, st));
      CK(run_steps(T->jvp, ctx->d_err, st, &ctx->prof, &ctx->launches));
      CK(run_steps(T->pchain, ctx->d_err, st, &ctx->prof, &ctx->launches));
      CK(data_grad(ctx, od, shape, T->zd, nullptr, ctx->gf, ctx->tmp, ctx->sv.fsum));
      CK(launch_red_update(n, per, ctx->sv_nblk, T->zd, ctx->gf, T->hvp, uk, up, p->lambda,
                           p->tau, ctx->sv.status, ctx->sv.part_s, ctx->sv.part_x, st, v));
      CK(launch_finalize(n, ctx->sv_nblk, ctx->sv, 1 - par, ap->beta, INFINITY, ap->tol,
                         ap->max_iter, 0.f, 1, 0, st));
      ctx->launches += 3;
      if ((it & 1) == 1 && it + 1 < ap->max_iter) {
        CK(cudaMemcpyAsync(ctx->h_running, ctx->sv.n_running, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (*ctx->h_running == 0) break;
      }
    }
    CK(launch_gather_parity(n, per, ctx->sv.parity, ctx->xb[0], ctx->xb[1], ctx->ubuf, st));
  } else {
    CK(cudaMemcpyAsync(ctx->ubuf, v, bytes, cudaMemcpyDeviceToDevice, st));
    CK(launch_solver_init(n, ctx->sv, 0.f, st));
  }
  // dl/dlambda = -tau <u, grad g(xbar)>
  CK(launch_dot((long long)n * per, ctx->ubuf, T->grad, -p->tau, ctx->dot_part, dl_dlambda, st));
  // dl/dtheta = -tau lambda d<u, grad g_theta(xbar)>/dtheta = +tau lambda gW(rdot, r)
  CK(cudaMemcpyAsync(T->zd, ctx->ubuf, bytes, cudaMemcpyDeviceToDevice, st));
  CK(run_steps(T->jvp, ctx->d_err, st, &ctx->prof, &ctx->launches));
  CK(run_steps(T->pchain, ctx->d_err, st, &ctx->prof, &ctx->launches));
  CK(cudaMemsetAsync(dl_dtheta, 0, ctx->w->nparams * 4, st));
  CK(T->run_wgrad(dl_dtheta, p->tau * p->lambda, true, st, &ctx->launches, ctx->d_err));
  // undo the scaling of v
  CK(launch_ldexp(ctx->w->nparams, dl_dtheta, ctx->adj_ms, 0, 1, dl_dtheta, st));
  CK(launch_ldexp(1, dl_dlambda, ctx->adj_ms, 0, 1, dl_dlambda, st));
  ctx->launches += 4;
  if (info) CK(launch_fill_info(n, ctx->sv, *info, st));
  if ((s = check_timeout(ctx)) != IDEQ_OK) return s;
  if (ap->mode == IDEQ_ADJ_IMPLICIT) {
    std::vector<int> hs(n);
    CK(cudaMemcpy(hs.data(), ctx->sv.status, n * 4, cudaMemcpyDeviceToHost));
    for (int v : hs)
      if (v != IDEQ_IMG_CONVERGED) return fail(ctx, IDEQ_ADJ_MAXITER, "adjoint solve did not converge");
  }
  return IDEQ_OK;
}

ideq_status ideq_train_step(ideq_ctx* ctx, const ideq_operator* op, ideq_shape shape,
                            const float* y, const float* x_true, const ideq_params* p,
                            const ideq_adj_params* ap, float lr, float* x_out,
                            float* dl_dtheta, float* dl_dlambda, double* loss, ideq_info* info) {
  clear_stale_cuda_error();
  if (!ctx || !y || !x_true || !x_out || !ap || !shape_ok(shape) || !(lr >= 0.f))
    return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  const long long np = ctx->w->nparams;
  const size_t bytes = (size_t)shape.n * shape.c * shape.h * shape.w * 4;
  if (!ctx->reg_m) {
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMalloc((void**)&ctx->reg_m, np * 4));
    CK(cudaMalloc((void**)&ctx->reg_v, np * 4));
    CK(cudaMalloc((void**)&ctx->reg_g, np * 4));
    CK(cudaMalloc((void**)&ctx->reg_loss, 16));
    CK(cudaMalloc((void**)&ctx->reg_dlam, 16));
    CK(cudaMemsetAsync(ctx->reg_m, 0, np * 4, ctx->stream));
    CK(cudaMemsetAsync(ctx->reg_v, 0, np * 4, ctx->stream));
    ctx->reg_t = 0;
  }
  if (ctx->reg_cot_bytes < bytes) {
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->reg_cot) cudaFree(ctx->reg_cot);
    ctx->reg_cot = nullptr;
    ctx->reg_cot_bytes = 0;
    CK(cudaMalloc((void**)&ctx->reg_cot, bytes));
    ctx->reg_cot_bytes = bytes;
  }
  // forward: x_hat, the fixed point (Algorithm 1); a solve that did not converge
  // stops the step before any weight changes
  ideq_status s = ideq_solve(ctx, op, shape, y, nullptr, x_out, p, info);
  if (s != IDEQ_OK) return s;
  cudaStream_t st = ctx->stream;
  // l = mean((x_hat - x*)^2) and dl/dx_hat
  double* lp = loss ? loss : ctx->reg_loss;
  CK(launch_mse_grad((long long)bytes / 4, x_out, x_true, ctx->reg_cot, ctx->dot_part, lp, st));
  ctx->launches += 2;
  // implicit backward (App. D.1.2): dl/dtheta, dl/dlambda
  float* dl = dl_dlambda ? dl_dlambda : ctx->reg_dlam;
  s = ideq_solve_backward(ctx, op, shape, y, x_out, ctx->reg_cot, p, ap, ctx->reg_g, dl, nullptr);
  if (s != IDEQ_OK) return s;
  if (dl_dtheta) CK(cudaMemcpyAsync(dl_dtheta, ctx->reg_g, np * 4, cudaMemcpyDeviceToDevice, st));
  // one Adam step on theta, then the weight forms of the convolutions
  ctx->reg_t += 1;
  CK(launch_adam(np, ctx->w->master, ctx->reg_g, ctx->reg_m, ctx->reg_v, ctx->reg_t, lr, 0.9f,
                 0.999f, 1e-8f, st));
  CK(ctx->w->reform(st));
  ctx->launches += 1 + 2 * (long long)ctx->w->layers.size();
  return IDEQ_OK;
}

ideq_status ideq_time_wgrad(ideq_ctx* ctx, int reps, double* ms, double* flops,
                            int64_t* tc_convs) {
  clear_stale_cuda_error();
  if (!ctx || reps < 1 || !ms) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  TrainPlan* T = ctx->train.get();
  if (!T) return fail(ctx, IDEQ_ERR_ARG, "no training plan yet: run ideq_solve_backward first");
  float* dst = ensure_scratch(ctx, (size_t)ctx->w->nparams * 4);
  if (!dst) return fail(ctx, IDEQ_ERR_NOMEM, "scratch");
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r)
    e = T->run_wgrad(dst, 1.f, true, st, &ctx->launches, ctx->d_err);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ideq_time_wgrad");
  double fl = 0;
  long long ntc = 0;
  for (const WgStep& g : T->wg) {
    fl += 2.0 * g.a.flops();  // the dual form: two products per conv
    ntc += g.tc[0] != nullptr;
  }
  *ms = t;
  if (flops) *flops = fl * reps;
  if (tc_convs) *tc_convs = ntc;
  return check_timeout(ctx);
}

ideq_status ideq_warm_set(ideq_ctx* ctx, const ideq_net_desc* net, const float* weights) {
  clear_stale_cuda_error();
  if (!ctx || !net || !weights) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  if (net->kind != IDEQ_NET_CNN) return fail(ctx, IDEQ_ERR_ARG, "warm start must be a plain CNN");
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->warm_plan.reset();
  for (float* p : {ctx->warm_m, ctx->warm_v, ctx->warm_g})
    if (p) cudaFree(p);
  ctx->warm_m = ctx->warm_v = ctx->warm_g = nullptr;
  std::unique_ptr<NetWeights> w(new NetWeights());
  std::string e;
  if (!w->build(*net, &e)) return fail(ctx, IDEQ_ERR_ARG, "warm start: " + e);
  CK(w->upload(weights, ctx->stream));
  const size_t b = (size_t)w->nparams * 4;
  CK(cudaMalloc((void**)&ctx->warm_m, b));
  CK(cudaMalloc((void**)&ctx->warm_v, b));
  CK(cudaMalloc((void**)&ctx->warm_g, b));
  CK(cudaMemsetAsync(ctx->warm_m, 0, b, ctx->stream));
  CK(cudaMemsetAsync(ctx->warm_v, 0, b, ctx->stream));
  ctx->warm_t = 0;
  ctx->warm_w = std::move(w);
  return IDEQ_OK;
}

ideq_status ideq_warm_forward(ideq_ctx* ctx, ideq_shape shape, const float* aty, float* x0) {
  clear_stale_cuda_error();
  if (!ctx || !aty || !x0 || !shape_ok(shape)) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  return warm_forward(ctx, shape, aty, x0);
}

ideq_status ideq_warm_train_step(ideq_ctx* ctx, ideq_shape shape, const float* aty,
                                 const float* target, float lr, double* loss) {
  clear_stale_cuda_error();
  if (!ctx || !aty || !target || !shape_ok(shape) || !(lr > 0.f))
    return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  ideq_status s = warm_forward(ctx, shape, aty, nullptr);
  if (s != IDEQ_OK) return s;
  TrainPlan* T = ctx->warm_plan.get();
  NetWeights* W = ctx->warm_w.get();
  cudaStream_t st = ctx->stream;
  const long long numel = (long long)shape.n * shape.c * shape.h * shape.w;
  double* part = nullptr;
  // the loss kernel needs 128 doubles of partials: reuse the solver's if sized, else scratch
  float* scr = ensure_scratch(ctx, 128 * 8);
  if (!scr) return fail(ctx, IDEQ_ERR_NOMEM, "scratch");
  part = (double*)scr;
  CK(launch_mse_grad(numel, T->out_img, target, T->cot_img, part, loss, st));
  // the reverse chain runs on 2^k dl/dx0, 2^k ~ numel (exact): the mean's 1/numel
  // would leave 16-bit cotangents subnormal; the gradient is scaled back by 2^-k
  int k = 0;
  while ((1LL << (k + 1)) <= numel && k < 60) ++k;
  CK(launch_ldexp(numel, T->cot_img, nullptr, k, 1, T->cot_img, st));
  CK(run_steps(T->tchain, ctx->d_err, st, &ctx->prof, &ctx->launches));
  CK(cudaMemsetAsync(ctx->warm_g, 0, W->nparams * 4, st));
  CK(T->run_wgrad(ctx->warm_g, 1.f, false, st, &ctx->launches, ctx->d_err));
  CK(launch_ldexp(W->nparams, ctx->warm_g, nullptr, k, -1, ctx->warm_g, st));
  ctx->warm_t += 1;
  CK(launch_adam(W->nparams, W->master, ctx->warm_g, ctx->warm_m, ctx->warm_v, ctx->warm_t, lr,
                 0.9f, 0.999f, 1e-8f, st));
  CK(W->reform(st));
  ctx->launches += 3 + 2 * (long long)W->layers.size();
  return IDEQ_OK;
}

ideq_status ideq_warm_get(ideq_ctx* ctx, float* weights) {
  clear_stale_cuda_error();
  if (!ctx || !weights) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  if (!ctx->warm_w) return fail(ctx, IDEQ_ERR_ARG, "no warm-start network");
  CK(cudaMemcpyAsync(weights, ctx->warm_w->master, ctx->warm_w->nparams * 4,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  return IDEQ_OK;
}

ideq_status ideq_prof_enable(ideq_ctx* ctx, int on) {
  if (!ctx) return IDEQ_ERR_ARG;
  ctx->prof.on = on != 0;
  return IDEQ_OK;
}

ideq_status ideq_prof_read(ideq_ctx* ctx, double* ms, int64_t* launches, double* flops) {
  clear_stale_cuda_error();
  if (!ctx) return IDEQ_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  double t = 0;
  for (size_t i = 0; i + 1 < ctx->prof.used; i += 2) {
    float m = 0.f;
    cudaEventElapsedTime(&m, ctx->prof.ev[i], ctx->prof.ev[i + 1]);
    t += m;
  }
  if (ms) *ms = t;
  if (launches) *launches = ctx->prof.launches;
  if (flops) *flops = ctx->prof.flops;
  ctx->prof.used = 0;
  ctx->prof.launches = 0;
  ctx->prof.flops = 0;
  return IDEQ_OK;
}

ideq_status ideq_time_convs(ideq_ctx* ctx, int reps, double* ms, int64_t* launches,
                            double* flops) {
  clear_stale_cuda_error();
  if (!ctx || reps < 1 || !ms) return fail(ctx, IDEQ_ERR_ARG, "bad arguments");
  NetPlan* P = ctx->plan.get();
  if (!P) return fail(ctx, IDEQ_ERR_ARG, "no plan yet: run a solve, step or grad_reg first");
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  long long nl = 0;
  double fl = 0;
  cudaError_t e = cudaMemsetAsync(ctx->sv.skip, 0, P->n * sizeof(int), st);  // every image
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r)
    for (const std::vector<Step>* list : {&P->fwd, &P->vjp})
      for (const Step& s : *list) {
        if (!s.tc || s.quant_n > 0 || e != cudaSuccess) continue;
        e = launch_conv_tc(s.tc, s.a, ctx->d_err, st);
        nl += 1;
        fl += s.a.flops();
      }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ideq_time_convs");
  ctx->launches += nl;
  *ms = t;
  if (launches) *launches = nl;
  if (flops) *flops = fl;
  return check_timeout(ctx);
}

ideq_status ideq_plan_flops(ideq_ctx* ctx, double* per_iteration) {
  if (!ctx || !per_iteration) return IDEQ_ERR_ARG;
  NetPlan* P = ctx->plan.get();
  if (!P) return fail(ctx, IDEQ_ERR_ARG, "no plan yet: run a solve, step or grad_reg first");
  *per_iteration = P->fwd_flops + P->vjp_flops;
  return IDEQ_OK;
}

ideq_status ideq_launch_count(ideq_ctx* ctx, int64_t* count) {
  if (!ctx || !count) return IDEQ_ERR_ARG;
  *count = ctx->launches;
  ctx->launches = 0;
  return IDEQ_OK;
}

ideq_status ideq_solve_graphed(ideq_ctx* ctx, int* graphed) {
  if (!ctx || !graphed) return IDEQ_ERR_ARG;
  *graphed = ctx->last_graphed ? 1 : 0;
  return IDEQ_OK;
}

}  // extern "C"
