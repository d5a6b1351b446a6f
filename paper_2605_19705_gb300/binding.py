"""Thin ctypes binding of libideq.so (the C ABI declared in include/ideq.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (device memory and the current stream
come from PyTorch); each wrapper checks dtype, device and contiguity, passes raw
pointers and raises IdeqError on a non-OK status.  There is no CPU fallback: if
the shared library is missing or cannot be loaded, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libideq.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback)")
_lib = ctypes.CDLL(LIB_PATH)

c_int, c_float, c_double, c_void_p = ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_void_p

# status / enum values (include/ideq.h)
IDEQ_OK, IDEQ_ERR_ARG, IDEQ_ERR_CUDA, IDEQ_ERR_NOMEM, IDEQ_ERR_UNSUPPORTED = 0, 1, 2, 3, 4
IDEQ_MAXITER, IDEQ_DIVERGED, IDEQ_ADJ_MAXITER, IDEQ_ERR_TIMEOUT = 5, 6, 7, 8
IDEQ_IMG_RUNNING, IDEQ_IMG_CONVERGED, IDEQ_IMG_MAXITER, IDEQ_IMG_DIVERGED = 0, 1, 2, 3
IDEQ_NET_CNN, IDEQ_NET_UNET = 0, 1
IDEQ_ACT_SOFTPLUS, IDEQ_ACT_RELU = 0, 1
IDEQ_OP_BLUR, IDEQ_OP_MASK, IDEQ_OP_SATBLUR, IDEQ_OP_MRI, IDEQ_OP_RICIAN = 0, 1, 2, 3, 4
IDEQ_FP32, IDEQ_BF16, IDEQ_BF16_FP8, IDEQ_FP16, IDEQ_FP16_FP8 = 0, 1, 2, 3, 4
IDEQ_INIT_ATY, IDEQ_INIT_X0, IDEQ_INIT_WARM = 0, 1, 2
IDEQ_ADJ_JFB, IDEQ_ADJ_IMPLICIT = 0, 1


class NetDesc(ctypes.Structure):
    _fields_ = [("kind", c_int), ("act", c_int), ("in_ch", c_int), ("n_levels", c_int),
                ("n_rb", c_int), ("depth", c_int), ("widths", c_int * 16)]


class Shape(ctypes.Structure):
    _fields_ = [("n", c_int), ("c", c_int), ("h", c_int), ("w", c_int)]


class Operator(ctypes.Structure):
    _fields_ = [("kind", c_int), ("kh", c_int), ("kw", c_int), ("kernel", c_void_p),
                ("mask", c_void_p), ("sat_gain", c_float), ("sigma", c_float)]


class Params(ctypes.Structure):
    _fields_ = [("lam", c_float), ("tau", c_float), ("beta", c_float), ("restart_B", c_float),
                ("tol", c_double), ("max_iter", c_int), ("init", c_int), ("average", c_int),
                ("prox", c_int)]


class Info(ctypes.Structure):
    _fields_ = [("iters", c_void_p), ("restarts", c_void_p), ("status", c_void_p),
                ("rel_res", c_void_p), ("energy", c_void_p), ("k0", c_void_p)]


class AdjParams(ctypes.Structure):
    _fields_ = [("mode", c_int), ("tol", c_double), ("max_iter", c_int), ("beta", c_float)]


P = ctypes.POINTER
_sig = {
    "ideq_create": [P(c_void_p), P(NetDesc), c_void_p, c_int, c_void_p],
    "ideq_destroy": [c_void_p],
    "ideq_set_weights": [c_void_p, c_void_p],
    "ideq_set_precision": [c_void_p, c_int],
    "ideq_set_stream": [c_void_p, c_void_p],
    "ideq_num_params": [P(NetDesc), P(ctypes.c_int64)],
    "ideq_apply_A": [c_void_p, P(Operator), Shape, c_void_p, c_void_p],
    "ideq_apply_AT": [c_void_p, P(Operator), Shape, c_void_p, c_void_p, c_void_p],
    "ideq_grad_reg": [c_void_p, Shape, c_void_p, c_void_p, c_void_p],
    "ideq_step": [c_void_p, P(Operator), Shape, c_void_p, c_void_p, c_void_p, P(Params), P(Info)],
    "ideq_solve": [c_void_p, P(Operator), Shape, c_void_p, c_void_p, c_void_p, P(Params),
                   P(Info)],
    "ideq_solve_backward": [c_void_p, P(Operator), Shape, c_void_p, c_void_p, c_void_p,
                            P(Params), P(AdjParams), c_void_p, c_void_p, P(Info)],
    "ideq_train_step": [c_void_p, P(Operator), Shape, c_void_p, c_void_p, P(Params),
                        P(AdjParams), c_float, c_void_p, c_void_p, c_void_p, c_void_p, P(Info)],
    "ideq_time_wgrad": [c_void_p, c_int, P(c_double), P(c_double), P(ctypes.c_int64)],
    "ideq_warm_set": [c_void_p, P(NetDesc), c_void_p],
    "ideq_warm_forward": [c_void_p, Shape, c_void_p, c_void_p],
    "ideq_warm_train_step": [c_void_p, Shape, c_void_p, c_void_p, c_float, c_void_p],
    "ideq_warm_get": [c_void_p, c_void_p],
    "ideq_prof_enable": [c_void_p, c_int],
    "ideq_prof_read": [c_void_p, P(c_double), P(ctypes.c_int64), P(c_double)],
    "ideq_launch_count": [c_void_p, P(ctypes.c_int64)],
    "ideq_time_convs": [c_void_p, c_int, P(c_double), P(ctypes.c_int64), P(c_double)],
    "ideq_plan_flops": [c_void_p, P(c_double)],
    "ideq_fp32_fma_peak": [c_void_p, P(c_double)],
    "ideq_solve_graphed": [c_void_p, P(c_int)],
    "ideq_red_update_noalloc": [c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_float, c_float, c_void_p, c_void_p, c_void_p],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = c_int
_lib.ideq_last_error.argtypes = [c_void_p]
_lib.ideq_last_error.restype = ctypes.c_char_p

EXPORTED = sorted(list(_sig) + ["ideq_last_error"])


class IdeqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ideq status {status}: {msg}")
        self.status = status


def _ptr(t, dtype=None):
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise ValueError("tensor must be on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"tensor dtype {t.dtype}, expected {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def net_desc(net: dict, c: int) -> NetDesc:
    """NetDesc from a config dict ({"type": "unet"|"cnn", ...})."""
    d = NetDesc()
    d.act = IDEQ_ACT_RELU if net.get("act", "softplus") == "relu" else IDEQ_ACT_SOFTPLUS
    d.in_ch = c
    if net["type"] == "unet":
        d.kind = IDEQ_NET_UNET
        d.n_levels = len(net["widths"])
        d.n_rb = net.get("n_rb", 2)
        for i, v in enumerate(net["widths"]):
            d.widths[i] = v
    else:
        d.kind = IDEQ_NET_CNN
        d.depth = len(net["chans"]) - 1
        for i, v in enumerate(net["chans"]):
            d.widths[i] = v
    return d


def ideq_num_params(desc: NetDesc) -> int:
    n = ctypes.c_int64(0)
    st = _lib.ideq_num_params(ctypes.byref(desc), ctypes.byref(n))
    if st != IDEQ_OK:
        raise IdeqError(st, "bad network description")
    return int(n.value)


class Context:
    """Owns an ideq_ctx; all calls run on torch's current CUDA stream."""

    def __init__(self, desc: NetDesc, weights, precision=IDEQ_FP32):
        import torch
        self.desc = desc
        self.h = c_void_p()
        st = _lib.ideq_create(ctypes.byref(self.h), ctypes.byref(desc), _ptr(weights, torch.float32),
                              precision, _stream())
        if st != IDEQ_OK:
            raise IdeqError(st, "ideq_create failed")

    def check(self, st):
        if st not in (IDEQ_OK,):
            raise IdeqError(st, _lib.ideq_last_error(self.h).decode())
        return st

    def close(self):
        if self.h:
            _lib.ideq_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_operator(kind: int, kernel=None, mask=None, sat_gain: float = 2.0,
                  sigma: float = 0.0) -> Operator:
    """Operator struct; kernel (n,kh,kw) f32 / mask (n,h,w) u8 CUDA tensors stay owned
    by the caller and must outlive the calls that use it."""
    import torch
    op = Operator()
    op.kind = kind
    if kernel is not None:
        op.kh, op.kw = int(kernel.shape[-2]), int(kernel.shape[-1])
        op.kernel = _ptr(kernel, torch.float32)
    if mask is not None:
        op.mask = _ptr(mask, torch.uint8)
    op.sat_gain = sat_gain
    op.sigma = sigma
    op._keep = (kernel, mask)
    return op


def _shape(x) -> Shape:
    n, c, h, w = x.shape
    return Shape(n, c, h, w)


def ideq_set_weights(ctx: Context, weights):
    import torch
    ctx.check(_lib.ideq_set_weights(ctx.h, _ptr(weights, torch.float32)))


def ideq_set_precision(ctx: Context, precision: int):
    ctx.check(_lib.ideq_set_precision(ctx.h, precision))


def ideq_apply_A(ctx: Context, op: Operator, x, out=None):
    import torch
    out = torch.empty_like(x) if out is None else out
    ctx.check(_lib.ideq_apply_A(ctx.h, ctypes.byref(op), _shape(x), _ptr(x, torch.float32),
                                _ptr(out, torch.float32)))
    return out


def ideq_apply_AT(ctx: Context, op: Operator, r, lin_point=None, out=None):
    import torch
    out = torch.empty_like(r) if out is None else out
    ctx.check(_lib.ideq_apply_AT(ctx.h, ctypes.byref(op), _shape(r), _ptr(r, torch.float32),
                                 _ptr(lin_point, torch.float32), _ptr(out, torch.float32)))
    return out


def ideq_grad_reg(ctx: Context, z, grad=None, g_val=None):
    import torch
    grad = torch.empty_like(z) if grad is None else grad
    ctx.check(_lib.ideq_grad_reg(ctx.h, _shape(z), _ptr(z, torch.float32),
                                 _ptr(grad, torch.float32), _ptr(g_val, torch.float64)))
    return grad


def make_params(lam, tau, beta, B=float("inf"), tol=0.0, max_iter=50, init=IDEQ_INIT_ATY,
                average=False, prox=False):
    p = Params()
    p.lam, p.tau, p.beta, p.restart_B = lam, tau, beta, (B if B != float("inf") else 0.0)
    p.tol, p.max_iter, p.init, p.average = tol, max_iter, init, 1 if average else 0
    p.prox = 1 if prox else 0
    return p


class InfoBuffers:
    """Device arrays backing an ideq_info for n images."""

    def __init__(self, n, device="cuda"):
        import torch
        self.iters = torch.zeros(n, dtype=torch.int32, device=device)
        self.restarts = torch.zeros(n, dtype=torch.int32, device=device)
        self.status = torch.zeros(n, dtype=torch.int32, device=device)
        self.rel_res = torch.zeros(n, dtype=torch.float64, device=device)
        self.energy = torch.zeros(n, dtype=torch.float64, device=device)
        self.k0 = torch.zeros(n, dtype=torch.int32, device=device)
        self.s = Info(self.iters.data_ptr(), self.restarts.data_ptr(), self.status.data_ptr(),
                      self.rel_res.data_ptr(), self.energy.data_ptr(), self.k0.data_ptr())


def ideq_step(ctx: Context, op: Operator, y, x_k, x_km1, params: Params, info=None):
    import torch
    return ctx.check(_lib.ideq_step(ctx.h, ctypes.byref(op), _shape(y), _ptr(y, torch.float32),
                                    _ptr(x_k, torch.float32), _ptr(x_km1, torch.float32),
                                    ctypes.byref(params),
                                    ctypes.byref(info.s) if info is not None else None))


def ideq_solve(ctx: Context, op: Operator, y, params: Params, x0=None, out=None, info=None,
               allow_maxiter=False):
    """Solve; returns (x_hat, status).  IDEQ_MAXITER raises unless allow_maxiter."""
    import torch
    out = torch.empty_like(y) if out is None else out
    st = _lib.ideq_solve(ctx.h, ctypes.byref(op), _shape(y), _ptr(y, torch.float32),
                         _ptr(x0, torch.float32), _ptr(out, torch.float32), ctypes.byref(params),
                         ctypes.byref(info.s) if info is not None else None)
    if st == IDEQ_MAXITER and allow_maxiter:
        return out, st
    ctx.check(st)
    return out, st


def ideq_solve_backward(ctx: Context, op: Operator, y, x_bar, dl_dx, params: Params,
                        adj: AdjParams, dl_dtheta, dl_dlambda, info=None, allow_maxiter=False):
    """Implicit backward; returns the status (IDEQ_ADJ_MAXITER raises unless allowed)."""
    import torch
    st = _lib.ideq_solve_backward(
        ctx.h, ctypes.byref(op), _shape(y), _ptr(y, torch.float32), _ptr(x_bar, torch.float32),
        _ptr(dl_dx, torch.float32), ctypes.byref(params), ctypes.byref(adj),
        _ptr(dl_dtheta, torch.float32), _ptr(dl_dlambda, torch.float32),
        ctypes.byref(info.s) if info is not None else None)
    if st == IDEQ_ADJ_MAXITER and allow_maxiter:
        return st
    return ctx.check(st)


def ideq_train_step(ctx: Context, op: Operator, y, x_true, params: Params, adj: AdjParams,
                    lr: float, x_out=None, dl_dtheta=None, dl_dlambda=None, loss=None, info=None):
    """One training step (solve, MSE loss, implicit backward, Adam on theta); returns
    x_hat.  Raises IdeqError when the forward or the adjoint solve did not converge."""
    import torch
    x_out = torch.empty_like(y) if x_out is None else x_out
    ctx.check(_lib.ideq_train_step(
        ctx.h, ctypes.byref(op), _shape(y), _ptr(y, torch.float32), _ptr(x_true, torch.float32),
        ctypes.byref(params), ctypes.byref(adj), float(lr), _ptr(x_out, torch.float32),
        _ptr(dl_dtheta, torch.float32), _ptr(dl_dlambda, torch.float32),
        _ptr(loss, torch.float64), ctypes.byref(info.s) if info is not None else None))
    return x_out


def ideq_time_wgrad(ctx: Context, reps: int):
    """(ms, flops, tensor-core convs) of `reps` weight-gradient passes of the last
    implicit backward, timed with CUDA events on the context's stream."""
    ms, fl, n = c_double(0), c_double(0), ctypes.c_int64(0)
    ctx.check(_lib.ideq_time_wgrad(ctx.h, int(reps), ctypes.byref(ms), ctypes.byref(fl),
                                   ctypes.byref(n)))
    return ms.value, fl.value, int(n.value)


def make_adj(mode=IDEQ_ADJ_IMPLICIT, tol=1e-3, max_iter=500, beta=0.0) -> AdjParams:
    a = AdjParams()
    a.mode, a.tol, a.max_iter, a.beta = mode, tol, max_iter, beta
    return a


def ideq_prof_enable(ctx: Context, on: bool):
    ctx.check(_lib.ideq_prof_enable(ctx.h, 1 if on else 0))


def ideq_prof_read(ctx: Context):
    ms, n, fl = c_double(0), ctypes.c_int64(0), c_double(0)
    ctx.check(_lib.ideq_prof_read(ctx.h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)))
    return ms.value, int(n.value), fl.value


def ideq_time_convs(ctx: Context, reps: int):
    """(ms, launches, flops) of `reps` back-to-back repetitions of the plan's
    tensor-core conv launches, timed with CUDA events on the context's stream."""
    ms, n, fl = c_double(0), ctypes.c_int64(0), c_double(0)
    ctx.check(_lib.ideq_time_convs(ctx.h, int(reps), ctypes.byref(ms), ctypes.byref(n),
                                   ctypes.byref(fl)))
    return ms.value, int(n.value), fl.value


def ideq_plan_flops(ctx: Context) -> float:
    """Algorithmic FLOPs of all convolutions of one iteration of the current plan."""
    v = c_double(0)
    ctx.check(_lib.ideq_plan_flops(ctx.h, ctypes.byref(v)))
    return v.value


def ideq_fp32_fma_peak() -> float:
    """Measured FP32 FFMA throughput of the current GPU, TFLOP/s."""
    v = c_double(0)
    st = _lib.ideq_fp32_fma_peak(_stream(), ctypes.byref(v))
    if st != IDEQ_OK:
        raise IdeqError(st, "ideq_fp32_fma_peak failed")
    return v.value


def ideq_launch_count(ctx: Context) -> int:
    n = ctypes.c_int64(0)
    ctx.check(_lib.ideq_launch_count(ctx.h, ctypes.byref(n)))
    return int(n.value)


def ideq_solve_graphed(ctx: Context) -> bool:
    """Whether the last ideq_solve on ctx ran its loop in the device-driven graph."""
    g = c_int(0)
    ctx.check(_lib.ideq_solve_graphed(ctx.h, ctypes.byref(g)))
    return bool(g.value)


def ideq_red_update_noalloc(z, grad_f, grad_g, x, x_new, lam, tau, step_sq=None, x_sq=None):
    """Context-free RED update for callers that cannot allocate device memory.

    x_new = z - tau (grad_f + lam grad_g) with per-image ||x_new - x||^2 and ||x||^2
    (FP64 sums of FP32 partial sums over <= 16 elements); every tensor is a caller-owned CUDA tensor (images (n, c, h, w) f32,
    norms (n,) f64).  Runs on torch's current stream; allocates nothing."""
    import torch
    n = z.shape[0]
    per = z.numel() // n
    st = _lib.ideq_red_update_noalloc(n, per, _ptr(z, torch.float32), _ptr(grad_f, torch.float32),
                                      _ptr(grad_g, torch.float32), _ptr(x, torch.float32),
                                      _ptr(x_new, torch.float32), lam, tau,
                                      _ptr(step_sq, torch.float64), _ptr(x_sq, torch.float64),
                                      _stream())
    if st != IDEQ_OK:
        raise IdeqError(st, "ideq_red_update_noalloc failed")
