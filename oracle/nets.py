"""Regulariser network N and the GS potential g (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The learned regulariser is the Gradient-Step potential g(x) = 1/2 ||x - N(x)||^2
with denoiser D = Id - grad g (Sec. 2.2, Eq. GS), so that

    grad g(x) = r - J_N(x)^T r,            r = x - N(x).

N is a convolutional network with smooth (softplus) activations (Sec. 3.3); the
warm-start network uses ReLU.  A network is a list of ops over named values:

    ("conv3", w, src, dst)  3x3 convolution, zero "same" padding, stride 1
    ("down",  w, src, dst)  2x2 convolution, stride 2
    ("up",    w, src, dst)  2x2 transposed convolution, stride 2
    ("act",   kind, src, dst)   softplus or relu
    ("add",   a, b, dst)

Every op is evaluated per image (c, h, w).  Reverse passes are written out by hand
per op.  Second-order quantities (Hessian-vector products of g and the parameter
gradient of <u, grad g>) use the reverse pass of the dual-number forward map
(x, xdot) -> (N(x), J_N(x) xdot); per op that is

    linear y = W x:    xbar = W^T ybar,   xdotbar = W^T ydotbar,
                       Wbar += ybar x^T + ydotbar xdot^T
    a = sp(h), adot = s hdot (s = sigmoid(h)):
                       hbar = s abar + s (1 - s) hdot adotbar,   hdotbar = s adotbar
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------- topology


def unet_program(c, widths, n_rb=2, act="softplus"):
    """Op list and weight table of the residual U-Net (see synth.unet_layout).

    Returns (ops, wtab) with wtab = [(name, kind, shape)] in flat-vector order."""
    L = len(widths)
    ops, wtab = [], []

    def W(name, kind, shape):
        wtab.append((name, kind, shape))
        return name

    ops.append(("conv3", W("head", "conv3", (widths[0], c, 3, 3)), "in", "h"))
    cur = "h"
    cnt = [0]

    def new(tag):
        cnt[0] += 1
        return f"{tag}#{cnt[0]}"

    def rb(prefix, wd, x):
        for r in range(n_rb):
            t, a, u, o = new("t"), new("a"), new("u"), new("o")
            ops.append(("conv3", W(f"{prefix}.rb{r}.c1", "conv3", (wd, wd, 3, 3)), x, t))
            ops.append(("act", act, t, a))
            ops.append(("conv3", W(f"{prefix}.rb{r}.c2", "conv3", (wd, wd, 3, 3)), a, u))
            ops.append(("add", x, u, o))
            x = o
        return x

    skips = []
    for lv in range(L - 1):
        cur = rb(f"enc{lv}", widths[lv], cur)
        skips.append(cur)
        d = new("d")
        ops.append(("down", W(f"enc{lv}.down", "down", (widths[lv + 1], widths[lv], 2, 2)),
                    cur, d))
        cur = d
    cur = rb(f"mid{L - 1}", widths[L - 1], cur)
    for lv in range(L - 2, -1, -1):
        up, s = new("up"), new("s")
        ops.append(("up", W(f"dec{lv}.up", "up", (widths[lv + 1], widths[lv], 2, 2)), cur, up))
        ops.append(("add", up, skips[lv], s))
        cur = rb(f"dec{lv}", widths[lv], s)
    ops.append(("conv3", W("tail", "conv3", (c, widths[0], 3, 3)), cur, "out"))
    return ops, wtab


def cnn_program(chans, act="softplus"):
    """Plain 3x3 conv stack with an activation after every layer but the last."""
    ops, wtab = [], []
    cur = "in"
    n = len(chans) - 1
    for i in range(n):
        name = f"l{i}"
        wtab.append((name, "conv3", (chans[i + 1], chans[i], 3, 3)))
        dst = "out" if i == n - 1 else f"h{i}"
        ops.append(("conv3", name, cur, dst))
        if i < n - 1:
            ops.append(("act", act, dst, f"a{i}"))
            cur = f"a{i}"
    return ops, wtab


class Net:
    """A network program with its weights unpacked to float64 arrays."""

    def __init__(self, ops, wtab, flat):
        self.ops, self.wtab = ops, wtab
        flat = np.asarray(flat, dtype=np.float64)
        self.W = {}
        off = 0
        for name, _kind, shape in wtab:
            n = int(np.prod(shape))
            self.W[name] = flat[off:off + n].reshape(shape).copy()
            off += n
        if off != flat.size:
            raise ValueError(f"weight vector has {flat.size} entries, program needs {off}")
        self.nparams = off

    @staticmethod
    def from_config(netcfg, c, flat):
        if netcfg["type"] == "unet":
            ops, wtab = unet_program(c, netcfg["widths"], netcfg.get("n_rb", 2),
                                     netcfg.get("act", "softplus"))
        else:
            ops, wtab = cnn_program(netcfg["chans"], netcfg.get("act", "softplus"))
        return Net(ops, wtab, flat)

    def flatten(self, grads: dict) -> np.ndarray:
        return np.concatenate([grads[name].ravel() for name, _k, _s in self.wtab])


# ---------------------------------------------------------------- primitive ops


def _shift(x, dy, dx):
    """s[c,i,j] = x[c, i+dy, j+dx], zero outside the image."""
    c, h, w = x.shape
    out = np.zeros_like(x)
    ys, ye = max(0, -dy), min(h, h - dy)
    xs, xe = max(0, -dx), min(w, w - dx)
    if ys < ye and xs < xe:
        out[:, ys:ye, xs:xe] = x[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv3(x, W):
    """out[o,i,j] = sum_{c,u,v} W[o,c,u,v] x[c, i+u-1, j+v-1] (zero padding)."""
    c, h, w = x.shape
    out = np.zeros((W.shape[0], h * w))
    for u in range(3):
        for v in range(3):
            out += W[:, :, u, v] @ _shift(x, u - 1, v - 1).reshape(c, h * w)
    return out.reshape(W.shape[0], h, w)


def conv3_T(g, W):
    """Adjoint of conv3 in its input: sum_{u,v} shift^T(W[:,:,u,v]^T g)."""
    o, h, w = g.shape
    out = np.zeros((W.shape[1], h, w))
    gf = g.reshape(o, h * w)
    for u in range(3):
        for v in range(3):
            t = (W[:, :, u, v].T @ gf).reshape(W.shape[1], h, w)
            out += _shift(t, -(u - 1), -(v - 1))
    return out


def conv3_W(g, x):
    """Gradient in W of <g, conv3(x, W)>."""
    c, h, w = x.shape
    gf = g.reshape(g.shape[0], h * w)
    dW = np.zeros((g.shape[0], c, 3, 3))
    for u in range(3):
        for v in range(3):
            dW[:, :, u, v] = gf @ _shift(x, u - 1, v - 1).reshape(c, h * w).T
    return dW


def down(x, W):
    """out[o,i,j] = sum_{c,u,v} W[o,c,u,v] x[c, 2i+u, 2j+v]."""
    c, h, w = x.shape
    out = np.zeros((W.shape[0], (h // 2) * (w // 2)))
    for u in range(2):
        for v in range(2):
            out += W[:, :, u, v] @ x[:, u::2, v::2].reshape(c, -1)
    return out.reshape(W.shape[0], h // 2, w // 2)


def down_T(g, W):
    o, h2, w2 = g.shape
    out = np.zeros((W.shape[1], 2 * h2, 2 * w2))
    gf = g.reshape(o, -1)
    for u in range(2):
        for v in range(2):
            out[:, u::2, v::2] = (W[:, :, u, v].T @ gf).reshape(W.shape[1], h2, w2)
    return out


def down_W(g, x):
    c = x.shape[0]
    gf = g.reshape(g.shape[0], -1)
    dW = np.zeros((g.shape[0], c, 2, 2))
    for u in range(2):
        for v in range(2):
            dW[:, :, u, v] = gf @ x[:, u::2, v::2].reshape(c, -1).T
    return dW


def up(x, U):
    """Transposed conv, U[c_in, c_out, u, v]: out[o, 2i+u, 2j+v] = sum_c U[c,o,u,v] x[c,i,j]."""
    c, h, w = x.shape
    out = np.zeros((U.shape[1], 2 * h, 2 * w))
    xf = x.reshape(c, -1)
    for u in range(2):
        for v in range(2):
            out[:, u::2, v::2] = (U[:, :, u, v].T @ xf).reshape(U.shape[1], h, w)
    return out


def up_T(g, U):
    o = g.shape[0]
    h, w = g.shape[1] // 2, g.shape[2] // 2
    out = np.zeros((U.shape[0], h * w))
    for u in range(2):
        for v in range(2):
            out += U[:, :, u, v] @ g[:, u::2, v::2].reshape(o, -1)
    return out.reshape(U.shape[0], h, w)


def up_W(g, x):
    c = x.shape[0]
    xf = x.reshape(c, -1)
    dU = np.zeros((c, g.shape[0], 2, 2))
    for u in range(2):
        for v in range(2):
            dU[:, :, u, v] = xf @ g[:, u::2, v::2].reshape(g.shape[0], -1).T
    return dU


_LIN = {"conv3": (conv3, conv3_T, conv3_W), "down": (down, down_T, down_W),
        "up": (up, up_T, up_W)}


def softplus(h):
    return np.logaddexp(0.0, h)


def sigmoid(h):
    return 0.5 * (1.0 + np.tanh(0.5 * h))


def _act(kind, h):
    if kind == "softplus":
        return softplus(h), sigmoid(h)
    if kind == "relu":
        return np.maximum(h, 0.0), (h > 0).astype(np.float64)
    raise ValueError(kind)


def _act_d2(kind, h):
    """Second derivative of the activation."""
    if kind == "softplus":
        s = sigmoid(h)
        return s * (1.0 - s)
    return np.zeros_like(h)


# ------------------------------------------------------------------ passes


def forward(net: Net, x):
    """N(x); returns (out, vals) with every named value kept."""
    v = {"in": np.asarray(x, dtype=np.float64)}
    for op in net.ops:
        if op[0] in _LIN:
            v[op[3]] = _LIN[op[0]][0](v[op[2]], net.W[op[1]])
        elif op[0] == "act":
            v[op[3]] = _act(op[1], v[op[2]])[0]
        else:
            v[op[3]] = v[op[1]] + v[op[2]]
    return v["out"], v


def jvp(net: Net, vals, xdot):
    """Tangents of every value for input tangent xdot (J_N(x) xdot is t['out'])."""
    t = {"in": np.asarray(xdot, dtype=np.float64)}
    for op in net.ops:
        if op[0] in _LIN:
            t[op[3]] = _LIN[op[0]][0](t[op[2]], net.W[op[1]])
        elif op[0] == "act":
            t[op[3]] = _act(op[1], vals[op[2]])[1] * t[op[2]]
        else:
            t[op[3]] = t[op[1]] + t[op[2]]
    return t


def _accum(d, k, g):
    if k in d:
        d[k] = d[k] + g
    else:
        d[k] = g


def vjp(net: Net, vals, cot, want_w=False):
    """J_N(x)^T cot (and the weight gradient of <cot, N(x)> if want_w)."""
    bar = {"out": np.asarray(cot, dtype=np.float64)}
    gW = {}
    for op in reversed(net.ops):
        if op[0] in _LIN:
            gb = bar.pop(op[3])
            f, fT, fW = _LIN[op[0]]
            _accum(bar, op[2], fT(gb, net.W[op[1]]))
            if want_w:
                gW[op[1]] = fW(gb, vals[op[2]])
        elif op[0] == "act":
            gb = bar.pop(op[3])
            _accum(bar, op[2], _act(op[1], vals[op[2]])[1] * gb)
        else:
            gb = bar.pop(op[3])
            _accum(bar, op[1], gb)
            _accum(bar, op[2], gb)
    return bar["in"], gW


def dual_reverse(net: Net, vals, tans, cot_p, cot_t, want_w=False):
    """Reverse pass of (x, xdot) -> (N(x), J_N(x) xdot).

    Output cotangents cot_p (for N) and cot_t (for J_N xdot).  Returns
    (xbar, xdotbar, gW) with
        xbar    = J_N^T cot_p + (d/dx [J_N(x) xdot])^T cot_t,
        xdotbar = J_N^T cot_t,
        gW      = gradient in the weights of <cot_p, N> + <cot_t, J_N xdot>."""
    pb = {"out": np.asarray(cot_p, dtype=np.float64)}
    tb = {"out": np.asarray(cot_t, dtype=np.float64)}
    gW = {}
    for op in reversed(net.ops):
        if op[0] in _LIN:
            a, b = pb.pop(op[3]), tb.pop(op[3])
            f, fT, fW = _LIN[op[0]]
            Wt = net.W[op[1]]
            _accum(pb, op[2], fT(a, Wt))
            _accum(tb, op[2], fT(b, Wt))
            if want_w:
                gW[op[1]] = fW(a, vals[op[2]]) + fW(b, tans[op[2]])
        elif op[0] == "act":
            a, b = pb.pop(op[3]), tb.pop(op[3])
            h, hd = vals[op[2]], tans[op[2]]
            s = _act(op[1], h)[1]
            _accum(pb, op[2], s * a + _act_d2(op[1], h) * hd * b)
            _accum(tb, op[2], s * b)
        else:
            a, b = pb.pop(op[3]), tb.pop(op[3])
            for k in (op[1], op[2]):
                _accum(pb, k, a)
                _accum(tb, k, b)
    return pb["in"], tb["in"], gW


# ----------------------------------------------------------- GS potential g


def g_value(net: Net, x) -> float:
    """g(x) = 1/2 ||x - N(x)||^2 (Eq. GS)."""
    out, _ = forward(net, x)
    r = x - out
    return 0.5 * float(np.sum(r * r))


def grad_g(net: Net, x):
    """(grad g(x), g(x)) with grad g = r - J_N(x)^T r, r = x - N(x)."""
    x = np.asarray(x, dtype=np.float64)
    out, vals = forward(net, x)
    r = x - out
    jt, _ = vjp(net, vals, r)
    return r - jt, 0.5 * float(np.sum(r * r))


def hvp_g(net: Net, x, w):
    """Hessian of g at x applied to w.

    With rdot = w - J_N w, the tangent of grad g in direction w is
    rdot - J_N^T rdot - (d/dx[J_N w])^T r, i.e. rdot - xbar of the dual reverse
    pass with cotangents (rdot, r)."""
    x = np.asarray(x, dtype=np.float64)
    out, vals = forward(net, x)
    tans = jvp(net, vals, w)
    r = x - out
    rdot = w - tans["out"]
    xbar, _, _ = dual_reverse(net, vals, tans, rdot, r)
    return rdot - xbar


def grad_theta_dot(net: Net, x, u):
    """Gradient in the weights of <u, grad g_theta(x)> (flat vector).

    <u, grad g> = <r, rdot> with r = x - N(x), rdot = u - J_N(x) u, so the
    cotangents of (N, J_N u) are (-rdot, -r)."""
    x = np.asarray(x, dtype=np.float64)
    out, vals = forward(net, x)
    tans = jvp(net, vals, u)
    r = x - out
    rdot = u - tans["out"]
    _, _, gW = dual_reverse(net, vals, tans, -rdot, -r, want_w=True)
    return net.flatten(gW)


def grad_theta_out(net: Net, x, cot):
    """Gradient in the weights of <cot, N(x)> (flat vector)."""
    _, vals = forward(net, x)
    _, gW = vjp(net, vals, cot, want_w=True)
    return net.flatten(gW)


def estimate_lipschitz(net: Net, x, iters=30, seed=0) -> float:
    """Power-iteration estimate of ||Hess g(x)||_2 (an L_g estimate)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(x.shape)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        hv = hvp_g(net, x, v)
        lam = float(np.linalg.norm(hv))
        v = hv / max(lam, 1e-300)
    return lam
