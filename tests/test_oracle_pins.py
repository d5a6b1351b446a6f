"""Pins of the FP64 oracle against facts independent of it (CPU only).

Each test ties one part of the oracle to something other than itself: a library
routine (torch.nn.functional, numpy.fft), torch.autograd, central finite
differences, an adjoint identity, a closed form, or a brute-force loop.
"""
import math

import numpy as np
import pytest

from oracle import adjoint, nets, operators, solver, warmstart
from synth import generators as G
from synth import get_config, workload

RNG = np.random.default_rng(1234)


def rnd(*shape):
    return RNG.standard_normal(shape)


def tiny_unet(c=3, widths=(4, 8, 8, 16), seed=7):
    layout = G.unet_layout(c, list(widths), 2)
    flat = G.init_weights(seed, layout)
    ops, wtab = nets.unet_program(c, list(widths), 2)
    return nets.Net(ops, wtab, flat), layout, flat


def tiny_cnn(chans=(1, 6, 6, 1), seed=3, act="softplus"):
    layout = G.cnn_layout(list(chans))
    flat = G.init_weights(seed, layout)
    ops, wtab = nets.cnn_program(list(chans), act)
    return nets.Net(ops, wtab, flat), layout, flat


# ------------------------------------------------------------ primitive convs


def test_conv_primitives_match_torch(torch64):
    torch = torch64
    F = torch.nn.functional
    x = rnd(5, 12, 10)
    W3 = rnd(7, 5, 3, 3)
    Wd = rnd(7, 5, 2, 2)
    U = rnd(5, 7, 2, 2)
    tx = torch.tensor(x)[None]
    np.testing.assert_allclose(nets.conv3(x, W3), F.conv2d(tx, torch.tensor(W3), padding=1)[0],
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(nets.down(x, Wd), F.conv2d(tx, torch.tensor(Wd), stride=2)[0],
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(nets.up(x, U),
                               F.conv_transpose2d(tx, torch.tensor(U), stride=2)[0],
                               rtol=1e-12, atol=1e-12)


def test_conv3_brute_force():
    x = rnd(2, 5, 4)
    W = rnd(3, 2, 3, 3)
    ref = np.zeros((3, 5, 4))
    for o in range(3):
        for i in range(5):
            for j in range(4):
                for c in range(2):
                    for u in range(3):
                        for v in range(3):
                            ii, jj = i + u - 1, j + v - 1
                            if 0 <= ii < 5 and 0 <= jj < 4:
                                ref[o, i, j] += W[o, c, u, v] * x[c, ii, jj]
    np.testing.assert_allclose(nets.conv3(x, W), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", ["conv3", "down", "up"])
def test_conv_adjoint_identities(kind):
    f, fT, fW = nets._LIN[kind]
    if kind == "conv3":
        x, W = rnd(4, 9, 7), rnd(6, 4, 3, 3)
    elif kind == "down":
        x, W = rnd(4, 8, 6), rnd(6, 4, 2, 2)
    else:
        x, W = rnd(4, 5, 3), rnd(4, 6, 2, 2)
    y = f(x, W)
    g = rnd(*y.shape)
    lhs = float(np.sum(y * g))
    assert abs(lhs - float(np.sum(x * fT(g, W)))) < 1e-12 * max(1.0, abs(lhs))
    assert abs(lhs - float(np.sum(W * fW(g, x)))) < 1e-12 * max(1.0, abs(lhs))


# ------------------------------------------------------------ network + g


def test_weight_tables_match_synth_layouts():
    for widths in ([64, 128, 256, 512], [32, 64, 128, 256]):
        lay = G.unet_layout(3, widths, 2)
        _, wtab = nets.unet_program(3, widths, 2)
        assert [(a, b, tuple(c)) for a, b, c, *_ in lay] == [(a, b, tuple(c)) for a, b, c in wtab]
    lay = G.cnn_layout([3, 48, 48, 48, 48, 48, 3])
    _, wtab = nets.cnn_program([3, 48, 48, 48, 48, 48, 3], "relu")
    assert [(a, tuple(c)) for a, _, c, *_ in lay] == [(a, tuple(c)) for a, _, c in wtab]
    assert sum(int(np.prod(s)) for _, _, s, *_ in G.unet_layout(3, [64, 128, 256, 512])) == 17010048


def test_unet_forward_matches_torch(torch64):
    import torch_ref
    torch = torch64
    net, layout, flat = tiny_unet()
    x = rnd(3, 16, 24)
    out, _ = nets.forward(net, x)
    W = torch_ref.unpack(flat, layout)
    ref = torch_ref.unet(W, torch.tensor(x)[None], [4, 8, 8, 16])[0]
    np.testing.assert_allclose(out, ref.numpy(), rtol=1e-11, atol=1e-12)


def test_grad_g_matches_finite_differences():
    net, _, _ = tiny_cnn()
    x = RNG.uniform(0, 1, (1, 8, 8))
    gg, _ = nets.grad_g(net, x)
    h = 1e-6
    fd = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        e = np.zeros_like(x)
        e[idx] = h
        fd[idx] = (nets.g_value(net, x + e) - nets.g_value(net, x - e)) / (2 * h)
    assert np.max(np.abs(fd - gg)) / np.max(np.abs(gg)) < 1e-8


def test_grad_g_unet_finite_differences_sampled():
    net, _, _ = tiny_unet()
    x = RNG.uniform(0, 1, (3, 16, 16))
    gg, _ = nets.grad_g(net, x)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 7, 9), (2, 15, 15), (0, 3, 12), (2, 8, 0), (1, 0, 15)]:
        e = np.zeros_like(x)
        e[idx] = h
        fd = (nets.g_value(net, x + e) - nets.g_value(net, x - e)) / (2 * h)
        assert abs(fd - gg[idx]) < 1e-7 * max(1.0, np.max(np.abs(gg)))


def test_grad_hvp_and_param_grads_match_autograd(torch64):
    import torch_ref
    torch = torch64
    net, layout, flat = tiny_unet()
    x = RNG.uniform(0, 1, (3, 16, 16))
    u = rnd(3, 16, 16)
    W = torch_ref.unpack(flat, layout)
    for t in W.values():
        t.requires_grad_(True)
    tx = torch.tensor(x)[None].requires_grad_(True)
    g = torch_ref.g_of(lambda z: torch_ref.unet(W, z, [4, 8, 8, 16]), tx)
    (gx,) = torch.autograd.grad(g, tx, create_graph=True)
    tu = torch.tensor(u)[None]
    dot = (gx * tu).sum()
    grads = torch.autograd.grad(dot, [tx] + list(W.values()))
    hv_ref = grads[0][0].detach().numpy()
    gth_ref = np.concatenate([t.detach().numpy().ravel() for t in grads[1:]])

    gg, gval = nets.grad_g(net, x)
    np.testing.assert_allclose(gval, float(g.detach()), rtol=1e-12)
    np.testing.assert_allclose(gg, gx[0].detach().numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(nets.hvp_g(net, x, u), hv_ref, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(nets.grad_theta_dot(net, x, u), gth_ref, rtol=1e-9, atol=1e-11)


def test_hvp_symmetric_and_matches_fd_of_gradient():
    net, _, _ = tiny_unet()
    x = RNG.uniform(0, 1, (3, 16, 16))
    a, b = rnd(3, 16, 16), rnd(3, 16, 16)
    ha, hb = nets.hvp_g(net, x, a), nets.hvp_g(net, x, b)
    assert abs(np.sum(ha * b) - np.sum(a * hb)) < 1e-10 * abs(np.sum(ha * b))
    h = 1e-5
    fd = (nets.grad_g(net, x + h * a)[0] - nets.grad_g(net, x - h * a)[0]) / (2 * h)
    assert np.max(np.abs(fd - ha)) < 1e-7 * np.max(np.abs(ha))


# ------------------------------------------------------------ forward models


@pytest.mark.parametrize("kind", ["blur", "mask", "satblur", "mri"])
def test_operator_adjoint_identity(kind):
    k = G.motion_kernel(5, 9)
    m = G.cartesian_mask(1, 12, 10, 2, 0.2) if kind == "mri" else G.bernoulli_mask(1, 12, 10, 0.3)
    op = operators.Operator(kind, kern=k, mask=m)
    c = 2 if kind == "mri" else 3
    x, r = rnd(c, 12, 10), rnd(c, 12, 10)
    lin = (lambda v: operators.conv_circ(v, op.k)) if kind == "satblur" else op.A
    lhs = float(np.sum(lin(x) * r))
    assert abs(lhs - float(np.sum(x * op.AT(r)))) < 1e-13 * max(1.0, abs(lhs))
    xl = RNG.uniform(0, 1, (c, 12, 10))
    lhs = float(np.sum(op.JA(xl, x) * r))
    assert abs(lhs - float(np.sum(x * op.JAT(xl, r)))) < 1e-13 * max(1.0, abs(lhs))


def test_blur_is_circular_convolution_by_fft():
    x = rnd(2, 16, 12)
    k = G.motion_kernel(11, 7).astype(np.float64)
    kp = np.zeros((16, 12))
    kp[:7, :7] = k
    kp = np.roll(kp, (-3, -3), axis=(0, 1))
    ref = np.real(np.fft.ifft2(np.fft.fft2(x) * np.fft.fft2(kp)[None]))
    np.testing.assert_allclose(operators.conv_circ(x, k), ref, atol=1e-13)


def test_saturation_jacobian_and_hessian_fd():
    op = operators.Operator("satblur", kern=G.gaussian_kernel(5, 1.0), gain=2.0)
    x = RNG.uniform(0, 1, (3, 9, 8))
    y = op.A(RNG.uniform(0, 1, (3, 9, 8))) + 0.05 * rnd(3, 9, 8)
    w = rnd(3, 9, 8)
    h = 1e-6
    fd = (op.A(x + h * w) - op.A(x - h * w)) / (2 * h)
    assert np.max(np.abs(fd - op.JA(x, w))) < 1e-8
    fdg = (op.grad_f(x + h * w, y) - op.grad_f(x - h * w, y)) / (2 * h)
    assert np.max(np.abs(fdg - op.hvp_f(x, y, w))) < 1e-7
    e = np.zeros_like(x)
    e[1, 4, 4] = h
    assert abs((op.f(x + e, y) - op.f(x - e, y)) / (2 * h) - op.grad_f(x, y)[1, 4, 4]) < 1e-8


def test_inpainting_gradient_closed_form():
    m = G.bernoulli_mask(2, 6, 5, 0.3)
    op = operators.Operator("mask", mask=m)
    x, y = rnd(3, 6, 5), rnd(3, 6, 5)
    # App. E: grad f = M^T (M x - y) = M (x - y) for a 0/1 diagonal M (on masked y)
    np.testing.assert_allclose(op.grad_f(x, m * y), m * (x - y), atol=1e-15)


# ------------------------------------------------------------ iteration


def zero_tail_unet(c=1, widths=(4, 8, 8, 16)):
    """U-Net whose tail weights are zero: N == 0, g = 1/2||x||^2, grad g = x."""
    net, layout, flat = tiny_unet(c, widths)
    net.W["tail"][:] = 0.0
    return net


def fourier_heavy_ball(Kf, Yf, X0f, lam, tau, beta, B, tol, max_iter, hw):
    """Independent Fourier-domain run of the iteration for N == 0 and circular blur.

    Each frequency obeys X_{k+1} = Z_k - tau((|K|^2 + lam) Z_k - conj(K) Y),
    Z_k = X_k + beta (X_k - X_{k-1}); norms use Parseval (||x||^2 = sum|X|^2 / hw)."""
    q = 1.0 - tau * (np.abs(Kf) ** 2 + lam)
    b = tau * np.conj(Kf) * Yf
    X, Xp = X0f.copy(), X0f.copy()
    k, S, total, restarts = 0, 0.0, 0, 0
    while total < max_iter:
        Z = X + beta * (X - Xp)
        Xn = q * Z + b
        s = float(np.sum(np.abs(Xn - X) ** 2)) / hw
        nx = float(np.sum(np.abs(X) ** 2)) / hw
        Xp, X = X, Xn
        k += 1
        total += 1
        S += s
        if tol > 0 and math.sqrt(s) < tol * math.sqrt(nx):
            break
        if k * S > B * B:
            Xp = X.copy()
            k, S = 0, 0.0
            restarts += 1
    return X, total, restarts


@pytest.mark.parametrize("beta,B,tol", [(0.8, math.inf, 0.0), (0.8, 0.35, 0.0), (0.8, 0.05, 0.0),
                                        (0.5, 1.0, 1e-6), (0.0, math.inf, 1e-5)])
def test_iteration_matches_fourier_closed_form(beta, B, tol):
    net = zero_tail_unet()
    h = w = 16
    k = G.motion_kernel(21, 7).astype(np.float64)
    op = operators.Operator("blur", kern=k)
    x_true = G.synth_image(3, 1, h, w).astype(np.float64)
    y = op.A(x_true) + 0.02 * rnd(1, h, w)
    x0 = op.AT(y)
    lam, tau, max_iter = 0.1, 0.75, 120
    x, info = solver.solve_image(net, op, y, x0, lam, tau, beta, B, tol, max_iter)
    kp = np.zeros((h, w))
    kp[:7, :7] = k
    kp = np.roll(kp, (-3, -3), axis=(0, 1))
    Kf = np.fft.fft2(kp)
    X, total, restarts = fourier_heavy_ball(Kf, np.fft.fft2(y[0]), np.fft.fft2(x0[0]), lam, tau,
                                            beta, B, tol, max_iter, h * w)
    assert info["iters"] == total
    assert info["restarts"] == restarts
    if B < math.inf and tol == 0:
        assert restarts >= 1
    np.testing.assert_allclose(x[0], np.real(np.fft.ifft2(X)), atol=1e-11)


def test_stopping_test_divides_by_the_old_iterate():
    """Stop when ||x^{k+1} - x^k|| < tol ||x^k|| (App. D.1.3): pick tol between the
    ratios taken against x^k and against x^{k+1} after the first step."""
    net = zero_tail_unet()
    op = operators.Operator("blur", kern=G.gaussian_kernel(5, 1.0))
    y = op.A(G.synth_image(4, 1, 16, 16).astype(np.float64))
    x0 = 3.0 * op.AT(y)  # far from the fixed point: ||x^1|| << ||x^0||
    x1 = solver.red_step(net, op, y, x0, 0.1, 0.75)[0]
    d = np.linalg.norm(x1 - x0)
    r_old, r_new = d / np.linalg.norm(x0), d / np.linalg.norm(x1)
    assert r_old < r_new
    _, info = solver.solve_image(net, op, y, x0, 0.1, 0.75, 0.8, math.inf,
                                 0.5 * (r_old + r_new), 50)
    assert info["iters"] == 1 and info["status"] == solver.CONVERGED


def test_tikhonov_fixed_point_blur_and_mask():
    lam, tau = 0.1, 0.75
    net = zero_tail_unet(c=1)
    h = w = 16
    k = G.gaussian_kernel(5, 1.2).astype(np.float64)
    op = operators.Operator("blur", kern=k)
    y = rnd(1, h, w)
    x, info = solver.solve_image(net, op, y, op.AT(y), lam, tau, 0.8, math.inf, 1e-13, 5000)
    kp = np.zeros((h, w))
    kp[:5, :5] = k
    kp = np.roll(kp, (-2, -2), axis=(0, 1))
    Kf = np.fft.fft2(kp)
    ref = np.real(np.fft.ifft2(np.conj(Kf) * np.fft.fft2(y[0]) / (np.abs(Kf) ** 2 + lam)))
    np.testing.assert_allclose(x[0], ref, atol=1e-10)
    m = G.bernoulli_mask(9, h, w, 0.3)
    opm = operators.Operator("mask", mask=m)
    ym = m * rnd(1, h, w)
    x, info = solver.solve_image(net, opm, ym, opm.AT(ym), lam, tau, 0.8, math.inf, 1e-13, 5000)
    np.testing.assert_allclose(x, m * ym / (m + lam), atol=1e-10)


def test_gradient_descent_special_case_decreases_energy():
    """beta = 0 is RED = gradient descent on F; F decreases for tau < 1/L."""
    net, _, _ = tiny_unet(c=3)
    k = G.gaussian_kernel(5, 1.5)
    op = operators.Operator("blur", kern=k)
    x_true = G.synth_image(5, 3, 16, 16).astype(np.float64)
    y = op.A(x_true) + 0.02 * rnd(3, 16, 16)
    x, info = solver.solve_image(net, op, y, op.AT(y), 0.1, 0.5, 0.0, math.inf, 0.0, 30,
                                 keep_history=True)
    e = np.array(info["energy_hist"])
    assert np.all(np.diff(e) <= 1e-12)
    # RED step equals x - tau grad F with F = f + lam g (Eq. RED_operator)
    z = op.AT(y)
    nxt = solver.red_step(net, op, y, z, 0.1, 0.5)[0]
    gF = op.grad_f(z, y) + 0.1 * nets.grad_g(net, z)[0]
    np.testing.assert_allclose(nxt, z - 0.5 * gF, atol=1e-14)


def test_psnr_value():
    assert abs(solver.psnr(np.full(4, 0.1), np.zeros(4)) - 20.0) < 1e-12


# ------------------------------------------------------------ differentiation


def _tiny_problem(seed=0):
    net, layout, flat = tiny_cnn((1, 4, 4, 1), seed=seed)
    k = G.gaussian_kernel(3, 0.8)
    op = operators.Operator("blur", kern=k)
    x_true = G.synth_image(seed + 40, 1, 8, 8).astype(np.float64)
    y = op.A(x_true) + 0.02 * RNG.standard_normal((1, 8, 8))
    return net, layout, flat, op, x_true, y


def _solve_loss(net, op, y, x_true, lam, tau):
    x, info = solver.solve_image(net, op, y, op.AT(y), lam, tau, 0.8, math.inf, 1e-14, 20000)
    assert info["status"] == solver.CONVERGED
    return adjoint.mse_loss_grad(x, x_true)[0], x


def test_implicit_gradient_matches_finite_differences():
    net, layout, flat, op, x_true, y = _tiny_problem()
    lam, tau = 0.1, 0.7
    loss, xbar = _solve_loss(net, op, y, x_true, lam, tau)
    v = adjoint.mse_loss_grad(xbar, x_true)[1]
    gth, glam, info = adjoint.backward_image(net, op, y, xbar, v, lam, tau, "implicit",
                                             tol=1e-13, max_iter=20000)
    assert info["adj_converged"]
    h = 1e-5
    lp = _solve_loss(net, op, y, x_true, lam + h, tau)[0]
    lm = _solve_loss(net, op, y, x_true, lam - h, tau)[0]
    assert abs((lp - lm) / (2 * h) - glam) < 1e-6 * max(abs(glam), 1e-3)
    flat64 = np.asarray(flat, np.float64)
    idx = np.random.default_rng(5).choice(flat64.size, 8, replace=False)
    for i in idx:
        fp, fm = flat64.copy(), flat64.copy()
        fp[i] += h
        fm[i] -= h
        netp = nets.Net(net.ops, net.wtab, fp)
        netm = nets.Net(net.ops, net.wtab, fm)
        fd = (_solve_loss(netp, op, y, x_true, lam, tau)[0]
              - _solve_loss(netm, op, y, x_true, lam, tau)[0]) / (2 * h)
        assert abs(fd - gth[i]) < 1e-6 * max(np.max(np.abs(gth)), 1e-6), (i, fd, gth[i])


def test_implicit_gradient_matches_unrolled_autograd(torch64):
    import torch_ref
    torch = torch64
    net, layout, flat, op, x_true, y = _tiny_problem(seed=1)
    lam, tau, beta = 0.1, 0.7, 0.8
    loss, xbar = _solve_loss(net, op, y, x_true, lam, tau)
    v = adjoint.mse_loss_grad(xbar, x_true)[1]
    gth, glam, _ = adjoint.backward_image(net, op, y, xbar, v, lam, tau, "implicit",
                                          tol=1e-13, max_iter=20000)
    W = torch_ref.unpack(flat, layout)
    for t in W.values():
        t.requires_grad_(True)
    tl = torch.tensor(lam, requires_grad=True)
    k = torch.tensor(op.k)
    ty = torch.tensor(y)

    def A(x):  # circular convolution as explicit roll sums
        out = torch.zeros_like(x)
        for a in range(3):
            for b in range(3):
                out = out + k[a, b] * torch.roll(x, (a - 1, b - 1), (-2, -1))
        return out

    def AT(x):
        out = torch.zeros_like(x)
        for a in range(3):
            for b in range(3):
                out = out + k[a, b] * torch.roll(x, (1 - a, 1 - b), (-2, -1))
        return out

    def grad_g(z):
        zz = z.detach().requires_grad_(True) if not z.requires_grad else z
        g = torch_ref.g_of(lambda q: torch_ref.cnn(W, q[None], 3)[0], zz)
        return torch.autograd.grad(g, zz, create_graph=True)[0]

    x = AT(ty)
    xp = x
    for _ in range(400):
        z = x + beta * (x - xp)
        xn = z - tau * (AT(A(z) - ty) + tl * grad_g(z))
        xp, x = x, xn
    loss_t = ((x - torch.tensor(x_true)) ** 2).mean()
    grads = torch.autograd.grad(loss_t, [tl] + list(W.values()))
    g_unrolled = np.concatenate([t.detach().numpy().ravel() for t in grads[1:]])
    assert abs(float(grads[0]) - glam) < 1e-6 * max(abs(glam), 1e-4)
    np.testing.assert_allclose(g_unrolled, gth, atol=1e-6 * np.max(np.abs(gth)))


def test_lambda_gradient_closed_form_tikhonov():
    """N == 0: xbar = (A^T A + lam I)^{-1} A^T y, dl/dlam = -v^T (A^T A + lam I)^{-1} xbar."""
    net = zero_tail_unet(c=1)
    h = w = 16
    k = G.gaussian_kernel(5, 1.2).astype(np.float64)
    op = operators.Operator("blur", kern=k)
    x_true = G.synth_image(8, 1, h, w).astype(np.float64)
    y = op.A(x_true) + 0.02 * rnd(1, h, w)
    lam, tau = 0.1, 0.75
    xbar, _ = solver.solve_image(net, op, y, op.AT(y), lam, tau, 0.8, math.inf, 1e-14, 20000)
    v = adjoint.mse_loss_grad(xbar, x_true)[1]
    _, glam, info = adjoint.backward_image(net, op, y, xbar, v, lam, tau, "implicit", 1e-14, 20000)
    kp = np.zeros((h, w))
    kp[:5, :5] = k
    kp = np.roll(kp, (-2, -2), axis=(0, 1))
    D = np.abs(np.fft.fft2(kp)) ** 2 + lam
    sol = np.real(np.fft.ifft2(np.fft.fft2(xbar[0]) / D))
    ref = -float(np.sum(v[0] * sol))
    assert abs(glam - ref) < 1e-9 * abs(ref)


# ------------------------------------------------------------ warm start


def test_adam_matches_torch(torch64):
    torch = torch64
    p0 = rnd(10)
    opt_o = warmstart.Adam(10, lr=1e-2)
    tp = torch.tensor(p0, requires_grad=True)
    opt_t = torch.optim.Adam([tp], lr=1e-2)
    p = p0.copy()
    for it in range(5):
        g = rnd(10)
        p = opt_o.step(p, g)
        opt_t.zero_grad()
        tp.grad = torch.tensor(g)
        opt_t.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_warm_start_gradient_matches_autograd(torch64):
    import torch_ref
    torch = torch64
    chans = [3, 5, 5, 3]
    net, layout, flat = tiny_cnn(tuple(chans), act="relu")
    atys = RNG.uniform(0, 1, (2, 3, 8, 8))
    tg = RNG.uniform(0, 1, (2, 3, 8, 8))
    loss, grad = warmstart.warm_loss_grad(net, atys, tg)
    W = torch_ref.unpack(flat, layout)
    for t in W.values():
        t.requires_grad_(True)
    ta = torch.tensor(atys)
    out = ta + torch_ref.cnn(W, ta, 3, act="relu")
    lt = ((out - torch.tensor(tg)) ** 2).mean()
    grads = torch.autograd.grad(lt, list(W.values()))
    np.testing.assert_allclose(loss, float(lt), rtol=1e-12)
    np.testing.assert_allclose(grad, np.concatenate([t.numpy().ravel() for t in grads]),
                               rtol=1e-10, atol=1e-13)


def test_workload_is_deterministic_and_shaped():
    cfg = get_config("C1a", n=2, h=32, w=32)
    a, b = workload(cfg), workload(cfg)
    assert np.array_equal(a["x_true"], b["x_true"]) and np.array_equal(a["kern"], b["kern"])
    assert a["kern"].shape == (2, 25, 25)
    assert abs(float(a["kern"][0].sum()) - 1.0) < 1e-5
    assert a["x_true"].min() >= 0 and a["x_true"].max() <= 1


def fourier_heavy_ball_average(Kf, Yf, X0f, lam, tau, beta, K, hw):
    """Averaging step of Algorithm 1 in the Fourier domain (N == 0, circular blur,
    no restart): run K updates keeping Z_k and the step norms, K0 = first
    minimiser of the step over floor(K/2) < k < K-1, x_hat = mean(Z_0..Z_K0)."""
    q = 1.0 - tau * (np.abs(Kf) ** 2 + lam)
    b = tau * np.conj(Kf) * Yf
    X, Xp = X0f.copy(), X0f.copy()
    Zs, steps = [], []
    for _ in range(K):
        Z = X + beta * (X - Xp)
        Xn = q * Z + b
        Zs.append(Z)
        steps.append(math.sqrt(float(np.sum(np.abs(Xn - X) ** 2)) / hw))
        Xp, X = X, Xn
    best = None
    for k in range(K // 2 + 1, K - 1):
        if best is None or steps[k] < steps[best]:
            best = k
    return sum(Zs[:best + 1]) / (best + 1), best


@pytest.mark.parametrize("K,beta", [(5, 0.8), (12, 0.8), (40, 0.5), (41, 0.95)])
def test_averaging_step_matches_fourier_closed_form(K, beta):
    """x_hat of the averaging step (Algorithm 1) against an independent per-frequency
    run: same K0 and the same average of the extrapolated points z^k."""
    net = zero_tail_unet()
    h = w = 16
    k = G.motion_kernel(21, 7).astype(np.float64)
    op = operators.Operator("blur", kern=k)
    x_true = G.synth_image(5, 1, h, w).astype(np.float64)
    y = op.A(x_true) + 0.02 * rnd(1, h, w)
    x0 = op.AT(y)
    lam, tau = 0.1, 0.75
    x, info = solver.solve_image(net, op, y, x0, lam, tau, beta, math.inf, 0.0, K, average=True)
    kp = np.zeros((h, w))
    kp[:7, :7] = k
    kp = np.roll(kp, (-3, -3), axis=(0, 1))
    Kf = np.fft.fft2(kp)
    Xa, K0 = fourier_heavy_ball_average(Kf, np.fft.fft2(y[0]), np.fft.fft2(x0[0]), lam, tau,
                                        beta, K, h * w)
    assert info["K0"] == K0 and K // 2 < K0 < K - 1
    np.testing.assert_allclose(x[0], np.real(np.fft.ifft2(Xa)), atol=1e-11)


def test_averaging_step_of_a_constant_sequence_is_that_point():
    """At a fixed point every z^k is that point, so is their average; K0 is the
    first minimiser inside floor(K/2) < k < K-1; the window is empty below K = 5."""
    zs = [np.full((2, 3), 0.25)] * 7
    x, K0 = solver.averaging_step(zs, [1.0, 0.5, 0.4, 0.3, 0.3, 0.2, 0.1])
    assert K0 == 5  # window {4, 5}; k = 6 (the last step, 0.1) is outside it
    np.testing.assert_array_equal(x, zs[0])
    _, K0 = solver.averaging_step(zs, [1.0, 0.5, 0.4, 0.3, 0.2, 0.2, 0.1])
    assert K0 == 4  # tie: the first minimiser
    with pytest.raises(ValueError):
        solver.averaging_step(zs[:4], [1.0, 0.5, 0.4, 0.3])


def test_inpainting_prox_optimality_condition():
    """prox_{tau f}(v) for the mask is the minimiser: its gradient condition
    (x - v)/tau + M^T(M x - y) = 0 holds, and a perturbation raises the objective."""
    rng = np.random.default_rng(21)
    m = G.bernoulli_mask(4, 12, 10, 0.3)
    op = operators.Operator("mask", mask=m)
    y = m * rng.standard_normal((3, 12, 10))
    v = rng.standard_normal((3, 12, 10))
    tau = 0.7
    x = op.prox_f(v, y, tau)
    np.testing.assert_allclose((x - v) / tau + op.AT(op.A(x) - y), 0.0, atol=1e-13)
    obj = lambda u: op.f(u, y) + 0.5 / tau * float(np.sum((u - v) ** 2))
    assert obj(x) < obj(x + 1e-3 * rng.standard_normal(x.shape))
    np.testing.assert_array_equal(x[:, m[0] == 0] if m.ndim == 3 else x[:, m == 0],
                                  v[:, m[0] == 0] if m.ndim == 3 else v[:, m == 0])


def test_proximal_variant_reaches_tikhonov_fixed_point():
    """With N == 0 (g = 1/2||x||^2) the fixed point of x = prox_{tau f}(x - tau lam x)
    is M y / (M + lam), the same Tikhonov point as the gradient form."""
    lam, tau = 0.1, 0.75
    net = zero_tail_unet(c=1)
    m = G.bernoulli_mask(9, 16, 16, 0.3)
    op = operators.Operator("mask", mask=m)
    y = m * rnd(1, 16, 16)
    x, info = solver.solve_image(net, op, y, op.AT(y), lam, tau, 0.8, math.inf, 1e-13, 5000,
                                 prox=True)
    assert info["status"] == solver.CONVERGED
    np.testing.assert_allclose(x, m * y / (m + lam), atol=1e-10)


def test_mri_operator_is_masked_unitary_dft_brute_force():
    """A x = M . F x with F the orthonormal DFT, written out as a double sum over
    pixels (no FFT) on an 8 x 6 complex image stored as (re, im) planes."""
    h, w = 8, 6
    m = G.cartesian_mask(3, h, w, 2, 0.2)
    op = operators.Operator("mri", mask=m)
    x = rnd(2, h, w)
    xc = x[0] + 1j * x[1]
    ref = np.zeros((h, w), complex)
    for u in range(h):
        for v in range(w):
            s = 0j
            for a in range(h):
                for b in range(w):
                    s += xc[a, b] * np.exp(-2j * np.pi * (u * a / h + v * b / w))
            ref[u, v] = m[u, v] * s / np.sqrt(h * w)
    np.testing.assert_allclose(op.A(x), np.stack([ref.real, ref.imag]), atol=1e-12)
    # F unitary and M a projection: ||A x|| <= ||x||, equality on a fully sampled mask
    full = operators.Operator("mri", mask=np.ones((h, w)))
    assert abs(np.linalg.norm(full.A(x)) - np.linalg.norm(x)) < 1e-12
    assert np.linalg.norm(op.A(x)) <= np.linalg.norm(x) + 1e-12


def test_mri_prox_and_tikhonov_fixed_point():
    """prox_{tau f} for MRI meets its optimality condition, and with N == 0 the
    inertial solve reaches the Tikhonov point F^{-1}(M y / (M + lambda))."""
    h, w = 16, 16
    m = G.cartesian_mask(5, h, w, 4, 0.125)
    op = operators.Operator("mri", mask=m)
    y = op.A(rnd(2, h, w)) + m * 0.05 * rnd(2, h, w)
    v = rnd(2, h, w)
    tau, lam = 0.7, 0.1
    x = op.prox_f(v, y, tau)
    np.testing.assert_allclose((x - v) / tau + op.AT(op.A(x) - y), 0.0, atol=1e-12)
    net = zero_tail_unet(c=2)
    ref = np.fft.ifft2(m * (y[0] + 1j * y[1]) / (m + lam), norm="ortho")
    for prox in (False, True):
        xs, info = solver.solve_image(net, op, y, op.AT(y), lam, 0.75, 0.8, math.inf, 1e-13,
                                      5000, prox=prox)
        assert info["status"] == solver.CONVERGED
        np.testing.assert_allclose(xs, np.stack([ref.real, ref.imag]), atol=1e-10)


def test_rician_data_term_is_the_negative_log_likelihood():
    """f(x, y) + y^2/(2 s^2) - log(y / s^2) is -log p(y | x) of the Rician density
    (App. E): exp of its negative integrates to 1 over y >= 0, for several x."""
    from scipy.integrate import quad
    s = 0.1
    op = operators.Operator("rician", sigma=s)
    for xv in (0.0, 0.05, 0.3, 0.9):
        dens = lambda y: math.exp(-(op.f(np.array([xv]), np.array([y])) + y * y / (2 * s * s)
                                    - math.log(y / (s * s)))) if y > 0 else 0.0
        total, _ = quad(dens, 0.0, xv + 12 * s, limit=200)
        assert abs(total - 1.0) < 1e-7, (xv, total)


def test_rician_gradient_and_hessian_finite_differences():
    s = 0.1
    op = operators.Operator("rician", sigma=s)
    x = RNG.uniform(0.05, 1.0, (1, 6, 5))
    y = np.sqrt((x + s * rnd(1, 6, 5)) ** 2 + (s * rnd(1, 6, 5)) ** 2)
    g = op.grad_f(x, y)
    h = 1e-7
    for idx in [(0, 0, 0), (0, 3, 2), (0, 5, 4)]:
        e = np.zeros_like(x)
        e[idx] = h
        fd = (op.f(x + e, y) - op.f(x - e, y)) / (2 * h)
        assert abs(fd - g[idx]) < 1e-6 * max(1.0, abs(g[idx]))
    u = rnd(1, 6, 5)
    eps = 1e-6
    fd = (op.grad_f(x + eps * u, y) - op.grad_f(x - eps * u, y)) / (2 * eps)
    np.testing.assert_allclose(op.hvp_f(x, y, u), fd, rtol=1e-6, atol=1e-4)
    # special case: y = 0 leaves the quadratic term only
    np.testing.assert_allclose(op.grad_f(x, np.zeros_like(x)), x / s ** 2, rtol=1e-15)
