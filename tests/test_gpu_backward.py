"""Implicit backward (App. D.1.2) on the GPU vs the FP64 oracle, through the C ABI.

The fixed point xbar is computed by the oracle (FP64, tight tolerance) and rounded
to float32; both sides then differentiate the loss l = mean((xbar - x*)^2) at the
same point.  Tolerances: FP32 convolutions 1e-4 relative on the parameter gradient
(sums of ~1e5 products per weight in FP32) and on dl/dlambda; FP16 convolutions
2e-2 (the second-order reverse pass multiplies two rounded activations).
"""
import numpy as np
import pytest

from gpu_common import ctx_for, op_for, rel, setup, to_np
from oracle import adjoint, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_19705_gb300 import build
    build.build()


def B():
    from paper_2605_19705_gb300 import binding
    return binding


def _problem(name="C3", **over):
    cfg, wl, net, ops, ys = setup(name, **over)
    x0 = np.stack([ops[i].AT(ys[i].astype(np.float64)) for i in range(len(ops))])
    xb, infos = solver.solve_batch(net, ops, ys.astype(np.float64), x0, cfg["lam"], cfg["tau"],
                                   cfg["beta"], np.inf, 1e-10, 3000)
    xbar = xb.astype(np.float32)
    loss, v = adjoint.mse_loss_grad(xbar.astype(np.float64), wl["x_true"])
    return cfg, wl, net, ops, ys, xbar, v


def _gpu_backward(cfg, wl, ys, xbar, v, prec, mode, tol=1e-7, max_iter=3000, beta=0.0,
                  allow_maxiter=False):
    b = B()
    ctx = ctx_for(cfg, wl, prec)
    op = op_for(cfg, wl)
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"])
    adj = b.make_adj(mode, tol, max_iter, beta)
    nparams = wl["weights"].size
    dth = torch.zeros(nparams, device="cuda")
    dlam = torch.zeros(1, device="cuda")
    info = b.InfoBuffers(ys.shape[0])
    st = b.ideq_solve_backward(ctx, op, torch.tensor(ys, device="cuda"),
                               torch.tensor(xbar, device="cuda"),
                               torch.tensor(v.astype(np.float32), device="cuda"), params, adj,
                               dth, dlam, info, allow_maxiter=allow_maxiter)
    torch.cuda.synchronize()
    return dth.double().cpu().numpy(), float(dlam.item()), info, st


def _oracle_backward(cfg, net, ops, ys, xbar, v, mode, tol=1e-9, max_iter=5000, beta=0.0):
    return adjoint.backward_batch(net, ops, ys.astype(np.float64), xbar.astype(np.float64), v,
                                  cfg["lam"], cfg["tau"], mode, tol, max_iter, beta)


@pytest.mark.parametrize("name,over", [("C3", dict(n=1, h=32, w=32)),
                                       ("C0", dict(n=2, h=24, w=32))])
def test_jfb_gradient_matches_oracle(name, over):
    cfg, wl, net, ops, ys, xbar, v = _problem(name, **over)
    gth, glam, infos = _oracle_backward(cfg, net, ops, ys, xbar, v, "jfb")
    dth, dlam, info, st = _gpu_backward(cfg, wl, ys, xbar, v, B().IDEQ_FP32, B().IDEQ_ADJ_JFB)
    assert rel(dth, gth) < 1e-4, rel(dth, gth)
    assert abs(dlam - glam) < 1e-4 * abs(glam)


def test_one_adjoint_iteration_is_the_hessian_vector_product():
    """max_iter = 1: u = v + J_R^T v exactly -- pins H_f v + lambda H_g v."""
    cfg, wl, net, ops, ys, xbar, v = _problem("C3", n=1, h=32, w=32)
    gth, glam, infos = _oracle_backward(cfg, net, ops, ys, xbar, v, "implicit", tol=1e-300,
                                        max_iter=1)
    dth, dlam, info, st = _gpu_backward(cfg, wl, ys, xbar, v, B().IDEQ_FP32,
                                        B().IDEQ_ADJ_IMPLICIT, tol=1e-300, max_iter=1,
                                        allow_maxiter=True)
    assert st == B().IDEQ_ADJ_MAXITER
    assert rel(dth, gth) < 1e-4, rel(dth, gth)
    assert abs(dlam - glam) < 1e-4 * abs(glam)


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_implicit_gradient_matches_oracle(beta):
    cfg, wl, net, ops, ys, xbar, v = _problem("C3", n=2, h=32, w=32)
    gth, glam, infos = _oracle_backward(cfg, net, ops, ys, xbar, v, "implicit", tol=1e-9,
                                        beta=beta)
    dth, dlam, info, st = _gpu_backward(cfg, wl, ys, xbar, v, B().IDEQ_FP32,
                                        B().IDEQ_ADJ_IMPLICIT, tol=1e-6, beta=beta)
    assert st == B().IDEQ_OK
    assert all(int(s) == 1 for s in info.status.cpu())
    assert rel(dth, gth) < 1e-4, rel(dth, gth)
    assert abs(dlam - glam) < 1e-4 * abs(glam)


def test_implicit_gradient_fp16_matches_oracle():
    cfg, wl, net, ops, ys, xbar, v = _problem("C3", n=1, h=64, w=64)
    gth, glam, infos = _oracle_backward(cfg, net, ops, ys, xbar, v, "implicit", tol=1e-7)
    dth, dlam, info, st = _gpu_backward(cfg, wl, ys, xbar, v, B().IDEQ_FP16,
                                        B().IDEQ_ADJ_IMPLICIT, tol=1e-4)
    assert rel(dth, gth) < 2e-2, rel(dth, gth)
    assert abs(dlam - glam) < 2e-2 * abs(glam)


def test_batch_gradient_is_the_sum_of_image_gradients_at_full_size():
    """C3 shape (128^2 RGB, half-width U-Net): the gradient of a batch of two images
    equals the sum of the two single-image gradients (images never interact)."""
    cfg, wl, net, ops, ys = setup("C3", n=2)
    b = B()
    rng = np.random.default_rng(2)
    xbar = np.clip(ys + 0.02 * rng.standard_normal(ys.shape), 0, 1).astype(np.float32)
    v = (2.0 * (xbar - wl["x_true"]) / xbar.size).astype(np.float64)
    d2, l2, _, _ = _gpu_backward(cfg, wl, ys, xbar, v, b.IDEQ_FP32, b.IDEQ_ADJ_IMPLICIT, tol=1e-4)
    parts = []
    for i in range(2):
        wl1 = dict(wl)
        wl1["kern"] = wl["kern"][i:i + 1]
        cfg1 = dict(cfg, n=1)
        parts.append(_gpu_backward(cfg1, wl1, ys[i:i + 1], xbar[i:i + 1], v[i:i + 1],
                                   b.IDEQ_FP32, b.IDEQ_ADJ_IMPLICIT, tol=1e-4))
    assert rel(d2, parts[0][0] + parts[1][0]) < 1e-4
    assert abs(l2 - (parts[0][1] + parts[1][1])) < 1e-4 * abs(l2)


def test_lambda_gradient_matches_finite_differences_of_gpu_solves():
    """dl/dlambda from the backward vs central differences of FP32 GPU solves."""
    cfg, wl, net, ops, ys = setup("C3", n=1, h=32, w=32)
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    op = op_for(cfg, wl)
    ty = torch.tensor(ys, device="cuda")
    xt = torch.tensor(wl["x_true"], device="cuda", dtype=torch.float64)

    def loss(lam):
        p = b.make_params(lam, cfg["tau"], cfg["beta"], tol=1e-6, max_iter=5000)
        x, _ = b.ideq_solve(ctx, op, ty, p, allow_maxiter=True)
        return float(((x.double() - xt) ** 2).mean()), x

    l0, x = loss(cfg["lam"])
    v = (2.0 * (x.double() - xt) / x.numel()).float().contiguous()
    adj = b.make_adj(b.IDEQ_ADJ_IMPLICIT, 1e-6, 5000, 0.0)
    dth = torch.zeros(wl["weights"].size, device="cuda")
    dlam = torch.zeros(1, device="cuda")
    b.ideq_solve_backward(ctx, op, ty, x, v, b.make_params(cfg["lam"], cfg["tau"], cfg["beta"]),
                          adj, dth, dlam)
    h = 2e-3
    fd = (loss(cfg["lam"] + h)[0] - loss(cfg["lam"] - h)[0]) / (2 * h)
    assert abs(fd - float(dlam)) < 3e-2 * abs(fd), (fd, float(dlam))


def test_autograd_function_backward_equals_direct_call():
    from paper_2605_19705_gb300 import autograd as IA
    cfg, wl, net, ops, ys = setup("C3", n=1, h=32, w=32)
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    op = op_for(cfg, wl)
    w = torch.tensor(wl["weights"], device="cuda", requires_grad=True)
    lam = torch.tensor(cfg["lam"], device="cuda", requires_grad=True)
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], tol=1e-6, max_iter=3000)
    adj = IA.make_adj(b.IDEQ_ADJ_IMPLICIT, 1e-6, 3000)
    ty = torch.tensor(ys, device="cuda")
    x = IA.ideq_restore(w, lam, ty, ctx, op, params, adj)
    xt = torch.tensor(wl["x_true"], device="cuda")
    loss = ((x - xt) ** 2).mean()
    gw, gl = torch.autograd.grad(loss, [w, lam])
    v = (2.0 * (x.detach() - xt) / x.numel()).contiguous()
    dth = torch.zeros_like(w)
    dlam = torch.zeros(1, device="cuda")
    b.ideq_solve_backward(ctx, op, ty, x.detach().contiguous(), v, params, adj, dth, dlam)
    assert torch.allclose(gw, dth, rtol=1e-5, atol=1e-12)
    assert abs(float(gl) - float(dlam)) <= 1e-5 * abs(float(dlam))


@pytest.mark.parametrize("name,over", [("C1a", dict(n=2, h=64, w=64)),
                                       ("C1a", dict(n=1, h=40, w=56)),
                                       ("C3", dict(n=2, h=64, w=64))])
def test_tensor_core_weight_gradient_matches_simt(name, over):
    """The tcgen05 weight gradient (3x3 and stride-2 2x2 convs with 64k input and
    output channels, MN-major operands, split-K with a fixed-order reduction) against
    the SIMT weight-gradient kernel on the same FP16 activations and cotangents
    (IDEQ_WGRAD_TC=0 keeps a context on the SIMT kernel): both accumulate in FP32
    over the pixels, so only the summation order differs.  JFB mode, the dual
    (pcot x input + tcot x tangent) form of App. D.1.2's parameter gradient.  The
    ragged 40 x 56 case has partial 64-pixel boxes and levels narrower than a box."""
    import os
    cfg, wl, net, ops, ys = setup(name, **over)
    b = B()
    rng = np.random.default_rng(9)
    xbar = np.clip(ys + 0.05 * rng.standard_normal(ys.shape), 0, 1).astype(np.float32)
    v = (2.0 * (xbar - wl["x_true"]) / xbar.size).astype(np.float64)
    out = []
    for simt in (False, True):
        if simt:
            os.environ["IDEQ_WGRAD_TC"] = "0"
        try:
            out.append(_gpu_backward(cfg, wl, ys, xbar, v, b.IDEQ_FP16, b.IDEQ_ADJ_JFB))
        finally:
            os.environ.pop("IDEQ_WGRAD_TC", None)
    (d_tc, l_tc, _, _), (d_simt, l_simt, _, _) = out
    assert np.isfinite(d_tc).all()
    assert rel(d_tc, d_simt) < 1e-4, rel(d_tc, d_simt)
    assert l_tc == l_simt  # dl/dlambda does not involve the weight gradient


def test_train_step_is_solve_backward_and_adam():
    """ideq_train_step = ideq_solve + MSE loss + ideq_solve_backward + one Adam step
    on theta: its gradient equals the direct calls' on a fresh context with the same
    weights, its loss equals mean((x_hat - x*)^2), and the new weights equal
    torch.optim.Adam's step on that gradient."""
    cfg, wl, net, ops, ys = setup("C3", n=2, h=32, w=32)
    b = B()
    op = op_for(cfg, wl)
    ty = torch.tensor(ys, device="cuda")
    xt = torch.tensor(wl["x_true"], device="cuda")
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], tol=1e-5, max_iter=3000)
    adj = b.make_adj(b.IDEQ_ADJ_IMPLICIT, 1e-5, 3000, 0.0)
    w0 = torch.tensor(wl["weights"], device="cuda")
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    g = torch.zeros_like(w0)
    dlam = torch.zeros(1, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    lr = 1e-3
    x = b.ideq_train_step(ctx, op, ty, xt, params, adj, lr, dl_dtheta=g, dl_dlambda=dlam,
                          loss=loss)
    # the same gradient from the direct calls on a fresh context
    ref = ctx_for(cfg, wl, b.IDEQ_FP32)
    xr, _ = b.ideq_solve(ref, op, ty, params)
    v = (2.0 * (xr - xt) / xr.numel()).contiguous()
    gr = torch.zeros_like(w0)
    lr_ = torch.zeros(1, device="cuda")
    b.ideq_solve_backward(ref, op, ty, xr, v, params, adj, gr, lr_)
    torch.cuda.synchronize()
    assert torch.equal(x, xr)
    lo = float(((xr.double() - xt.double()) ** 2).mean())
    assert abs(float(loss) - lo) < 1e-9 * lo  # two FP64 reductions in different orders
    assert torch.allclose(g, gr, rtol=1e-5, atol=1e-12)
    assert abs(float(dlam) - float(lr_)) <= 1e-5 * abs(float(lr_))
    # weights after the step: torch's Adam on the same gradient
    p = w0.clone().requires_grad_(True)
    opt = torch.optim.Adam([p], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    p.grad = gr.clone()
    opt.step()
    # the context now solves with the updated weights: compare through a solve
    ctx_new = b.Context(b.net_desc(cfg["net"], cfg["c"]), p.detach().contiguous(), b.IDEQ_FP32)
    x1, _ = b.ideq_solve(ctx, op, ty, params)
    x2, _ = b.ideq_solve(ctx_new, op, ty, params)
    assert rel(to_np(x1), to_np(x2)) < 1e-5


def test_autograd_raises_on_unconverged_adjoint():
    """A capped implicit adjoint solve is reported, not silently differentiated."""
    from paper_2605_19705_gb300 import autograd as IA
    cfg, wl, net, ops, ys = setup("C3", n=1, h=32, w=32)
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    op = op_for(cfg, wl)
    w = torch.tensor(wl["weights"], device="cuda", requires_grad=True)
    lam = torch.tensor(cfg["lam"], device="cuda", requires_grad=True)
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], tol=1e-6, max_iter=3000)
    adj = IA.make_adj(b.IDEQ_ADJ_IMPLICIT, 1e-12, 2)  # two adjoint iterations at most
    x = IA.ideq_restore(w, lam, torch.tensor(ys, device="cuda"), ctx, op, params, adj)
    loss = ((x - torch.tensor(wl["x_true"], device="cuda")) ** 2).mean()
    with pytest.raises(b.IdeqError) as e:
        torch.autograd.grad(loss, [w, lam])
    assert e.value.status == b.IDEQ_ADJ_MAXITER
