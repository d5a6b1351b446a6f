"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative 2-norm error against the oracle):
  FP32 arithmetic: 1e-5 for operators, the regulariser gradient, single steps and
    full solves (float32 rounding, ~6e-8 per operation, accumulated over a few
    hundred dependent operations per output and damped by the contractive
    iteration).
  BF16 network convolutions: BF16 rounds every activation to 8 significant bits
    (relative error <= 2^-9); about 70 rounded layers in the forward and reverse
    passes accumulate to ~1% of N(z) and J_N^T r, which are ~0.2-0.4 of ||grad g||,
    hence 1e-2 on grad g; the solve damps it by lambda tau, hence 2e-3 on x_hat
    and PSNR within 0.05 dB.
  FP16 network convolutions: 11 significant bits (relative error <= 2^-12), 8x
    finer than BF16: 2e-3 on grad g, 2e-3 on x_hat, PSNR within 0.05 dB.
"""
import math

import numpy as np
import pytest

from gpu_common import ctx_for, op_for, rel, setup, to_np
from oracle import nets, solver

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


PREC = {"fp32": lambda: B().IDEQ_FP32, "bf16": lambda: B().IDEQ_BF16,
        "fp16": lambda: B().IDEQ_FP16, "fp16_fp8": lambda: B().IDEQ_FP16_FP8,
        "bf16_fp8": lambda: B().IDEQ_BF16_FP8}


# ---------------------------------------------------------------- operators


@pytest.mark.parametrize("name,over", [
    ("C1a", dict(n=2, h=40, w=56)),                                   # 25x25 motion, ragged tiles
    ("C1b", dict(n=2, h=40, w=56)),                                   # mask
    ("C4", dict(n=2, h=40, w=56)),                                    # saturation after 15x15 blur
    ("C0", dict(n=1)),                                                # 9x9 Gaussian, grey
])
def test_operators_match_oracle(name, over):
    cfg, wl, net, ops, ys = setup(name, **over)
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    op = op_for(cfg, wl)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, ys.shape).astype(np.float32)
    r = rng.standard_normal(ys.shape).astype(np.float32)
    tx, tr = torch.tensor(x, device="cuda"), torch.tensor(r, device="cuda")
    Ax = to_np(b.ideq_apply_A(ctx, op, tx))
    ATr = to_np(b.ideq_apply_AT(ctx, op, tr))
    ref_A = np.stack([ops[i].A(x[i].astype(np.float64)) for i in range(len(ops))])
    ref_AT = np.stack([ops[i].AT(r[i].astype(np.float64)) for i in range(len(ops))])
    assert rel(Ax, ref_A) < 1e-6
    assert rel(ATr, ref_AT) < 1e-6
    if cfg["op"] == "satblur":
        JT = to_np(b.ideq_apply_AT(ctx, op, tr, lin_point=tx))
        ref = np.stack([ops[i].JAT(x[i].astype(np.float64), r[i].astype(np.float64))
                        for i in range(len(ops))])
        assert rel(JT, ref) < 1e-6


def test_operator_argument_errors():
    cfg, wl, net, ops, ys = setup("C0")
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    k = torch.ones(1, 4, 4, device="cuda")  # even kernel size is rejected
    op = b.make_operator(b.IDEQ_OP_BLUR, k)
    x = torch.zeros(1, 1, 64, 64, device="cuda")
    with pytest.raises(b.IdeqError) as e:
        b.ideq_apply_A(ctx, op, x)
    assert e.value.status == b.IDEQ_ERR_ARG
    with pytest.raises(b.IdeqError):
        b.ideq_grad_reg(ctx, torch.zeros(1, 3, 64, 64, device="cuda"))  # wrong channels


# ---------------------------------------------------------------- regulariser


@pytest.mark.parametrize("name,over,prec,tol", [
    ("C0", dict(n=1), "fp32", 1e-5),
    ("C0", dict(n=2, h=37, w=45), "fp32", 1e-5),
    ("C1a", dict(n=1, h=64, w=64), "fp32", 1e-5),
    ("C1a", dict(n=2, h=40, w=56), "fp32", 1e-5),
    ("C1a", dict(n=1, h=64, w=64), "bf16", 1e-2),
    ("C1a", dict(n=2, h=40, w=56), "bf16", 1e-2),
    ("C1a", dict(n=1, h=64, w=64), "fp16", 2e-3),
    ("C1a", dict(n=2, h=40, w=56), "fp16", 2e-3),
    ("C1a", dict(n=1), "fp16", 2e-3),           # 256^2: halo form of the 64-channel convs
    ("C1a", dict(n=1), "bf16", 1e-2),
    ("C1a", dict(n=1, h=136, w=200), "fp16", 2e-3),  # halo tiles with ragged row ends
    ("C3", dict(n=1, h=32, w=32), "fp32", 1e-5),
    # half-width U-Net: 32-channel layers on 64-byte K rows and 32-wide N tiles
    ("C3", dict(n=1, h=64, w=64), "fp16", 2e-3),
    ("C3", dict(n=2, h=40, w=56), "bf16", 1e-2),
    ("C3", dict(n=1), "fp16", 2e-3),
    ("C3", dict(n=1), "bf16", 1e-2),
    ("C3", dict(n=1, h=136, w=200), "fp16", 2e-3),  # 32-channel halo tiles, ragged rows
    ("C5", dict(n=1), "fp16", 2e-3),            # 2-channel (complex) input and output
    # e4m3 operands (unit roundoff 2^-4) on the 256- and 512-channel convs, averaged
    # over K >= 1024 terms and damped by the 0.1 residual gains: measured 1.2e-2
    ("C1a", dict(n=1, h=64, w=64), "fp16_fp8", 3e-2),
    ("C1a", dict(n=1), "fp16_fp8", 3e-2),
    ("C1a", dict(n=2, h=40, w=56), "bf16_fp8", 3e-2),
])
def test_grad_reg_matches_oracle(name, over, prec, tol):
    cfg, wl, net, ops, ys = setup(name, **over)
    b = B()
    ctx = ctx_for(cfg, wl, PREC[prec]())
    z = np.random.default_rng(5).uniform(0, 1, ys.shape).astype(np.float32)
    gval = torch.zeros(z.shape[0], dtype=torch.float64, device="cuda")
    g = to_np(b.ideq_grad_reg(ctx, torch.tensor(z, device="cuda"), g_val=gval))
    for i in range(z.shape[0]):
        ref, gv = nets.grad_g(net, z[i].astype(np.float64))
        assert rel(g[i], ref) < tol, (i, rel(g[i], ref))
        assert abs(float(gval[i]) - gv) < tol * gv


# ---------------------------------------------------------------- iteration


def _oracle_solve(cfg, net, ops, ys, **kw):
    x0 = np.stack([ops[i].AT(ys[i].astype(np.float64)) for i in range(len(ops))])
    p = dict(lam=cfg["lam"], tau=cfg["tau"], beta=cfg["beta"], B=cfg["B"], tol=cfg["tol"],
             max_iter=cfg["max_iter"])
    p.update(kw)
    return solver.solve_batch(net, ops, ys.astype(np.float64), x0, p["lam"], p["tau"], p["beta"],
                              p["B"], p["tol"], p["max_iter"])


def _gpu_solve(cfg, wl, ys, prec, **kw):
    b = B()
    ctx = ctx_for(cfg, wl, prec)
    op = op_for(cfg, wl)
    p = dict(lam=cfg["lam"], tau=cfg["tau"], beta=cfg["beta"], B=cfg["B"], tol=cfg["tol"],
             max_iter=cfg["max_iter"])
    p.update(kw)
    params = b.make_params(p["lam"], p["tau"], p["beta"], p["B"], p["tol"], p["max_iter"])
    info = b.InfoBuffers(ys.shape[0])
    x, st = b.ideq_solve(ctx, op, torch.tensor(ys, device="cuda"), params, info=info,
                         allow_maxiter=True)
    torch.cuda.synchronize()
    return to_np(x), info, st


def test_solve_c0_fixed_50_steps_fp32():
    cfg, wl, net, ops, ys = setup("C0")
    xo, infos = _oracle_solve(cfg, net, ops, ys)
    xg, info, st = _gpu_solve(cfg, wl, ys, B().IDEQ_FP32)
    assert int(info.iters[0]) == 50 == infos[0]["iters"]
    assert rel(xg, xo) < 1e-5
    assert abs(float(info.energy[0]) - infos[0]["energy"]) < 1e-5 * abs(infos[0]["energy"])


@pytest.mark.parametrize("B_,tol", [(0.05, 1e-4), (math.inf, 1e-4)])
def test_solve_c0_restart_and_stopping_fp32(B_, tol):
    cfg, wl, net, ops, ys = setup("C0", n=2, h=48, w=40)
    xo, infos = _oracle_solve(cfg, net, ops, ys, B=B_, tol=tol, max_iter=400)
    xg, info, st = _gpu_solve(cfg, wl, ys, B().IDEQ_FP32, B=B_, tol=tol, max_iter=400)
    for i in range(2):
        it = int(info.iters[i])
        assert abs(it - infos[i]["iters"]) <= 1
        assert int(info.restarts[i]) == infos[i]["restarts"]
        assert int(info.status[i]) == infos[i]["status"]
        # the FP32 iterate against the oracle run for exactly the GPU's number of
        # updates (same restarts; the stopping test may flip by one update between
        # FP32 and FP64, so the oracle's own stopping iterate is not the reference)
        xo_i, inf_i = solver.solve_image(net, ops[i], ys[i].astype(np.float64),
                                         ops[i].AT(ys[i].astype(np.float64)), cfg["lam"],
                                         cfg["tau"], cfg["beta"], B_, 0.0, it)
        assert inf_i["restarts"] == int(info.restarts[i])
        assert rel(xg[i], xo_i) < 1e-5, (i, rel(xg[i], xo_i))
    if B_ < math.inf:
        assert min(int(v) for v in info.restarts.cpu()) >= 1


@pytest.mark.parametrize("name", ["C1a", "C1b"])
def test_solve_unet_fp32(name):
    cfg, wl, net, ops, ys = setup(name, n=1, h=64, w=64)
    xg, info, st = _gpu_solve(cfg, wl, ys, B().IDEQ_FP32, max_iter=300)
    it = int(info.iters[0])
    assert int(info.status[0]) == solver.CONVERGED
    # oracle run for exactly the same number of updates (the stopping test may
    # flip by one iteration between FP32 and FP64)
    xo, infos = _oracle_solve(cfg, net, ops, ys, tol=0.0, max_iter=it)
    assert rel(xg, xo) < 1e-5
    xo2, infos2 = _oracle_solve(cfg, net, ops, ys, max_iter=300)
    assert abs(infos2[0]["iters"] - it) <= 1


@pytest.mark.parametrize("name,n,h,w", [("C0", 1, 64, 64), ("C0", 3, 40, 56)])
def test_solve_averaging_step_fp32(name, n, h, w):
    """Averaging step of Algorithm 1 over a fixed run of 50 updates: the same K0
    as the oracle (or, where FP32 iterates reorder two step norms closer than
    1e-4 relative, a K0 the oracle ranks as tied) and x_hat within 1e-5 of the
    oracle's average of z^0 .. z^K0 for that K0."""
    cfg, wl, net, ops, ys = setup(name, n=n, h=h, w=w)
    b = B()
    x0 = np.stack([ops[i].AT(ys[i].astype(np.float64)) for i in range(n)])
    outs = [solver.solve_image(net, ops[i], ys[i].astype(np.float64), x0[i], cfg["lam"],
                               cfg["tau"], cfg["beta"], math.inf, 0.0, 50, keep_history=True,
                               average=True) for i in range(n)]
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], max_iter=50, average=True)
    info = b.InfoBuffers(n)
    x, st = b.ideq_solve(ctx, op_for(cfg, wl), torch.tensor(ys, device="cuda"), params,
                         info=info, allow_maxiter=True)
    xg = to_np(x)
    for i in range(n):
        xo, inf = outs[i]
        k0 = int(info.k0[i])
        assert 25 < k0 < 49
        if k0 != inf["K0"]:
            s = inf["step_hist"]
            assert abs(s[k0] - s[inf["K0"]]) < 1e-4 * s[inf["K0"]]
            xo = np.mean(np.stack(inf["z_hist"][:k0 + 1]), axis=0)
        assert rel(xg[i], xo) < 1e-5


@pytest.mark.parametrize("tol,max_iter", [(1e-4, 400), (0.0, 37), (0.0, 3)])
def test_device_driven_loop_matches_host_loop(tol, max_iter):
    """The solve's CUDA graph (a while node repeating two iterations until no image
    runs) gives the same iterates, counts and statuses as the host-driven loop
    (forced here by recording per-launch profiler events)."""
    cfg, wl, net, ops, ys = setup("C0", n=2, h=48, w=40)
    b = B()
    y = torch.tensor(ys, device="cuda")
    out = []
    for host in (False, True):
        ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
        b.ideq_prof_enable(ctx, host)
        params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], tol=tol, max_iter=max_iter)
        info = b.InfoBuffers(2)
        op = op_for(cfg, wl)
        for _ in range(2):  # the second solve reuses the graph built by the first
            x, st = b.ideq_solve(ctx, op, y, params, info=info, allow_maxiter=True)
        torch.cuda.synchronize()
        out.append((to_np(x), info.iters.cpu().numpy(), info.status.cpu().numpy()))
    (xg, ig, sg), (xh, ih, sh) = out
    assert np.array_equal(ig, ih) and np.array_equal(sg, sh)
    assert np.array_equal(xg, xh)
    if tol == 0.0:
        assert list(ig) == [max_iter, max_iter]


def test_solve_graph_holds_tensor_core_convs():
    """The 16-bit U-Net solve (tcgen05 convs launched with programmatic stream
    serialisation) runs its loop in the device-driven graph and matches the
    host-driven loop bit for bit."""
    cfg, wl, net, ops, ys = setup("C1a", n=2, h=64, w=64)
    b = B()
    y = torch.tensor(ys, device="cuda")
    out = []
    for host in (False, True):
        ctx = ctx_for(cfg, wl, b.IDEQ_FP16)
        b.ideq_prof_enable(ctx, host)
        params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], tol=cfg["tol"], max_iter=60)
        info = b.InfoBuffers(2)
        x, st = b.ideq_solve(ctx, op_for(cfg, wl), y, params, info=info, allow_maxiter=True)
        torch.cuda.synchronize()
        assert b.ideq_solve_graphed(ctx) == (not host)
        out.append((to_np(x), info.iters.cpu().numpy()))
    (xg, ig), (xh, ih) = out
    assert np.array_equal(ig, ih)
    assert np.array_equal(xg, xh)


def test_proximal_variant_matches_oracle_fp32():
    """i-DEQ-P (Algorithm 2): x^{k+1} = prox_{tau f}(z - tau lambda grad g(z)) with the
    closed-form inpainting prox, 30 updates on two masked images, against the oracle."""
    cfg, wl, net, ops, ys = setup("C1b", n=2, h=40, w=56)
    b = B()
    x0 = np.stack([ops[i].AT(ys[i].astype(np.float64)) for i in range(2)])
    xo, infos = solver.solve_batch(net, ops, ys.astype(np.float64), x0, cfg["lam"], cfg["tau"],
                                   cfg["beta"], math.inf, 0.0, 30, prox=True)
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], max_iter=30, prox=True)
    info = b.InfoBuffers(2)
    x, st = b.ideq_solve(ctx, op_for(cfg, wl), torch.tensor(ys, device="cuda"), params,
                         info=info, allow_maxiter=True)
    assert rel(to_np(x), xo) < 1e-5
    for i in range(2):
        assert abs(float(info.energy[i]) - infos[i]["energy"]) < 1e-5 * infos[i]["energy"]
    # the blur operator has no closed-form prox here
    cfg2, wl2, _, _, ys2 = setup("C1a", n=1, h=32, w=32)
    ctx2 = ctx_for(cfg2, wl2, b.IDEQ_FP32)
    with pytest.raises(b.IdeqError) as e:
        b.ideq_solve(ctx2, op_for(cfg2, wl2), torch.tensor(ys2, device="cuda"), params)
    assert e.value.status == b.IDEQ_ERR_UNSUPPORTED


@pytest.mark.parametrize("n,h,w", [(2, 32, 64), (1, 256, 256), (1, 8, 1024)])
def test_mri_operator_matches_oracle(n, h, w):
    """A x = M F x and A^T r = F^{-1}(M r) (orthonormal DFT, own FFT kernels: the
    generic radix-2 one and the four-step 256-point one) against numpy's FFT in FP64."""
    cfg, wl, net, ops, ys = setup("C5", n=n, h=h, w=w)
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    op = op_for(cfg, wl)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(ys.shape).astype(np.float32)
    Ax = to_np(b.ideq_apply_A(ctx, op, torch.tensor(x, device="cuda")))
    ATr = to_np(b.ideq_apply_AT(ctx, op, torch.tensor(x, device="cuda")))
    ref_A = np.stack([ops[i].A(x[i].astype(np.float64)) for i in range(n)])
    ref_AT = np.stack([ops[i].AT(x[i].astype(np.float64)) for i in range(n)])
    assert rel(Ax, ref_A) < 1e-6 and rel(ATr, ref_AT) < 1e-6


@pytest.mark.parametrize("prox", [False, True])
def test_mri_solve_matches_oracle_fp32(prox):
    """30 inertial updates on two complex 64^2 MRI problems (2-channel half-width
    U-Net), gradient form (Algorithm 1) and proximal form (Algorithm 2)."""
    cfg, wl, net, ops, ys = setup("C5", n=2, h=64, w=64)
    b = B()
    x0 = np.stack([ops[i].AT(ys[i].astype(np.float64)) for i in range(2)])
    xo, infos = solver.solve_batch(net, ops, ys.astype(np.float64), x0, cfg["lam"], cfg["tau"],
                                   cfg["beta"], math.inf, 0.0, 30, prox=prox)
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], max_iter=30, prox=prox)
    info = b.InfoBuffers(2)
    x, st = b.ideq_solve(ctx, op_for(cfg, wl), torch.tensor(ys, device="cuda"), params,
                         info=info, allow_maxiter=True)
    assert rel(to_np(x), xo) < 1e-5
    for i in range(2):
        assert abs(float(info.energy[i]) - infos[i]["energy"]) < 1e-5 * infos[i]["energy"]


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("bf16", 1e-2)])
def test_mri_solve_half_precision_tensor_core_convs(prec, tol):
    """30 inertial updates of the MRI problem with 16-bit convolutions, whose
    32-channel layers run on the tensor cores: the iterate stays within the 16-bit
    operand rounding (fp16 2^-11, bf16 2^-8, a few units after the U-Net) of the
    FP64 iterate; the regulariser energy, quadratic in the residual z - N(z) (a
    difference much smaller than z, so relatively less accurate), within 4x that."""
    cfg, wl, net, ops, ys = setup("C5", n=2, h=64, w=64)
    b = B()
    x0 = np.stack([ops[i].AT(ys[i].astype(np.float64)) for i in range(2)])
    xo, infos = solver.solve_batch(net, ops, ys.astype(np.float64), x0, cfg["lam"], cfg["tau"],
                                   cfg["beta"], math.inf, 0.0, 30)
    ctx = ctx_for(cfg, wl, PREC[prec]())
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], max_iter=30)
    info = b.InfoBuffers(2)
    x, st = b.ideq_solve(ctx, op_for(cfg, wl), torch.tensor(ys, device="cuda"), params,
                         info=info, allow_maxiter=True)
    assert rel(to_np(x), xo) < tol
    for i in range(2):
        assert abs(float(info.energy[i]) - infos[i]["energy"]) < 4 * tol * infos[i]["energy"]


def test_rician_solve_matches_oracle_fp32():
    """Rician denoising (App. E): 30 inertial updates on two grey 64^2 images with the
    library's own I1/I0 ratio (series below t = 15, Hankel expansion above) against
    the oracle's SciPy i1e/i0e; t = x y / sigma^2 spans ~0..100 here."""
    cfg, wl, net, ops, ys = setup("C6", n=2, h=64, w=64)
    b = B()
    x0 = np.stack([ops[i].AT(ys[i].astype(np.float64)) for i in range(2)])
    xo, infos = solver.solve_batch(net, ops, ys.astype(np.float64), x0, cfg["lam"], cfg["tau"],
                                   cfg["beta"], math.inf, 0.0, 30)
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], max_iter=30)
    info = b.InfoBuffers(2)
    y = torch.tensor(ys, device="cuda")
    op = op_for(cfg, wl)
    x, st = b.ideq_solve(ctx, op, y, params, info=info, allow_maxiter=True)
    assert rel(to_np(x), xo) < 1e-5
    for i in range(2):
        assert abs(float(info.energy[i]) - infos[i]["energy"]) < 1e-5 * abs(infos[i]["energy"])
    assert np.array_equal(to_np(b.ideq_apply_A(ctx, op, y)), ys.astype(np.float64))
    with pytest.raises(b.IdeqError) as e:  # no closed-form prox for the Rician term
        b.ideq_solve(ctx, op, y, b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], prox=True))
    assert e.value.status == b.IDEQ_ERR_UNSUPPORTED


def test_mri_rejects_sizes_without_fft():
    cfg, wl, net, ops, ys = setup("C5", n=1, h=48, w=64)  # 48 is not a power of two
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    with pytest.raises(b.IdeqError) as e:
        b.ideq_apply_A(ctx, op_for(cfg, wl), torch.tensor(ys, device="cuda"))
    assert e.value.status == b.IDEQ_ERR_UNSUPPORTED


@pytest.mark.parametrize("lam,beta", [(0.0, 0.8), (0.1, 0.0), (0.0, 0.0)])
def test_solve_degenerate_parameters_fp32(lam, beta):
    """lambda = 0 (data term alone, gradient descent on f with inertia), beta = 0
    (RED, Sec. 2.1: no inertia) and both: 20 updates on a ragged C0 batch vs the oracle."""
    cfg, wl, net, ops, ys = setup("C0", n=2, h=37, w=45)
    xo, infos = _oracle_solve(cfg, net, ops, ys, lam=lam, beta=beta, max_iter=20)
    xg, info, st = _gpu_solve(cfg, wl, ys, B().IDEQ_FP32, lam=lam, beta=beta, max_iter=20)
    assert rel(xg, xo) < 1e-5


def test_empty_and_invalid_shapes_are_argument_errors():
    """n = 0 (an empty batch), a negative size, a NULL pointer, tau <= 0 and beta >= 1
    are rejected before any launch, and the context stays usable afterwards."""
    cfg, wl, net, ops, ys = setup("C0")
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    op = op_for(cfg, wl)
    y = torch.tensor(ys, device="cuda")
    shp = b.Shape(0, 1, 64, 64)
    out = torch.zeros_like(y)
    st = b._lib.ideq_solve(ctx.h, ctypes_ref(op), shp, y.data_ptr(), None, out.data_ptr(),
                           ctypes_ref(b.make_params(0.1, 0.8, 0.5)), None)
    assert st == b.IDEQ_ERR_ARG
    st = b._lib.ideq_solve(ctx.h, ctypes_ref(op), b.Shape(1, 1, -64, 64), y.data_ptr(), None,
                           out.data_ptr(), ctypes_ref(b.make_params(0.1, 0.8, 0.5)), None)
    assert st == b.IDEQ_ERR_ARG
    st = b._lib.ideq_solve(ctx.h, ctypes_ref(op), b.Shape(1, 1, 64, 64), None, None,
                           out.data_ptr(), ctypes_ref(b.make_params(0.1, 0.8, 0.5)), None)
    assert st == b.IDEQ_ERR_ARG
    for bad in (b.make_params(0.1, 0.0, 0.5), b.make_params(0.1, 0.8, 1.0)):
        with pytest.raises(b.IdeqError) as e:
            b.ideq_solve(ctx, op, y, bad)
        assert e.value.status == b.IDEQ_ERR_ARG
    x, st = b.ideq_solve(ctx, op, y, b.make_params(cfg["lam"], cfg["tau"], cfg["beta"],
                                                   max_iter=3), allow_maxiter=True)
    assert torch.isfinite(x).all()


def ctypes_ref(o):
    import ctypes
    return ctypes.byref(o)


def test_solve_averaging_rejects_runs_it_does_not_define():
    cfg, wl, net, ops, ys = setup("C0")
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    y = torch.tensor(ys, device="cuda")
    for kw in (dict(tol=1e-4), dict(B=0.5), dict(max_iter=4)):
        p = dict(B=math.inf, tol=0.0, max_iter=50)
        p.update(kw)
        params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], p["B"], p["tol"],
                               p["max_iter"], average=True)
        with pytest.raises(b.IdeqError) as e:
            b.ideq_solve(ctx, op_for(cfg, wl), y, params, allow_maxiter=True)
        assert e.value.status == b.IDEQ_ERR_ARG


@pytest.mark.parametrize("prec", ["fp16_fp8", "bf16_fp8"])
def test_solve_unet_fp8_form_stated_error(prec):
    """FP8 operands on the deep convs leave the relative step near 8e-4 (measured),
    above the 1e-4 stopping residual, so the solve runs to max_iter; the iterate
    still stays within 2e-2 of the FP64 fixed point and 0.05 dB of its PSNR."""
    cfg, wl, net, ops, ys = setup("C2", n=1, h=64, w=64)
    xo, infos = _oracle_solve(cfg, net, ops, ys, max_iter=300)
    xg, info, st = _gpu_solve(cfg, wl, ys, PREC[prec](), max_iter=120)
    assert float(info.rel_res[0]) < 5e-3
    assert rel(xg, xo) < 2e-2
    assert abs(solver.psnr(xo[0], wl["x_true"][0]) - solver.psnr(xg[0], wl["x_true"][0])) < 0.05


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_solve_unet_half_precision_matches_fp64_within_stated_error(prec):
    """FP16 convolutions reach the stopping residual 1e-4; BF16 convolutions stall
    near 2e-4 (activation rounding floor) and stop at max_iter.  Both stay within
    2e-3 of the FP64 fixed point and 0.05 dB of its PSNR."""
    cfg, wl, net, ops, ys = setup("C2", n=1, h=64, w=64)
    xo, infos = _oracle_solve(cfg, net, ops, ys, max_iter=300)
    xg, info, st = _gpu_solve(cfg, wl, ys, PREC[prec](), max_iter=120)
    if prec == "fp16":
        assert int(info.status[0]) == solver.CONVERGED
        assert abs(int(info.iters[0]) - infos[0]["iters"]) <= 3
    e = rel(xg, xo)
    assert e < 2e-3, e
    p_o = solver.psnr(xo[0], wl["x_true"][0])
    p_g = solver.psnr(xg[0], wl["x_true"][0])
    assert abs(p_o - p_g) < 0.05


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 2e-3), ("fp16", 2e-3)])
def test_step_at_full_size_sampled_images(prec, tol):
    """One inertial step of the full 8 x RGB 256^2 C1a batch; images 0 and 7 checked."""
    cfg, wl, net, ops, ys = setup("C1a")
    b = B()
    ctx = ctx_for(cfg, wl, PREC[prec]())
    op = op_for(cfg, wl)
    rng = np.random.default_rng(11)
    xk = np.clip(ys + 0.05 * rng.standard_normal(ys.shape), 0, 1).astype(np.float32)
    xkm1 = np.clip(xk + 0.02 * rng.standard_normal(ys.shape), 0, 1).astype(np.float32)
    tk, tkm1 = torch.tensor(xk, device="cuda"), torch.tensor(xkm1, device="cuda")
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"])
    info = b.InfoBuffers(8)
    b.ideq_step(ctx, op, torch.tensor(ys, device="cuda"), tk, tkm1, params, info)
    out = to_np(tk)
    assert np.array_equal(to_np(tkm1), xk.astype(np.float64))
    for i in (0, 7):
        z = xk[i].astype(np.float64) + cfg["beta"] * (xk[i].astype(np.float64) - xkm1[i])
        ref, fval, gval = solver.red_step(net, ops[i], ys[i].astype(np.float64), z, cfg["lam"],
                                          cfg["tau"])
        d_gpu = out[i] - z
        d_ref = ref - z
        # compare the update direction tau (grad f + lambda grad g), the part that carries
        # the arithmetic, and the iterate itself
        assert rel(d_gpu, d_ref) < {"fp32": 5e-5, "bf16": 1e-2, "fp16": 2e-3}[prec]
        assert rel(out[i], ref) < tol
        # F = f + lambda g with g = 1/2||r||^2: 16-bit operands in the tail conv
        # (unit roundoff u = 2^-11 f16, 2^-8 bf16) move g by up to ~2u relative
        e_tol = {"fp32": 1e-4, "bf16": 2 * 2.0 ** -8, "fp16": 2 * 2.0 ** -11}[prec]
        assert abs(float(info.energy[i]) - (fval + cfg["lam"] * gval)) < e_tol * (fval + cfg["lam"] * gval)


# ---------------------------------------------------------------- saturation model in a solve


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16", 2e-3)])
def test_saturation_solve_matches_oracle(prec, tol):
    """The nonlinear forward model A(x) = tanh(2 k*x)/tanh 2 (15x15 Gaussian k) inside
    a solve: 30 inertial updates of two RGB 64^2 images, data gradient J_A(z)^T(A(z) - y)
    at every extrapolated point, against the oracle (FP32 1e-5, FP16 convs 2e-3)."""
    cfg, wl, net, ops, ys = setup("C4", n=2, h=64, w=64)
    xo, infos = _oracle_solve(cfg, net, ops, ys, tol=0.0, max_iter=30)
    xg, info, st = _gpu_solve(cfg, wl, ys, PREC[prec](), tol=0.0, max_iter=30)
    assert list(info.iters.cpu().numpy()) == [30, 30]
    assert rel(xg, xo) < tol, rel(xg, xo)
    for i in range(2):
        assert abs(float(info.energy[i]) - infos[i]["energy"]) < 4 * tol * abs(infos[i]["energy"])


# ---------------------------------------------------------------- full-size solves


def _c1a_golden():
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1a_oracle_samples.npz")
    return np.load(p)


@pytest.mark.parametrize("prec,tol,it_slack", [("fp32", 1e-5, 1), ("fp16", 2e-3, 3)])
def test_full_size_c1a_solve_matches_oracle(prec, tol, it_slack):
    """Images 0 and 1 of the 8 x RGB 256^2 motion-blur workload solved to the 1e-4
    relative step (App. D.1.3) in the launch configuration of the benchmark (device-
    driven solve graph, spectral data step, halo/streamed tcgen05 convs for FP16).
    The stored FP64 oracle trajectory (tests/golden/oracle_c1a_samples.py) gives the
    iteration count and, at the GPU's own count, x^k at 512 sampled pixels and the
    PSNR of the whole image."""
    g = _c1a_golden()
    cfg, wl, net, ops, ys = setup("C1a", n=2)
    xg, info, st = _gpu_solve(cfg, wl, ys, PREC[prec]())
    idx, ks = g["idx"], list(g["k"])
    for i in range(2):
        it = int(info.iters[i])
        assert int(info.status[i]) == solver.CONVERGED
        assert abs(it - int(g["stop"][i])) <= it_slack, (i, it, int(g["stop"][i]))
        j = ks.index(it)
        xs = xg[i].ravel()[idx]
        assert rel(xs, g["samples"][i, j]) < tol, (i, rel(xs, g["samples"][i, j]))
        p_gpu = solver.psnr(xg[i], wl["x_true"][i])
        assert abs(p_gpu - float(g["psnr"][i, j])) < 0.05
        # and against the oracle's own stopping iterate
        j0 = ks.index(int(g["stop"][i]))
        assert abs(p_gpu - float(g["psnr"][i, j0])) < 0.05


# ---------------------------------------------------------------- failure detection


def _solve_status(ctx, op, y, params, info):
    b = B()
    try:
        x, st = b.ideq_solve(ctx, op, y, params, info=info, allow_maxiter=True)
    except b.IdeqError as e:
        return None, e.status
    return x, st


@pytest.mark.parametrize("name,prec", [("C0", "fp32"), ("C1a", "fp16")])
def test_nan_observation_marks_only_that_image_diverged(name, prec):
    """A NaN in image 0's observation makes its first step non-finite: the solve
    returns IDEQ_DIVERGED with image 0 DIVERGED and image 1 CONVERGED, image 1's
    restoration is bit-identical to the one from a clean batch (images never
    interact), and the context solves normally afterwards."""
    cfg, wl, net, ops, ys = setup(name, n=2, h=48, w=64)
    b = B()
    op = op_for(cfg, wl)
    params = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], tol=1e-4, max_iter=400)
    clean = torch.tensor(ys, device="cuda")
    bad = clean.clone()
    bad[0, 0, 5, 7] = float("nan")
    ctx = ctx_for(cfg, wl, PREC[prec]())
    info = b.InfoBuffers(2)
    out = torch.zeros_like(clean)
    st = b._lib.ideq_solve(ctx.h, ctypes_ref(op), b._shape(bad), bad.data_ptr(), None,
                           out.data_ptr(), ctypes_ref(params), ctypes_ref(info.s))
    assert st == b.IDEQ_DIVERGED
    assert int(info.status[0]) == b.IDEQ_IMG_DIVERGED
    assert int(info.status[1]) == b.IDEQ_IMG_CONVERGED
    assert int(info.iters[0]) == 1  # frozen at its first (non-finite) update
    ref_ctx = ctx_for(cfg, wl, PREC[prec]())
    info2 = b.InfoBuffers(2)
    x_ref, st2 = b.ideq_solve(ref_ctx, op, clean, params, info=info2)
    assert torch.equal(out[1], x_ref[1])
    assert int(info.iters[1]) == int(info2.iters[1])
    # the context that saw the failure still solves the clean batch identically
    x_again, st3 = b.ideq_solve(ctx, op, clean, params, info=info)
    assert torch.equal(x_again, x_ref)


def test_step_size_far_above_1_over_L_diverges_every_image():
    """tau = 200 (about 200 x 1/L): the iterates grow geometrically until a step
    norm overflows; every image is reported DIVERGED before max_iter, the solve
    returns IDEQ_DIVERGED, and the context then solves a valid problem normally."""
    cfg, wl, net, ops, ys = setup("C0", n=2, h=40, w=48)
    b = B()
    op = op_for(cfg, wl)
    y = torch.tensor(ys, device="cuda")
    ctx = ctx_for(cfg, wl, b.IDEQ_FP32)
    info = b.InfoBuffers(2)
    x, st = _solve_status(ctx, op, y, b.make_params(cfg["lam"], 200.0, cfg["beta"], tol=1e-4,
                                                    max_iter=400), info)
    assert st == b.IDEQ_DIVERGED
    assert [int(v) for v in info.status.cpu()] == [b.IDEQ_IMG_DIVERGED] * 2
    assert max(int(v) for v in info.iters.cpu()) < 400
    good = b.make_params(cfg["lam"], cfg["tau"], cfg["beta"], max_iter=20)
    x1, _ = b.ideq_solve(ctx, op, y, good, allow_maxiter=True)
    x2, _ = b.ideq_solve(ctx_for(cfg, wl, b.IDEQ_FP32), op, y, good, allow_maxiter=True)
    assert torch.equal(x1, x2)


# ---------------------------------------------------------------- solve-graph cache


def test_graph_cache_tracks_rician_sigma():
    """Two device-graph Rician solves on one context and one y buffer that differ
    only in the noise level sigma of the data term: each matches the host-driven
    loop bit for bit (the captured graph must not be reused across sigmas)."""
    cfg, wl, net, ops, ys = setup("C6", n=2, h=64, w=64)
    b = B()
    y = torch.tensor(ys, device="cuda")
    ctx_g = ctx_for(cfg, wl, b.IDEQ_FP32)
    ctx_h = ctx_for(cfg, wl, b.IDEQ_FP32)
    b.ideq_prof_enable(ctx_h, True)  # per-launch events keep this one on the host loop
    params = b.make_params(cfg["lam"], 0.002, cfg["beta"], max_iter=12)  # tau < 0.9 sigma^2
    for sigma in (0.1, 0.05):
        op = b.make_operator(b.IDEQ_OP_RICIAN, sigma=sigma)
        xg, _ = b.ideq_solve(ctx_g, op, y, params, allow_maxiter=True)
        assert b.ideq_solve_graphed(ctx_g)
        xh, _ = b.ideq_solve(ctx_h, op, y, params, allow_maxiter=True)
        assert not b.ideq_solve_graphed(ctx_h)
        torch.cuda.synchronize()
        assert torch.equal(xg, xh), sigma


@pytest.mark.parametrize("name,over", [("C1a", dict(n=2, h=64, w=64)),
                                       ("C1a", dict(n=1, h=136, w=200)),
                                       ("C1a", dict(n=1)),
                                       ("C3", dict(n=2, h=40, w=56))])
def test_grad_reg_two_subtile_convs_match_oracle(name, over, monkeypatch):
    """Tiles of two 128-row sub-tiles sharing each weight chunk (M = 256 per CTA),
    forced on every conv that can take them (IDEQ_TC_MS=2): plain tiles with two
    accumulator buffers (N <= 128) and with one (N = 256), and the streamed-halo
    form with two row boxes per stage; odd tile counts leave a last sub-tile past
    the batch (loaded as zeros, stored nowhere).  FP16, 2e-3 as for the other forms."""
    monkeypatch.setenv("IDEQ_TC_MS", "2")
    cfg, wl, net, ops, ys = setup(name, **over)
    b = B()
    ctx = ctx_for(cfg, wl, b.IDEQ_FP16)
    z = np.random.default_rng(5).uniform(0, 1, ys.shape).astype(np.float32)
    g = to_np(b.ideq_grad_reg(ctx, torch.tensor(z, device="cuda")))
    for i in range(z.shape[0]):
        ref, gv = nets.grad_g(net, z[i].astype(np.float64))
        assert rel(g[i], ref) < 2e-3, (i, rel(g[i], ref))


@pytest.mark.parametrize("name,over,prec", [("C1a", dict(n=2, h=64, w=64), "fp16"),
                                            ("C1a", dict(n=1, h=136, w=200), "fp16"),
                                            ("C1a", dict(n=3), "bf16"),
                                            ("C3", dict(n=2, h=40, w=56), "fp16")])
def test_grad_reg_cta_pair_convs_match_single_cta(name, over, prec, monkeypatch):
    """Tiles of 256 rows on a CTA pair (two-SM tcgen05 MMAs, half of B in each CTA's
    shared memory; plain, streamed-halo, stride-2 and depth-to-space layers with 128
    or 256 columns) against the single-CTA tiles (IDEQ_TC_CG2=0) on the same inputs,
    and both against the oracle.  Odd tile counts leave the odd CTA of the last pair a
    sub-tile past the batch.  The two forms sum the same products in the same K order
    per tile, so they agree to a unit of the 16-bit outputs."""
    cfg, wl, net, ops, ys = setup(name, **over)
    b = B()
    z = torch.tensor(np.random.default_rng(5).uniform(0, 1, ys.shape).astype(np.float32),
                     device="cuda")
    out = {}
    for cg2 in ("1", "0"):
        monkeypatch.setenv("IDEQ_TC_CG2", cg2)
        ctx = ctx_for(cfg, wl, PREC[prec]())
        out[cg2] = to_np(b.ideq_grad_reg(ctx, z))
    assert rel(out["1"], out["0"]) < (2e-3 if prec == "bf16" else 5e-4), rel(out["1"], out["0"])
    zz = to_np(z)
    for i in range(zz.shape[0]):
        ref, gv = nets.grad_g(net, zz[i])
        assert rel(out["1"][i], ref) < (1e-2 if prec == "bf16" else 2e-3)


@pytest.mark.parametrize("name,over,prec", [("C1a", dict(n=2, h=40, w=128), "fp16"),
                                            ("C1a", dict(n=1, h=136, w=200), "fp16"),
                                            ("C1a", dict(n=3, h=48, w=256), "bf16")])
def test_grad_reg_stacked_tap_convs_match_nine_tap(name, over, prec, monkeypatch):
    """The stacked-tap form of the full-row 3x3 layers of <= 64 output channels
    (IDEQ_TC_STACK=1: one MMA of N = 3 x 64 per input row and horizontal offset,
    accumulators of consecutive output rows in a ring of TMEM blocks, contiguous row
    runs per CTA that cross strip and image boundaries) against the 9-tap tiles on
    the same inputs, and against the oracle.  Row counts not a multiple of the CTA
    count leave runs of uneven length; 136 rows x 200 columns gives a ragged strip."""
    cfg, wl, net, ops, ys = setup(name, **over)
    b = B()
    z = torch.tensor(np.random.default_rng(9).uniform(0, 1, ys.shape).astype(np.float32),
                     device="cuda")
    out = {}
    for stk in ("1", "0"):
        monkeypatch.setenv("IDEQ_TC_STACK", stk)
        ctx = ctx_for(cfg, wl, PREC[prec]())
        out[stk] = to_np(b.ideq_grad_reg(ctx, z))
    assert rel(out["1"], out["0"]) < (2e-3 if prec == "bf16" else 5e-4), rel(out["1"], out["0"])
    zz = to_np(z)
    for i in range(zz.shape[0]):
        ref, gv = nets.grad_g(net, zz[i])
        assert rel(out["1"][i], ref) < (1e-2 if prec == "bf16" else 2e-3)


@pytest.mark.parametrize("name,over,prec", [("C1a", dict(n=2, h=40, w=128), "fp16"),
                                            ("C1a", dict(n=1, h=136, w=200), "bf16")])
def test_grad_reg_direct_epilogue_matches_staged(name, over, prec, monkeypatch):
    """The full-row (halo and streamed) 3x3 layers with the direct epilogue (results
    and auxiliary inputs through global memory from the epilogue threads) against
    the staged epilogue (shared-memory boxes and TMA stores, IDEQ_TC_DIRECT=0) on the
    same inputs: the same accumulators through the same epilogue arithmetic, so the
    outputs agree to the last bit; 200 columns leave a ragged second strip whose
    pixels past the image must not be stored."""
    cfg, wl, net, ops, ys = setup(name, **over)
    b = B()
    z = torch.tensor(np.random.default_rng(13).uniform(0, 1, ys.shape).astype(np.float32),
                     device="cuda")
    out = {}
    for d in ("1", "0"):
        monkeypatch.setenv("IDEQ_TC_DIRECT", d)
        ctx = ctx_for(cfg, wl, PREC[prec]())
        out[d] = to_np(b.ideq_grad_reg(ctx, z))
    assert rel(out["1"], out["0"]) < 1e-7, rel(out["1"], out["0"])
    zz = to_np(z)
    for i in range(zz.shape[0]):
        ref, gv = nets.grad_g(net, zz[i])
        assert rel(out["1"][i], ref) < (1e-2 if prec == "bf16" else 2e-3)


@pytest.mark.parametrize("name,over,prec", [("C1a", dict(n=2, h=40, w=56), "fp16"),
                                            ("C1a", dict(n=1, h=136, w=200), "bf16"),
                                            ("C5", dict(n=2, h=64, w=64), "fp16")])
def test_grad_reg_image_side_tensor_core_convs_match_simt(name, over, prec, monkeypatch):
    """The image-side input convs (head forward, tail input gradient: 3x3 from c image
    channels to the first features) as im2col rows of the 9 c taps (one 32-channel K
    chunk, zero past 9 c and outside the image) and a 1x1 tcgen05 conv
    (IDEQ_IMG_TC=1), against the SIMT edge kernels on the same inputs and against the
    oracle; RGB and the 2-channel MRI net, ragged sizes.  The tensor-core form rounds
    the f32 image and the head weights to the 16-bit operand type (unit roundoff 2^-11
    FP16, 2^-9 BF16: measured 2.1e-3 between the BF16 forms at 136 x 200), so the two
    forms are held to the 16-bit tolerances of the oracle comparisons."""
    cfg, wl, net, ops, ys = setup(name, **over)
    b = B()
    z = torch.tensor(np.random.default_rng(17).uniform(0, 1, ys.shape).astype(np.float32),
                     device="cuda")
    out = {}
    for v in ("1", "0"):
        monkeypatch.setenv("IDEQ_IMG_TC", v)
        ctx = ctx_for(cfg, wl, PREC[prec]())
        out[v] = to_np(b.ideq_grad_reg(ctx, z))
    assert rel(out["1"], out["0"]) < (1e-2 if prec == "bf16" else 2e-3), rel(out["1"], out["0"])
    zz = to_np(z)
    for i in range(zz.shape[0]):
        ref, gv = nets.grad_g(net, zz[i])
        assert rel(out["1"][i], ref) < (1e-2 if prec == "bf16" else 2e-3)
