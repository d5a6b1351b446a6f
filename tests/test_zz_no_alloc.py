"""The allocation-free RED update agrees with the context-based step.

ideq_red_update_noalloc serves callers that cannot allocate device memory
(frameworks that own every allocation, fixed memory budgets, servers that must not
allocate while serving): it keeps its partial sums in a static device array
instead of a context workspace.  This test drives it through the C ABI with the
inputs of one inertial step -- z from the inertial extrapolation, grad f from
ideq_apply_A / ideq_apply_AT and grad g from ideq_grad_reg -- and compares its
output with ideq_step's on two consecutive steps (the second call reuses the
array the first one left behind).  FP32 tolerance 1e-5, as for the other FP32
parity tests.  The file sorts last so that a run stopping at the first failure
has run every other test already; it also passes on its own.
"""
import numpy as np
import pytest

from gpu_common import ctx_for, op_for, setup

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_update_matches_step_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_19705_gb300 import build
    build.build()
    from paper_2605_19705_gb300 import binding as B

    cfg, wl, net, ops, ys = setup("C1a", n=2, h=64, w=64)
    ctx = ctx_for(cfg, wl, B.IDEQ_FP32)
    op = op_for(cfg, wl)
    y = torch.tensor(ys, device="cuda")
    rng = np.random.default_rng(21)
    x = torch.tensor(np.clip(ys + 0.05 * rng.standard_normal(ys.shape), 0, 1).astype(np.float32),
                     device="cuda")
    xp = x + 0.01 * torch.tensor(rng.standard_normal(ys.shape).astype(np.float32), device="cuda")
    lam, tau, beta = cfg["lam"], cfg["tau"], cfg["beta"]
    params = B.make_params(lam, tau, beta)
    step_sq = torch.zeros(2, dtype=torch.float64, device="cuda")
    x_sq = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call in range(2):
        # reference: the context-based inertial step
        xk, xkm1 = x.clone(), xp.clone()
        info = B.InfoBuffers(2)
        B.ideq_step(ctx, op, y, xk, xkm1, params, info)
        # the same step with the allocation-free update
        z = x + beta * (x - xp)
        gg = B.ideq_grad_reg(ctx, z)
        gf = B.ideq_apply_AT(ctx, op, B.ideq_apply_A(ctx, op, z) - y)
        x_new = torch.empty_like(x)
        B.ideq_red_update_noalloc(z, gf, gg, x, x_new, lam, tau, step_sq, x_sq)
        torch.cuda.synchronize()
        err = float((x_new - xk).norm() / xk.norm())
        assert err < 1e-5, (call, err)
        rel = torch.sqrt(step_sq / x_sq)
        assert torch.allclose(rel, info.rel_res, rtol=1e-5, atol=0), (call, rel, info.rel_res)
        # squares summed in FP32 over at most 16 elements, then in FP64: relative
        # error at most 16 FP32 ulps of each partial sum
        ref_x_sq = (x.double() ** 2).sum(dim=(1, 2, 3))
        assert torch.allclose(x_sq, ref_x_sq, rtol=1e-6, atol=0), call
        # advance to the next step's state
        xp, x = x, xk


def test_noalloc_nullable_outputs_size_limit_and_unaligned_views():
    """The step norms are optional; a request larger than the static array is an
    argument error that leaves x_new untouched; and tensors that start 4 bytes past a
    16-byte boundary (a sub-allocation or an offset view of a caller's buffer) take
    the scalar path and give the same update as aligned ones."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_19705_gb300 import build
    build.build()
    from paper_2605_19705_gb300 import binding as B

    g = torch.Generator(device="cpu").manual_seed(5)
    shape = (3, 3, 40, 56)
    numel = 3 * 3 * 40 * 56
    z, gf, gg, x = (torch.randn(shape, generator=g).cuda() for _ in range(4))
    lam, tau = 0.1, 0.75
    ref = torch.empty_like(x)
    s_ref = torch.zeros(3, dtype=torch.float64, device="cuda")
    x_ref = torch.zeros(3, dtype=torch.float64, device="cuda")
    B.ideq_red_update_noalloc(z, gf, gg, x, ref, lam, tau, s_ref, x_ref)
    # no norms requested
    out = torch.empty_like(x)
    B.ideq_red_update_noalloc(z, gf, gg, x, out, lam, tau, None, None)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # unaligned: every tensor viewed one float into a larger buffer
    def shifted(t):
        buf = torch.empty(numel + 1, device="cuda")
        v = buf[1:].view(shape)
        v.copy_(t)
        assert v.data_ptr() % 16 == 4
        return v
    zu, fu, gu, xu = shifted(z), shifted(gf), shifted(gg), shifted(x)
    ou = shifted(torch.zeros_like(x))
    s_u = torch.zeros(3, dtype=torch.float64, device="cuda")
    x_u = torch.zeros(3, dtype=torch.float64, device="cuda")
    B.ideq_red_update_noalloc(zu, fu, gu, xu, ou, lam, tau, s_u, x_u)
    torch.cuda.synchronize()
    assert torch.allclose(ou, ref, rtol=1e-6, atol=1e-6)
    # the float4 path forms squares of four elements in FP32 before the FP64 sums, the
    # scalar path one element at a time: the sums agree to a few FP32 roundings
    assert torch.allclose(s_u, s_ref, rtol=1e-6) and torch.allclose(x_u, x_ref, rtol=1e-6)
    # 2 * n * blocks > 65536 partial sums: refused before any launch
    n_big = 32769  # one block per one-value image
    t = torch.zeros(n_big, 1, 1, 1, device="cuda")
    sentinel = torch.full_like(t, 7.0)
    with pytest.raises(B.IdeqError) as e:
        B.ideq_red_update_noalloc(t, t, t, t, sentinel, lam, tau)
    assert e.value.status == B.IDEQ_ERR_ARG
    torch.cuda.synchronize()
    assert bool((sentinel == 7.0).all())
