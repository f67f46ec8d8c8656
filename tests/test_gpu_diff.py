"""Differentiable filter: forward and adjoint kernels against the FP64 oracle.

The oracle's gradient is itself pinned by central finite differences in
tests/test_oracle_pins.py.  Tolerances: colours 1e-4 on the [0, 1] scale (as
for the filter); colour gradients 1e-4 of their largest magnitude; dL/dalpha
and dL/dsigma 1e-4 relative (float32 iterates, float64 sums over 3N terms).
Recomputed checkpoint segments run the same kernels, so checkpointing must
not change a single bit.
"""
import numpy as np
import pytest
import torch

from oracle import fgbd_oracle as orc
from paper_2401_09721_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    build.build()
    from paper_2401_09721_gb300 import fgbd
    return fgbd


def _frame(kind):
    if kind == "shell":
        xyz = synth.torso_points(60000, 8, 7)
        y = synth.add_noise_f32(synth.piecewise_colors(xyz, 8, 7, as_float=True), 30.0, 7)
        return xyz, y, 8
    rng = np.random.default_rng(8)
    xyz = rng.integers(0, 64, size=(12289, 3)).astype(np.int32)
    return xyz, rng.uniform(0, 255, size=(12289, 3)).astype(np.float32), 6


def _graph(F, xyz, bits):
    ctx = F.Context(len(xyz), bits=bits)
    ctx.build_graph(torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.int32)).cuda())
    codes = orc.scan_line_codes(xyz, bits)
    edges = orc.slg_edges(orc.scan_orders(codes), 1)
    row_ptr, col = orc.adjacency_csr(edges, len(xyz))
    return ctx, row_ptr, col


def _fwd_bwd(F, ctx, y, gout, q, alpha, sigma, checkpoint):
    yt = torch.from_numpy(y).cuda()
    out = torch.empty_like(yt)
    n = len(y)
    F.fgbd_filter_forward(ctx.handle, yt, q, alpha, sigma, checkpoint, out, n)
    gin = torch.empty_like(yt)
    gp = torch.zeros(2, dtype=torch.float64, device="cuda")
    F.fgbd_filter_backward(ctx.handle, torch.from_numpy(gout).cuda(), gin, gp, n)
    torch.cuda.synchronize()
    return out.cpu().numpy(), gin.cpu().numpy(), gp.cpu().numpy()


@pytest.mark.parametrize("kind", ["shell", "random"])
@pytest.mark.parametrize("q,alpha,sigma_scale", [(0, 0.5, 1.0), (1, 0.5, 0.0), (4, 0.3, 1.5), (9, 0.7, 0.8)])
def test_forward_and_gradients_match_the_oracle(F, kind, q, alpha, sigma_scale):
    xyz, y, bits = _frame(kind)
    ctx, row_ptr, col = _graph(F, xyz, bits)
    sg = orc.sigma_g(xyz, row_ptr, col)
    sigma = sigma_scale * sg            # 0 asks the library for sigma_g itself
    s_used = sigma if sigma > 0 else sg
    gout = np.random.default_rng(q).normal(size=y.shape).astype(np.float32)
    out, gin, gp = _fwd_bwd(F, ctx, y, gout, q, alpha, sigma, 1)
    ref = orc.param_filter(xyz, row_ptr, col, y, q, alpha, s_used)[-1]
    assert np.abs(out - ref).max() <= 1e-4 * 255
    gy, da, ds = orc.param_filter_vjp(xyz, row_ptr, col, y, q, alpha, s_used, gout.astype(np.float64))
    assert np.abs(gin - gy).max() <= 1e-4 * max(np.abs(gy).max(), 1e-12)
    if q == 0:
        assert gp[0] == 0.0 and gp[1] == 0.0
    else:
        assert gp[0] == pytest.approx(da, rel=1e-4)
        assert gp[1] == pytest.approx(ds, rel=1e-4)
    ctx.close()


def test_checkpointing_changes_no_bit(F):
    xyz, y, bits = _frame("shell")
    ctx, _, _ = _graph(F, xyz, bits)
    gout = np.random.default_rng(1).normal(size=y.shape).astype(np.float32)
    ref = _fwd_bwd(F, ctx, y, gout, 10, 0.5, 0.0, 1)
    for c in (2, 3, 10, 64):
        got = _fwd_bwd(F, ctx, y, gout, 10, 0.5, 0.0, c)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
    ctx.close()


def test_paper_parameters_give_the_eq5_filter(F):
    xyz, y, bits = _frame("shell")
    ctx, _, _ = _graph(F, xyz, bits)
    yt = torch.from_numpy(y).cuda()
    for q in (1, 3):
        out = ctx.filter(yt, 0.5, 0.0, q)
        plain = ctx.denoise(yt, q, out_dtype=torch.float32)
        assert (out - plain).abs().max().item() <= 1e-4 * 255
    ctx.close()


def test_autograd_function(F):
    xyz, y, bits = _frame("random")
    ctx, row_ptr, col = _graph(F, xyz, bits)
    sg = orc.sigma_g(xyz, row_ptr, col)
    yt = torch.from_numpy(y).cuda().requires_grad_(True)
    alpha = torch.tensor(0.45, dtype=torch.float64, requires_grad=True)
    sigma = torch.tensor(1.2 * sg, dtype=torch.float64, requires_grad=True)
    w = torch.from_numpy(np.random.default_rng(3).normal(size=y.shape).astype(np.float32)).cuda()
    out = ctx.filter(yt, alpha, sigma, q=3)
    (out * w).sum().backward()
    gy, da, ds = orc.param_filter_vjp(xyz, row_ptr, col, y, 3, 0.45, 1.2 * sg, w.cpu().numpy().astype(np.float64))
    assert np.abs(yt.grad.cpu().numpy() - gy).max() <= 1e-4 * np.abs(gy).max()
    assert alpha.grad.item() == pytest.approx(da, rel=1e-4)
    assert sigma.grad.item() == pytest.approx(ds, rel=1e-4)
    ctx.close()


def test_backward_needs_its_forward(F):
    xyz, y, bits = _frame("random")
    ctx = F.Context(len(xyz), bits=bits)
    x = torch.from_numpy(xyz).cuda()
    ctx.build_graph(x)
    g = torch.zeros((len(xyz), 3), dtype=torch.float32, device="cuda")
    gp = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FgbdError):
        F.fgbd_filter_backward(ctx.handle, g, g.clone(), gp, len(xyz))     # no forward yet
    yt = torch.from_numpy(y).cuda()
    F.fgbd_filter_forward(ctx.handle, yt, 2, 0.5, 0.0, 1, torch.empty_like(yt), len(xyz))
    ctx.build_graph(x)                                                      # a new graph drops the forward state
    with pytest.raises(F.FgbdError):
        F.fgbd_filter_backward(ctx.handle, g, g.clone(), gp, len(xyz))
    ctx.close()
