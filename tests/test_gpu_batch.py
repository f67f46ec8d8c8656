"""Batched path: fgbd_run_batch against fgbd_run and the oracle.

Each frame of a batch runs the same kernels as fgbd_run in its own context,
so its graph, statistics and output must equal the plain run's bit for bit;
the plain path is in turn checked against the oracle elsewhere, and two small
frames are checked against the oracle here directly.  The batch is also
captured into a CUDA graph and replayed on new colours.
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


def _frames():
    out = []
    fr = synth.sphere_frame(20500, 9, 20.0, 0)
    out.append((fr.xyz, fr.noisy, 9))
    xyz = synth.torso_points(60000, 8, 1)
    out.append((xyz, synth.add_noise_u8(synth.piecewise_colors(xyz, 8, 1), 30.0, 2), 8))
    rng = np.random.default_rng(3)
    xyz = rng.integers(0, 1024, size=(12289, 3)).astype(np.int32)
    out.append((xyz, rng.integers(0, 256, size=(12289, 3)).astype(np.uint8), 10))
    xyz = synth.torso_points(30000, 8, 3)
    out.append((xyz, synth.add_noise_f32(synth.piecewise_colors(xyz, 8, 3, as_float=True), 25.0, 3), 8))
    out.append((np.zeros((0, 3), np.int32), np.zeros((0, 3), np.uint8), 10))   # an empty frame
    return out


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _plain(F, xyz, rgb, bits, window=1):
    ctx = F.Context(max(len(xyz), 1), bits=bits, window=window)
    out = ctx.run(_dev(xyz.astype(np.int32)), _dev(rgb), out_dtype=torch.float32)
    ctx.sync()
    res = (out.cpu().numpy(), ctx.stats(), ctx.orders().cpu().numpy())
    ctx.close()
    return res


def test_batch_equals_plain_runs(F):
    frames = _frames()
    ctxs = [F.Context(max(len(x), 1), bits=b) for x, _, b in frames]
    xs = [_dev(x.astype(np.int32)) for x, _, _ in frames]
    cs = [_dev(c) for _, c, _ in frames]
    outs = F.Context.run_batch(ctxs, xs, cs, out_dtype=torch.float32)
    torch.cuda.synchronize()
    for ctx, out, (xyz, rgb, bits) in zip(ctxs, outs, frames):
        ctx.sync()
        ref_out, ref_st, ref_orders = _plain(F, xyz, rgb, bits)
        st = ctx.stats()
        assert np.array_equal(out.cpu().numpy(), ref_out)
        for key in ("n", "n_edges", "sigma_g", "n_patches", "m", "q", "sigma_est", "n_keep"):
            assert st[key] == ref_st[key], key
        if len(xyz):
            assert np.array_equal(ctx.orders().cpu().numpy(), ref_orders)
    for ctx in ctxs:
        ctx.close()


def test_batch_of_mixed_windows_equals_plain_runs(F):
    """Contexts of windows 1, 2 and 3 in one batch, run directly, then recorded
    and replayed: every frame equals its own plain run bit for bit."""
    frames = _frames()[:4]
    windows = [2, 3, 1, 2]
    ctxs = [F.Context(len(x), bits=b, window=w) for (x, _, b), w in zip(frames, windows)]
    xs = [_dev(x.astype(np.int32)) for x, _, _ in frames]
    cs = [_dev(c) for _, c, _ in frames]
    outs = [torch.empty((len(x), 3), dtype=torch.float32, device="cuda") for x, _, _ in frames]
    refs = [_plain(F, xyz, rgb, bits, w) for (xyz, rgb, bits), w in zip(frames, windows)]
    for _ in range(3):   # direct, recorded, replayed
        for o in outs:
            o.fill_(-1.0)
        F.Context.run_batch(ctxs, xs, cs, outs=outs)
        torch.cuda.synchronize()
        for ctx, out, (ref_out, ref_st, _), w in zip(ctxs, outs, refs, windows):
            ctx.sync()
            st = ctx.stats()
            assert np.array_equal(out.cpu().numpy(), ref_out), w
            assert st["patch_dim"] == 3 * (6 * w + 1)
            for key in ("n_edges", "n_patches", "m", "q", "sigma_est", "n_keep"):
                assert st[key] == ref_st[key], (w, key)
    for ctx in ctxs:
        ctx.close()


def test_batch_frames_match_the_oracle(F):
    frames = _frames()[:3]
    ctxs = [F.Context(len(x), bits=b) for x, _, b in frames]
    outs = F.Context.run_batch(ctxs, [_dev(x.astype(np.int32)) for x, _, _ in frames], [_dev(c) for _, c, _ in frames])
    for ctx, out, (xyz, rgb, bits) in zip(ctxs, outs, frames):
        ctx.sync()
        res = orc.fgbd(xyz, rgb, orc.Params(bits=bits))
        row_ptr, col, _ = ctx.graph_csr()
        assert np.array_equal(row_ptr.cpu().numpy(), res.row_ptr)
        assert np.array_equal(col.cpu().numpy(), res.col.astype(np.int32))
        st = ctx.stats()
        assert st["sigma_est"] == pytest.approx(res.noise["sigma_est"], rel=1e-5)
        if st["q"] == res.q:
            assert np.abs(out.cpu().numpy() - res.out).max() <= 1e-4 * 255
        ctx.close()


def test_batch_argument_checks(F):
    xyz = _dev(np.zeros((4, 3), np.int32))
    rgb = _dev(np.zeros((4, 3), np.uint8))
    out = torch.empty((4, 3), dtype=torch.float32, device="cuda")
    ctx = F.Context(4, bits=4)
    with pytest.raises(F.FgbdError):
        F.fgbd_run_batch([ctx.handle, ctx.handle], [xyz, xyz], [rgb, rgb], [out, out])   # one frame per context
    small = F.Context(2, bits=4)
    with pytest.raises(F.FgbdError):
        F.fgbd_run_batch([small.handle], [xyz], [rgb], [out])                          # above capacity
    F.fgbd_run_batch([], [], [], [])                                                   # nothing to do
    ctx.close()
    small.close()


def test_batch_captured_in_a_cuda_graph(F):
    frames = _frames()[:4]
    ctxs = [F.Context(len(x), bits=b) for x, _, b in frames]
    xs = [_dev(x.astype(np.int32)) for x, _, _ in frames]
    cs = [_dev(c) for _, c, _ in frames]
    outs = [torch.empty((len(x), 3), dtype=torch.float32, device="cuda") for x, _, _ in frames]
    F.Context.run_batch(ctxs, xs, cs, outs=outs)      # first run outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.Context.run_batch(ctxs, xs, cs, outs=outs)
    # new noise on every frame, written into the captured input buffers
    new = []
    for k, (xyz, rgb, bits) in enumerate(frames):
        if rgb.dtype == np.uint8:
            noisy = synth.add_noise_u8(rgb, 10.0, 50 + k)
        else:
            noisy = synth.add_noise_f32(rgb, 10.0, 50 + k)
        cs[k].copy_(_dev(noisy))
        new.append(noisy)
    g.replay()
    torch.cuda.synchronize()
    for ctx, out, (xyz, _, bits), noisy in zip(ctxs, outs, frames, new):
        ctx.sync()
        ref_out, ref_st, _ = _plain(F, xyz, noisy, bits)
        assert np.array_equal(out.cpu().numpy(), ref_out)
        assert ctx.stats()["q"] == ref_st["q"]
        ctx.close()


def test_repeated_batches_replay_their_graph(F):
    """The second call with the same contexts and buffers records a CUDA graph of
    the batch and later calls launch it: new contents in the same buffers give
    the plain results every time; a context destroyed and replaced (its address
    may come back) never meets a graph recorded for the old one."""
    frames = _frames()[:3]
    ctxs = [F.Context(len(x), bits=b) for x, _, b in frames]
    xs = [_dev(x.astype(np.int32)) for x, _, _ in frames]
    cs = [_dev(c) for _, c, _ in frames]
    outs = [torch.empty((len(x), 3), dtype=torch.float32, device="cuda") for x, _, _ in frames]
    for call in range(4):
        new = []
        for k, (xyz, rgb, bits) in enumerate(frames):
            noisy = (synth.add_noise_u8(rgb, 8.0, 70 + 10 * call + k) if rgb.dtype == np.uint8
                     else synth.add_noise_f32(rgb, 8.0, 70 + 10 * call + k))
            cs[k].copy_(_dev(noisy))
            new.append(noisy)
        if call == 3:
            # replace the middle context by a new one of the same shape
            ctxs[1].close()
            ctxs[1] = F.Context(len(frames[1][0]), bits=frames[1][2])
        F.Context.run_batch(ctxs, xs, cs, outs=outs)
        torch.cuda.synchronize()
        for ctx, out, (xyz, _, bits), noisy in zip(ctxs, outs, frames, new):
            ctx.sync()
            ref_out, ref_st, _ = _plain(F, xyz, noisy, bits)
            assert np.array_equal(out.cpu().numpy(), ref_out), call
            assert ctx.stats()["q"] == ref_st["q"]
    for ctx in ctxs:
        ctx.close()
