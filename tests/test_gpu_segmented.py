"""Segmented batches: one launch per stage over the frames of a batch.

A batch whose frames share window 1, the ablation switches and the colour type
runs every stage as one launch over up to 16 frames, each frame with the same
kernels and block counts as fgbd_run (or, for the tunable block shapes, code
whose results do not depend on the shape).  So every frame's output, graph and
statistics must equal a plain fgbd_run bit for bit, under every block shape the
tuner may choose, in a chunked batch of more than 16 frames, under the
ablation switches, and replayed from a CUDA graph.  That the segmented path
ran is seen in the launch counts: it counts every launch in the stats of
the first context of each chunk of frames, none in the others'.
"""
import numpy as np
import pytest
import torch

from oracle import fgbd_oracle as orc
from paper_2401_09721_gb300 import build, synth

pytestmark = pytest.mark.gpu


SHAPES = [
    dict(seg_frames=16, scatter_threads=512, filter_threads=512, filter_blocks_per_sm=2),   # the defaults
    dict(seg_frames=16, scatter_threads=256, filter_threads=256, filter_blocks_per_sm=4),
    dict(seg_frames=16, scatter_threads=1024, filter_threads=512, filter_blocks_per_sm=1),
    dict(seg_frames=4, scatter_threads=256, filter_threads=256, filter_blocks_per_sm=2),
]


@pytest.fixture(scope="module")
def F():
    build.build()
    from paper_2401_09721_gb300 import fgbd
    return fgbd


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _frames(dtype="u8"):
    rng = np.random.default_rng(11)
    out = []
    fr = synth.sphere_frame(20500, 9, 20.0, 0)
    out.append((fr.xyz, fr.noisy, 9))
    xyz = synth.torso_points(70000, 8, 1)
    out.append((xyz, synth.add_noise_u8(synth.piecewise_colors(xyz, 8, 1), 30.0, 2), 8))
    for n, b in ((1, 4), (2, 4), (7, 3), (4097, 10), (12289, 6)):
        xyz = rng.integers(0, 1 << b, size=(n, 3)).astype(np.int32)
        out.append((xyz, rng.integers(0, 256, size=(n, 3)).astype(np.uint8), b))
    if dtype == "f32":
        out = [(x, (c.astype(np.float32) + rng.normal(0, 0.3, c.shape)).astype(np.float32), b) for x, c, b in out]
    return out


def _plain(F, xyz, rgb, bits, variant=0):
    ctx = F.Context(max(len(xyz), 1), bits=bits, variant=variant)
    out = ctx.run(_dev(xyz.astype(np.int32)), _dev(rgb), out_dtype=torch.float32)
    ctx.sync()
    res = (out.cpu().numpy(), ctx.stats(), ctx.orders().cpu().numpy())
    ctx.close()
    return res


def _check_batch(F, frames, variant=0, shape=None, replays=1):
    shape = shape or SHAPES[0]
    mean = int(np.mean([max(len(x), 1) for x, _, _ in frames]))
    F.fgbd_set_batch_shape(torch.cuda.current_device(), mean, shape)
    chunk = shape["seg_frames"]
    try:
        ctxs = [F.Context(len(x), bits=b, variant=variant) for x, _, b in frames]
        xs = [_dev(x.astype(np.int32)) for x, _, _ in frames]
        cs = [_dev(c) for _, c, _ in frames]
        outs = [torch.empty((len(x), 3), dtype=torch.float32, device="cuda") for x, _, _ in frames]
        refs = [_plain(F, xyz, rgb, bits, variant) for xyz, rgb, bits in frames]
        for call in range(replays):   # direct, recorded, replayed
            for o in outs:
                o.fill_(-1.0)
            before = [c.stats()["launches"] for c in ctxs]
            F.Context.run_batch(ctxs, xs, cs, outs=outs)
            torch.cuda.synchronize()
            after = [c.stats()["launches"] for c in ctxs]
            # every launch is counted in the first context of each chunk
            for f in range(len(ctxs)):
                assert (after[f] > before[f]) == (f % chunk == 0), "the segmented path did not run"
            for ctx, out, (ref_out, ref_st, ref_orders) in zip(ctxs, outs, refs):
                ctx.sync()
                st = ctx.stats()
                assert np.array_equal(out.cpu().numpy(), ref_out)
                for key in ("n", "n_edges", "sigma_g", "n_patches", "m", "q", "sigma_est", "n_keep", "eigenvalues"):
                    assert st[key] == ref_st[key], key
                assert np.array_equal(ctx.orders().cpu().numpy(), ref_orders)
        for c in ctxs:
            c.close()
    finally:
        F.fgbd_set_batch_shape(torch.cuda.current_device(), mean, None)


@pytest.mark.parametrize("shape", SHAPES)
def test_segmented_batch_equals_plain_runs_under_every_shape(F, shape):
    _check_batch(F, _frames(), shape=shape)


def test_segmented_batch_of_float_colours(F):
    _check_batch(F, _frames("f32"))


@pytest.mark.parametrize("variant", [1, 2, 4])   # no FSLR, unsorted patches, same-line links
def test_segmented_batch_under_the_ablation_switches(F, variant):
    _check_batch(F, _frames()[:4], variant=variant)


def test_segmented_batch_recorded_and_replayed(F):
    _check_batch(F, _frames()[:5], replays=3)


def test_more_frames_than_one_launch_holds(F):
    """19 frames: two chunks (16 + 3), each one launch per stage."""
    rng = np.random.default_rng(5)
    frames = []
    for k in range(19):
        n = int(rng.integers(3000, 9000))
        xyz = rng.integers(0, 64, size=(n, 3)).astype(np.int32)
        frames.append((xyz, rng.integers(0, 256, size=(n, 3)).astype(np.uint8), 6))
    _check_batch(F, frames)


def test_segmented_frames_match_the_oracle(F):
    frames = _frames()[:2]
    ctxs = [F.Context(len(x), bits=b) for x, _, b in frames]
    outs = F.Context.run_batch(ctxs, [_dev(x.astype(np.int32)) for x, _, _ in frames],
                               [_dev(c) for _, c, _ in frames])
    for ctx, out, (xyz, rgb, bits) in zip(ctxs, outs, frames):
        ctx.sync()
        res = orc.fgbd(xyz, rgb, orc.Params(bits=bits))
        row_ptr, col, _ = ctx.graph_csr()
        assert np.array_equal(row_ptr.cpu().numpy(), res.row_ptr)
        assert np.array_equal(col.cpu().numpy(), res.col.astype(np.int32))
        st = ctx.stats()
        assert st["sigma_est"] == pytest.approx(res.noise["sigma_est"], rel=1e-5)
        assert st["q"] == res.q
        assert np.abs(out.cpu().numpy() - res.out).max() <= 1e-4 * 255
        ctx.close()


def test_tuner_keeps_a_valid_shape_and_the_results(F):
    frames = _frames()
    ctxs = [F.Context(len(x), bits=b) for x, _, b in frames]
    xs = [_dev(x.astype(np.int32)) for x, _, _ in frames]
    cs = [_dev(c) for _, c, _ in frames]
    mean = int(np.mean([len(x) for x, _, _ in frames]))
    dev = torch.cuda.current_device()
    try:
        shape, outs = F.Context.tune_batch(ctxs, xs, cs)
        torch.cuda.synchronize()
        assert shape["seg_frames"] in (0, 2, 4, 8, 16) and shape["ms"] > 0
        assert shape["scatter_threads"] in (256, 512, 1024) and shape["filter_threads"] in (256, 512)
        kept = F.fgbd_get_batch_shape(dev, mean)
        for k in ("seg_frames", "scatter_threads", "filter_threads", "filter_blocks_per_sm"):
            assert kept[k] == shape[k]
        for out, (xyz, rgb, bits) in zip(outs, frames):
            assert np.array_equal(out.cpu().numpy(), _plain(F, xyz, rgb, bits)[0])
        # a batch the segmented path does not take (an empty frame) has nothing to tune
        e_ctx = F.Context(1, bits=4)
        e_out = torch.empty((0, 3), dtype=torch.float32, device="cuda")
        none = F.fgbd_tune_batch([ctxs[0].handle, e_ctx.handle], [xs[0], _dev(np.zeros((0, 3), np.int32))],
                                 [cs[0], _dev(np.zeros((0, 3), np.uint8))],
                                 [torch.empty((len(frames[0][0]), 3), dtype=torch.float32, device="cuda"), e_out])
        assert none["seg_frames"] == -1
        e_ctx.close()
        with pytest.raises(F.FgbdError):
            F.fgbd_set_batch_shape(dev, mean, dict(scatter_threads=384, filter_threads=512, filter_blocks_per_sm=2))
    finally:
        F.fgbd_set_batch_shape(dev, mean, None)
        for c in ctxs:
            c.close()
