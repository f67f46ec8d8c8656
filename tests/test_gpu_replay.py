"""fgbd_run replays a CUDA graph when called again with the same arguments.

The buffers' contents change between the calls here; every call's output and
statistics must equal a fresh context's direct run on the same contents (the
kernels are the same, so the bits are).
"""
import numpy as np
import pytest
import torch

from paper_2401_09721_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    build.build()
    from paper_2401_09721_gb300 import fgbd
    return fgbd


def _direct(F, xyz, rgb, bits):
    ctx = F.Context(len(xyz), bits=bits)
    ctx.set_timing(True)            # per-kernel timing keeps the direct path
    out = ctx.run(torch.from_numpy(xyz).cuda(), torch.from_numpy(rgb).cuda(), out_dtype=torch.uint8)
    ctx.sync()
    res = out.cpu().numpy(), ctx.stats()
    ctx.close()
    return res


def test_replayed_runs_follow_the_buffer_contents(F):
    xyz = synth.torso_points(60000, 8, 2)
    clean = synth.piecewise_colors(xyz, 8, 2)
    x = torch.from_numpy(xyz).cuda()
    c = torch.empty((len(xyz), 3), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(c)
    ctx = F.Context(len(xyz), bits=8)
    for k, sigma in enumerate([10.0, 30.0, 50.0, 20.0, 40.0]):   # direct, capture, replay, replay, replay
        noisy = synth.add_noise_u8(clean, sigma, 70 + k)
        c.copy_(torch.from_numpy(noisy))
        ctx.run(x, c, out=out)
        ctx.sync()
        ref_out, ref_st = _direct(F, xyz, noisy, 8)
        st = ctx.stats()
        assert np.array_equal(out.cpu().numpy(), ref_out)
        for key in ("n", "n_edges", "sigma_g", "n_patches", "m", "q", "sigma_est", "n_keep"):
            assert st[key] == ref_st[key], (k, key)
    # new geometry in the same buffers (same n): the replay must rebuild the graph
    xyz2 = synth.torso_points(60000, 8, 3)
    x.copy_(torch.from_numpy(xyz2))
    noisy = synth.add_noise_u8(synth.piecewise_colors(xyz2, 8, 3), 25.0, 80)
    c.copy_(torch.from_numpy(noisy))
    ctx.run(x, c, out=out)
    ctx.sync()
    ref_out, ref_st = _direct(F, xyz2, noisy, 8)
    assert np.array_equal(out.cpu().numpy(), ref_out)
    assert ctx.stats()["n_edges"] == ref_st["n_edges"]
    # other buffers and another n: a new graph; the orders of the new frame are there
    xyz3 = synth.torso_points(30000, 8, 4)
    noisy3 = synth.add_noise_u8(synth.piecewise_colors(xyz3, 8, 4), 25.0, 81)
    for _ in range(3):
        out3 = ctx.run(torch.from_numpy(xyz3).cuda(), torch.from_numpy(noisy3).cuda(), out_dtype=torch.uint8)
        ctx.sync()
        assert np.array_equal(out3.cpu().numpy(), _direct(F, xyz3, noisy3, 8)[0])
    assert ctx.orders().shape == (3, len(xyz3))
    ctx.close()
