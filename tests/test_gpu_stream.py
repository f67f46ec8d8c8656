"""Streaming mode (Section 3 (2)): frames that reuse the previous frame's q.

fgbd_run_reuse builds the new frame's graph and filters it with the q the
context selected last, read on the device.  Its output must equal an explicit
fgbd_denoise with that q on the same graph bit for bit (same kernel, same q),
and the oracle's Eq. 5 filter with that q within the colour tolerance.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_reuse_needs_a_selected_q(F):
    ctx = F.Context(16, bits=4)
    x = _dev(np.zeros((16, 3), np.int32))
    c = _dev(np.zeros((16, 3), np.uint8))
    with pytest.raises(F.FgbdError):
        ctx.run_reuse(x, c)
    ctx.close()


def test_reuse_filters_the_new_frame_with_the_previous_q(F):
    seq = synth.StreamSequence(frames=300, samples=70000, bits=8, sigma=25.0, seed=3)
    a, b = seq.frame(0), seq.frame(5)
    ctx = F.Context(max(a.n, b.n), bits=8)
    ctx.run(_dev(a.xyz), _dev(a.noisy))
    ctx.sync()
    q_a = ctx.stats()["q"]
    assert q_a >= 1
    out = ctx.run_reuse(_dev(b.xyz), _dev(b.noisy), out_dtype=torch.float32)
    ctx.sync()
    st = ctx.stats()
    assert st["q"] == q_a and st["n"] == b.n
    got = out.cpu().numpy()
    # the same frame through an explicit fixed-q filter: identical bits
    ref_ctx = F.Context(b.n, bits=8)
    ref_ctx.build_graph(_dev(b.xyz))
    same = ref_ctx.denoise(_dev(b.noisy), q_a, out_dtype=torch.float32).cpu().numpy()
    assert np.array_equal(got, same)
    assert st["sigma_g"] == ref_ctx.stats()["sigma_g"]
    # and the oracle's filter with that q
    res = orc.fgbd(b.xyz, b.noisy, orc.Params(bits=8), q=q_a)
    assert np.abs(got - res.out).max() <= 1e-4 * 255
    ctx.close()
    ref_ctx.close()


def test_reuse_keeps_q_across_frames_and_empty_frames(F):
    seq = synth.StreamSequence(frames=300, samples=40000, bits=8, sigma=40.0, seed=4)
    ctx = F.Context(50000, bits=8)
    f0 = seq.frame(0)
    ctx.run(_dev(f0.xyz), _dev(f0.noisy))
    ctx.sync()
    q0 = ctx.stats()["q"]
    ctx.run_reuse(_dev(np.zeros((0, 3), np.int32)), _dev(np.zeros((0, 3), np.uint8)))   # an empty frame
    for t in (1, 2):
        f = seq.frame(t)
        ctx.run_reuse(_dev(f.xyz), _dev(f.noisy))
        ctx.sync()
        assert ctx.stats()["q"] == q0
    ctx.close()
