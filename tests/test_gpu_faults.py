"""Failure detection without a GPU fault: every device-side wait is bounded.
A zero wait limit makes the grid barriers give up; the next synchronising call
reports FGBD_ETIMEOUT and the context then works again."""
import numpy as np
import pytest
import torch

from paper_2401_09721_gb300 import build, synth

pytestmark = pytest.mark.gpu

FGBD_ETIMEOUT = 5


@pytest.fixture(scope="module")
def F():
    build.build()
    from paper_2401_09721_gb300 import fgbd
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    return fgbd


@pytest.mark.parametrize("flags", [0, 1])
def test_barrier_timeout_is_reported_and_the_context_recovers(F, flags):
    fr = synth.sphere_frame(60000, 9, 40.0, 70)
    ctx = F.Context(fr.n, bits=9, flags=flags)
    x = torch.from_numpy(fr.xyz).cuda()
    c = torch.from_numpy(fr.noisy).cuda()
    ref = ctx.run(x, c).cpu().numpy()
    ctx.sync()
    ctx.set_wait_limit(0)
    ctx.run(x, c)
    with pytest.raises(F.FgbdError) as err:
        ctx.sync()
    assert err.value.status == FGBD_ETIMEOUT
    ctx.sync()  # the latched flag was cleared when it was reported
    ctx.set_wait_limit(2_000_000_000)
    for _ in range(3):  # direct, captured and replayed runs
        out = ctx.run(x, c).cpu().numpy()
        ctx.sync()
        assert np.array_equal(out, ref)
    ctx.close()


def test_negative_limit_is_rejected(F):
    ctx = F.Context(100, bits=9)
    with pytest.raises(F.FgbdError):
        ctx.set_wait_limit(-1)
    ctx.close()
