"""fgbd_run_host: the same results as fgbd_run on device buffers, for pinned
and pageable host memory, with consecutive calls in flight (two staging
slots) and outputs read after fgbd_sync."""
import numpy as np
import pytest
import torch

from paper_2401_09721_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    build.build()
    from paper_2401_09721_gb300 import fgbd
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    return fgbd


@pytest.mark.parametrize("pinned", [True, False])
def test_host_runs_match_device_runs(F, pinned):
    frames = [synth.sphere_frame(30000, 9, s, 40 + i) for i, s in enumerate((15.0, 25.0, 35.0, 45.0, 20.0))]
    n = max(fr.n for fr in frames)
    ref_ctx = F.Context(n, bits=9)
    refs = []
    for fr in frames:
        x = torch.from_numpy(fr.xyz).cuda()
        c = torch.from_numpy(fr.noisy).cuda()
        refs.append(ref_ctx.run(x, c, out_dtype=torch.uint8).cpu().numpy())
    ctx = F.Context(n, bits=9)
    hx = [torch.from_numpy(fr.xyz) for fr in frames]
    hc = [torch.from_numpy(fr.noisy) for fr in frames]
    if pinned:
        hx = [t.pin_memory() for t in hx]
        hc = [t.pin_memory() for t in hc]
    outs = [torch.empty((fr.n, 3), dtype=torch.uint8) for fr in frames]
    if pinned:
        outs = [o.pin_memory() for o in outs]
    # twice over the frames: the second pass replays captured graphs on the staging slots
    for rep in range(2):
        for i in range(len(frames)):
            ctx.run_host(hx[i], hc[i], outs[i])
        ctx.sync()
        for i in range(len(frames)):
            assert np.array_equal(outs[i].numpy(), refs[i]), (rep, i)
    ctx.close()
    ref_ctx.close()


def test_host_run_float_output_and_empty_frame(F):
    fr = synth.sphere_frame(20500, 9, 30.0, 50)
    ctx = F.Context(fr.n, bits=9)
    ref = ctx.run(torch.from_numpy(fr.xyz).cuda(), torch.from_numpy(fr.noisy).cuda()).cpu().numpy()
    out = torch.empty((fr.n, 3), dtype=torch.float32).pin_memory()
    ctx.run_host(torch.from_numpy(fr.xyz).pin_memory(), torch.from_numpy(fr.noisy).pin_memory(), out)
    ctx.sync()
    assert np.array_equal(out.numpy(), ref)
    empty = torch.empty((0, 3), dtype=torch.int32)
    ctx.run_host(empty, torch.empty((0, 3), dtype=torch.uint8), torch.empty((0, 3), dtype=torch.uint8))
    ctx.sync()
    assert ctx.stats()["n"] == 0
    ctx.close()
