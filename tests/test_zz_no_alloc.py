"""The allocation-free scan orders agree with the context-based ones and the oracle.

``fgbd_scan_orders_static`` is for callers that cannot allocate device memory
when they need the scan orders (a real-time frame loop where an allocation
would stall the frame, or a host application that owns all device memory).
Its scratch is one fixed device array shared by every call, so this test makes
two calls in a row, the second on a smaller cloud with another bit width, and
checks each against ``fgbd_build_graph`` + ``fgbd_get_orders`` on the same
input and against the oracle's stable sorts of the three codes.  Orders are
integers, so the comparisons are exact, as in the other parity tests.  A
coordinate out of range must set status bit 1.  The file name sorts last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import fgbd_oracle as orc
from paper_2401_09721_gb300 import build, synth

pytestmark = pytest.mark.gpu

MAX_POINTS = 32768  # FGBD_STATIC_MAX_POINTS


def _call(lib, x, n, bits, out, status, stream):
    return lib.fgbd_scan_orders_static(ctypes.c_void_p(x.data_ptr()), n, bits, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_static_orders_match_context_orders_on_two_calls():
    build.build()
    from paper_2401_09721_gb300 import fgbd

    lib = fgbd.lib()
    stream = torch.cuda.current_stream()
    cases = [
        (synth.torso_points(MAX_POINTS, 10, 21), 10),                                        # the maximum size
        (np.random.default_rng(5).integers(0, 512, size=(20001, 3)).astype(np.int32), 9),    # smaller, repeats
    ]
    for xyz, bits in cases:
        n = xyz.shape[0]
        x = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.int32)).cuda()
        got = torch.full((3, n), -1, dtype=torch.int32, device="cuda")
        status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
        assert _call(lib, x, n, bits, got, status, stream) == 0
        ctx = fgbd.Context(n, bits=bits)
        ctx.build_graph(x)
        want = ctx.orders()
        torch.cuda.synchronize()
        assert status.item() == 0
        assert torch.equal(got, want)
        ctx.close()
        ref = orc.scan_orders(orc.scan_line_codes(xyz, bits)).astype(np.int32)
        assert np.array_equal(got.cpu().numpy(), ref)


def test_static_orders_flag_a_coordinate_out_of_range():
    build.build()
    from paper_2401_09721_gb300 import fgbd

    lib = fgbd.lib()
    stream = torch.cuda.current_stream()
    xyz = np.random.default_rng(9).integers(0, 256, size=(5000, 3)).astype(np.int32)
    xyz[1234, 1] = 256                                                         # y = 2^bits
    x = torch.from_numpy(xyz).cuda()
    got = torch.empty((3, xyz.shape[0]), dtype=torch.int32, device="cuda")
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    assert _call(lib, x, xyz.shape[0], 8, got, status, stream) == 0
    torch.cuda.synchronize()
    assert status.item() & 1
    # the next call on valid input clears the bit
    x = torch.from_numpy(np.clip(xyz, 0, 255)).cuda()
    assert _call(lib, x, xyz.shape[0], 8, got, status, stream) == 0
    torch.cuda.synchronize()
    assert status.item() == 0


def test_static_orders_reject_sizes_beyond_the_maximum():
    build.build()
    from paper_2401_09721_gb300 import fgbd

    lib = fgbd.lib()
    assert lib.fgbd_scan_orders_static(None, MAX_POINTS + 1, 10, None, None, None) == 1   # FGBD_EINVAL
    assert lib.fgbd_scan_orders_static(None, -1, 10, None, None, None) == 1
    assert lib.fgbd_scan_orders_static(None, 100, 11, None, None, None) == 1
