"""Patch moments of the noise estimate (Section 2.3), bit for bit.

With uint8 colours the library sums the patches' entries (centred on 128) on
the tensor pipe: float16 tiles, float32 accumulation moved to int64 before any
partial sum could leave float32's exact-integer range.  These tests compare its
sums with the exact integer sums of the oracle's patches, entry by entry, at
windows 1, 2 and 3, with sorted and link-order patches, on frames whose tiles
of 16 and 32 patches end raggedly, and with long runs of the extreme colour
values (0 and 255, the largest products)."""
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
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    return fgbd


def oracle_sums(xyz, rgb, bits, window, unsorted=False):
    codes = orc.scan_line_codes(xyz, bits)
    orders = orc.scan_orders(codes)
    row_ptr, col = orc.adjacency_csr(orc.slg_edges(orders, window), len(xyz))
    A, _ = orc.patch_vectors(xyz, rgb, row_ptr, col, 6 * window, orders if unsorted else None)
    a = np.rint(A).astype(np.int64) - 128
    s2 = np.triu(a.T @ a)
    return s2, a.sum(axis=0), a.shape[0]


def gpu_sums(F, xyz, rgb, bits, window, variant=0):
    ctx = F.Context(len(xyz), bits=bits, window=window, variant=variant)
    ctx.build_graph(torch.from_numpy(xyz).cuda())
    ctx.estimate_noise(torch.from_numpy(rgb).cuda())
    out = ctx.debug_moments()
    ctx.close()
    return out


def check(F, xyz, rgb, bits, window, variant=0):
    s2, s1, n = gpu_sums(F, xyz, rgb, bits, window, variant)
    r2, r1, rn = oracle_sums(xyz, rgb, bits, window, unsorted=bool(variant & F.VARIANT_UNSORTED_PATCH))
    assert n == rn and n > 0
    assert np.array_equal(s1, r1)
    assert np.array_equal(s2, r2)


@pytest.mark.parametrize("window", [1, 2, 3])
def test_moments_torso_shell(F, window):
    xyz = synth.torso_points(40000, 8, 50 + window)
    rgb = synth.add_noise_u8(synth.piecewise_colors(xyz, 8, 50 + window), 30.0, 60 + window)
    check(F, xyz, rgb, 8, window)


@pytest.mark.parametrize("window,n,bits,seed", [(1, 37, 3, 1), (1, 4133, 6, 2), (1, 70001, 9, 3),
                                                (2, 4133, 6, 4), (3, 9001, 7, 5)])
def test_moments_random_clouds(F, window, n, bits, seed):
    rng = np.random.default_rng(seed)
    xyz = rng.integers(0, 1 << bits, size=(n, 3)).astype(np.int32)
    rgb = rng.integers(0, 256, size=(n, 3)).astype(np.uint8)
    check(F, xyz, rgb, bits, window)


@pytest.mark.parametrize("window", [1, 3])
def test_moments_extreme_colours(F, window):
    """Only 0 and 255: every product is +-2^14 or near it, the largest partial sums."""
    xyz = synth.torso_points(60000, 8, 70 + window)
    rng = np.random.default_rng(71)
    rgb = np.where(rng.random((len(xyz), 3)) < 0.5, 0, 255).astype(np.uint8)
    rgb[: len(xyz) // 2] = 0   # a long run of equal extremes
    check(F, xyz, rgb, 8, window)


def test_moments_unsorted_patches(F):
    xyz = synth.torso_points(30000, 8, 80)
    rgb = synth.add_noise_u8(synth.piecewise_colors(xyz, 8, 80), 20.0, 81)
    check(F, xyz, rgb, 8, 1, variant=F.VARIANT_UNSORTED_PATCH)


def test_moments_full_size_frame(F):
    """The benchmarked 1M-point torso frame (b = 10), against the oracle's sums."""
    xyz = synth.torso_points(1_000_000, 10, 0)
    rgb = synth.add_noise_u8(synth.piecewise_colors(xyz, 10, 0), 30.0, 11)
    check(F, xyz, rgb, 10, 1)
