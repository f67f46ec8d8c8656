"""Pins for the FP64 oracle: each checks it against something other than itself.

Sources of truth used here: hand-derived cases under ``tests/golden`` (each
with its citation), the pure-Python brute force in ``brute_force.py``, closed
forms, the spectral identity of Eq. 5, invariances that follow from Eq. 1-3,
and statistical recovery of a known noise level.
"""
import json
import math
import os

import numpy as np
import pytest

import brute_force as bf
from oracle import fgbd_oracle as orc
from paper_2401_09721_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def graph_of(xyz, bits, window=1):
    codes = orc.scan_line_codes(xyz, bits)
    orders = orc.scan_orders(codes)
    edges = orc.slg_edges(orders, window)
    row_ptr, col = orc.adjacency_csr(edges, len(xyz))
    return codes, orders, edges, row_ptr, col


def csr_sets(row_ptr, col):
    return [set(col[row_ptr[i]:row_ptr[i + 1]].tolist()) for i in range(len(row_ptr) - 1)]


def random_cloud(rng, n, bits, dup_frac=0.0):
    side = 1 << bits
    xyz = rng.integers(0, side, size=(n, 3))
    if dup_frac > 0 and n > 2:
        ndup = max(1, int(dup_frac * n))
        src = rng.integers(0, n, size=ndup)
        dst = rng.integers(0, n, size=ndup)
        xyz[dst] = xyz[src]
    return xyz.astype(np.int32)


# ---------------------------------------------------------------- SLG, Section 2.2

def test_codes_orders_edges_hand_example():
    gd = load("slg_six_points.json")
    xyz = np.array(gd["xyz"])
    codes, orders, edges, row_ptr, col = graph_of(xyz, gd["bits"])
    assert codes.tolist() == gd["codes"]
    assert orders.tolist() == gd["orders"]
    assert edges.tolist() == gd["edges"]
    assert [sorted(s) for s in csr_sets(row_ptr, col)] == gd["neighbours"]
    t = gd["sigma_g_terms"]
    expect = (t["ones"] + t["sqrt2"] * math.sqrt(2) + t["sqrt3"] * math.sqrt(3)
              + t["sqrt5"] * math.sqrt(5)) / t["edges"]
    assert orc.sigma_g(xyz, row_ptr, col) == pytest.approx(expect, rel=1e-15)


def test_same_line_links_hand_example():
    """Four points on a 2x2 square in the z = 0 plane: along C1 and C3 the
    middle pair (1, 2) is a jump to the next scan line, along C2 the pair
    (2, 1); with the jumps kept the graph is the square plus the diagonal 1-2,
    without them the square alone."""
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.int32)
    codes = orc.scan_line_codes(xyz, 2)
    orders = orc.scan_orders(codes)
    assert orders.tolist() == [[0, 1, 2, 3], [0, 2, 1, 3], [0, 1, 2, 3]]
    assert orc.slg_edges(orders).tolist() == [[0, 1], [0, 2], [1, 2], [1, 3], [2, 3]]
    assert orc.slg_edges(orders, 1, codes, 2).tolist() == [[0, 1], [0, 2], [1, 3], [2, 3]]


@pytest.mark.parametrize("seed", range(8))
def test_same_line_graph_matches_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 60))
    bits = int(rng.integers(1, 4))
    xyz = random_cloud(rng, n, bits, dup_frac=0.15 if seed % 2 else 0.0)
    pts = [tuple(int(v) for v in p) for p in xyz]
    codes = orc.scan_line_codes(xyz, bits)
    edges = orc.slg_edges(orc.scan_orders(codes), 1, codes, bits)
    row_ptr, col = orc.adjacency_csr(edges, n)
    assert csr_sets(row_ptr, col) == bf.neighbour_sets(pts, 1, same_line=True)


@pytest.mark.parametrize("seed", range(12))
def test_graph_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 45))
    bits = int(rng.integers(1, 5))
    window = 1 if seed % 3 else 2
    xyz = random_cloud(rng, n, bits, dup_frac=0.15 if seed % 2 else 0.0)
    pts = [tuple(int(v) for v in p) for p in xyz]
    _, orders, _, row_ptr, col = graph_of(xyz, bits, window)
    assert orders.tolist() == bf.orders(pts)
    nb = bf.neighbour_sets(pts, window)
    assert csr_sets(row_ptr, col) == nb
    assert orc.sigma_g(xyz, row_ptr, col) == pytest.approx(bf.sigma_g(pts, nb), rel=1e-12)


@pytest.mark.parametrize("window", [1, 2, 3])
def test_graph_invariants(window):
    rng = np.random.default_rng(5)
    xyz = random_cloud(rng, 400, 5, dup_frac=0.05)
    _, _, edges, row_ptr, col = graph_of(xyz, 5, window)
    n = len(xyz)
    A = np.zeros((n, n), int)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    A[rows, col] = 1
    assert (A == A.T).all()                 # symmetric
    assert np.trace(A) == 0                 # no self loops
    assert np.diff(row_ptr).max() <= 6 * window   # at most 2w neighbours x 3 codes
    assert (np.diff(row_ptr) >= 1).all()    # n >= 2: every point is linked
    for i in range(n):                      # rows sorted by column
        r = col[row_ptr[i]:row_ptr[i + 1]]
        assert (np.diff(r) > 0).all()


def test_axis_rotation_permutes_codes_graph_invariant():
    # (x,y,z) -> (y,z,x) maps the code family {C1,C2,C3} onto itself (Eq. 1-3),
    # so the union graph is unchanged.
    rng = np.random.default_rng(11)
    xyz = random_cloud(rng, 300, 6)
    rot = xyz[:, [1, 2, 0]]
    _, o1, e1, _, _ = graph_of(xyz, 6)
    _, o2, e2, _, _ = graph_of(rot, 6)
    assert e1.tolist() == e2.tolist()
    assert o1[0].tolist() == o2[2].tolist()
    assert o1[1].tolist() == o2[0].tolist()
    assert o1[2].tolist() == o2[1].tolist()


def test_point_permutation_equivariance():
    rng = np.random.default_rng(12)
    xyz = np.unique(random_cloud(rng, 500, 6), axis=0)  # distinct voxels: no index ties
    perm = rng.permutation(len(xyz))
    _, _, e1, _, _ = graph_of(xyz, 6)
    _, _, e2, _, _ = graph_of(xyz[perm], 6)
    mapped = np.sort(perm[e2], axis=1)
    mapped = mapped[np.lexsort((mapped[:, 1], mapped[:, 0]))]
    assert mapped.tolist() == e1.tolist()


def test_translation_invariance():
    rng = np.random.default_rng(13)
    xyz = random_cloud(rng, 300, 5)
    _, _, e1, rp1, c1 = graph_of(xyz, 6)
    _, _, e2, rp2, c2 = graph_of(xyz + 17, 6)
    assert e1.tolist() == e2.tolist()
    assert orc.sigma_g(xyz, rp1, c1) == orc.sigma_g(xyz + 17, rp2, c2)


# ---------------------------------------------------------------- weights, Eq. 4

def test_weights_hand_example_and_normalisation():
    gd = load("slg_six_points.json")
    xyz = np.array(gd["xyz"])
    _, _, _, row_ptr, col = graph_of(xyz, gd["bits"])
    sg = orc.sigma_g(xyz, row_ptr, col)
    w = orc.edge_weights(xyz, row_ptr, col, sg)
    rows = np.repeat(np.arange(len(xyz)), np.diff(row_ptr))
    for r, c, wv in zip(rows, col, w):
        key = f"{min(r, c)}-{max(r, c)}"
        assert wv == pytest.approx(math.exp(-gd["edge_sq_len"][key] / sg ** 2), rel=1e-15)
    rw = orc.random_walk_weights(xyz, row_ptr, col, sg)
    deg = np.bincount(rows, weights=w)
    assert np.allclose(rw, w / deg[rows], rtol=1e-14)
    assert np.allclose(np.bincount(rows, weights=rw), 1.0, rtol=1e-14)


def test_random_walk_weights_survive_underflow():
    # Two far clusters joined only by scan-line jumps: plain weights of a long
    # edge underflow, the row-normalised ones do not.
    xyz = np.array([[0, 0, 0], [1, 0, 0], [1023, 1023, 1023], [1022, 1023, 1023]])
    _, _, _, row_ptr, col = graph_of(xyz, 10)
    sg = 1.0
    rw = orc.random_walk_weights(xyz, row_ptr, col, sg)
    rows = np.repeat(np.arange(4), np.diff(row_ptr))
    assert np.isfinite(rw).all()
    assert np.allclose(np.bincount(rows, weights=rw), 1.0)
    w = orc.edge_weights(xyz, row_ptr, col, sg)
    assert (w == 0).any()


# ---------------------------------------------------------------- filter, Eq. 5

def test_filter_one_step_hand_example():
    gd = load("filter_small.json")["path3"]
    xyz = np.array(gd["xyz"])
    _, _, _, row_ptr, col = graph_of(xyz, gd["bits"])
    sg = orc.sigma_g(xyz, row_ptr, col)
    assert sg == gd["sigma_g"]
    rw = orc.random_walk_weights(xyz, row_ptr, col, sg)
    f = np.zeros((3, 3))
    f[:, 0] = gd["red"]
    x1 = orc.lowpass(f, row_ptr, col, rw, 1)
    a, b = math.exp(-4 / 9), math.exp(-16 / 9)
    expect1 = 10 + (10 * a + 40 * b) / (2 * (a + b))
    assert x1[:, 0] == pytest.approx([15.0, expect1, 30.0], rel=1e-14)
    assert (x1[:, 1:] == 0).all()


def test_filter_brute_force_and_identities():
    rng = np.random.default_rng(21)
    xyz = random_cloud(rng, 40, 4)
    pts = [tuple(int(v) for v in p) for p in xyz]
    f = rng.uniform(0, 255, size=(40, 3))
    _, _, _, row_ptr, col = graph_of(xyz, 4)
    sg = orc.sigma_g(xyz, row_ptr, col)
    rw = orc.random_walk_weights(xyz, row_ptr, col, sg)
    nb = bf.neighbour_sets(pts)
    for q in (0, 1, 3):
        got = orc.lowpass(f, row_ptr, col, rw, q)
        ref = np.array(bf.filter_power(pts, f.tolist(), nb, sg, q))
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-10)
    assert np.array_equal(orc.lowpass(f, row_ptr, col, rw, 0), f)       # q = 0 is the identity
    const = np.full((40, 3), 77.25)
    assert np.allclose(orc.lowpass(const, row_ptr, col, rw, 9), 77.25)   # row-stochastic


def test_filter_spectral_response():
    # Eq. 5 has graph-frequency response h_q(lambda) = (1 - lambda/2)^q, lambda the
    # eigenvalues of the random-walk Laplacian I - D^{-1}W.  Computed here through
    # the symmetric normalised Laplacian and eigh, a route independent of the
    # oracle's vertex-domain iteration.
    rng = np.random.default_rng(3)
    xyz = np.unique(random_cloud(rng, 150, 5), axis=0)
    n = len(xyz)
    _, _, _, row_ptr, col = graph_of(xyz, 5)
    sg = orc.sigma_g(xyz, row_ptr, col)
    w = orc.edge_weights(xyz, row_ptr, col, sg)
    rw = orc.random_walk_weights(xyz, row_ptr, col, sg)
    W = np.zeros((n, n))
    W[np.repeat(np.arange(n), np.diff(row_ptr)), col] = w
    d = W.sum(1)
    Lsym = np.eye(n) - W / np.sqrt(np.outer(d, d))
    lam, U = np.linalg.eigh(Lsym)
    assert lam.min() > -1e-10 and lam.max() < 2 + 1e-10
    f = rng.uniform(0, 255, size=(n, 3))
    for q in (1, 2, 5):
        H = np.diag((1 - lam / 2) ** q)
        spectral = np.diag(d ** -0.5) @ U @ H @ U.T @ np.diag(d ** 0.5) @ f
        assert np.allclose(orc.lowpass(f, row_ptr, col, rw, q), spectral, rtol=1e-9, atol=1e-8)


# ---------------------------------------------------------------- selection, Eq. 6

def test_select_q_pair_closed_form():
    gd = load("filter_small.json")["pair"]
    xyz = np.array(gd["xyz"])
    y = np.array(gd["colors"], float)
    _, _, _, row_ptr, col = graph_of(xyz, gd["bits"])
    rw = orc.random_walk_weights(xyz, row_ptr, col, orc.sigma_g(xyz, row_ptr, col))
    keep = np.ones(2, bool)
    for case in gd["cases"]:
        q, xq, J = orc.select_q(y, row_ptr, col, rw, keep, case["sigma"], q_max=10)
        assert q == case["q"]
        assert J == pytest.approx(case["J"], abs=1e-12)


def test_select_q_constant_and_q0():
    rng = np.random.default_rng(4)
    xyz = random_cloud(rng, 200, 5)
    _, _, _, row_ptr, col = graph_of(xyz, 5)
    rw = orc.random_walk_weights(xyz, row_ptr, col, orc.sigma_g(xyz, row_ptr, col))
    const = np.full((200, 3), 100.0)
    q, xq, J = orc.select_q(const, row_ptr, col, rw, np.ones(200, bool), 7.0)
    assert q == 0 and J[0] == 49.0 and J[1] == pytest.approx(49.0, abs=1e-9)
    y = rng.uniform(0, 255, size=(200, 3))
    assert orc.selection_objective(y, y, np.ones(200, bool), 3.0) == 9.0   # J(0) = sigma^2


def test_selection_objective_limited_region():
    y = np.array([[10.0, 0, 0], [20.0, 0, 0], [30.0, 0, 0]])
    x = np.array([[11.0, 0, 0], [19.0, 0, 0], [0.0, 0, 0]])
    keep = np.array([True, True, False])
    # kept power lost: (100 - 121) + (400 - 361) = 18 over 3 channels x 2 points
    assert orc.selection_objective(y, x, keep, 2.0) == pytest.approx(abs(4 - 18 / 6))


# ---------------------------------------------------------------- FSLR, Section 2.4

def test_spread_hand_example_and_brute_force():
    gd = load("slg_six_points.json")
    xyz = np.array(gd["xyz"])
    colors = np.array(gd["colors"], float)
    _, _, _, row_ptr, col = graph_of(xyz, gd["bits"])
    s = orc.fslr_spread(colors, row_ptr, col)
    assert s[3] == pytest.approx((math.sqrt(6) + math.sqrt(8)) / 3, rel=1e-14)
    nb = [set(map(int, col[row_ptr[i]:row_ptr[i + 1]])) for i in range(len(xyz))]
    for i in range(len(xyz)):
        assert s[i] == pytest.approx(bf.spread(colors.tolist(), nb, i), rel=1e-12, abs=1e-12)


# ---------------------------------------------------------------- ablations (Tables 4 and 5)

@pytest.mark.parametrize("seed", range(3))
def test_unsorted_patches_brute_force(seed):
    # "NE-GBP w/o sort": the oracle's link-order patches equal the brute-force ones,
    # they hold the same colours per patch as the sorted ones (a permutation of the
    # neighbour blocks), and so the mean over the six neighbour blocks of mu agrees
    rng = np.random.default_rng(300 + seed)
    xyz = random_cloud(rng, 80, 3, dup_frac=0.05 if seed == 2 else 0.0)
    colors = rng.integers(0, 256, size=(80, 3))
    pts = [tuple(int(v) for v in p) for p in xyz]
    _, orders, _, row_ptr, col = graph_of(xyz, 3)
    A_u, idx_u = orc.patch_vectors(xyz, colors, row_ptr, col, 6, orders=orders)
    A_s, idx_s = orc.patch_vectors(xyz, colors, row_ptr, col, 6)
    nb = bf.neighbour_sets(pts)
    ref = bf.link_order_patches(pts, colors.tolist(), nb, 6)
    assert A_u.shape[0] == len(ref) > 5 and np.array_equal(A_u, np.array(ref))
    assert np.array_equal(idx_u, idx_s)
    blocks_u = np.sort(A_u[:, 3:].reshape(-1, 6, 3), axis=1)
    blocks_s = np.sort(A_s[:, 3:].reshape(-1, 6, 3), axis=1)
    assert np.array_equal(blocks_u, blocks_s)
    _, mu_u = orc.patch_covariance(A_u)
    _, mu_s = orc.patch_covariance(A_s)
    assert np.allclose(mu_u[3:].reshape(6, 3).mean(axis=0), mu_s[3:].reshape(6, 3).mean(axis=0), rtol=1e-12)
    assert np.allclose(mu_u[:3], mu_s[:3], rtol=0, atol=0)


def test_no_fslr_objective_brute_force():
    # "FGBD w/o FSLR": every point enters Eq. 6; J(q) recomputed from the
    # brute-force filter over all points with the oracle's sigma_est
    g = np.array([(x, y, z) for x in range(12) for y in range(6) for z in range(2)], np.int32)
    rng = np.random.default_rng(7)
    f = np.where(g[:, 0:1] < 6, 60.0, 190.0) * np.ones((1, 3)) + rng.normal(0, 8, size=(g.shape[0], 3))
    res = orc.fgbd(g, f, orc.Params(bits=4, fslr=False, q_max=6))
    full = orc.fgbd(g, f, orc.Params(bits=4, q_max=6))
    assert res.keep.all() and not full.keep.all()
    pts = [tuple(int(v) for v in p) for p in g]
    nb = bf.neighbour_sets(pts)
    sg = bf.sigma_g(pts, nb)
    s2 = res.noise["sigma_est"] ** 2
    y = f.tolist()
    for q in range(len(res.J)):
        x = bf.filter_power(pts, y, nb, sg, q)
        p = sum(y[i][c] ** 2 - x[i][c] ** 2 for i in range(len(pts)) for c in range(3))
        assert res.J[q] == pytest.approx(abs(s2 - p / (3 * len(pts))), rel=1e-9, abs=1e-9)


def test_fslr_keep_rule():
    s = np.array([0.0, 3.9, 4.0, 4.1])
    assert orc.fslr_keep(s, 2.0, 2.0).tolist() == [True, True, True, False]   # strict ">" excludes
    assert orc.fslr_keep(np.array([9.0, 9.0]), 1.0, 2.0).tolist() == [True, True]  # none left: all


def test_fslr_masks_sharp_edge():
    # A colour step across the middle of a dense slab: points on the step get a
    # large patch spread and are left out, flat points are kept.
    g = np.array([(x, y, z) for x in range(16) for y in range(16) for z in range(2)], np.int32)
    f = np.where(g[:, 0:1] < 8, 50.0, 200.0) * np.ones((1, 3))
    _, _, _, row_ptr, col = graph_of(g, 4)
    s = orc.fslr_spread(f, row_ptr, col)
    keep = orc.fslr_keep(s, 5.0, 2.0)
    near = (g[:, 0] == 7) | (g[:, 0] == 8)
    assert not keep[near].all()
    assert keep[(g[:, 0] < 5) | (g[:, 0] > 10)].sum() > 0.8 * ((g[:, 0] < 5) | (g[:, 0] > 10)).sum()


# ---------------------------------------------------------------- NE-GBP, Section 2.3

@pytest.mark.parametrize("seed", range(4))
def test_patches_and_covariance_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    xyz = random_cloud(rng, 70, 3, dup_frac=0.1 if seed == 3 else 0.0)
    colors = rng.integers(0, 256, size=(70, 3))
    pts = [tuple(int(v) for v in p) for p in xyz]
    _, _, _, row_ptr, col = graph_of(xyz, 3)
    A, idx = orc.patch_vectors(xyz, colors, row_ptr, col, 6)
    nb = bf.neighbour_sets(pts)
    ref = bf.patches(pts, colors.tolist(), nb, 6)
    assert len(ref) == A.shape[0] and A.shape[0] > 5
    assert np.array_equal(A, np.array(ref))
    S, mu = orc.patch_covariance(A)
    Sref, muref = bf.patch_covariance(ref)
    assert np.allclose(S, np.array(Sref), rtol=1e-12, atol=1e-9)
    assert np.allclose(mu, muref, rtol=1e-14)


@pytest.mark.parametrize("window,seed", [(2, 0), (2, 1), (3, 2), (3, 3)])
def test_patches_wider_windows_brute_force(window, seed):
    """Windows w > 1: K = 6w neighbours, D = 3 (6w + 1) patch entries, each
    patch in increasing distance order, against the brute-force construction."""
    rng = np.random.default_rng(200 + seed)
    xyz = random_cloud(rng, 150, 3, dup_frac=0.05 if seed % 2 else 0.0)
    colors = rng.integers(0, 256, size=(150, 3))
    pts = [tuple(int(v) for v in p) for p in xyz]
    _, _, _, row_ptr, col = graph_of(xyz, 3, window)
    k = 6 * window
    A, idx = orc.patch_vectors(xyz, colors, row_ptr, col, k)
    nb = bf.neighbour_sets(pts, window)
    ref = bf.patches(pts, colors.tolist(), nb, k)
    assert A.shape[1] == 3 * (k + 1)
    assert len(ref) == A.shape[0] and A.shape[0] > 5
    assert np.array_equal(A, np.array(ref))
    res = orc.fgbd(xyz, colors.astype(np.uint8), orc.Params(bits=3, window=window))
    assert res.noise["n_patches"] == A.shape[0] and len(res.noise["eigenvalues"]) == 3 * (k + 1)


def test_tail_rule_hand_cases():
    for case in load("tail_rule.json")["cases"]:
        m, tau, s = orc.tail_rule(np.array(case["lambda"], float))
        assert (m, tau) == (case["m"], case["tau"]), case["why"]
        assert s == pytest.approx(math.sqrt(case["tau"]), rel=1e-15)


def test_eigen_tail_closed_form_spectrum():
    # Sigma with a rank-3 signal above an isotropic floor sigma^2: the tail rule
    # strips exactly the signal and returns sigma.
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((21, 21)))
    lam = np.array([5000.0, 900.0, 300.0] + [144.0] * 18)
    S = Q @ np.diag(lam) @ Q.T
    got = orc.eigenvalues_desc((S + S.T) / 2)
    assert np.allclose(got, lam, rtol=1e-10)
    m, tau, s = orc.tail_rule(got)
    assert m == 3 and s == pytest.approx(12.0, rel=1e-10)


def test_rank_deficient_covariance_gives_exact_zeros():
    # fewer patches than the patch dimension: Sigma has rank <= N' - 1, and
    # the remaining eigenvalues are exactly 0, not rounding noise
    rng = np.random.default_rng(17)
    A = rng.uniform(0, 255, size=(12, 21))
    S, _ = orc.patch_covariance(A)
    lam = orc.eigenvalues_desc(S)
    assert (lam[11:] == 0.0).all() and (lam[:11] > 0).all()
    ref = np.linalg.svd(A - A.mean(0), compute_uv=False) ** 2 / 12
    assert np.allclose(lam[:11], ref[:11], rtol=1e-10)
    # a channel without variation removes its 7 patch entries
    B = rng.uniform(0, 255, size=(500, 21))
    B[:, 1::3] = 77.0
    lamb = orc.eigenvalues_desc(orc.patch_covariance(B)[0])
    assert (lamb[14:] == 0.0).all() and (lamb[:14] > 0).all()
    # all patches equal: every eigenvalue and the estimate are 0
    C = np.tile(rng.uniform(0, 255, size=(1, 21)), (40, 1))
    lamc = orc.eigenvalues_desc(orc.patch_covariance(C)[0])
    assert (lamc == 0).all() and orc.tail_rule(lamc)[2] == 0.0


def _noise_recovery(sigma, seed, smooth):
    xyz = synth.sphere_points(20500, 9, seed)
    base = synth.smooth_colors(xyz, 9, seed, as_float=True) if smooth else np.full((len(xyz), 3), 128.0)
    f = synth.add_noise_f32(base, sigma, seed)
    _, _, _, row_ptr, col = graph_of(xyz, 9)
    return orc.estimate_noise(xyz, f, row_ptr, col, 6)


@pytest.mark.parametrize("sigma", [5.0, 10.0, 20.0, 30.0, 50.0])
def test_noise_recovery_white(sigma):
    r = _noise_recovery(sigma, 1, smooth=False)
    assert r["n_patches"] > 15000
    assert abs(r["sigma_est"] - sigma) / sigma < 0.03


_SHELL = {}


def _shell():
    # a densely voxelized body-like shell (8 bits, 60k voxels): the kind of
    # surface the paper evaluates on, where scan-line neighbours are mostly
    # adjacent voxels
    if not _SHELL:
        xyz = synth.torso_points(60000, 8, 0)
        _, _, _, row_ptr, col = graph_of(xyz, 8)
        _SHELL.update(xyz=xyz, row_ptr=row_ptr, col=col)
    return _SHELL


@pytest.mark.parametrize("sigma", [10.0, 20.0, 30.0])
def test_noise_recovery_piecewise_signal(sigma):
    sh = _shell()
    base = synth.piecewise_colors(sh["xyz"], 8, 0, as_float=True)
    f = synth.add_noise_f32(base, sigma, 1)
    r = orc.estimate_noise(sh["xyz"], f, sh["row_ptr"], sh["col"], 6)
    assert r["n_patches"] > 50000
    assert abs(r["sigma_est"] - sigma) / sigma < 0.05


def test_noise_estimate_degenerate():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]])
    f = np.array([[1.0, 2, 3], [4, 5, 6], [7, 8, 9]])
    _, _, _, row_ptr, col = graph_of(xyz, 2)
    r = orc.estimate_noise(xyz, f, row_ptr, col, 6)
    assert r["n_patches"] == 0 and r["sigma_est"] == 0.0


# ---------------------------------------------------------------- whole path

def _psnr(a, b):
    mse = ((a.astype(float) - b.astype(float)) ** 2).mean()
    return 10 * math.log10(255.0 ** 2 / mse)


@pytest.mark.parametrize("sigma", [10.0, 20.0, 30.0])
def test_fgbd_improves_psnr_on_dense_shell(sigma):
    sh = _shell()
    clean = synth.piecewise_colors(sh["xyz"], 8, 0)
    noisy = synth.add_noise_u8(clean, sigma, 0)
    res = orc.fgbd(sh["xyz"], noisy, orc.Params(bits=8))
    noisy_db = _psnr(noisy, clean)
    assert abs(noisy_db - 20 * math.log10(255.0 / sigma)) < 0.6   # PSNR convention: all channels, peak 255
    assert res.q >= 1 and _psnr(res.out, clean) > noisy_db + 3.0
    assert abs(res.noise["sigma_est"] - sigma) / sigma < 0.1
    assert res.J[0] == pytest.approx(res.noise["sigma_est"] ** 2, rel=1e-12)


def test_fgbd_sparse_sphere_runs():
    # the small frame is a sparse sample of a sphere; its scan-line neighbours
    # are mostly long jumps, so the estimate is high, but every step is defined
    fr = synth.sphere_frame(20500, 9, 20.0, 0)
    res = orc.fgbd(fr.xyz, fr.noisy, orc.Params(bits=9))
    assert res.noise["n_patches"] > 15000 and res.q >= 1
    assert res.J[0] == pytest.approx(res.noise["sigma_est"] ** 2, rel=1e-12)
    assert np.isfinite(res.out).all()


# ---------------------------------------------------------------- differentiable filter

def _diff_case(seed=0, n=150, bits=4):
    rng = np.random.default_rng(500 + seed)
    xyz = random_cloud(rng, n, bits)
    y = rng.uniform(0, 255, size=(n, 3))
    _, _, _, row_ptr, col = graph_of(xyz, bits)
    return xyz, y, row_ptr, col, rng


def test_param_filter_reduces_to_eq5():
    xyz, y, row_ptr, col, _ = _diff_case(0)
    sg = orc.sigma_g(xyz, row_ptr, col)
    rw = orc.random_walk_weights(xyz, row_ptr, col, sg)
    for q in (0, 1, 3):
        assert np.allclose(orc.param_filter(xyz, row_ptr, col, y, q, 0.5, sg)[-1],
                           orc.lowpass(y, row_ptr, col, rw, q), rtol=1e-13, atol=1e-11)


@pytest.mark.parametrize("seed", range(3))
def test_param_filter_gradient_finite_differences(seed):
    xyz, y, row_ptr, col, rng = _diff_case(seed)
    q, alpha = 4, 0.35 + 0.1 * seed
    sigma = orc.sigma_g(xyz, row_ptr, col) * (0.8 + 0.2 * seed)
    gout = rng.normal(size=y.shape)
    loss = lambda yy, a, s: float(np.sum(gout * orc.param_filter(xyz, row_ptr, col, yy, q, a, s)[-1]))
    gy, da, ds = orc.param_filter_vjp(xyz, row_ptr, col, y, q, alpha, sigma, gout)
    h = 1e-3

    def central(f, h):   # central differences at steps h and h/2, Richardson-combined (error O(h^4))
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    fd_a = central(lambda d: loss(y, alpha + d, sigma), h)
    fd_s = central(lambda d: loss(y, alpha, sigma + d), h)
    assert da == pytest.approx(fd_a, rel=1e-8, abs=1e-6)
    assert ds == pytest.approx(fd_s, rel=1e-7, abs=1e-6)
    for _ in range(16):   # random colour entries
        i, c = int(rng.integers(len(y))), int(rng.integers(3))
        yp, ym = y.copy(), y.copy()
        yp[i, c] += h
        ym[i, c] -= h
        assert gy[i, c] == pytest.approx((loss(yp, alpha, sigma) - loss(ym, alpha, sigma)) / (2 * h), rel=1e-6, abs=1e-8)


def test_param_filter_adjoint_identity():
    # <P^q y, g> = <y, (P^T)^q g>: the colour gradient of a linear loss
    xyz, y, row_ptr, col, rng = _diff_case(3)
    sg = orc.sigma_g(xyz, row_ptr, col)
    gout = rng.normal(size=y.shape)
    xq = orc.param_filter(xyz, row_ptr, col, y, 5, 0.5, sg)[-1]
    gy, _, _ = orc.param_filter_vjp(xyz, row_ptr, col, y, 5, 0.5, sg, gout)
    assert np.sum(xq * gout) == pytest.approx(np.sum(y * gy), rel=1e-12)


# ---------------------------------------------------------------- alternative readings

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sigma_g_readings_brute_force(seed):
    """node-mean sigma_g and the per-point bandwidths of the pair reading
    against loops over the brute-force neighbour sets."""
    rng = np.random.default_rng(40 + seed)
    xyz = random_cloud(rng, 60, 4, dup_frac=0.1)
    pts = [tuple(int(v) for v in p) for p in xyz]
    nb = bf.neighbour_sets(pts)
    _, _, _, row_ptr, col = graph_of(xyz, 4)
    per, mean = bf.node_sigma(pts, nb)
    assert np.allclose(orc.node_mean_lengths(xyz, row_ptr, col), per, rtol=1e-13, atol=0)
    assert orc.sigma_g_node(xyz, row_ptr, col) == pytest.approx(mean, rel=1e-13)
    # edge and node means differ unless every point has the same mean edge length
    assert orc.sigma_g(xyz, row_ptr, col) != pytest.approx(mean, rel=1e-6)
    scale = orc.pair_scale(xyz, row_ptr, col)
    rows = np.repeat(np.arange(len(pts)), np.diff(row_ptr))
    assert np.allclose(scale, [per[i] * per[j] for i, j in zip(rows, col)], rtol=1e-13, atol=0)


def test_sigma_g_node_hand_example():
    # a path of four points along x with edge lengths 1, 3 and 5: the edge
    # mean is 3; the points' mean edge lengths are 1, 2, 4 and 5, whose mean
    # is 3 as well.  A path 0-1-2 with lengths 1 and 8 separates the readings:
    # edge mean 4.5, point means 1, 4.5 and 8, node mean 13.5 / 3 = 4.5 -- equal
    # again (a path always gives equal means); a star does not: centre linked
    # to leaves at 1, 1 and 4 has edge mean 2 and point means 2, 1, 1, 4,
    # node mean 2; leaves at 2, 2 and 8: edge mean 4, point means 4, 2, 2, 8,
    # node mean 4.  With a second centre the weights differ: see the random clouds.
    xyz4 = np.array([[0, 0, 0], [1, 0, 0], [4, 0, 0], [9, 0, 0]])
    row_ptr4 = np.array([0, 1, 3, 5, 6])
    col4 = np.array([1, 0, 2, 1, 3, 2])
    assert orc.sigma_g(xyz4, row_ptr4, col4) == 3.0
    assert orc.node_mean_lengths(xyz4, row_ptr4, col4).tolist() == [1.0, 2.0, 4.0, 5.0]
    assert orc.sigma_g_node(xyz4, row_ptr4, col4) == 3.0
    # two stars sharing a leaf: centres a (0) and b (4); a has leaves at 1 and 1
    # (points 1, 2), b has the leaf 3 at distance 2 and shares leaf 1 (distance
    # from b to point 1 is 3).  Edges: a-1 (1), a-2 (1), b-3 (2), b-1 (3):
    # edge mean 7 / 4 = 1.75; point means a 1, point 1 (1 + 3) / 2 = 2,
    # point 2 1, b (2 + 3) / 2 = 2.5, point 3 2: node mean 8.5 / 5 = 1.7.
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [4, 0, 0], [4, 2, 0]])
    edges = [(0, 1), (0, 2), (3, 4), (3, 1)]
    nbs = [[] for _ in range(5)]
    for a, b in edges:
        nbs[a].append(b)
        nbs[b].append(a)
    row_ptr = np.cumsum([0] + [len(v) for v in nbs])
    col = np.array([c for v in nbs for c in sorted(v)])
    assert orc.sigma_g(xyz, row_ptr, col) == pytest.approx(1.75)
    assert orc.node_mean_lengths(xyz, row_ptr, col).tolist() == [1.0, 2.0, 1.0, 2.5, 2.0]
    assert orc.sigma_g_node(xyz, row_ptr, col) == pytest.approx(1.7)


@pytest.mark.parametrize("seed", [0, 1])
def test_pair_weights_filter_brute_force(seed):
    rng = np.random.default_rng(60 + seed)
    xyz = random_cloud(rng, 40, 4)
    pts = [tuple(int(v) for v in p) for p in xyz]
    f = rng.uniform(0, 255, size=(40, 3))
    _, _, _, row_ptr, col = graph_of(xyz, 4)
    per, _ = bf.node_sigma(pts, bf.neighbour_sets(pts))
    rw = orc.random_walk_weights(xyz, row_ptr, col, 0.0, orc.pair_scale(xyz, row_ptr, col))
    nb = bf.neighbour_sets(pts)
    for q in (1, 3):
        got = orc.lowpass(f, row_ptr, col, rw, q)
        ref = np.array(bf.filter_power(pts, f.tolist(), nb, 0.0, q, pair=per))
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-10)
    res = orc.fgbd(xyz, np.clip(f, 0, 255).astype(np.uint8), orc.Params(bits=4, sigma_g_mode="pair"))
    assert np.allclose(res.rw, rw, rtol=1e-13)


@pytest.mark.parametrize("seed", [0, 1])
def test_pooled_patches_brute_force(seed):
    rng = np.random.default_rng(80 + seed)
    xyz = synth.sphere_points(3000, 6, seed)
    f = rng.integers(0, 256, size=(len(xyz), 3)).astype(np.uint8)
    _, _, _, row_ptr, col = graph_of(xyz, 6)
    pts = [tuple(int(v) for v in p) for p in xyz]
    nb = bf.neighbour_sets(pts)
    vecs = bf.patches(pts, f.tolist(), nb)
    cov, mu = bf.pooled_covariance(vecs)
    A, _ = orc.patch_vectors(xyz, f, row_ptr, col, 6)
    S, m = orc.patch_covariance(orc.pooled_patches(A))
    assert S.shape == (7, 7) and np.allclose(S, cov, rtol=1e-10, atol=1e-9) and np.allclose(m, mu)
    r = orc.estimate_noise(xyz, f, row_ptr, col, 6, pooled=True)
    assert r["eigenvalues"].size == 7 and r["n_patches"] == len(vecs)
    # the pooled covariance is the channel average of the 7x7 diagonal blocks of
    # the RGB covariance, plus the spread of the channel means
    S21, mu21 = orc.patch_covariance(A)
    blocks = [S21[c::3, c::3] for c in range(3)]
    means = [mu21[c::3] for c in range(3)]
    mbar = sum(means) / 3
    rebuilt = sum(blocks) / 3 + sum(np.outer(mc - mbar, mc - mbar) for mc in means) / 3
    assert np.allclose(S, rebuilt, rtol=1e-10, atol=1e-9)


def test_pooled_patches_recover_white_noise():
    rng = np.random.default_rng(7)
    xyz = synth.sphere_points(20500, 9, 0)
    f = (128.0 + rng.normal(0, 20.0, size=(len(xyz), 3)))
    _, _, _, row_ptr, col = graph_of(xyz, 9)
    r = orc.estimate_noise(xyz, f, row_ptr, col, 6, pooled=True)
    assert abs(r["sigma_est"] - 20.0) / 20.0 < 0.03


def test_select_q_global_argmin_brute_force():
    """The global rule against J computed for every q with dense powers of D^-1 W."""
    rng = np.random.default_rng(9)
    xyz = np.unique(random_cloud(rng, 120, 5), axis=0)
    n = len(xyz)
    _, _, _, row_ptr, col = graph_of(xyz, 5)
    rw = orc.random_walk_weights(xyz, row_ptr, col, orc.sigma_g(xyz, row_ptr, col))
    R = np.zeros((n, n))
    R[np.repeat(np.arange(n), np.diff(row_ptr)), col] = rw
    P = 0.5 * np.eye(n) + 0.5 * R
    y = rng.uniform(0, 255, size=(n, 3))
    keep = rng.uniform(size=n) < 0.7
    for sigma in (3.0, 15.0, 40.0):
        Js, x = [], y.copy()
        for q in range(0, 13):
            Js.append(abs(sigma ** 2 - ((y[keep] ** 2).sum() - (x[keep] ** 2).sum()) / (3 * keep.sum())))
            x = P @ x
        q, xq, J = orc.select_q(y, row_ptr, col, rw, keep, sigma, q_max=12, rule="global")
        assert len(J) == 13 and np.allclose(J, Js, rtol=1e-9, atol=1e-9)
        assert q == int(np.argmin(Js))
        assert np.allclose(xq, np.linalg.matrix_power(P, q) @ y, rtol=1e-9, atol=1e-8)
        qf, _, Jf = orc.select_q(y, row_ptr, col, rw, keep, sigma, q_max=12)
        # the first local minimum is never below the global one, and the rules agree on a convex curve
        assert Js[qf] >= Js[q]
