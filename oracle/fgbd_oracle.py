"""FP64 CPU oracle for the FGBD per-frame path.  TEST INFRASTRUCTURE ONLY.

A plain, slow, NumPy (float64) restatement of the method of Watanabe, Nonaka,
Pavez, Kobayashi and Ortega, "Fast Graph-Based Denoising for Point Cloud Color
Information" (ICASSP 2024), written from the paper's definitions:

  step 1  SLG scan-line graph          Section 2.2, Eq. 1-3 (codes), Eq. 4 (weights)
  step 2  NE-GBP noise estimate        Section 2.3
  step 3  FSLR filter selection        Section 2.4, Eq. 6 and the limited-region rule
  step 4  graph low-pass filter        Section 2.4, Eq. 5

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The CUDA library never calls it, and it
shares no code with the library: the two meet only at the seeded inputs from
``paper_2401_09721_gb300.synth`` (which holds none of the method's arithmetic).

Where the paper is silent or ambiguous, the reading taken is stated at the
function that implements it.  Every function here is pinned by a ``-m "not gpu"``
test against something other than itself (hand-derived cases, brute force,
closed forms, spectral identities or statistical recovery).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Params",
    "scan_line_codes",
    "scan_orders",
    "slg_edges",
    "adjacency_csr",
    "sigma_g",
    "node_mean_lengths",
    "sigma_g_node",
    "pair_scale",
    "edge_weights",
    "random_walk_weights",
    "patch_vectors",
    "patch_covariance",
    "pooled_patches",
    "eigenvalues_desc",
    "tail_rule",
    "estimate_noise",
    "fslr_spread",
    "fslr_keep",
    "lowpass_step",
    "lowpass",
    "selection_objective",
    "select_q",
    "fgbd",
    "OracleResult",
]


@dataclass
class Params:
    bits: int = 10           # b: coordinate bits (Section 2.2)
    window: int = 1          # linked positions on each side along a scan line (Section 2.2: 1)
    fslr_factor: float = 2.0  # points with mean patch std > factor * sigma_est are skipped (Section 2.4)
    q_max: int = 64          # largest filter power searched (the paper gives none; a reading)
    # ablations of Section 3 (Tables 4 and 5); the defaults are the method as published
    fslr: bool = True             # False: "FGBD w/o FSLR", Eq. 6 over every point
    sorted_patches: bool = True   # False: "NE-GBP w/o sort", patch entries in link order
    # a reading, not the paper's: links only between points of the same scan line
    same_line: bool = False       # True: no link joins the end of one scan line to the next
    # alternative readings where the paper leaves a choice open (the defaults are the readings taken)
    sigma_g_mode: str = "edge"    # sigma_g of Eq. 4 (Section 2.2): "edge" the mean length over the edges;
                                  # "node" the mean over the points of each point's mean edge length;
                                  # "pair" a bandwidth per point, w_ij = exp(-d_ij^2 / (sigma_i sigma_j))
    pooled_patch: bool = False    # Section 2.3: True takes D = K + 1 per colour channel and pools the
                                  # three channels' patches in one covariance (False: D = 3 (K + 1))
    q_rule: str = "first"         # Section 2.4: "first" stops at the first q whose J is not below the
                                  # previous one; "global" takes the argmin of J over q = 0..q_max


# --------------------------------------------------------------------------
# Step 1: SLG graph (Section 2.2)
# --------------------------------------------------------------------------

def scan_line_codes(g: np.ndarray, bits: int) -> np.ndarray:
    """Eq. 1-3: the three raster scan-line codes of each voxel.

    C1 = 2^{2b} z + 2^b y + x,  C2 = 2^{2b} x + 2^b z + y,  C3 = 2^{2b} y + 2^b x + z.
    Returns int64 [3, N].
    """
    g = np.asarray(g, dtype=np.int64)
    x, y, z = g[:, 0], g[:, 1], g[:, 2]
    s1 = np.int64(2) ** bits
    s2 = np.int64(2) ** (2 * bits)
    c1 = s2 * z + s1 * y + x
    c2 = s2 * x + s1 * z + y
    c3 = s2 * y + s1 * x + z
    return np.stack([c1, c2, c3])


def scan_orders(codes: np.ndarray) -> np.ndarray:
    """Section 2.2: points ordered along each scan-line code.

    The paper uses a radix sort; any stable sort yields the same order.  Equal
    codes (repeated voxels) keep their input order (reading: ties by index).
    Returns int64 [3, N]; row l lists point indices in ascending code l.
    """
    return np.stack([np.argsort(c, kind="stable") for c in codes])


def slg_edges(orders: np.ndarray, window: int = 1, codes: np.ndarray | None = None,
              bits: int | None = None) -> np.ndarray:
    """Section 2.2: points consecutive along a code are linked, independently per code.

    With window w, positions k and k+d (1 <= d <= w) are linked; the paper uses
    w = 1 ("two consecutive points"), giving 2 neighbours per code.
    Reading: links are taken in the global sorted order, so they also join the
    end of one scan line to the start of the next (the paper keeps these
    "distant connections").  Reading: the union over codes is a set, so a pair
    linked by several codes is one edge.
    With ``codes`` and ``bits`` given (the same-line ablation), a pair is linked
    along code l only if both points lie on the same scan line of that code,
    i.e. their codes agree in all but the low b bits (the minor coordinate).
    Returns int64 [E, 2] undirected edges (i < j), lexicographically sorted.
    """
    parts = []
    for l, order in enumerate(orders):
        for d in range(1, window + 1):
            a = order[:-d]
            b = order[d:]
            if codes is not None:
                line = codes[l] >> bits
                same = line[a] == line[b]
                a, b = a[same], b[same]
            parts.append(np.stack([np.minimum(a, b), np.maximum(a, b)], axis=1))
    if not parts:
        return np.zeros((0, 2), np.int64)
    e = np.concatenate(parts)
    if e.shape[0] == 0:
        return np.zeros((0, 2), np.int64)
    return np.unique(e, axis=0)


def adjacency_csr(edges: np.ndarray, n: int):
    """Symmetric adjacency of the undirected edge set as CSR (rows sorted by column).

    Returns (row_ptr int64 [n+1], col int64 [2E]).
    """
    rows = np.concatenate([edges[:, 0], edges[:, 1]])
    cols = np.concatenate([edges[:, 1], edges[:, 0]])
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return row_ptr, cols


def _row_index(row_ptr: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(row_ptr.size - 1), np.diff(row_ptr))


def _sq_dist(g: np.ndarray, row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    g = np.asarray(g, dtype=np.int64)
    diff = g[col] - g[_row_index(row_ptr)]
    return (diff * diff).sum(axis=1)  # exact integers


def sigma_g(g: np.ndarray, row_ptr: np.ndarray, col: np.ndarray) -> float:
    """Section 2.2: sigma_g, the average Euclidean distance between points and their neighbours.

    Reading: one global scalar, the mean of ||g_i - g_j|| over all directed
    adjacency entries (equivalently over undirected edges), line-jump edges
    included.  With no edges the value is 0.
    """
    if col.size == 0:
        return 0.0
    return float(np.sqrt(_sq_dist(g, row_ptr, col).astype(np.float64)).mean())


def node_mean_lengths(g: np.ndarray, row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """sigma_i: the mean Euclidean length of point i's edges (0 for a point without edges).

    The per-point bandwidth of the "pair" reading of sigma_g (Section 2.2
    speaks of the average distance between points and their neighbours).
    """
    n = row_ptr.size - 1
    deg = np.diff(row_ptr)
    lengths = np.sqrt(_sq_dist(g, row_ptr, col).astype(np.float64))
    s = np.bincount(_row_index(row_ptr), weights=lengths, minlength=n)
    out = np.zeros(n)
    out[deg > 0] = s[deg > 0] / deg[deg > 0]
    return out


def sigma_g_node(g: np.ndarray, row_ptr: np.ndarray, col: np.ndarray) -> float:
    """The "node" reading of sigma_g (Section 2.2): the mean over the points that
    have edges of their mean edge length (0 without edges)."""
    deg = np.diff(row_ptr)
    if not (deg > 0).any():
        return 0.0
    return float(node_mean_lengths(g, row_ptr, col)[deg > 0].mean())


def pair_scale(g: np.ndarray, row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """sigma_i sigma_j per adjacency entry (the "pair" reading of Eq. 4's sigma_g^2)."""
    si = node_mean_lengths(g, row_ptr, col)
    return si[_row_index(row_ptr)] * si[col]


def edge_weights(g: np.ndarray, row_ptr: np.ndarray, col: np.ndarray, sg: float) -> np.ndarray:
    """Eq. 4: w_ij = exp(-||g_i - g_j||^2 / sigma_g^2) per adjacency entry (float64).

    Reading: (g_i - g_j)^2 in Eq. 4 is the squared Euclidean norm.  If sigma_g
    is 0 (every edge has length 0) all weights are 1.  Long edges may underflow
    to 0 here; ``random_walk_weights`` is the underflow-free row-normalised form.
    """
    d2 = _sq_dist(g, row_ptr, col).astype(np.float64)
    if sg == 0.0:
        return np.ones_like(d2)
    return np.exp(-d2 / (sg * sg))


def random_walk_weights(g: np.ndarray, row_ptr: np.ndarray, col: np.ndarray, sg: float,
                        scale: np.ndarray | None = None) -> np.ndarray:
    """Entries of D^{-1} W (rows of Eq. 4's W divided by their degree d_i = sum_j w_ij).

    Computed as exp(-(d2_ij - min_k d2_ik)/sigma_g^2) / sum_k exp(-(d2_ik - min_k d2_ik)/sigma_g^2),
    which equals w_ij / d_i exactly in real arithmetic (the common factor
    exp(-min d2 / sigma_g^2) cancels) and stays defined when every w_ij of a
    row underflows in floating point.  With ``scale`` (per adjacency entry,
    the "pair" reading: sigma_i sigma_j) the exponents are d2_ij / scale_ij,
    shifted by their row minimum the same way; an entry with scale 0 has
    length 0 (its points' mean edge length is 0) and exponent 0.
    """
    d2 = _sq_dist(g, row_ptr, col).astype(np.float64)
    n = row_ptr.size - 1
    rows = _row_index(row_ptr)
    if d2.size == 0:
        return d2
    if scale is None:
        a = np.zeros_like(d2) if sg == 0.0 else d2 / (sg * sg)
    else:
        a = np.zeros_like(d2)
        pos = scale > 0
        a[pos] = d2[pos] / scale[pos]
    amin = np.full(n, np.inf)
    np.minimum.at(amin, rows, a)
    e = np.exp(-(a - amin[rows]))
    s = np.bincount(rows, weights=e, minlength=n)
    return e / s[rows]


# --------------------------------------------------------------------------
# Step 2: NE-GBP (Section 2.3)
# --------------------------------------------------------------------------

def link_order_neighbours(orders: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """The neighbours of points idx in the order the scan-line graph links them.

    For each code l = 1, 2, 3 (window 1): the point before and the point after
    along the order of C_l.  Returns int64 [len(idx), 6].  Used by the "NE-GBP
    w/o sort" ablation (Section 3 (4), Table 4), whose patch entries are not
    ordered by distance; reading: "not sorted" is this link order.
    """
    n = orders.shape[1]
    out = np.empty((idx.size, 6), dtype=np.int64)
    for l in range(3):
        pos = np.empty(n, dtype=np.int64)
        pos[orders[l]] = np.arange(n)
        p = pos[idx]
        out[:, 2 * l] = orders[l][np.clip(p - 1, 0, n - 1)]
        out[:, 2 * l + 1] = orders[l][np.clip(p + 1, 0, n - 1)]
    return out


def patch_vectors(g: np.ndarray, f: np.ndarray, row_ptr: np.ndarray, col: np.ndarray, k: int,
                  orders: np.ndarray | None = None):
    """Section 2.3: graph-based patches a_i, entries ordered by distance from the query point.

    a_i = [f_i, f_{n1}, ..., f_{nk}] with the neighbours in increasing distance.
    Reading: D = 3 (k + 1) (three colour channels per node, node-major), and only
    points with exactly k distinct neighbours (k = 6w) give a patch; points with
    fewer (the ends of the scan orders, pairs linked by two codes) are left out.
    Reading: equal distances are ordered by the offset g_j - g_i compared as
    (dz, dy, dx) ascending, then by neighbour index.
    With ``orders`` given (window 1 only), the neighbours are not sorted but
    taken in link order (``link_order_neighbours``): the "w/o sort" ablation.
    Returns (A float64 [N', D], idx int64 [N']): the patches and their point indices.
    """
    g = np.asarray(g, dtype=np.int64)
    f = np.asarray(f, dtype=np.float64)
    deg = np.diff(row_ptr)
    idx = np.nonzero(deg == k)[0]
    if idx.size == 0:
        return np.zeros((0, 3 * (k + 1))), idx
    if orders is not None:
        assert k == 6, "link order is defined for window 1"
        members = np.concatenate([idx[:, None], link_order_neighbours(orders, idx)], axis=1)
        return f[members].reshape(idx.size, 3 * (k + 1)), idx
    nb = col[row_ptr[idx][:, None] + np.arange(k)[None, :]]          # [N', k]
    off = g[nb] - g[idx][:, None, :]                                  # [N', k, 3]
    d2 = (off * off).sum(axis=2)
    # lexicographic (d2, dz, dy, dx, j) inside each row; lexsort keys are given last-major
    order = np.lexsort((nb, off[:, :, 0], off[:, :, 1], off[:, :, 2], d2), axis=1)
    nb_sorted = np.take_along_axis(nb, order, axis=1)
    members = np.concatenate([idx[:, None], nb_sorted], axis=1)        # [N', k+1]
    A = f[members].reshape(idx.size, 3 * (k + 1))
    return A, idx


def patch_covariance(A: np.ndarray):
    """Section 2.3: Sigma = (1/N) sum_i (a_i - mu)(a_i - mu)^T with mu the mean patch."""
    n = A.shape[0]
    mu = A.mean(axis=0)
    C = A - mu
    return (C.T @ C) / n, mu


def pooled_patches(A: np.ndarray) -> np.ndarray:
    """The "pooled" reading of Section 2.3's patch dimension: each RGB patch
    (node-major, channel-minor, D = 3 (K + 1)) becomes three single-channel
    patches of K + 1 entries, one per channel, all in one sample: [3 N', K + 1]."""
    n, d = A.shape
    k1 = d // 3
    return A.reshape(n, k1, 3).transpose(0, 2, 1).reshape(3 * n, k1)


ZERO_EIG_REL = 1e-9


def eigenvalues_desc(S: np.ndarray) -> np.ndarray:
    """Section 2.3: eigenvalues of the symmetric covariance, lambda_1 >= ... >= lambda_D.

    Reading: an eigenvalue whose magnitude is below 1e-9 max(lambda_1, 1)
    (colours on the 0..255 scale) is a numerical zero and is returned as
    exactly 0.  Such values only occur when the covariance is rank-deficient
    (fewer patches than D, a colour channel without variation, identical
    patches); any solver returns them as rounding noise of either sign, and
    the tail rule must not decide on that noise.
    """
    lam = np.linalg.eigvalsh(S)[::-1].copy()
    top = lam[0] if lam.size else 0.0
    lam[np.abs(lam) < ZERO_EIG_REL * max(top, 1.0)] = 0.0
    return lam


def tail_rule(lam: np.ndarray):
    """Section 2.3: pick the noise subspace S_H = {lambda_{m+1..D}} and sigma_est = sqrt(tau).

    tau(m) is the mean of lambda_{m+1}..lambda_D.  The paper states the test
    against the median of the same values following Chen et al. (ICCV 2015):
    eigenvalues that carry signal lift the mean of the tail above its median,
    so leading eigenvalues are dropped until that stops.  Reading: m* is the
    smallest m in [0, D-1] with tau(m) <= median(lambda_{m+1..D}); the mean
    divides by the D - m values it averages; the median of an even count is the
    mean of its two middle values.  m = D - 1 always passes.
    Returns (m*, tau, sigma_est).
    """
    lam = np.asarray(lam, dtype=np.float64)
    D = lam.size
    for m in range(D):
        tail = lam[m:]
        tau = tail.mean()
        if tau <= np.median(tail):
            return m, float(tau), float(np.sqrt(max(tau, 0.0)))
    raise AssertionError("unreachable: a single value is its own median")


def estimate_noise(g, f, row_ptr, col, k: int = 6, orders: np.ndarray | None = None, pooled: bool = False):
    """NE-GBP (Section 2.3): patches -> covariance -> eigenvalues -> sigma_est.

    With no complete patch the estimate is 0 (reading: nothing to estimate from).
    ``orders`` selects the unsorted (link-order) patches of the ablation;
    ``pooled`` the per-channel patches of D = k + 1 pooled over the channels.
    Returns a dict with sigma_est, tau, m, eigenvalues, n_patches, covariance.
    """
    A, idx = patch_vectors(g, f, row_ptr, col, k, orders)
    D = 3 * (k + 1)
    if pooled:
        D = k + 1
        n_points = A.shape[0]
        A = pooled_patches(A) if n_points else np.zeros((0, D))
        if n_points == 0:
            return dict(sigma_est=0.0, tau=0.0, m=0, eigenvalues=np.zeros(D), n_patches=0,
                        covariance=np.zeros((D, D)), mean=np.zeros(D))
        S, mu = patch_covariance(A)
        lam = eigenvalues_desc(S)
        m, tau, s = tail_rule(lam)
        return dict(sigma_est=s, tau=tau, m=m, eigenvalues=lam, n_patches=int(n_points),
                    covariance=S, mean=mu)
    if A.shape[0] == 0:
        return dict(sigma_est=0.0, tau=0.0, m=0, eigenvalues=np.zeros(D), n_patches=0,
                    covariance=np.zeros((D, D)), mean=np.zeros(D))
    S, mu = patch_covariance(A)
    lam = eigenvalues_desc(S)
    m, tau, s = tail_rule(lam)
    return dict(sigma_est=s, tau=tau, m=m, eigenvalues=lam, n_patches=int(A.shape[0]),
                covariance=S, mean=mu)


# --------------------------------------------------------------------------
# Step 3/4: filter and FSLR selection (Section 2.4)
# --------------------------------------------------------------------------

def fslr_spread(f: np.ndarray, row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Section 2.4: (sigma_R(i) + sigma_G(i) + sigma_B(i)) / 3 over the patch of point i.

    Reading: the patch of i is i and all its graph neighbours (whatever the
    degree); each sigma is the population standard deviation (divisor n, as
    in the covariance of Section 2.3) of that channel over the patch.
    """
    f = np.asarray(f, dtype=np.float64)
    n = f.shape[0]
    rows = _row_index(row_ptr)
    cnt = np.diff(row_ptr).astype(np.float64) + 1.0
    mean = (f + np.stack([np.bincount(rows, weights=f[col, c], minlength=n) for c in range(3)], 1)) / cnt[:, None]
    dev_self = (f - mean) ** 2
    dev_nb = (f[col] - mean[rows]) ** 2
    var = (dev_self + np.stack([np.bincount(rows, weights=dev_nb[:, c], minlength=n) for c in range(3)], 1)) / cnt[:, None]
    return np.sqrt(var).mean(axis=1)


def fslr_keep(spread: np.ndarray, sigma_est: float, factor: float = 2.0) -> np.ndarray:
    """Section 2.4: points whose spread exceeds factor * sigma_est (factor 2) are not used.

    Reading: if this would leave no point, every point is used.
    """
    keep = ~(spread > factor * sigma_est)
    if not keep.any():
        keep[:] = True
    return keep


def _rw_matrix(row_ptr, col, rw):
    n = row_ptr.size - 1
    return sp.csr_matrix((rw, col, row_ptr), shape=(n, n))


def lowpass_step(x: np.ndarray, rwm) -> np.ndarray:
    """One application of D_g^{-1} W_g with W_g = D + W and D_g = 2 D (Eq. 5).

    D_g^{-1} W_g = (2D)^{-1}(D + W) = I/2 + D^{-1} W / 2.  A point without
    neighbours (only possible when N = 1) keeps its value.
    """
    y = rwm @ x
    isolated = np.diff(rwm.indptr) == 0
    y[isolated] = x[isolated]
    return 0.5 * x + 0.5 * y


def lowpass(f_in: np.ndarray, row_ptr, col, rw, q: int) -> np.ndarray:
    """Eq. 5: f_out = (D_g^{-1} W_g)^q f_in, computed on the vertex domain."""
    x = np.asarray(f_in, dtype=np.float64).copy()
    M = _rw_matrix(row_ptr, col, rw)
    for _ in range(q):
        x = lowpass_step(x, M)
    return x


# --------------------------------------------------------------------------
# Differentiable filter (an extension for parameter tuning; Eq. 4-5 generalised)
# --------------------------------------------------------------------------

def param_filter(g, row_ptr, col, y, q: int, alpha: float, sigma: float):
    """x_0 = y, x_{t+1} = (1 - alpha) x_t + alpha R x_t with R = D^{-1} W(sigma) of Eq. 4.

    alpha = 1/2 and sigma = sigma_g give Eq. 5 (``lowpass``).  A point without
    neighbours has R x = x, as in Eq. 5.  Returns the iterates [x_0 .. x_q].
    """
    rw = random_walk_weights(g, row_ptr, col, sigma)
    R = _rw_matrix(row_ptr, col, rw)
    isolated = np.diff(row_ptr) == 0
    xs = [np.asarray(y, dtype=np.float64).copy()]
    for _ in range(q):
        x = xs[-1]
        rx = R @ x
        rx[isolated] = x[isolated]
        xs.append((1.0 - alpha) * x + alpha * rx)
    return xs


def param_filter_vjp(g, row_ptr, col, y, q: int, alpha: float, sigma: float, grad_out):
    """Gradient of L(x_q) for ``param_filter``, given grad_out = dL/dx_q.

    With P = (1 - alpha) I + alpha R and u_t = dL/dx_t:
      u_t = P^T u_{t+1};  dL/dy = u_0;
      dL/dalpha = sum_t u_{t+1} . (R x_t - x_t);
      dL/dsigma = sum_t alpha u_{t+1} . (dR/dsigma) x_t,
    where R_ij = w_ij / sum_k w_ik and w_ij = exp(-d_ij^2 / sigma^2) give
      dR_ij/dsigma = (2 / sigma^3) R_ij (d_ij^2 - sum_k R_ik d_ik^2).
    Returns (dL/dy [N, 3], dL/dalpha, dL/dsigma).
    """
    xs = param_filter(g, row_ptr, col, y, q, alpha, sigma)
    rw = random_walk_weights(g, row_ptr, col, sigma)
    n = row_ptr.size - 1
    rows = _row_index(row_ptr)
    d2 = _sq_dist(g, row_ptr, col).astype(np.float64)
    isolated = np.diff(row_ptr) == 0
    R = _rw_matrix(row_ptr, col, rw)
    e = np.bincount(rows, weights=rw * d2, minlength=n)
    dR = _rw_matrix(row_ptr, col, (2.0 / sigma ** 3) * rw * (d2 - e[rows]))
    RT = R.T.tocsr()
    u = np.asarray(grad_out, dtype=np.float64).copy()
    da = 0.0
    ds = 0.0
    for t in range(q - 1, -1, -1):
        x = xs[t]
        rx = R @ x
        rx[isolated] = x[isolated]
        da += float(np.sum(u * (rx - x)))
        ds += float(alpha * np.sum(u * (dR @ x)))
        ru = RT @ u
        ru[isolated] = u[isolated]
        u = (1.0 - alpha) * u + alpha * ru
    return u, da, ds


def selection_objective(y: np.ndarray, xq: np.ndarray, keep: np.ndarray, sigma_est: float) -> float:
    """Eq. 6 over the limited region: |sigma_est^2 - (sum y^2 - sum x_q^2) / N|.

    Reading: the signals have three channels and the noise level is per
    scalar, so the sums run over the kept points and their 3 channels and N is
    3 times the number of kept points.
    """
    y = np.asarray(y, dtype=np.float64)[keep]
    xq = np.asarray(xq, dtype=np.float64)[keep]
    lost = ((y - xq) * (y + xq)).sum()
    return abs(sigma_est * sigma_est - lost / (3.0 * keep.sum()))


def select_q(y, row_ptr, col, rw, keep, sigma_est: float, q_max: int = 64, rule: str = "first"):
    """Section 2.4: the integer q minimising Eq. 6, and x_q.

    Reading ("first"): q is searched upward from 0 and the search stops at the
    first q whose objective is not below the previous one (J(q) >= J(q-1));
    q* = q - 1.  Equal objectives go to the smaller q.  The search ends at q_max.
    Alternative reading ("global"): J is evaluated for every q = 0..q_max and
    q* is its argmin (the smallest q among equal minima).
    Returns (q*, x_{q*} float64 [N, 3], J list for q = 0..last evaluated).
    """
    if rule not in ("first", "global"):
        raise ValueError(rule)
    y = np.asarray(y, dtype=np.float64)
    M = _rw_matrix(row_ptr, col, rw)
    x_prev = y.copy()
    J = [selection_objective(y, x_prev, keep, sigma_est)]
    best_q, best_x = 0, x_prev
    for q in range(1, q_max + 1):
        x = lowpass_step(x_prev, M)
        J.append(selection_objective(y, x, keep, sigma_est))
        if rule == "first":
            if J[q] >= J[q - 1]:
                return q - 1, x_prev, J
        elif J[q] < J[best_q]:
            best_q, best_x = q, x
        x_prev = x
    if rule == "global":
        return best_q, best_x, J
    return q_max, x_prev, J


# --------------------------------------------------------------------------
# whole path
# --------------------------------------------------------------------------

@dataclass
class OracleResult:
    orders: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    sigma_g: float
    w: np.ndarray
    rw: np.ndarray
    noise: dict
    spread: np.ndarray
    keep: np.ndarray
    q: int
    J: list
    out: np.ndarray
    extra: dict = field(default_factory=dict)


def fgbd(g: np.ndarray, f: np.ndarray, params: Params = Params(), q: int | None = None) -> OracleResult:
    """The four steps of Section 2.1 in order: SLG, NE-GBP, FSLR, low-pass filter.

    With ``q`` given, the filter power is fixed and the selection is skipped.
    """
    g = np.asarray(g)
    n = g.shape[0]
    codes = scan_line_codes(g, params.bits)
    orders = scan_orders(codes)
    edges = slg_edges(orders, params.window, codes if params.same_line else None, params.bits)
    row_ptr, col = adjacency_csr(edges, n)
    if params.sigma_g_mode not in ("edge", "node", "pair"):
        raise ValueError(params.sigma_g_mode)
    sg = sigma_g_node(g, row_ptr, col) if params.sigma_g_mode == "node" else sigma_g(g, row_ptr, col)
    if params.sigma_g_mode == "pair":
        scale = pair_scale(g, row_ptr, col)
        d2 = _sq_dist(g, row_ptr, col).astype(np.float64)
        w = np.ones_like(d2)
        w[scale > 0] = np.exp(-d2[scale > 0] / scale[scale > 0])
        rw = random_walk_weights(g, row_ptr, col, sg, scale)
    else:
        w = edge_weights(g, row_ptr, col, sg)
        rw = random_walk_weights(g, row_ptr, col, sg)
    noise = estimate_noise(g, f, row_ptr, col, k=6 * params.window,
                           orders=None if params.sorted_patches else orders, pooled=params.pooled_patch)
    spread = fslr_spread(f, row_ptr, col)
    if params.fslr:
        keep = fslr_keep(spread, noise["sigma_est"], params.fslr_factor)
    else:
        keep = np.ones(n, dtype=bool)   # "FGBD w/o FSLR": Eq. 6 over every point
    if q is None:
        qs, out, J = select_q(f, row_ptr, col, rw, keep, noise["sigma_est"], params.q_max, params.q_rule)
    else:
        qs, out, J = q, lowpass(f, row_ptr, col, rw, q), []
    return OracleResult(orders, row_ptr, col, sg, w, rw, noise, spread, keep, qs, J, out)
