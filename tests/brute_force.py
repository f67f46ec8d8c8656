"""Pure-Python brute force for tiny clouds, used to pin the oracle.

Written with plain loops and tuples, independently of ``oracle/fgbd_oracle.py``
(no NumPy in the arithmetic), so that a vectorisation mistake in the oracle
(a transposed operand, a wrong axis, a dropped term) shows up as a mismatch.
Each function restates one definition of the paper:

* ``orders``            Section 2.2, Eq. 1-3: sorting by C1/C2/C3 is sorting by the
                        coordinate tuples (z,y,x), (x,z,y), (y,x,z); ties by index.
* ``neighbour_sets``    Section 2.2: consecutive points along each order are linked
                        (optionally only within one scan line: the same-line ablation).
* ``patch_covariance``  Section 2.3: Sigma = 1/N sum (a - mu)(a - mu)^T, element by element.
* ``link_order_patches`` the "NE-GBP w/o sort" ablation (Table 4): patch entries
                        in the order the scan lines link them.
* ``spread``            Section 2.4: mean over channels of the population std in a patch.
* ``filter_power``      Eq. 5: x <- x/2 + (sum_j w_ij x_j)/(2 sum_j w_ij), q times
                        (``pair`` bandwidths: w_ij = exp(-d^2 / (s_i s_j))).
* ``node_sigma``        the alternative readings of sigma_g: each point's mean edge
                        length, and their mean over the points with edges.
* ``pooled_covariance`` the pooled reading of the patch dimension: every channel of
                        every patch one sample of K + 1 entries.
"""
from __future__ import annotations

import math


def orders(points, window=1):
    """Index orders along the three scan directions, ties broken by index."""
    n = len(points)
    keys = [
        lambda i: (points[i][2], points[i][1], points[i][0], i),  # C1: z, y, x
        lambda i: (points[i][0], points[i][2], points[i][1], i),  # C2: x, z, y
        lambda i: (points[i][1], points[i][0], points[i][2], i),  # C3: y, x, z
    ]
    return [sorted(range(n), key=k) for k in keys]


# the two coordinates a scan line of each code holds fixed: C1 (z, y), C2 (x, z), C3 (y, x)
LINE_AXES = [(2, 1), (0, 2), (1, 0)]


def neighbour_sets(points, window=1, same_line=False):
    """With same_line, two points are linked along a code only if they lie on
    one scan line of it (equal in that code's two major coordinates)."""
    n = len(points)
    nb = [set() for _ in range(n)]
    for l, order in enumerate(orders(points)):
        for k in range(n):
            for d in range(1, window + 1):
                if k + d < n:
                    a, b = order[k], order[k + d]
                    if same_line and any(points[a][ax] != points[b][ax] for ax in LINE_AXES[l]):
                        continue
                    if a != b:
                        nb[a].add(b)
                        nb[b].add(a)
    return nb


def sq_dist(p, q):
    return sum((p[c] - q[c]) ** 2 for c in range(3))


def sigma_g(points, nb):
    total = 0.0
    count = 0
    for i in range(len(points)):
        for j in nb[i]:
            total += math.sqrt(sq_dist(points[i], points[j]))
            count += 1
    return total / count if count else 0.0


def patches(points, colors, nb, k=6):
    """Patch vectors of the points with exactly k neighbours, neighbours by distance."""
    out = []
    for i in range(len(points)):
        if len(nb[i]) != k:
            continue

        def key(j):
            off = [points[j][c] - points[i][c] for c in range(3)]
            return (sq_dist(points[i], points[j]), off[2], off[1], off[0], j)

        members = [i] + sorted(nb[i], key=key)
        vec = []
        for m in members:
            vec.extend(float(colors[m][c]) for c in range(3))
        out.append(vec)
    return out


def link_order_patches(points, colors, nb, k=6):
    """Patch vectors in link order (the "w/o sort" ablation, window 1).

    Members: the point, then its predecessor and successor along C1, along C2
    and along C3, for the points with exactly k = 6 neighbours.
    """
    ords = orders(points)
    pos = []
    for order in ords:
        p = [0] * len(points)
        for r, i in enumerate(order):
            p[i] = r
        pos.append(p)
    out = []
    for i in range(len(points)):
        if len(nb[i]) != k:
            continue
        members = [i]
        for l in range(3):
            r = pos[l][i]
            members.append(ords[l][r - 1])
            members.append(ords[l][r + 1])
        vec = []
        for m in members:
            vec.extend(float(colors[m][c]) for c in range(3))
        out.append(vec)
    return out


def patch_covariance(vectors):
    n = len(vectors)
    d = len(vectors[0])
    mu = [sum(v[r] for v in vectors) / n for r in range(d)]
    cov = [[0.0] * d for _ in range(d)]
    for r in range(d):
        for c in range(d):
            s = 0.0
            for v in vectors:
                s += (v[r] - mu[r]) * (v[c] - mu[c])
            cov[r][c] = s / n
    return cov, mu


def spread(colors, nb, i):
    members = [i] + sorted(nb[i])
    n = len(members)
    total = 0.0
    for c in range(3):
        vals = [float(colors[m][c]) for m in members]
        mean = sum(vals) / n
        total += math.sqrt(sum((v - mean) ** 2 for v in vals) / n)
    return total / 3.0


def node_sigma(points, nb):
    """(per-point mean edge length list, mean of it over the points with edges)."""
    per = []
    for i in range(len(points)):
        if nb[i]:
            per.append(sum(math.sqrt(sq_dist(points[i], points[j])) for j in nb[i]) / len(nb[i]))
        else:
            per.append(0.0)
    with_edges = [per[i] for i in range(len(points)) if nb[i]]
    return per, (sum(with_edges) / len(with_edges) if with_edges else 0.0)


def pooled_covariance(vectors):
    """Each RGB patch (point-major, channel-minor) as three single-channel samples."""
    samples = []
    for v in vectors:
        k1 = len(v) // 3
        for c in range(3):
            samples.append([v[3 * m + c] for m in range(k1)])
    return patch_covariance(samples)


def filter_power(points, colors, nb, sg, q, pair=None):
    n = len(points)
    x = [[float(colors[i][c]) for c in range(3)] for i in range(n)]
    for _ in range(q):
        new = []
        for i in range(n):
            if not nb[i]:
                new.append(list(x[i]))
                continue
            if pair is not None:
                # the common factor exp(-min_j a_ij) cancels in the row; taken out so nothing underflows
                a = {j: (sq_dist(points[i], points[j]) / (pair[i] * pair[j]) if pair[i] * pair[j] > 0 else 0.0)
                     for j in nb[i]}
                amin = min(a.values())
                ws = {j: math.exp(-(a[j] - amin)) for j in nb[i]}
            else:
                ws = {j: math.exp(-sq_dist(points[i], points[j]) / (sg * sg)) for j in nb[i]}
            dsum = sum(ws.values())
            row = []
            for c in range(3):
                avg = sum(ws[j] * x[j][c] for j in nb[i]) / dsum
                row.append(0.5 * x[i][c] + 0.5 * avg)
            new.append(row)
        x = new
    return x
