"""Seeded synthetic point-cloud frames shaped like the ones FGBD is evaluated on.

The paper evaluates on voxelized human-body sequences (8iVFBv2 at 10 bits and
MVUB at 9 bits, "around 1 million points" per frame; Section 4.1 and the
introduction) perturbed by additive Gaussian colour noise with standard
deviation 10, 20 or 30 on the 0-255 scale.  Those datasets are not available
here, so these generators stand in for them.

This module draws geometry, colour fields and noise only.  It contains no step
of the denoising method (no scan-line codes, graphs, estimates or filters), so
both the CUDA library's tests and the CPU oracle's tests can take their inputs
from it without sharing any of the method's arithmetic.

Every function is deterministic for a given seed (``numpy.random.default_rng``).
Point order is shuffled after voxelization so that no input arrives already
sorted along a scan direction.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Frame",
    "sphere_points",
    "torso_points",
    "smooth_colors",
    "piecewise_colors",
    "add_noise_u8",
    "add_noise_f32",
    "sphere_frame",
    "torso_frame",
]


class Frame:
    """One synthetic frame: int32 voxel coordinates and colour arrays."""

    def __init__(self, xyz, clean, noisy, sigma, bits, name):
        self.xyz = xyz          # int32 [N, 3], each coordinate in [0, 2**bits)
        self.clean = clean      # uint8 [N, 3] (or float32) noise-free colours
        self.noisy = noisy      # same dtype as clean, noisy colours
        self.sigma = sigma      # noise standard deviation on the 0-255 scale
        self.bits = bits
        self.name = name

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    def __repr__(self) -> str:
        return f"Frame({self.name}, n={self.n}, bits={self.bits}, sigma={self.sigma})"


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def _voxelize(p01: np.ndarray, bits: int, rng: np.random.Generator) -> np.ndarray:
    """Quantize points of [0,1]^3 to a 2**bits grid, drop repeated voxels, shuffle."""
    side = 1 << bits
    g = np.floor(p01 * side).astype(np.int64)
    np.clip(g, 0, side - 1, out=g)
    lin = np.ravel_multi_index((g[:, 0], g[:, 1], g[:, 2]), (side, side, side))
    lin = np.unique(lin)
    gx, gy, gz = np.unravel_index(lin, (side, side, side))
    g = np.stack([gx, gy, gz], axis=1).astype(np.int32)
    return g[rng.permutation(g.shape[0])]


def sphere_points(n_samples: int = 20500, bits: int = 9, seed: int = 0) -> np.ndarray:
    """Points drawn uniformly on the unit sphere, voxelized to a 2**bits grid.

    With 20,500 samples on a 2**9 grid about 20k distinct voxels remain.
    """
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n_samples, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return _voxelize(v * 0.5 + 0.5, bits, rng)


def _sample_ellipsoid(center, radii, m, rng):
    """Area-uniform samples on an ellipsoid surface (rejection on the area element)."""
    out = []
    a, b, c = radii
    inv2 = np.array([1.0 / a**2, 1.0 / b**2, 1.0 / c**2])
    gmax = a * b * c * np.sqrt(inv2.max())
    need = m
    while need > 0:
        u = rng.standard_normal((2 * need + 64, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        gscale = a * b * c * np.sqrt((u * u) @ inv2)
        keep = rng.random(u.shape[0]) * gmax < gscale
        u = u[keep][:need]
        out.append(center + u * np.array(radii))
        need -= u.shape[0]
    return np.concatenate(out)


def _ellipsoid_area(radii):
    # Knud Thomsen's approximation; only used to split the sample budget.
    a, b, c = radii
    p = 1.6075
    return 4 * np.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p)


def _orthonormal_frame(axis):
    axis = axis / np.linalg.norm(axis)
    helper = np.array([1.0, 0.0, 0.0]) if abs(axis[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(axis, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(axis, e1)
    return axis, e1, e2


def _sample_capsule(p0, p1, r, m, rng):
    """Area-uniform samples on a capped cylinder (cylinder side + two hemispheres)."""
    p0 = np.asarray(p0, float)
    p1 = np.asarray(p1, float)
    axis = p1 - p0
    length = np.linalg.norm(axis)
    ax, e1, e2 = _orthonormal_frame(axis)
    side_area = 2 * np.pi * r * length
    cap_area = 4 * np.pi * r * r
    m_side = int(round(m * side_area / (side_area + cap_area)))
    m_cap = m - m_side
    t = rng.random(m_side) * length
    phi = rng.random(m_side) * 2 * np.pi
    side = p0 + np.outer(t, ax) + r * (np.outer(np.cos(phi), e1) + np.outer(np.sin(phi), e2))
    u = rng.standard_normal((m_cap, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    along = u @ ax
    cap = np.where((along < 0)[:, None], p0 + r * u, p1 + r * u)
    return np.concatenate([side, cap])


def _capsule_area(p0, p1, r):
    return 2 * np.pi * r * np.linalg.norm(np.asarray(p1) - np.asarray(p0)) + 4 * np.pi * r * r


def _inside_ellipsoid(p, center, radii, eps):
    q = (p - center) / np.asarray(radii)
    return (q * q).sum(axis=1) < 1.0 - eps


def _inside_capsule(p, p0, p1, r, eps):
    p0 = np.asarray(p0, float)
    p1 = np.asarray(p1, float)
    d = p1 - p0
    t = np.clip(((p - p0) @ d) / (d @ d), 0.0, 1.0)
    closest = p0 + t[:, None] * d
    return np.linalg.norm(p - closest, axis=1) < r * (1.0 - eps)


def _torso_layout(rng):
    """Six ellipsoids and four capped cylinders with standing-body extents.

    The body stands along +y inside the unit cube.  Centres and radii are
    jittered by the seed so different seeds give different shapes.
    """
    def jit(v, s):
        return np.asarray(v, float) * (1.0 + s * (rng.random(len(v)) * 2 - 1))

    ell = [
        ((0.50, 0.885, 0.50), (0.065, 0.085, 0.075)),   # head
        ((0.50, 0.640, 0.50), (0.165, 0.150, 0.095)),   # chest
        ((0.50, 0.480, 0.50), (0.145, 0.110, 0.088)),   # abdomen
        ((0.50, 0.360, 0.50), (0.155, 0.075, 0.095)),   # pelvis
        ((0.335, 0.730, 0.50), (0.060, 0.048, 0.058)),  # left shoulder
        ((0.665, 0.730, 0.50), (0.060, 0.048, 0.058)),  # right shoulder
    ]
    ell = [(jit(c, 0.02), jit(r, 0.10)) for c, r in ell]
    caps = [
        ((0.300, 0.715, 0.50), (0.230, 0.400, 0.53), 0.036),  # left arm
        ((0.700, 0.715, 0.50), (0.770, 0.400, 0.53), 0.036),  # right arm
        ((0.440, 0.320, 0.50), (0.420, 0.035, 0.51), 0.056),  # left leg
        ((0.560, 0.320, 0.50), (0.580, 0.035, 0.51), 0.056),  # right leg
    ]
    caps = [(jit(a, 0.02), jit(b, 0.02), float(jit([r], 0.10)[0])) for a, b, r in caps]
    return ell, caps


def torso_points(target: int = 1_000_000, bits: int = 10, seed: int = 0,
                 oversample: float = 3.0) -> np.ndarray:
    """A densely voxelized union of 6 ellipsoids and 4 capped cylinders.

    Surface samples lying strictly inside another primitive are dropped, so
    only the outer shell of the union remains.  The layout is scaled about the
    cube centre so the shell holds at least ``target`` voxels, and then a
    seeded random subset of exactly ``target`` voxels is kept.
    """
    rng = np.random.default_rng(seed)
    ell, caps = _torso_layout(rng)
    side = float(1 << bits)
    area01 = sum(_ellipsoid_area(r) for _, r in ell) + sum(_capsule_area(a, b, r) for a, b, r in caps)
    # a dense one-voxel shell holds roughly 1.15 voxels per unit of surface area
    scale = min(1.0, np.sqrt(target * 1.08 / (1.15 * area01 * side * side)))
    for _attempt in range(6):
        prims_e = [((np.asarray(c) - 0.5) * scale + 0.5, np.asarray(r) * scale) for c, r in ell]
        prims_c = [((np.asarray(a) - 0.5) * scale + 0.5, (np.asarray(b) - 0.5) * scale + 0.5, r * scale)
                   for a, b, r in caps]
        total_area = (sum(_ellipsoid_area(r) for _, r in prims_e)
                      + sum(_capsule_area(a, b, r) for a, b, r in prims_c))
        budget = oversample * total_area * side * side
        pts = []
        owners = []
        for idx, (c, r) in enumerate(prims_e):
            m = int(budget * _ellipsoid_area(r) / total_area) + 1
            pts.append(_sample_ellipsoid(c, r, m, rng))
            owners.append(np.full(m, idx))
        for idx, (a, b, r) in enumerate(prims_c):
            m = int(budget * _capsule_area(a, b, r) / total_area) + 1
            pts.append(_sample_capsule(a, b, r, m, rng))
            owners.append(np.full(m, len(prims_e) + idx))
        p = np.concatenate(pts)
        owner = np.concatenate(owners)
        inside = np.zeros(p.shape[0], bool)
        for idx, (c, r) in enumerate(prims_e):
            inside |= (owner != idx) & _inside_ellipsoid(p, c, r, 1e-3)
        for idx, (a, b, r) in enumerate(prims_c):
            inside |= (owner != len(prims_e) + idx) & _inside_capsule(p, a, b, r, 1e-3)
        p = p[~inside]
        p = p[np.all((p >= 0.0) & (p < 1.0), axis=1)]
        g = _voxelize(p, bits, rng)
        if g.shape[0] >= target:
            return g[:target]  # already shuffled: a seeded random subset
        scale *= np.sqrt(target * 1.03 / g.shape[0])
    raise RuntimeError("torso_points: could not reach the requested point count")


# --------------------------------------------------------------------------
# colours and noise
# --------------------------------------------------------------------------

def smooth_colors(xyz: np.ndarray, bits: int, seed: int = 0, as_float: bool = False) -> np.ndarray:
    """Smooth procedural RGB: per channel 127.5 + sum of 3 random-phase sinusoids.

    Channel c at voxel g is 127.5 + sum_k 40 sin(2 pi w_ck . g / 2**bits + phi_ck)
    with w_ck ~ U[-3, 3]^3 and phi_ck ~ U[0, 2 pi).
    """
    rng = np.random.default_rng(seed + 7919)
    w = rng.uniform(-3.0, 3.0, size=(3, 3, 3))      # [channel, term, axis]
    phi = rng.uniform(0.0, 2 * np.pi, size=(3, 3))  # [channel, term]
    u = xyz.astype(np.float64) / float(1 << bits)
    col = np.empty((xyz.shape[0], 3))
    for c in range(3):
        arg = 2 * np.pi * (u @ w[c].T) + phi[c]
        col[:, c] = 127.5 + 40.0 * np.sin(arg).sum(axis=1)
    col = np.clip(col, 0.0, 255.0)
    return col.astype(np.float32) if as_float else np.rint(col).astype(np.uint8)


def piecewise_colors(xyz: np.ndarray, bits: int, seed: int = 0, n_planes: int = 8,
                     as_float: bool = False) -> np.ndarray:
    """Smooth field plus ``n_planes`` sharp colour boundaries.

    Each boundary is a random plane n.g > t; every voxel on its positive side
    gets an offset drawn from U[-60, 60]^3.  The result is clipped to [0, 255].
    """
    base = smooth_colors(xyz, bits, seed, as_float=True).astype(np.float64)
    rng = np.random.default_rng(seed + 104729)
    u = xyz.astype(np.float64) / float(1 << bits)
    for _ in range(n_planes):
        nrm = rng.standard_normal(3)
        nrm /= np.linalg.norm(nrm)
        t = nrm @ rng.uniform(0.3, 0.7, size=3)
        off = rng.uniform(-60.0, 60.0, size=3)
        base[(u @ nrm) > t] += off
    base = np.clip(base, 0.0, 255.0)
    return base.astype(np.float32) if as_float else np.rint(base).astype(np.uint8)


def add_noise_u8(clean: np.ndarray, sigma: float, seed: int = 0) -> np.ndarray:
    """y = clip(rint(c + N(0, sigma^2)), 0, 255) as uint8 (the paper's noisy frames)."""
    rng = np.random.default_rng(seed + 15485863)
    y = clean.astype(np.float64) + rng.standard_normal(clean.shape) * sigma
    return np.clip(np.rint(y), 0, 255).astype(np.uint8)


def add_noise_f32(clean: np.ndarray, sigma: float, seed: int = 0) -> np.ndarray:
    """y = c + N(0, sigma^2) as float32, neither rounded nor clipped."""
    rng = np.random.default_rng(seed + 15485863)
    return (clean.astype(np.float64) + rng.standard_normal(clean.shape) * sigma).astype(np.float32)


# --------------------------------------------------------------------------
# whole frames
# --------------------------------------------------------------------------

def sphere_frame(n_samples: int = 20500, bits: int = 9, sigma: float = 20.0, seed: int = 0) -> Frame:
    """The small plain-method frame: ~20k sphere voxels at 9 bits, smooth colour, uint8."""
    xyz = sphere_points(n_samples, bits, seed)
    clean = smooth_colors(xyz, bits, seed)
    noisy = add_noise_u8(clean, sigma, seed)
    return Frame(xyz, clean, noisy, sigma, bits, f"sphere{xyz.shape[0]}_b{bits}_s{sigma:g}")


def torso_frame(target: int = 1_000_000, bits: int = 10, sigma: float = 20.0, seed: int = 0,
                noise_seed: int | None = None) -> Frame:
    """The large plain-method frame: ~1M torso-shell voxels at 10 bits, piecewise colour."""
    xyz = torso_points(target, bits, seed)
    clean = piecewise_colors(xyz, bits, seed)
    noisy = add_noise_u8(clean, sigma, seed if noise_seed is None else noise_seed)
    return Frame(xyz, clean, noisy, sigma, bits, f"torso{xyz.shape[0]}_b{bits}_s{sigma:g}")


def batch_frame(f: int, lo: int = 200_000, hi: int = 1_200_000, seed: int = 1, bits: int = 10) -> Frame:
    """Frame f of ``batch_frames``: seed seed + f, N_f ~ U[lo, hi] sphere voxels
    at `bits` bits (sampled 1.5x, voxelized and trimmed to N_f), smooth colour,
    and uint8 noise with sigma_f ~ U[10, 50]."""
    s = seed + f
    rng = np.random.default_rng(s)
    target = int(rng.integers(lo, hi + 1))
    sigma = float(rng.uniform(10.0, 50.0))
    samples = int(target * 1.5) + 1024
    xyz = sphere_points(samples, bits, s)
    while xyz.shape[0] < target:
        samples *= 2
        xyz = sphere_points(samples, bits, s)
    xyz = np.ascontiguousarray(xyz[:target])
    clean = smooth_colors(xyz, bits, s)
    noisy = add_noise_u8(clean, sigma, s)
    return Frame(xyz, clean, noisy, sigma, bits, f"sphere{target}_b{bits}_s{sigma:.1f}")


def batch_frames(count: int = 16, lo: int = 200_000, hi: int = 1_200_000, seed: int = 1,
                 bits: int = 10) -> list:
    """Frames of uneven sizes for the batched path: ``batch_frame`` f for f = 0..count-1."""
    return [batch_frame(f, lo, hi, seed, bits) for f in range(count)]


def tuning_pairs(count: int = 8, n: int = 300_000, sigma: float = 30.0, seed: int = 101, bits: int = 9) -> list:
    """Clean/noisy pairs for filter-parameter tuning: pair k (seed seed + k) is an
    n-point sphere frame at `bits` bits with smooth colour and float32 noise of
    the given sigma (unrounded, unclipped)."""
    frames = []
    for k in range(count):
        s = seed + k
        samples = int(n * 1.6) + 1024
        xyz = sphere_points(samples, bits, s)
        while xyz.shape[0] < n:
            samples *= 2
            xyz = sphere_points(samples, bits, s)
        xyz = np.ascontiguousarray(xyz[:n])
        clean = smooth_colors(xyz, bits, s, as_float=True)
        noisy = add_noise_f32(clean, sigma, s)
        frames.append(Frame(xyz, clean, noisy, sigma, bits, f"sphere{n}_b{bits}_s{sigma:g}_pair{k}"))
    return frames


class StreamSequence:
    """A moving, jittered sphere for the streaming mode: frame t of `frames`.

    The base is `samples` points on a sphere of radius 0.35 (in units of the
    grid side) around the grid centre.  Frame t rotates it by t * omega about
    a random axis (omega ~ U[0.2, 0.5] degrees per frame), translates it by
    40 sin(2 pi t / frames) * d voxels of a 2^10 grid (d a random unit vector;
    at most about 0.84 voxel per frame), voxelizes at `bits` bits, adds an integer jitter in
    {-1, 0, 1} to each coordinate and drops repeated voxels.  Colour: the smooth
    field of ``smooth_colors`` with every phase advanced by 2 pi t / frames;
    uint8 noise of the given sigma.  Everything is seeded by (seed, t).
    """

    def __init__(self, frames: int = 300, samples: int = 1_150_000, bits: int = 10, sigma: float = 25.0,
                 seed: int = 0):
        self.frames, self.bits, self.sigma, self.seed = frames, bits, sigma, seed
        rng = np.random.default_rng(seed)
        v = rng.standard_normal((samples, 3))
        self.base = v / np.linalg.norm(v, axis=1, keepdims=True) * 0.35
        axis = rng.standard_normal(3)
        self.axis = axis / np.linalg.norm(axis)
        self.omega = np.deg2rad(rng.uniform(0.2, 0.5))
        d = rng.standard_normal(3)
        self.dir = d / np.linalg.norm(d)
        crng = np.random.default_rng(seed + 7919)
        self.w = crng.uniform(-3.0, 3.0, size=(3, 3, 3))      # [channel, k, xyz]
        self.phi = crng.uniform(0.0, 2.0 * np.pi, size=(3, 3))

    def _rotation(self, angle):
        k = self.axis
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)

    def frame(self, t: int) -> Frame:
        side = 1 << self.bits
        rng = np.random.default_rng([self.seed, t])
        p = self.base @ self._rotation(t * self.omega).T
        shift = 40.0 * (side / 1024.0) * np.sin(2 * np.pi * t / self.frames) * self.dir
        g = np.floor((p + 0.5) * side + shift).astype(np.int64)
        g += rng.integers(-1, 2, size=g.shape)
        np.clip(g, 0, side - 1, out=g)
        lin = np.sort(np.ravel_multi_index((g[:, 0], g[:, 1], g[:, 2]), (side, side, side)))
        lin = lin[np.concatenate(([True], lin[1:] != lin[:-1]))]   # drop repeated voxels
        gx, gy, gz = np.unravel_index(lin, (side, side, side))
        xyz = np.stack([gx, gy, gz], axis=1).astype(np.int32)
        xyz = np.ascontiguousarray(xyz[rng.permutation(xyz.shape[0])])
        gf = xyz.astype(np.float64) / side
        phase = 2 * np.pi * t / self.frames
        clean = np.empty(xyz.shape, dtype=np.float64)
        for c in range(3):
            acc = np.full(xyz.shape[0], 127.5)
            for k in range(3):
                acc += 40.0 * np.sin(2 * np.pi * (gf @ self.w[c, k]) + self.phi[c, k] + phase)
            clean[:, c] = acc
        clean = np.clip(np.rint(clean), 0, 255).astype(np.uint8)
        noisy = add_noise_u8(clean, self.sigma, self.seed * 100003 + t)
        return Frame(xyz, clean, noisy, self.sigma, self.bits, f"stream{t}_n{xyz.shape[0]}")
