"""Seeded synthetic templates, rotation sets and tomograms.

Conventions shared by every consumer (they are data conventions, not method
arithmetic):

* Volumes are float32 arrays indexed ``[z, y, x]`` (x fastest in memory).
  Spatial vectors are written ``(x, y, z)``.
* A template box has edge ``s``; its centre is voxel ``floor(s/2)`` on every
  axis; the binary mask is the ball of radius ``r`` about that centre.
* Quaternions are ``(a, b, c, d)`` with the real part first; the rotation of a
  unit quaternion q acts on column vectors ``(x, y, z)`` as ``v -> q v q*``.
* A copy of template ``t`` planted at voxel ``p`` with rotation ``R`` adds
  ``t(c + R^-1 (u - c))`` to voxel ``p + (u - c)`` for every box voxel ``u``
  (trilinear interpolation, zero outside the box) -- the rotated-template
  convention ``t_R = O_{R^-1} t`` of Sec. 2 of the paper.
"""

from __future__ import annotations

import concurrent.futures
import dataclasses
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
from scipy import ndimage

# --------------------------------------------------------------------------
# rotation sets
# --------------------------------------------------------------------------

# psi is the real root > 1 of psi**4 = psi + 4 (Alexa, "Super-Fibonacci
# Spirals: Fast, Low-Discrepancy Sampling of SO(3)", CVPR 2022).
_SF_PHI = math.sqrt(2.0)
_SF_PSI = 1.533751168755204288118041


def super_fibonacci_quaternions(n: int) -> np.ndarray:
    """``n`` near-uniform unit quaternions on S^3 (super-Fibonacci spiral).

    Point i uses s = i + 1/2, radii sqrt(s/n) and sqrt(1 - s/n) for the two
    complex planes, and angles 2*pi*s/phi and 2*pi*s/psi.  Returns float64
    ``(n, 4)``.  Because every quantity of the method is even in q (q and -q
    are the same rotation), a set covering all of S^3 with equal weights is a
    quadrature for the normalised Haar measure of SO(3).
    """
    if n <= 0:
        return np.zeros((0, 4))
    s = np.arange(n, dtype=np.float64) + 0.5
    r = np.sqrt(s / n)
    big_r = np.sqrt(1.0 - s / n)
    alpha = 2.0 * np.pi * s / _SF_PHI
    beta = 2.0 * np.pi * s / _SF_PSI
    q = np.stack([r * np.sin(alpha), r * np.cos(alpha),
                  big_r * np.sin(beta), big_r * np.cos(beta)], axis=1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def shoemake_quaternions(n: int, seed: int) -> np.ndarray:
    """``n`` uniformly random unit quaternions (Shoemake 1992), float64."""
    rng = np.random.default_rng(seed)
    u1, u2, u3 = rng.random((3, n))
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=1)
    return q


def _rotation_matrix(q: np.ndarray) -> np.ndarray:
    """3x3 matrix of v -> q v q* for a unit quaternion (a, b, c, d)."""
    a, b, c, d = q / np.linalg.norm(q)
    return np.array([
        [a*a + b*b - c*c - d*d, 2*(b*c - a*d), 2*(b*d + a*c)],
        [2*(b*c + a*d), a*a - b*b + c*c - d*d, 2*(c*d - a*b)],
        [2*(b*d - a*c), 2*(c*d + a*b), a*a - b*b - c*c + d*d],
    ])


# --------------------------------------------------------------------------
# templates and masks
# --------------------------------------------------------------------------

def default_mask_radius(s: int) -> int:
    """Mask radius for a box of edge s: (s-1)/2 if s is odd, s/2-1 if even."""
    return (s - 1) // 2 if s % 2 else s // 2 - 1


def ball_mask(s: int, r: Optional[float] = None) -> np.ndarray:
    """Binary ball of radius r about voxel floor(s/2) in an s^3 box (float32)."""
    if r is None:
        r = default_mask_radius(s)
    c = s // 2
    z, y, x = np.meshgrid(*(np.arange(s) - c,) * 3, indexing="ij")
    return ((x * x + y * y + z * z) <= r * r + 1e-9).astype(np.float32)


def soft_ball_mask(s: int, r: float, edge: float) -> np.ndarray:
    """Raised-cosine ball about the box centre: 1 within r - edge of it,
    falling as cos^2 to 0 at r (a soft mask: weights in [0, 1])."""
    c = s // 2
    zz, yy, xx = np.meshgrid(np.arange(s), np.arange(s), np.arange(s), indexing="ij")
    d = np.sqrt((xx - c) ** 2 + (yy - c) ** 2 + (zz - c) ** 2)
    t = np.clip((d - (r - edge)) / edge, 0.0, 1.0)
    return np.where(t >= 1.0, 0.0, np.cos(0.5 * np.pi * t) ** 2).astype(np.float32)


def blob_template(s: int, n_blobs: int, seed: int,
                  lowpass_sigma: Optional[float] = None) -> np.ndarray:
    """Asymmetric object: a sum of anisotropic Gaussian blobs (float32 s^3).

    Blob centres are uniform in the ball of radius r/2 about the box centre;
    per-axis widths are U[1, 2.5] * s/15 voxels along a random orthonormal
    frame; amplitudes are U[0.5, 1].  Optionally smoothed by a Gaussian of
    ``lowpass_sigma`` voxels (zero outside the box).
    """
    rng = np.random.default_rng(seed)
    r = default_mask_radius(s)
    c = s // 2
    z, y, x = np.meshgrid(*(np.arange(s, dtype=np.float64) - c,) * 3, indexing="ij")
    pts = np.stack([x, y, z], axis=-1)
    t = np.zeros((s, s, s))
    for _ in range(n_blobs):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        centre = d * (r / 2.0) * rng.random() ** (1.0 / 3.0)
        sig = rng.uniform(1.0, 2.5, size=3) * (s / 15.0)
        frame = _rotation_matrix(shoemake_quaternions(1, int(rng.integers(1 << 31)))[0])
        amp = rng.uniform(0.5, 1.0)
        local = (pts - centre) @ frame
        t += amp * np.exp(-0.5 * np.sum((local / sig) ** 2, axis=-1))
    if lowpass_sigma:
        t = ndimage.gaussian_filter(t, lowpass_sigma, mode="constant", cval=0.0)
    return t.astype(np.float32)


def rotated_copy(t: np.ndarray, q: np.ndarray) -> np.ndarray:
    """t_R(u) = t(c + R^-1 (u - c)), trilinear, zero outside the box (float64).

    Implemented with scipy's linear spline resampling so that it shares no
    code with either implementation of the method.
    """
    s = t.shape[0]
    c = s // 2
    rot = _rotation_matrix(np.asarray(q, dtype=np.float64))
    z, y, x = np.meshgrid(*(np.arange(s, dtype=np.float64) - c,) * 3, indexing="ij")
    v = np.stack([x.ravel(), y.ravel(), z.ravel()])       # (3, s^3) as (x, y, z)
    p = rot.T @ v + c                                      # R^-1 = R^T
    coords = np.stack([p[2], p[1], p[0]])                  # array order z, y, x
    out = ndimage.map_coordinates(t.astype(np.float64), coords, order=1,
                                  mode="grid-constant", cval=0.0, prefilter=False)
    return out.reshape(s, s, s)


# --------------------------------------------------------------------------
# tomograms
# --------------------------------------------------------------------------

def plant_copies(shape_zyx: Sequence[int], t: np.ndarray, quats: np.ndarray,
                 positions_xyz: np.ndarray) -> np.ndarray:
    """Noise-free volume (float64) with a rotated copy of t at every position."""
    vol = np.zeros(tuple(shape_zyx))
    s = t.shape[0]
    c = s // 2
    quats = np.asarray(quats).reshape(-1, 4)
    positions_xyz = np.asarray(positions_xyz).reshape(-1, 3)
    # the copies are resampled in worker threads, a bounded window ahead, and
    # added in their own order (the sum is the same as one copy at a time)
    workers = min(8, os.cpu_count() or 1)
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        for i0 in range(0, len(quats), 4 * workers):
            chunk = list(ex.map(lambda q: rotated_copy(t, q), quats[i0:i0 + 4 * workers]))
            for copy, p in zip(chunk, positions_xyz[i0:i0 + 4 * workers]):
                x0, y0, z0 = (int(p[0]) - c, int(p[1]) - c, int(p[2]) - c)
                vol[z0:z0 + s, y0:y0 + s, x0:x0 + s] += copy
    return vol


def _random_positions(shape_zyx: Sequence[int], s: int, count: int,
                      min_dist: float, rng: np.random.Generator) -> np.ndarray:
    """Integer positions whose whole s^3 box is inside the volume, spaced apart."""
    c = s // 2
    lo = np.array([c, c, c])
    hi = np.array([shape_zyx[2] - s + c, shape_zyx[1] - s + c, shape_zyx[0] - s + c])
    if np.any(hi < lo):
        raise ValueError("volume smaller than the template box")
    pts = np.zeros((count, 3), dtype=np.int64)
    n = 0
    tries = 0
    dist = float(min_dist)
    while n < count:
        p = np.array([rng.integers(lo[i], hi[i] + 1) for i in range(3)])
        if n == 0 or np.min(np.sum((pts[:n] - p) ** 2, axis=1)) >= dist * dist:
            pts[n] = p
            n += 1
            tries = 0
        else:
            tries += 1
            if tries > 2000:           # crowded: relax the spacing a little
                dist *= 0.9
                tries = 0
    return pts


@dataclasses.dataclass
class Workload:
    """One synthetic (volume, template) matching problem."""
    name: str
    volume: np.ndarray            # float32 [z, y, x]
    template: np.ndarray          # float32 [s, s, s]
    mask: np.ndarray              # float32 [s, s, s], binary ball
    radius: int
    n_order: int
    quadrature: np.ndarray        # float32 (n_rot, 4) rotation set for the tensor template
    weights: np.ndarray           # float64 (n_rot,), sums to 1
    positions: np.ndarray         # int64 (P, 3) planted centres (x, y, z)
    planted_quats: np.ndarray     # float32 (P, 4)
    noise_sigma: float
    snr: float

    @property
    def shape(self) -> Tuple[int, int, int]:
        return tuple(self.volume.shape)  # type: ignore[return-value]


# Every config of the benchmark plan, written as the data it generates.
CONFIGS: Dict[str, dict] = {
    # 64^3, 15^3 template of 5 blobs, 4 copies, SNR 1, order 4
    "c1": dict(shape_zyx=(64, 64, 64), s=15, n_blobs=5, lowpass=None, copies=4,
               snr=1.0, n_order=4, n_rot=10000),
    # 256^3, 32^3 lowpassed 30-blob template, 50 copies, SNR 0.5, order 4
    "c2": dict(shape_zyx=(256, 256, 256), s=32, n_blobs=30, lowpass=1.0, copies=50,
               snr=0.5, n_order=4, n_rot=10000),
    # 512^3, 40^3 template, 200 copies, SNR 0.3, order 4
    "c3": dict(shape_zyx=(512, 512, 512), s=40, n_blobs=30, lowpass=1.0, copies=200,
               snr=0.3, n_order=4, n_rot=10000),
    # 928 x 928 x 464 (x, y, z), 64^3 template, 2000 copies, SNR 0.2, order 6
    "c5": dict(shape_zyx=(464, 928, 928), s=64, n_blobs=30, lowpass=1.0, copies=2000,
               snr=0.2, n_order=6, n_rot=20000),
}


def make_workload(shape_zyx: Sequence[int], s: int, n_blobs: int, copies: int,
                  snr: float, n_order: int, n_rot: int,
                  lowpass: Optional[float] = None, radius: Optional[int] = None,
                  seeds: Tuple[int, int, int] = (1, 2, 3), name: str = "custom",
                  noise: bool = True) -> Workload:
    """Build a seeded tomogram: planted rotated copies plus Gaussian noise.

    SNR is var(noise-free volume over the union of the planted mask balls)
    divided by the noise variance.  Seeds are (object, planting, noise).
    """
    obj_seed, plant_seed, noise_seed = seeds
    r = default_mask_radius(s) if radius is None else int(radius)
    t = blob_template(s, n_blobs, obj_seed, lowpass)
    m = ball_mask(s, r)
    rng = np.random.default_rng(plant_seed)
    pos = _random_positions(shape_zyx, s, copies, 2.0 * r, rng)
    pq = shoemake_quaternions(copies, int(rng.integers(1 << 31)))
    clean = plant_copies(shape_zyx, t, pq, pos)
    sigma = 0.0
    if noise and copies > 0 and snr > 0:
        union = np.zeros(clean.shape, dtype=bool)
        c = s // 2
        ball = m.astype(bool)
        for p in pos:
            x0, y0, z0 = (int(p[0]) - c, int(p[1]) - c, int(p[2]) - c)
            union[z0:z0 + s, y0:y0 + s, x0:x0 + s] |= ball
        sigma = float(np.sqrt(np.var(clean[union]) / snr))
        clean += np.random.default_rng(noise_seed).normal(0.0, sigma, size=clean.shape)
    quad = super_fibonacci_quaternions(n_rot)
    return Workload(name=name, volume=clean.astype(np.float32), template=t, mask=m,
                    radius=r, n_order=n_order, quadrature=quad.astype(np.float32),
                    weights=np.full(n_rot, 1.0 / n_rot), positions=pos,
                    planted_quats=pq.astype(np.float32), noise_sigma=sigma, snr=snr)


# Batch of uneven volumes x several templates (2*3*5-smooth extents).
BATCH_CONFIGS: Dict[str, dict] = {
    # 16 volumes (z, y, x) from 128^3 to 384 x 384 x 192, templates 24^3..48^3,
    # copies per (volume, template) = clamp(round(100 V / V_max), 20, 100), SNR 0.5
    "c4": dict(shapes_zyx=[(128, 128, 128), (128, 160, 160), (128, 192, 192), (192, 192, 192),
                           (128, 240, 240), (128, 256, 256), (160, 256, 256), (192, 256, 256),
                           (160, 288, 288), (128, 320, 320), (160, 320, 320), (192, 320, 320),
                           (160, 360, 360), (192, 360, 360), (160, 384, 384), (192, 384, 384)],
               sizes=(24, 32, 40, 48), n_blobs=30, lowpass=1.0, snr=0.5, n_order=4,
               n_rot=10000, copies_min=20, copies_max=100),
}


@dataclasses.dataclass
class BatchWorkload:
    """Several volumes, each holding planted copies of every template."""
    name: str
    volumes: List[np.ndarray]          # float32 [z, y, x] each
    templates: List[np.ndarray]        # float32 [s, s, s] each
    masks: List[np.ndarray]
    radii: List[int]
    n_order: int
    quadrature: np.ndarray
    weights: np.ndarray
    positions: List[List[np.ndarray]]  # [volume][template] -> (P, 3) centres (x, y, z)
    planted_quats: List[List[np.ndarray]]
    snr: float


def _spaced_positions(shape_zyx: Sequence[int], s: int, count: int, min_dist: float,
                      rng: np.random.Generator, taken: List[np.ndarray]) -> np.ndarray:
    """Like _random_positions, also keeping min_dist from the points in taken."""
    c = s // 2
    lo = np.array([c, c, c])
    hi = np.array([shape_zyx[2] - s + c, shape_zyx[1] - s + c, shape_zyx[0] - s + c])
    if np.any(hi < lo):
        raise ValueError("volume smaller than the template box")
    pts = np.zeros((len(taken) + count, 3), dtype=np.int64)
    if taken:
        pts[:len(taken)] = np.asarray(taken, dtype=np.int64).reshape(-1, 3)
    n = len(taken)
    dist, tries = float(min_dist), 0
    while n < len(pts):
        p = np.array([rng.integers(lo[i], hi[i] + 1) for i in range(3)])
        if n == 0 or np.min(np.sum((pts[:n] - p) ** 2, axis=1)) >= dist * dist:
            pts[n] = p
            n += 1
            tries = 0
        else:
            tries += 1
            if tries > 500:
                dist *= 0.9
                tries = 0
    return pts[len(taken):]


def make_batch(shapes_zyx: Sequence[Sequence[int]], sizes: Sequence[int], n_blobs: int,
               snr: float, n_order: int, n_rot: int, copies_min: int, copies_max: int,
               lowpass: Optional[float] = None, seed: int = 1, name: str = "batch",
               copies: Optional[Sequence[Sequence[int]]] = None) -> BatchWorkload:
    """Seeded batch: template k has object seed seed + k; volume v plants
    clamp(round(copies_max V_v / V_max), copies_min, copies_max) copies of
    every template (or copies[v][k]) at Shoemake rotations, then adds noise
    at the given SNR (over the union of all planted mask balls)."""
    templates = [blob_template(s, n_blobs, seed + k, lowpass) for k, s in enumerate(sizes)]
    radii = [default_mask_radius(s) for s in sizes]
    masks = [ball_mask(s, r) for s, r in zip(sizes, radii)]
    vmax = max(int(np.prod(sh)) for sh in shapes_zyx)
    vols, pos_all, quat_all = [], [], []
    for v, shape in enumerate(shapes_zyx):
        rng = np.random.default_rng(1000 * seed + v)
        n_cp = int(np.clip(round(copies_max * np.prod(shape) / vmax), copies_min, copies_max))
        clean = np.zeros(tuple(shape))
        union = np.zeros(tuple(shape), dtype=bool)
        taken: List[np.ndarray] = []
        pv, qv = [], []
        for k in sorted(range(len(sizes)), key=lambda k: -sizes[k]):
            count = n_cp if copies is None else int(copies[v][k])
            pos = _spaced_positions(shape, sizes[k], count, 2.0 * radii[k], rng, taken)
            taken.extend(list(pos))
            pq = shoemake_quaternions(count, int(rng.integers(1 << 31)))
            clean += plant_copies(shape, templates[k], pq, pos)
            c, sk, ball = sizes[k] // 2, sizes[k], masks[k].astype(bool)
            for p in pos:
                x0, y0, z0 = (int(p[0]) - c, int(p[1]) - c, int(p[2]) - c)
                union[z0:z0 + sk, y0:y0 + sk, x0:x0 + sk] |= ball
            pv.append((k, pos))
            qv.append((k, pq.astype(np.float32)))
        sigma = float(np.sqrt(np.var(clean[union]) / snr)) if union.any() and snr > 0 else 0.0
        clean += np.random.default_rng(1000 * seed + 500 + v).normal(0.0, sigma, size=clean.shape)
        vols.append(clean.astype(np.float32))
        pos_all.append([p for _, p in sorted(pv, key=lambda t: t[0])])
        quat_all.append([q for _, q in sorted(qv, key=lambda t: t[0])])
    quad = super_fibonacci_quaternions(n_rot)
    return BatchWorkload(name=name, volumes=vols, templates=templates, masks=masks, radii=radii,
                         n_order=n_order, quadrature=quad.astype(np.float32),
                         weights=np.full(n_rot, 1.0 / n_rot), positions=pos_all,
                         planted_quats=quat_all, snr=snr)


def batch_workload(key: str, **overrides) -> BatchWorkload:
    """Batch workload for one of BATCH_CONFIGS, with optional overrides."""
    cfg = dict(BATCH_CONFIGS[key])
    cfg.update(overrides)
    return make_batch(cfg["shapes_zyx"], cfg["sizes"], cfg["n_blobs"], cfg["snr"],
                      cfg["n_order"], cfg["n_rot"], cfg["copies_min"], cfg["copies_max"],
                      lowpass=cfg.get("lowpass"), seed=cfg.get("seed", 1), name=key,
                      copies=cfg.get("copies"))


def config_workload(key: str, **overrides) -> Workload:
    """Workload for one of CONFIGS, with optional overrides (e.g. n_rot)."""
    cfg = dict(CONFIGS[key])
    cfg.update(overrides)
    return make_workload(cfg["shape_zyx"], cfg["s"], cfg["n_blobs"], cfg["copies"],
                         cfg["snr"], cfg["n_order"], cfg["n_rot"],
                         lowpass=cfg.get("lowpass"), radius=cfg.get("radius"),
                         seeds=cfg.get("seeds", (1, 2, 3)), name=key,
                         noise=cfg.get("noise", True))
