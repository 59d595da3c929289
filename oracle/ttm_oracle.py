"""FP64 CPU oracle for tensorial template matching (TTM).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the CUDA path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and reference
legs) may import it; the product path never does, and this module imports
nothing from the product package.

Every function cites the passage of Almira, Phelippeau & Martinez-Sanchez,
"Fast Normalized Cross-Correlation for Template Matching with Rotations"
(arXiv 2311.07561) that it follows.  Arithmetic is float64 throughout.

Readings taken where the paper is silent:

* the low-pass filter h is the identity unless a Gaussian is asked for
  (lowpass: sampled, unit sum, zero outside the array; the paper allows any
  isotropic h with h*1 = 1, Sec. 2); the mask m is binary or soft;
* rotated templates use trilinear interpolation about the box centre
  floor(s/2), zero outside the box;
* each rotated copy is masked and S-normalised after rotation (Algorithm 1
  normalises then rotates; both agree in the continuum, and normalising every
  rotated copy keeps the discrete identities of the tests exact);
* the measure dR is the normalised Haar measure, discretised by a caller-given
  set of unit quaternions with weights summing to one;
* correlation values are defined on the interior only: voxels whose whole
  template box lies inside the volume; everything else is 0;
* the local variance is treated as zero (w = 0) when it is at most
  1e-6 * m_sum * var(f) with var(f) the variance of the whole volume;
* the per-voxel rotation is the dominant Z-eigenpair of C_n(x) (the global
  maximum of phi(Q) = C_n(x) . Q^(n) on the unit sphere), found by a dense
  search followed by SS-HOPM (Kolda & Mayo 2011) to convergence.

Parity pins: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, library routines, brute force,
identities of the paper); see tests/test_oracle_*.py.
"""

from __future__ import annotations

import functools
import itertools
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

# ==========================================================================
# Quaternions and rotations (Sec. 2: O_R t(z) = t(Rz), t_R = O_{R^-1} t;
# end of Sec. 2: unit quaternions, Re(xy) and <x, y> = Re(y^-1 x))
# ==========================================================================


def quat_mul(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Hamilton product of quaternions (a, b, c, d) = a + bi + cj + dk."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    pa, pv = p[..., 0], p[..., 1:]
    qa, qv = q[..., 0], q[..., 1:]
    a = pa * qa - np.sum(pv * qv, axis=-1)
    v = pa[..., None] * qv + qa[..., None] * pv + np.cross(pv, qv)
    return np.concatenate([a[..., None], v], axis=-1)


def quat_conj(q: np.ndarray) -> np.ndarray:
    q = np.asarray(q, dtype=np.float64)
    return q * np.array([1.0, -1.0, -1.0, -1.0])


def rotate_vectors(q: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Rotate column vectors v (..., 3) by unit quaternion q: v -> q v q*."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q)
    pure = np.concatenate([np.zeros(v.shape[:-1] + (1,)), v], axis=-1)
    return quat_mul(quat_mul(q, pure), quat_conj(q))[..., 1:]


def rotation_matrix(q: np.ndarray) -> np.ndarray:
    """3x3 matrix of v -> q v q*, built column by column from quat_mul."""
    return rotate_vectors(q, np.eye(3)).T


def rotate_template(t: np.ndarray, q: np.ndarray) -> np.ndarray:
    """t_R(u) = t(c + R^-1 (u - c)) for the rotation R of q (Sec. 2, t_R).

    Trilinear interpolation of the s^3 box ``t`` (indexed [z, y, x]) about the
    centre c = floor(s/2), reading 0 outside the box.  Returns float64.
    """
    t = np.asarray(t, dtype=np.float64)
    s = t.shape[0]
    c = s // 2
    z, y, x = np.meshgrid(*(np.arange(s, dtype=np.float64) - c,) * 3, indexing="ij")
    v = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=-1)
    p = rotate_vectors(quat_conj(q), v) + c          # R^-1 (u - c) + c, as (x, y, z)
    base = np.floor(p)
    frac = p - base
    base = base.astype(np.int64)
    out = np.zeros(p.shape[0])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ix, iy, iz = base[:, 0] + dx, base[:, 1] + dy, base[:, 2] + dz
                wgt = ((frac[:, 0] if dx else 1.0 - frac[:, 0])
                       * (frac[:, 1] if dy else 1.0 - frac[:, 1])
                       * (frac[:, 2] if dz else 1.0 - frac[:, 2]))
                ok = (ix >= 0) & (ix < s) & (iy >= 0) & (iy < s) & (iz >= 0) & (iz < s)
                val = np.zeros(p.shape[0])
                val[ok] = t[iz[ok], iy[ok], ix[ok]]
                out += wgt * val
    return out.reshape(s, s, s)


# ==========================================================================
# Symmetric tensors (Sec. 3.1)
# ==========================================================================


@functools.lru_cache(maxsize=None)
def multi_indices(n: int, d: int = 4) -> Tuple[Tuple[int, ...], ...]:
    """Independent components of S^n(R^d): sorted index tuples i1 <= ... <= in,
    in lexicographic order.  There are C(n+d-1, n) of them (Sec. 3.1)."""
    return tuple(itertools.combinations_with_replacement(range(d), n))


def multinomial(alpha: Sequence[int], d: int = 4) -> int:
    """Number of index tuples that sort to alpha: n! / prod(count_i!)."""
    counts = [list(alpha).count(i) for i in range(d)]
    out = math.factorial(len(alpha))
    for k in counts:
        out //= math.factorial(k)
    return out


def monomials(q: np.ndarray, n: int) -> np.ndarray:
    """q^alpha = q_{i1} ... q_{in} for every component alpha; q (..., 4) -> (..., K)."""
    q = np.asarray(q, dtype=np.float64)
    cols = [np.prod(q[..., list(a)], axis=-1) for a in multi_indices(n)]
    return np.stack(cols, axis=-1)


@functools.lru_cache(maxsize=None)
def _full_to_unique(n: int) -> np.ndarray:
    """For every full index tuple (i1..in) in C order, the position of its
    sorted tuple in multi_indices(n)."""
    pos = {a: k for k, a in enumerate(multi_indices(n))}
    return np.array([pos[tuple(sorted(ix))] for ix in itertools.product(range(4), repeat=n)])


def expand_full(C: np.ndarray, n: int) -> np.ndarray:
    """Symmetric tensor with every entry: (..., K) -> (..., 4, ..., 4)."""
    C = np.asarray(C, dtype=np.float64)
    return C[..., _full_to_unique(n)].reshape(C.shape[:-1] + (4,) * n)


def contract(A: np.ndarray, x: np.ndarray, times: int) -> np.ndarray:
    """A x^k of Sec. 3.1: contract the last ``times`` indices of A with x."""
    x = np.asarray(x, dtype=np.float64)
    lead = x.shape[:-1]
    out = np.asarray(A, dtype=np.float64).reshape((-1,) + A.shape[len(lead):])
    xx = x.reshape(-1, x.shape[-1])
    for _ in range(times):
        out = np.einsum("n...i,ni->n...", out, xx)
    return out.reshape(lead + out.shape[1:])


def phi_full(A: np.ndarray, Q: np.ndarray, n: int) -> np.ndarray:
    """phi(Q) = A . Q^(n) = sum over all index tuples of A_{i..} Q_i1..Q_in."""
    return contract(A, Q, n)


def frobenius(A: np.ndarray, n: int) -> np.ndarray:
    """Frobenius norm of a full tensor (..., 4, ..., 4) (Sec. 3.4)."""
    return np.sqrt(np.sum(A.reshape(A.shape[:A.ndim - n] + (-1,)) ** 2, axis=-1))


# ==========================================================================
# Optional isotropic low-pass filter h (Sec. 2: t' = h * t and f' = h * f with
# h * 1 = 1; identity unless asked for)
# ==========================================================================

def gaussian_kernel(sigma: float) -> np.ndarray:
    """Sampled Gaussian exp(-d^2 / (2 sigma^2)), d = -r..r with
    r = int(4 sigma + 0.5), normalised to unit sum (unit DC gain)."""
    r = int(4.0 * sigma + 0.5)
    d = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (d / sigma) ** 2)
    return k / k.sum()


def lowpass(x: np.ndarray, sigma: float) -> np.ndarray:
    """h * x for the Gaussian h of gaussian_kernel: the same 1D kernel along
    each axis in turn, linear convolution with zero outside the array."""
    y = np.asarray(x, dtype=np.float64)
    k = gaussian_kernel(sigma)
    r = (len(k) - 1) // 2
    for axis in range(y.ndim):
        n = y.shape[axis]
        out = np.zeros_like(y)
        for j, kj in enumerate(k):
            d = j - r                                  # out[i] += k[j] * y[i + d]
            lo, hi = max(0, -d), min(n, n - d)
            if hi <= lo:
                continue
            src = [slice(None)] * y.ndim
            dst = [slice(None)] * y.ndim
            src[axis] = slice(lo + d, hi + d)
            dst[axis] = slice(lo, hi)
            out[tuple(dst)] += kj * y[tuple(src)]
        y = out
    return y


# ==========================================================================
# Template normalisation and the tensor template
# (Sec. 2 formulas for ||P_S t||_S and <t, 1>_S; Algorithm 1 template block;
#  Sec. 3.2 definition T(z) = int R^(n) S(t)_R(z) dR)
# ==========================================================================


def normalise_under_mask(u: np.ndarray, m: np.ndarray) -> np.ndarray:
    """m * (u - <u,m>/<1,m>) / sqrt(<u^2,m> - <u,m>^2/<1,m>)  (Algorithm 1)."""
    u = np.asarray(u, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    m_sum = m.sum()
    t1 = np.sum(u * m)
    t2 = np.sum(u * u * m)
    return m * (u - t1 / m_sum) / np.sqrt(t2 - t1 * t1 / m_sum)


def rotated_normalised(t: np.ndarray, m: np.ndarray, q: np.ndarray) -> np.ndarray:
    """The S-normalised, masked copy of t rotated by q (one quadrature node)."""
    return normalise_under_mask(rotate_template(t, q), m)


def tensor_template(t: np.ndarray, m: np.ndarray, quats: np.ndarray,
                    weights: np.ndarray, n: int, chunk: int = 128) -> np.ndarray:
    """Unique components T_alpha(z) = sum_j w_j q_j^alpha t~_j(z)  (Sec. 3.2).

    Returns (K, s, s, s) float64 in the order of multi_indices(n).
    """
    s = t.shape[0]
    quats = np.asarray(quats, dtype=np.float64)
    weights = np.asarray(weights, dtype=np.float64)
    K = len(multi_indices(n))
    T = np.zeros((K, s ** 3))
    for j0 in range(0, len(quats), chunk):
        q = quats[j0:j0 + chunk]
        U = np.stack([rotated_normalised(t, m, qq).ravel() for qq in q])
        coeff = weights[j0:j0 + chunk, None] * monomials(q, n)      # (J, K)
        T += coeff.T @ U
    return T.reshape(K, s, s, s)


def tensor_template_full(t: np.ndarray, m: np.ndarray, quats: np.ndarray,
                         weights: np.ndarray, n: int) -> np.ndarray:
    """Every entry T_{i1..in}(z) = sum_j w_j q_j,i1 ... q_j,in t~_j(z).

    A second, independent construction (outer products of q with itself) used
    to check symmetry and the unique-component form.  Shape (4,)*n + (s,s,s).
    """
    s = t.shape[0]
    out = np.zeros((4,) * n + (s ** 3,))
    for q, w in zip(np.asarray(quats, dtype=np.float64), weights):
        power = np.array(1.0)
        for _ in range(n):
            power = np.multiply.outer(power, q)
        out += w * np.multiply.outer(power, rotated_normalised(t, m, q).ravel())
    return out.reshape((4,) * n + (s, s, s))


# ==========================================================================
# Correlation and local statistics
# (Sec. 2: (f * g)(x) = int f(z + x) g(z) dz; <f,g> via F^-1(F f . conj F g);
#  ||P_S tau_x f||_S^2 = <(tau_x f)^2, m> - <tau_x f, m>^2 / <1, m>;
#  Algorithm 1, image block)
# ==========================================================================


def interior_bounds(shape_zyx: Sequence[int], s: int) -> Tuple[Tuple[int, int], ...]:
    """Per axis (z, y, x) the inclusive range of voxels whose s^3 box fits."""
    c = s // 2
    return tuple((c, n - s + c) for n in shape_zyx)


def interior_mask(shape_zyx: Sequence[int], s: int) -> np.ndarray:
    out = np.zeros(tuple(shape_zyx), dtype=bool)
    (z0, z1), (y0, y1), (x0, x1) = interior_bounds(shape_zyx, s)
    if z1 >= z0 and y1 >= y0 and x1 >= x0:
        out[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] = True
    return out


def correlate_direct(f: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Corr[k](x) = sum_u f(x + u - c) T[k](u) on the interior, by direct sum.

    f is (Z, Y, X); T is (..., s, s, s).  Returns (..., Z, Y, X), 0 outside
    the interior.
    """
    f = np.asarray(f, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    lead = T.shape[:-3]
    s = T.shape[-1]
    Tf = T.reshape((-1, s, s, s))
    Z, Y, X = f.shape
    (z0, z1), (y0, y1), (x0, x1) = interior_bounds(f.shape, s)
    out = np.zeros((Tf.shape[0], Z, Y, X))
    if z1 < z0 or y1 < y0 or x1 < x0:
        return out.reshape(lead + (Z, Y, X))
    nz, ny, nx = z1 - z0 + 1, y1 - y0 + 1, x1 - x0 + 1
    acc = np.zeros((Tf.shape[0], nz, ny, nx))
    for uz, uy, ux in zip(*np.nonzero(np.any(Tf != 0, axis=0))):
        # voxel x + u - c for x - c starting at 0
        window = f[uz:uz + nz, uy:uy + ny, ux:ux + nx]
        acc += Tf[:, uz, uy, ux][:, None, None, None] * window[None]
    out[:, z0:z1 + 1, y0:y1 + 1, x0:x1 + 1] = acc
    return out.reshape(lead + (Z, Y, X))


def correlate_fft(f: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Same correlation through the FFT identity of Sec. 2 (circular), then
    restricted to the interior, where circular and linear sums coincide."""
    f = np.asarray(f, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    lead = T.shape[:-3]
    s = T.shape[-1]
    c = s // 2
    Tf = T.reshape((-1, s, s, s))
    F = np.fft.rfftn(f)
    keep = interior_mask(f.shape, s)
    out = np.zeros((Tf.shape[0],) + f.shape)
    for k in range(Tf.shape[0]):
        pad = np.zeros(f.shape)
        pad[:s, :s, :s] = Tf[k]
        pad = np.roll(pad, shift=(-c, -c, -c), axis=(0, 1, 2))   # pad[(u-c) mod N] = T[u]
        corr = np.fft.irfftn(F * np.conj(np.fft.rfftn(pad)), s=f.shape, axes=(0, 1, 2))
        out[k] = np.where(keep, corr, 0.0)
    return out.reshape(lead + f.shape)


W_EPS = 1e-6   # relative variance floor: w = 0 when V <= W_EPS * m_sum * var(f)


def inverse_norm(S1: np.ndarray, S2: np.ndarray, m_sum: float, var_f: float,
                 keep: np.ndarray) -> np.ndarray:
    """w = 1 / ||P_S tau_x f||_S = 1 / sqrt(S2 - S1^2 / m_sum)  (Algorithm 1),
    set to 0 outside ``keep`` and where the local variance is degenerate."""
    V = S2 - S1 * S1 / m_sum
    ok = keep & (V > W_EPS * m_sum * var_f)
    w = np.zeros_like(V)
    w[ok] = 1.0 / np.sqrt(V[ok])
    return w


def local_stats_direct(f: np.ndarray, m: np.ndarray):
    """S1 = <tau_x f, m>, S2 = <(tau_x f)^2, m> and w on the interior, summing
    over every mask voxel (plain definition).  Returns (S1, S2, w)."""
    f = np.asarray(f, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    S1 = correlate_direct(f, m)
    S2 = correlate_direct(f * f, m)
    keep = interior_mask(f.shape, m.shape[0])
    return S1, S2, inverse_norm(S1, S2, m.sum(), float(np.var(f)), keep)


def local_stats_fft(f: np.ndarray, m: np.ndarray):
    """The same statistics the way Algorithm 1 computes them: FFT of f and of
    f^2, multiplied by conj(FFT(m)), inverted (float64)."""
    f = np.asarray(f, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    S1 = correlate_fft(f, m)
    S2 = correlate_fft(f * f, m)
    keep = interior_mask(f.shape, m.shape[0])
    return S1, S2, inverse_norm(S1, S2, m.sum(), float(np.var(f)), keep)


def patches_at(f: np.ndarray, points_xyz: np.ndarray, s: int) -> np.ndarray:
    """The s^3 box of f around each point (x, y, z): (P, s^3) float64."""
    f = np.asarray(f, dtype=np.float64)
    c = s // 2
    out = np.empty((len(points_xyz), s ** 3))
    for i, (x, y, z) in enumerate(np.asarray(points_xyz, dtype=np.int64)):
        out[i] = f[z - c:z - c + s, y - c:y - c + s, x - c:x - c + s].ravel()
    return out


def components_at(f: np.ndarray, T: np.ndarray, m: np.ndarray,
                  points_xyz: np.ndarray, var_f: Optional[float] = None):
    """w(x) and C_alpha(x) = w(x) <tau_x f, T_alpha> at interior sample points,
    each by direct sum over its own box (Sec. 3.2).  Returns (w, C (P, K))."""
    s = m.shape[0]
    P = patches_at(f, points_xyz, s)
    mm = np.asarray(m, dtype=np.float64).ravel()
    S1 = P @ mm
    S2 = (P * P) @ mm
    if var_f is None:
        var_f = float(np.var(np.asarray(f, dtype=np.float64)))
    w = inverse_norm(S1, S2, mm.sum(), var_f, np.ones(len(P), dtype=bool))
    corr = P @ np.asarray(T, dtype=np.float64).reshape(T.shape[0], -1).T
    return w, w[:, None] * corr


def ttm_components(f: np.ndarray, T: np.ndarray, m: np.ndarray,
                   use_fft: bool = True):
    """C_n(x)_alpha = w(x) <tau_x f, T_alpha> on the whole interior (Sec. 3.2).
    Returns (w, C) with C of shape (K, Z, Y, X)."""
    stats = local_stats_fft if use_fft else local_stats_direct
    _, _, w = stats(f, m)
    corr = (correlate_fft if use_fft else correlate_direct)(f, T)
    return w, w[None] * corr


def frobenius_score(C: np.ndarray, n: int, axis: int = 0) -> np.ndarray:
    """||C_n(x)||_F of the full symmetric tensor (Sec. 3.4 position score)."""
    C = np.moveaxis(np.asarray(C, dtype=np.float64), axis, -1)
    return frobenius(expand_full(C, n), n)


# ==========================================================================
# Classical template matching (Algorithm 1, per rotation)
# ==========================================================================


def classical_ncc(f: np.ndarray, t: np.ndarray, m: np.ndarray,
                  quats: np.ndarray) -> np.ndarray:
    """c(x, R_j) = w(x) (f * S(t)_{R_j})(x) for every rotation j (Algorithm 1).
    Returns (J, Z, Y, X) on the interior (small inputs only)."""
    _, _, w = local_stats_fft(f, m)
    tj = np.stack([rotated_normalised(t, m, q) for q in np.asarray(quats, dtype=np.float64)])
    return w[None] * correlate_fft(f, tj)


def classical_best(f: np.ndarray, t: np.ndarray, m: np.ndarray, quats: np.ndarray):
    """max_j c(x, R_j) and the first j attaining it (Algorithm 1 over a set)."""
    _, _, w = local_stats_fft(f, m)
    best = np.full(f.shape, -np.inf)
    arg = np.zeros(f.shape, dtype=np.int64)
    for j, q in enumerate(np.asarray(quats, dtype=np.float64)):
        c = w * correlate_fft(f, rotated_normalised(t, m, q)[None])[0]
        better = c > best
        best[better] = c[better]
        arg[better] = j
    keep = interior_mask(f.shape, t.shape[0])
    return np.where(keep, best, 0.0), np.where(keep, arg, 0)


# ==========================================================================
# Rotation: dominant Z-eigenpair of C_n(x)
# (Sec. 3.1 Z-eigenpairs; Sec. 3.3 Theorem 3.1; Sec. 3.4 SS-HOPM)
# ==========================================================================


def ss_hopm(A: np.ndarray, x0: np.ndarray, n: int, shift: np.ndarray,
            tol: float = 1e-14, max_iter: int = 5000):
    """Shifted symmetric higher-order power method (Kolda & Mayo 2011).

    Repeats x <- (A x^{n-1} + shift * x) / ||A x^{n-1} + shift * x|| and stops
    a trajectory once its value lambda_k = A x_k^n changes by at most ``tol``
    (or after ``max_iter`` steps).  With shift at least
    (n-1) * max_x rho(A x^{n-2}) (Kolda & Mayo, Thm 4.4) the values increase
    monotonically to a local maximum on the sphere.  A is (N, 4, ..., 4),
    x0 (N, 4), shift (N,).  Returns (lambda, x, iterations).
    """
    N = A.shape[0]
    x = x0 / np.linalg.norm(x0, axis=-1, keepdims=True)
    lam = contract(A, x, n)
    act = np.arange(N)
    Aa, xa, sa, la = A, x.copy(), shift, lam.copy()
    it = 0
    while it < max_iter and len(act):
        g = contract(Aa, xa, n - 1) + sa[:, None] * xa
        gn = np.linalg.norm(g, axis=-1, keepdims=True)
        xa = np.where(gn > 0, g / np.where(gn > 0, gn, 1.0), xa)   # A = 0: stay put
        ln = contract(Aa, xa, n)
        done = np.abs(ln - la) <= tol
        la = ln
        it += 1
        if it % 16 == 0 or done.all() or it == max_iter:
            x[act], lam[act] = xa, la
            keep = ~done
            act, Aa, xa, sa, la = act[keep], Aa[keep], xa[keep], sa[keep], la[keep]
    x[act], lam[act] = xa, la
    return lam, x, it


def canonical_quaternion(q: np.ndarray) -> np.ndarray:
    """Representative of {q, -q}: real part positive (else the first non-zero
    component positive).  n is even, so phi(q) = phi(-q)."""
    q = np.array(q, dtype=np.float64)
    flat = q.reshape(-1, 4)
    for row in flat:
        nz = np.nonzero(np.abs(row) > 0)[0]
        if len(nz) and row[nz[0]] < 0:
            row *= -1.0
    return flat.reshape(q.shape)


@functools.lru_cache(maxsize=None)
def search_grid(G: int = 8192, k: int = 12, seed: int = 20231113):
    """The oracle's own dense search set on S^3 (uniform random, fixed seed)
    and, for each point, its k nearest neighbours under the q ~ -q
    identification (largest |<p, q>|)."""
    rng = np.random.default_rng(seed)
    pts = rng.normal(size=(G, 4))
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    nbr = np.empty((G, k), dtype=np.int64)
    for i0 in range(0, G, 1024):
        sim = np.abs(pts[i0:i0 + 1024] @ pts.T)
        sim[np.arange(sim.shape[0]), np.arange(i0, i0 + sim.shape[0])] = -1.0
        nbr[i0:i0 + 1024] = np.argsort(-sim, axis=1)[:, :k]
    return pts, nbr


def dominant_z_eigenpair(C: np.ndarray, n: int, n_candidates: int = 8,
                         grid_size: int = 8192):
    """lambda*(x) = max_{|Q|=1} phi(Q) and its maximiser q*(x) (Sec. 3.3, 3.4).

    phi is evaluated on the oracle's dense search set; every grid point at
    least as large as its neighbours is a candidate; the ``n_candidates``
    largest candidates are polished by SS-HOPM with the convexity shift
    (n-1)||C||_F (it bounds (n-1) rho(C x^{n-2}) on the unit sphere) and the
    largest result is kept.  C is (P, K) in the order of multi_indices(n).
    Returns (lambda (P,), q (P, 4) canonical).  C = 0 gives (0, identity).
    """
    C = np.atleast_2d(np.asarray(C, dtype=np.float64))
    P = C.shape[0]
    grid, nbr = search_grid(grid_size)
    Qn = grid
    for _ in range(n - 1):
        Qn = np.einsum("g...,gi->g...i", Qn, grid)
    Qn = Qn.reshape(grid.shape[0], -1)                      # (G, 4^n)
    m = min(n_candidates, grid.shape[0])
    lam_out = np.zeros(P)
    q_out = np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (P, 1))
    for p0 in range(0, P, 256):
        A = expand_full(C[p0:p0 + 256], n)
        B = A.shape[0]
        vals = A.reshape(B, -1) @ Qn.T                      # phi on the grid, (B, G)
        is_max = vals >= vals[:, nbr].max(axis=2)
        ranked = np.where(is_max, vals, -np.inf)
        top = np.argsort(-ranked, axis=1)[:, :m]
        valid = np.take_along_axis(ranked, top, axis=1) > -np.inf
        top = np.where(valid, top, top[:, :1])              # pad with the best one
        x0 = grid[top].reshape(B * m, 4)
        Ar = np.repeat(A, m, axis=0)
        shift = np.repeat((n - 1) * frobenius(A, n), m)
        lam, x, _ = ss_hopm(Ar, x0, n, shift)
        lam, x = lam.reshape(B, m), x.reshape(B, m, 4)
        best = np.argmax(lam, axis=1)
        nz = frobenius(A, n) > 0
        rows = np.arange(B)[nz]
        lam_out[p0 + rows] = lam[rows, best[nz]]
        q_out[p0 + rows] = x[rows, best[nz]]
    return lam_out, canonical_quaternion(q_out)


def phi_unique(C: np.ndarray, Q: np.ndarray, n: int) -> np.ndarray:
    """phi(Q) = C . Q^(n) evaluated through the full tensor; C (P, K), Q (P, 4)."""
    return phi_full(expand_full(C, n), np.asarray(Q, dtype=np.float64), n)


def rotation_angle_deg(q1: np.ndarray, q2: np.ndarray) -> np.ndarray:
    """Angle of the rotation taking q2 to q1, in degrees: 2 acos |<q1, q2>|."""
    d = np.abs(np.sum(np.asarray(q1, np.float64) * np.asarray(q2, np.float64), axis=-1))
    return np.rad2deg(2.0 * np.arccos(np.clip(d, 0.0, 1.0)))


# ==========================================================================
# Peaks of the position score (Sec. 3.4)
# ==========================================================================


def extract_peaks(score: np.ndarray, threshold: float, radius: int,
                  max_peaks: int) -> np.ndarray:
    """Voxels whose score exceeds ``threshold`` and beats every other voxel of
    the (2*radius+1)^3 cube around it (a tie goes to the lower linear index;
    the cube is clipped to the array).  Returns up to ``max_peaks`` linear
    indices, highest score first (ties: lower index first).

    Every voxel above the threshold is a candidate; each candidate is checked
    against every voxel of its cube, one cube offset at a time."""
    score = np.asarray(score, dtype=np.float64)
    Z, Y, X = score.shape
    flat = score.ravel()
    cand = np.nonzero(flat > threshold)[0]
    cz, rem = np.divmod(cand, Y * X)
    cy, cx = np.divmod(rem, X)
    ok = np.ones(len(cand), dtype=bool)
    for dz in range(-radius, radius + 1):
        for dy in range(-radius, radius + 1):
            for dx in range(-radius, radius + 1):
                if dz == 0 and dy == 0 and dx == 0:
                    continue
                nz, ny, nx = cz + dz, cy + dy, cx + dx
                inside = (nz >= 0) & (nz < Z) & (ny >= 0) & (ny < Y) & (nx >= 0) & (nx < X)
                nb = (np.clip(nz, 0, Z - 1) * Y + np.clip(ny, 0, Y - 1)) * X + np.clip(nx, 0, X - 1)
                u = flat[nb]
                beaten = inside & ((u > flat[cand]) | ((u == flat[cand]) & (nb < cand)))
                ok &= ~beaten
    idx = cand[ok]
    order = np.lexsort((idx, -flat[idx]))
    return idx[order][:max_peaks]


# ==========================================================================
# The S'-consistent normalisation (Sec. 3.3, proof of Theorem 3.1, and the
# false-positive discussion of Sec. 3.4).
#
# The proof of Theorem 3.1 shows phi(Q) = C_n(x) . Q^(n) = w(x) <tau_x f, t_Q>_S'
# with S' = S_2 o S and S_2(t) = (t (*) K)(I_d), K(R) = Re(R)^n: S_2 averages
# the rotated copies t_R of its argument with weight Re(R)^n (Re(R^-1) =
# Re(R)), so <f, g>_S' = int Re(R)^n <f, g_R>_S dR for a rotation-invariant
# mask.  TTM normalises with S (w(x) = 1/||P_S tau_x f||_S, ||t||_S = 1); the
# S'-consistent value divides phi(Q) / w(x) by ||P_S' tau_x f||_S' ||t_Q||_S'
# instead, which keeps it in [-1, 1] with 1 at a match.  Discretised with the
# caller's quadrature {q_j, w_j} and trilinear rotation (the readings above);
# h is the identity.
# ==========================================================================


def s2_apply(u: np.ndarray, quats: np.ndarray, weights: np.ndarray, n: int) -> np.ndarray:
    """S_2(u) = sum_j w_j Re(q_j)^n u_{R_j}: the Re(R)^n-weighted average of
    the rotated copies of the s^3 box u (rotate_template)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    for q, wj in zip(np.asarray(quats, dtype=np.float64), np.asarray(weights, dtype=np.float64)):
        a = q[0] / np.linalg.norm(q)
        out += wj * a ** n * rotate_template(u, q)
    return out


def sprime_inner(f: np.ndarray, g: np.ndarray, m: np.ndarray, quats: np.ndarray,
                 weights: np.ndarray, n: int) -> float:
    """<f, g>_S' = <f, S'(g)> with S'(g) = S_2(S(g)) = S_2(m g) (h = identity)."""
    m = np.asarray(m, dtype=np.float64)
    return float(np.sum(np.asarray(f, dtype=np.float64)
                        * s2_apply(m * np.asarray(g, dtype=np.float64), quats, weights, n)))


def sprime_projected_norm(patch: np.ndarray, m: np.ndarray, quats: np.ndarray,
                          weights: np.ndarray, n: int) -> float:
    """||P_S' p||_S' of an s^3 patch: P_S' p = p - (<p, 1>_S' / <1, 1>_S') 1
    removes the S'-mean (the projection of Sec. 2, taken in S')."""
    p = np.asarray(patch, dtype=np.float64)
    one = np.ones_like(p)
    mean = sprime_inner(p, one, m, quats, weights, n) / sprime_inner(one, one, m, quats, weights, n)
    g = p - mean
    return math.sqrt(max(sprime_inner(g, g, m, quats, weights, n), 0.0))


def sprime_ncc_at(f: np.ndarray, t: np.ndarray, m: np.ndarray, quats: np.ndarray,
                  weights: np.ndarray, n: int, points_xyz: np.ndarray,
                  Q: np.ndarray) -> np.ndarray:
    """The S'-consistent normalised correlation at each point x and rotation Q
    (one Q per point):  <P_S' tau_x f, t~_Q>_S' / (||P_S' tau_x f||_S' ||t~_Q||_S'),
    t~_Q the masked, S-normalised template rotated by Q (rotated_normalised)."""
    s = np.asarray(m).shape[0]
    P = patches_at(f, points_xyz, s).reshape(-1, s, s, s)
    out = np.empty(len(P))
    for i, (p, q) in enumerate(zip(P, np.asarray(Q, dtype=np.float64).reshape(-1, 4))):
        tq = rotated_normalised(t, m, q)
        one = np.ones_like(p)
        mean = sprime_inner(p, one, m, quats, weights, n) / sprime_inner(one, one, m, quats, weights, n)
        g = p - mean
        num = 0.5 * (sprime_inner(g, tq, m, quats, weights, n) + sprime_inner(tq, g, m, quats, weights, n))
        den = math.sqrt(max(sprime_inner(g, g, m, quats, weights, n), 0.0)
                        * max(sprime_inner(tq, tq, m, quats, weights, n), 0.0))
        out[i] = num / den if den > 0 else 0.0
    return out


def sprime_rescale_at(f: np.ndarray, t: np.ndarray, m: np.ndarray, quats: np.ndarray,
                      weights: np.ndarray, n: int, points_xyz: np.ndarray,
                      var_f: Optional[float] = None) -> np.ndarray:
    """The factor that turns TTM's S-normalised C_n(x) into the S'-consistent
    one at each point: rho(x) = ||P_S tau_x f||_S / (||P_S' tau_x f||_S' ||t~||_S'),
    so that rho(x) phi(Q) is phi(Q) / (w(x) ||P_S' tau_x f||_S' ||t~||_S') (the
    template's S'-norm is taken unrotated; it does not depend on Q in the
    continuum).  Scaling C_n(x) by rho(x) > 0 leaves its maximiser q unchanged
    and scales the score and lambda."""
    s = np.asarray(m).shape[0]
    P = patches_at(f, points_xyz, s).reshape(-1, s, s, s)
    w, _ = components_at(f, np.zeros((1, s, s, s)), m, points_xyz, var_f=var_f)
    tt = normalise_under_mask(t, m)
    tnorm = math.sqrt(max(sprime_inner(tt, tt, m, quats, weights, n), 0.0))
    out = np.zeros(len(P))
    for i, p in enumerate(P):
        if w[i] > 0:
            out[i] = (1.0 / w[i]) / (sprime_projected_norm(p, m, quats, weights, n) * tnorm)
    return out
