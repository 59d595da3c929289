"""Pins of the oracle's S'-consistent normalisation (Sec. 3.3, proof of
Theorem 3.1; Sec. 3.4, false positives).

On the 24 rotations of the cube (the octahedral group) trilinear rotation of
an odd box is an exact permutation that keeps the ball mask, so with the group
as the quadrature the discrete identities of the proof hold exactly:
phi(Q) = w(x) <tau_x f, t_Q>_S', S_2 is symmetric positive semidefinite (its
kernel Re(R)^n = (p . q)^n is a Gram kernel), the S'-normalised correlation is
1 at a match, and the S_2 weight of an isotropic patch is the Haar moment
E[a^n] of the unit sphere in R^4 (the group is a spherical 7-design).
"""

import itertools
import math

import numpy as np
import pytest

import synth
from oracle import ttm_oracle as o


def octahedral_group():
    """The 24 rotations of the cube as unit quaternions (a, b, c, d)."""
    q = [np.array([1.0, 0, 0, 0])]
    h = math.sqrt(0.5)
    for i in range(3):
        e = np.zeros(3)
        e[i] = 1.0
        for ang in (0.5 * math.pi, math.pi, 1.5 * math.pi):
            q.append(np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * e]))
    for sx, sy, sz in itertools.product((1, -1), repeat=3):
        if sx > 0:            # +-(1, +-1, +-1, +-1)/2: turns by 120 and 240 degrees
            q.append(0.5 * np.array([1.0, sx, sy, sz]))
            q.append(0.5 * np.array([1.0, -sx, -sy, -sz]))
    for i, j in ((0, 1), (0, 2), (1, 2)):
        for sgn in (1.0, -1.0):
            v = np.zeros(3)
            v[i], v[j] = h, sgn * h
            q.append(np.concatenate([[0.0], v]))
    G = np.array(q)
    assert len(G) == 24
    return G


G = octahedral_group()
WG = np.full(len(G), 1.0 / len(G))


def test_group_is_closed_and_permutes_the_grid():
    R = [o.rotation_matrix(q) for q in G]
    for a in R:
        assert np.allclose(a, np.round(a), atol=1e-12)
        for b in R:
            assert any(np.allclose(a @ b, c, atol=1e-12) for c in R)
    t = synth.blob_template(7, 3, seed=4).astype(np.float64)
    for q in G:
        r = o.rotate_template(t, q)
        assert np.allclose(np.sort(r.ravel()), np.sort(t.ravel()), atol=1e-12)


@pytest.mark.parametrize("n", [4, 6])
def test_isotropic_patch_weight_is_the_haar_moment(n):
    """For a patch invariant under the group, S_2 multiplies it by
    sum_j w_j a_j^n, which on the group equals E[a^n] on S^3:
    (n-1)!! / (4 * 6 * ... * (n + 2))."""
    s, c = 9, 4
    z, y, x = np.meshgrid(*(np.arange(s) - c,) * 3, indexing="ij")
    g = np.exp(-(x * x + y * y + z * z) / 6.0)
    m = synth.ball_mask(s, 4).astype(np.float64)
    moment = math.prod(range(n - 1, 0, -2)) / math.prod(range(4, n + 3, 2))
    assert np.sum(WG * G[:, 0] ** n) == pytest.approx(moment, rel=1e-12)
    assert np.allclose(o.s2_apply(m * g, G, WG, n), moment * m * g, atol=1e-14)
    assert o.sprime_inner(g, g, m, G, WG, n) == pytest.approx(moment * np.sum(m * g * g), rel=1e-12)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_s2_is_symmetric_positive_semidefinite(n):
    s = 7
    m = synth.ball_mask(s, 3).astype(np.float64)
    idx = np.flatnonzero(m.ravel())
    A = np.zeros((len(idx), len(idx)))
    for col, k in enumerate(idx):
        e = np.zeros(s ** 3)
        e[k] = 1.0
        A[:, col] = (m * o.s2_apply(m * e.reshape(s, s, s), G, WG, n)).ravel()[idx]
    assert np.allclose(A, A.T, atol=1e-14)
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() >= -1e-12


@pytest.fixture(scope="module")
def group_problem():
    s, r = 7, 3
    t = synth.blob_template(s, 4, seed=21)
    m = synth.ball_mask(s, r)
    rng = np.random.default_rng(22)
    f = rng.normal(size=(17, 16, 15))
    T = o.tensor_template(t, m, G, WG, 4)
    pts = np.array([[3, 3, 3], [7, 8, 9], [11, 12, 13], [5, 10, 6]])
    w, C = o.components_at(f, T, m, pts)
    return t, m, f, pts, w, C


def test_phi_is_the_sprime_correlation(group_problem):
    """phi(Q) = C_n(x) . Q^(n) = w(x) <tau_x f, t_Q>_S' (proof of Theorem 3.1)."""
    t, m, f, pts, w, C = group_problem
    P = o.patches_at(f, pts, 7).reshape(-1, 7, 7, 7)
    for i in range(len(pts)):
        for Q in G[::3]:
            tq = o.rotated_normalised(t, m, Q)
            lhs = o.phi_unique(C[i:i + 1], Q[None], 4)[0]
            rhs = w[i] * o.sprime_inner(P[i], tq, m, G, WG, 4)
            assert lhs == pytest.approx(rhs, abs=1e-12)


def test_sprime_mean_is_the_s_mean_and_rescale_matches_ncc(group_problem):
    """On the group the S'-mean of a patch is its S-mean (S_2 scales the
    constant), and rho(x) phi(Q) is the S'-normalised correlation."""
    t, m, f, pts, w, C = group_problem
    P = o.patches_at(f, pts, 7).reshape(-1, 7, 7, 7)
    mm = m.astype(np.float64)
    one = np.ones((7, 7, 7))
    for p in P:
        mean_sp = o.sprime_inner(p, one, m, G, WG, 4) / o.sprime_inner(one, one, m, G, WG, 4)
        assert mean_sp == pytest.approx(np.sum(mm * p) / mm.sum(), rel=1e-12)
    rho = o.sprime_rescale_at(f, t, m, G, WG, 4, pts)
    Q = G[[1, 5, 9, 14]]
    ncc = o.sprime_ncc_at(f, t, m, G, WG, 4, pts, Q)
    phi = np.array([o.phi_unique(C[i:i + 1], Q[i][None], 4)[0] for i in range(len(pts))])
    assert np.allclose(rho * phi, ncc, atol=1e-12)
    assert np.all(np.abs(ncc) <= 1.0 + 1e-12)


def test_sprime_ncc_is_one_at_a_match_and_affine_invariant():
    """Theorem 2.4 in the S' inner product: at a noise-free isolated copy
    planted with a group rotation the S'-normalised correlation is 1; an
    affine change of brightness (alpha > 0) keeps it, alpha < 0 flips it."""
    t = synth.blob_template(7, 4, seed=23)
    m = synth.ball_mask(7, 3)
    Q = G[7]
    vol = synth.plant_copies((19, 18, 17), t, Q[None], np.array([[8, 9, 9]]))
    pt = np.array([[8, 9, 9]])
    for a, b, expect in ((1.0, 0.0, 1.0), (2.5, 7.0, 1.0), (-2.0, 1.0, -1.0)):
        v = o.sprime_ncc_at(a * vol + b, t, m, G, WG, 4, pt, Q[None])[0]
        assert v == pytest.approx(expect, abs=1e-10)
    rng = np.random.default_rng(24)
    noise = rng.normal(size=(15, 15, 15))
    pts = rng.integers(3, 12, size=(6, 3))
    vals = o.sprime_ncc_at(noise, t, m, G, WG, 4, pts, G[rng.integers(0, 24, 6)])
    assert np.all(np.abs(vals) <= 1.0 + 1e-12)
