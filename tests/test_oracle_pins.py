"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to a closed form, a library routine, brute
force, or an identity the paper states.  They run on the CPU (no GPU marker).
"""

import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import synth
from oracle import ttm_oracle as o

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "paper_printed_values.json")))


def _closed_form_rotation(q):
    """Textbook matrix of v -> q v q* (written out independently of quat_mul)."""
    a, b, c, d = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)],
    ])


def _rand_quats(k, seed):
    q = np.random.default_rng(seed).normal(size=(k, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


# --------------------------------------------------------------------------
# Sec. 3.1: symmetric tensors
# --------------------------------------------------------------------------

def test_component_count_matches_paper_and_binomial():
    assert len(o.multi_indices(4)) == GOLDEN["dim_S4_R4"]["value"]
    assert 4 ** 4 == GOLDEN["dim_T4_R4"]["value"]
    for n in range(1, 9):
        assert len(o.multi_indices(n)) == math.comb(n + 3, n)
        assert len(set(o.multi_indices(n))) == len(o.multi_indices(n))
        # multinomial weights count every full index tuple exactly once
        assert sum(o.multinomial(a) for a in o.multi_indices(n)) == 4 ** n


@pytest.mark.parametrize("n", [2, 4, 6])
def test_tensor_power_inner_product(n):
    """x^(n) . y^(n) = (x . y)^n (Sec. 3.1), through the unique components
    with multinomial weights and through explicit outer products."""
    rng = np.random.default_rng(n)
    x, y = rng.normal(size=4), rng.normal(size=4)
    mu = np.array([o.multinomial(a) for a in o.multi_indices(n)])
    unique = np.sum(mu * o.monomials(x, n) * o.monomials(y, n))
    px, py = np.array(1.0), np.array(1.0)
    for _ in range(n):
        px, py = np.multiply.outer(px, x), np.multiply.outer(py, y)
    assert unique == pytest.approx(np.dot(x, y) ** n, rel=1e-12)
    assert np.sum(px * py) == pytest.approx(np.dot(x, y) ** n, rel=1e-12)
    # expand_full of the unique components of x^(n) is the outer power itself
    assert np.allclose(o.expand_full(o.monomials(x, n), n), px, rtol=1e-13, atol=0)


@pytest.mark.parametrize("n", [2, 4])
def test_expand_symmetric_and_gradient(n):
    rng = np.random.default_rng(10 + n)
    C = rng.normal(size=len(o.multi_indices(n)))
    A = o.expand_full(C, n)
    for perm in itertools.permutations(range(n)):
        assert np.array_equal(A, np.transpose(A, perm))
    x = rng.normal(size=4)
    # grad phi = n A x^{n-1} (Sec. 3.1), checked by central differences
    h = 1e-6
    num = np.array([(o.phi_full(A, x + h * e, n) - o.phi_full(A, x - h * e, n)) / (2 * h)
                    for e in np.eye(4)])
    assert np.allclose(num, n * o.contract(A, x, n - 1), rtol=1e-7, atol=1e-8)
    # Frobenius norm of the full tensor = sqrt(sum mu_alpha C_alpha^2)
    mu = np.array([o.multinomial(a) for a in o.multi_indices(n)])
    assert o.frobenius(A, n) == pytest.approx(np.sqrt(np.sum(mu * C * C)), rel=1e-13)


# --------------------------------------------------------------------------
# Sec. 2: rotations and quaternions
# --------------------------------------------------------------------------

def test_rotation_matrix_closed_form_and_composition():
    Q = _rand_quats(20, 1)
    for q in Q:
        R = o.rotation_matrix(q)
        assert np.allclose(R, _closed_form_rotation(q), atol=1e-14)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-13)
    for p, q in zip(Q[:10], Q[10:]):
        # O_{R1 R2} = O_{R2} o O_{R1}  <=>  R(pq) = R(p) R(q)
        assert np.allclose(o.rotation_matrix(o.quat_mul(p, q)),
                           o.rotation_matrix(p) @ o.rotation_matrix(q), atol=1e-14)
        # <x, y> = Re(y^-1 x) for unit quaternions (end of Sec. 2)
        assert o.quat_mul(o.quat_conj(q), p)[0] == pytest.approx(np.dot(p, q), abs=1e-14)


def test_rotate_template_matches_scipy_and_special_cases():
    t = synth.blob_template(11, 4, seed=7).astype(np.float64)
    for q in _rand_quats(5, 2):
        R = _closed_form_rotation(q)
        c = 5
        z, y, x = np.meshgrid(*(np.arange(11.0) - c,) * 3, indexing="ij")
        v = np.stack([x.ravel(), y.ravel(), z.ravel()])
        p = R.T @ v + c
        ref = ndimage.map_coordinates(t, np.stack([p[2], p[1], p[0]]), order=1,
                                      mode="grid-constant", cval=0.0, prefilter=False)
        assert np.allclose(o.rotate_template(t, q).ravel(), ref, atol=1e-12)
    # identity and a quarter turn about z are exact resamplings
    assert np.array_equal(o.rotate_template(t, np.array([1.0, 0, 0, 0])), t)
    qz = np.array([math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)])
    rot = o.rotate_template(t, qz)
    # t_R(u) = t(R^-1 u): a +90 deg turn about z maps (x, y) -> (y, -x) under R^-1
    expect = np.transpose(t, (0, 2, 1))[:, :, ::-1]
    assert np.allclose(rot, expect, atol=1e-12)


def test_quadrature_moments_match_uniform_s3():
    q = synth.super_fibonacci_quaternions(10000)
    mom = GOLDEN["uniform_S3_moments"]
    for i in range(4):
        assert np.mean(q[:, i] ** 2) == pytest.approx(mom["E_a2"], abs=2e-4)
        assert np.mean(q[:, i] ** 4) == pytest.approx(mom["E_a4"], abs=2e-4)
    assert np.mean(q[:, 0] ** 2 * q[:, 1] ** 2) == pytest.approx(mom["E_a2b2"], abs=2e-4)
    assert abs(np.mean(q[:, 0] ** 3 * q[:, 1])) < 2e-4


# --------------------------------------------------------------------------
# Sec. 3.2: tensor template
# --------------------------------------------------------------------------

def test_tensor_template_unique_matches_full_and_is_symmetric():
    s, n = 7, 4
    t = synth.blob_template(s, 3, seed=3)
    m = synth.ball_mask(s, 3)
    q = _rand_quats(6, 3)
    w = np.full(6, 1 / 6)
    T = o.tensor_template(t, m, q, w, n)
    F = o.tensor_template_full(t, m, q, w, n)
    for a_idx, a in enumerate(o.multi_indices(n)):
        for perm in set(itertools.permutations(a)):
            assert np.allclose(F[perm], T[a_idx], atol=1e-14)


def test_normalised_template_is_zero_mean_unit_norm():
    t = synth.blob_template(9, 3, seed=4)
    m = synth.ball_mask(9, 4)
    u = o.rotated_normalised(t, m, _rand_quats(1, 4)[0])
    assert np.sum(u * m) == pytest.approx(0.0, abs=1e-12)
    assert np.sum(u * u * m) == pytest.approx(1.0, rel=1e-12)
    assert np.all(u[m == 0] == 0)


def test_isotropic_template_tensor_is_moment_times_template():
    """For a rotation-invariant template, T_alpha = (sum_j w_j q_j^alpha) t~."""
    s, n = 9, 4
    c = s // 2
    z, y, x = np.meshgrid(*(np.arange(s) - c,) * 3, indexing="ij")
    t = np.exp(-(x * x + y * y + z * z) / 12.0)
    m = synth.ball_mask(s, 4)
    q = synth.super_fibonacci_quaternions(400)
    w = np.full(400, 1 / 400)
    T = o.tensor_template(t, m, q, w, n)
    tt = o.normalise_under_mask(t, m)
    mom = w @ o.monomials(q, n)
    # trilinear resampling of a Gaussian is not exactly isotropic; the error
    # is small compared with the template itself
    err = np.abs(T - mom[:, None, None, None] * tt[None]).max()
    assert err < 1e-2 * np.abs(tt).max()


# --------------------------------------------------------------------------
# Sec. 2: correlation, local statistics, NCC (Algorithm 1, Theorems 2.1, 2.4)
# --------------------------------------------------------------------------

def test_correlation_direct_fft_and_loops_agree():
    rng = np.random.default_rng(5)
    f = rng.normal(size=(14, 13, 12))
    T = rng.normal(size=(2, 5, 5, 5))
    d = o.correlate_direct(f, T)
    ff = o.correlate_fft(f, T)
    assert np.allclose(d, ff, atol=1e-12)
    # definition (f * g)(x) = sum_z f(z + x) g(z), with z = u - c
    c = 2
    for (xz, xy, xx) in [(2, 2, 2), (5, 7, 3), (11, 10, 9)]:
        acc = 0.0
        for uz, uy, ux in itertools.product(range(5), repeat=3):
            acc += f[xz + uz - c, xy + uy - c, xx + ux - c] * T[1, uz, uy, ux]
        assert d[1, xz, xy, xx] == pytest.approx(acc, abs=1e-12)
    assert np.all(d[:, :2] == 0) and np.all(d[:, :, :, -2:] == 0)


def test_local_stats_direct_fft_and_textbook_variance():
    rng = np.random.default_rng(6)
    f = rng.normal(size=(16, 15, 14)) + 3.0
    m = synth.ball_mask(7, 3)
    S1, S2, w = o.local_stats_direct(f, m)
    S1f, S2f, wf = o.local_stats_fft(f, m)
    assert np.allclose(S1, S1f, atol=1e-10) and np.allclose(S2, S2f, atol=1e-9)
    assert np.allclose(w, wf, rtol=1e-8)
    # w = 1 / ||P_S tau_x f||_S = 1 / (sqrt(m_sum) * population std over the ball)
    ball = m.astype(bool)
    for x, y, z in [(3, 3, 3), (7, 8, 9), (10, 11, 12)]:
        win = f[z - 3:z + 4, y - 3:y + 4, x - 3:x + 4][ball]
        assert w[z, y, x] == pytest.approx(1.0 / (math.sqrt(ball.sum()) * np.std(win)), rel=1e-12)


def test_ncc_is_pearson_and_bounded():
    rng = np.random.default_rng(8)
    f = rng.normal(size=(18, 18, 18))
    t = synth.blob_template(7, 3, seed=8)
    m = synth.ball_mask(7, 3)
    q = _rand_quats(3, 8)
    c = o.classical_ncc(f, t, m, q)
    assert np.abs(c).max() <= 1.0 + 1e-12
    ball = m.astype(bool)
    for j in range(3):
        tr = o.rotate_template(t, q[j])[ball]
        for (x, y, z) in [(3, 3, 3), (9, 10, 11), (14, 14, 14)]:
            win = f[z - 3:z + 4, y - 3:y + 4, x - 3:x + 4][ball]
            assert c[j, z, y, x] == pytest.approx(np.corrcoef(win, tr)[0, 1], abs=1e-12)


def test_ncc_equals_one_at_isolated_planted_copy():
    """Theorem 2.4 (b*): a noise-free isolated copy rotated by a rotation of
    the set gives NCC = 1 there.  The copy is planted by the input generator's
    own resampling code."""
    t = synth.blob_template(11, 4, seed=9)
    m = synth.ball_mask(11, 5)
    q = synth.super_fibonacci_quaternions(50)[17]
    vol = synth.plant_copies((30, 31, 32), t, q[None], np.array([[15, 14, 16]]))
    c = o.classical_ncc(vol, t, m, q[None])
    assert c[0, 16, 14, 15] == pytest.approx(1.0, abs=1e-10)
    assert c[0].max() == pytest.approx(1.0, abs=1e-10)


def test_ncc_affine_invariance():
    """Theorem 2.4, last claim, read for alpha*delta > 0; a negative factor flips the sign."""
    rng = np.random.default_rng(11)
    f = rng.normal(size=(16, 16, 16))
    t = synth.blob_template(7, 3, seed=11).astype(np.float64)
    m = synth.ball_mask(7, 3)
    q = _rand_quats(2, 11)
    c0 = o.classical_ncc(f, t, m, q)
    assert np.allclose(o.classical_ncc(2.5 * f + 7.0, 0.3 * t - 1.0, m, q), c0, atol=1e-10)
    assert np.allclose(o.classical_ncc(-2.0 * f + 1.0, t, m, q), -c0, atol=1e-10)


def test_degenerate_variance_gives_zero_weight():
    f = np.full((12, 12, 12), 3.25)
    _, _, w = o.local_stats_fft(f, synth.ball_mask(5, 2))
    assert np.all(w == 0)
    f[:, :, 6:] += np.random.default_rng(1).normal(size=(12, 12, 6))
    _, _, w = o.local_stats_direct(f, synth.ball_mask(5, 2))
    assert np.all(w[:, :, 2:4] == 0)          # windows entirely in the flat half
    assert np.all(w[2:10, 2:10, 6:10] > 0)


# --------------------------------------------------------------------------
# Sec. 3.2 / 3.3: TTM components, phi and the score
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_problem():
    wl = synth.make_workload((22, 21, 20), 9, 4, 2, 1.0, 4, 60, radius=4, seeds=(3, 4, 5))
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature, wl.weights, 4)
    w, C = o.ttm_components(wl.volume, T, wl.mask)
    cj = o.classical_ncc(wl.volume, wl.template, wl.mask, wl.quadrature)
    return wl, T, w, C, cj


def test_components_equal_weighted_sum_of_classical_ncc(small_problem):
    """C_alpha(x) = sum_j w_j q_j^alpha c(x, R_j): linearity of Sec. 3.2."""
    wl, T, w, C, cj = small_problem
    mono = o.monomials(wl.quadrature.astype(np.float64), 4)          # (J, K)
    expect = np.einsum("j,jk,jzyx->kzyx", wl.weights, mono, cj)
    assert np.allclose(C, expect, atol=1e-12)


def test_phi_equals_kernel_weighted_ncc(small_problem):
    """phi(Q) = sum_j w_j (Q . q_j)^n c(x, R_j): the first step of the proof
    of Theorem 3.1."""
    wl, T, w, C, cj = small_problem
    qj = wl.quadrature.astype(np.float64)
    Q = _rand_quats(5, 12)
    for (x, y, z) in [(5, 6, 7), (10, 10, 10), (14, 13, 12)]:
        Cx = C[:, z, y, x]
        for q in Q:
            direct = np.sum(wl.weights * (qj @ q) ** 4 * cj[:, z, y, x])
            assert o.phi_unique(Cx[None], q[None], 4)[0] == pytest.approx(direct, abs=1e-13)


def test_score_bounds(small_problem):
    """score <= 1 (|c| <= 1, probability weights); |phi| <= score (Cauchy-
    Schwarz); max |phi| >= score / 2^(n-1) (Sec. 3.4)."""
    wl, T, w, C, cj = small_problem
    score = o.frobenius_score(C, 4)
    assert score.max() <= 1.0 + 1e-12
    Cs = C.reshape(C.shape[0], -1).T[score.ravel() > 0][:40]
    sc = o.frobenius_score(Cs.T, 4)
    lam, q = o.dominant_z_eigenpair(Cs, 4)
    lam_neg, _ = o.dominant_z_eigenpair(-Cs, 4)
    base = GOLDEN["spectral_frobenius_bound_base"]["value"]
    assert np.all(lam <= sc + 1e-12)
    assert np.all(np.maximum(lam, lam_neg) >= sc / base ** 3 - 1e-12)


# --------------------------------------------------------------------------
# Sec. 3.3 / 3.4: dominant Z-eigenpair
# --------------------------------------------------------------------------

def test_dominant_eigenpair_order2_is_symmetric_eigenproblem():
    """For n = 2, phi(Q) = Q^T A Q: lambda* is the largest eigenvalue."""
    rng = np.random.default_rng(13)
    C = rng.normal(size=(30, 10))
    lam, q = o.dominant_z_eigenpair(C, 2)
    for k in range(30):
        A = o.expand_full(C[k], 2)
        ev, vec = np.linalg.eigh(A)
        assert lam[k] == pytest.approx(ev[-1], abs=1e-11)
        if ev[-1] - ev[-2] > 1e-2:
            assert abs(np.dot(q[k], vec[:, -1])) == pytest.approx(1.0, abs=1e-8)


@pytest.mark.parametrize("n", [4, 6])
def test_dominant_eigenpair_rank_one(n):
    """C = c q0^(n) with c > 0 has lambda* = c at q0 (Theorem 3.1 with one rotation)."""
    for k, q0 in enumerate(_rand_quats(6, 14 + n)):
        c = 0.3 + 0.1 * k
        lam, q = o.dominant_z_eigenpair(c * o.monomials(q0, n)[None], n)
        assert lam[0] == pytest.approx(c, rel=1e-10)
        assert abs(np.dot(q[0], q0)) == pytest.approx(1.0, abs=1e-7)
        assert q[0][0] >= 0


def test_dominant_eigenpair_beats_brute_force(small_problem):
    wl, T, w, C, cj = small_problem
    pts = np.random.default_rng(15).integers(4, 16, size=(24, 3))
    Cs = C[:, pts[:, 2], pts[:, 1], pts[:, 0]].T
    lam, q = o.dominant_z_eigenpair(Cs, 4)
    g = np.random.default_rng(16).normal(size=(300000, 4))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    A = o.expand_full(Cs, 4).reshape(len(Cs), -1)
    gn = np.einsum("gi,gj,gk,gl->gijkl", g, g, g, g).reshape(len(g), -1)
    bf = (A @ gn.T).max(axis=1)
    assert np.all(lam >= bf - 1e-12)
    assert np.all(lam - bf <= 1e-4)
    assert np.allclose(o.phi_unique(Cs, q, 4), lam, atol=1e-13)


def test_ss_hopm_is_monotone():
    rng = np.random.default_rng(17)
    C = rng.normal(size=(8, 35))
    A = o.expand_full(C, 4)
    x = _rand_quats(8, 18)
    shift = 3 * o.frobenius(A, 4)
    prev = o.contract(A, x, 4)
    for _ in range(50):
        lam, x, _ = o.ss_hopm(A, x, 4, shift, max_iter=1)
        assert np.all(lam >= prev - 1e-14)
        prev = lam


def test_rotation_recovered_at_noise_free_planted_copies():
    """Theorem 3.1: at a match the maximiser of phi is the planted rotation
    (exact in the continuum; here within quadrature and resampling error)."""
    wl = synth.make_workload((40, 40, 40), 15, 5, 3, 1.0, 4, 3000, seeds=(1, 2, 3),
                             noise=False)
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature, wl.weights, 4)
    p = wl.positions
    w, Cs = o.components_at(wl.volume, T, wl.mask, p)
    lam, q = o.dominant_z_eigenpair(Cs, 4)
    ang = o.rotation_angle_deg(q, wl.planted_quats.astype(np.float64))
    assert np.all(ang < 6.0), ang


# --------------------------------------------------------------------------
# Sec. 3.4: peaks
# --------------------------------------------------------------------------

def test_peaks_match_brute_force_with_ties():
    rng = np.random.default_rng(19)
    score = np.round(rng.random((9, 10, 11)), 1)     # many ties
    got = o.extract_peaks(score, 0.3, 2, 1000)
    Z, Y, X = score.shape
    expect = []
    for z, y, x in itertools.product(range(Z), range(Y), range(X)):
        v = score[z, y, x]
        if v <= 0.3:
            continue
        lin = (z * Y + y) * X + x
        ok = True
        for dz, dy, dx in itertools.product(range(-2, 3), repeat=3):
            zz, yy, xx = z + dz, y + dy, x + dx
            if (dz, dy, dx) == (0, 0, 0) or not (0 <= zz < Z and 0 <= yy < Y and 0 <= xx < X):
                continue
            u = score[zz, yy, xx]
            if u > v or (u == v and (zz * Y + yy) * X + xx < lin):
                ok = False
        if ok:
            expect.append((-v, lin))
    expect.sort()
    assert list(got) == [lin for _, lin in expect]


def _weighted_corr(a, b, wts):
    """Weighted Pearson correlation from numpy's weighted covariance."""
    cv = np.cov(np.stack([a, b]), aweights=wts, bias=True)
    return cv[0, 1] / math.sqrt(cv[0, 0] * cv[1, 1])


def test_soft_mask_ncc_is_weighted_pearson():
    """With a soft mask m (weights in [0, 1]) the NCC of Sec. 2's S-inner
    product is the m-weighted Pearson correlation of the window and the
    rotated template (numpy's weighted covariance as the reference), and it
    stays in [-1, 1]."""
    rng = np.random.default_rng(12)
    f = rng.normal(size=(20, 20, 20))
    t = synth.blob_template(9, 3, seed=12)
    m = synth.soft_ball_mask(9, 4, 1.5)
    assert np.any((m > 0) & (m < 1))
    q = _rand_quats(2, 12)
    c = o.classical_ncc(f, t, m, q)
    assert np.abs(c).max() <= 1.0 + 1e-12
    wts = m.ravel().astype(np.float64)
    sel = wts > 0
    for j in range(2):
        tr = o.rotate_template(t, q[j]).ravel()
        for (x, y, z) in [(4, 4, 4), (9, 11, 12), (15, 15, 15)]:
            win = f[z - 4:z + 5, y - 4:y + 5, x - 4:x + 5].ravel()
            ref = _weighted_corr(win[sel], tr[sel], wts[sel])
            assert c[j, z, y, x] == pytest.approx(ref, abs=1e-12)


def test_lowpass_is_scipy_gaussian_filter_with_unit_gain():
    """The optional prefilter h of Sec. 2: the oracle's separable Gaussian
    equals scipy.ndimage.gaussian_filter (zero outside, truncated at 4 sigma);
    h * 1 = 1 away from the borders (unit DC gain, Sec. 2) and h is even."""
    from scipy import ndimage
    rng = np.random.default_rng(21)
    x = rng.normal(size=(14, 17, 19))
    for sigma in (0.8, 1.0, 2.3):
        ref = ndimage.gaussian_filter(x, sigma, mode="constant", cval=0.0, truncate=4.0)
        assert np.abs(o.lowpass(x, sigma) - ref).max() <= 1e-12
        k = o.gaussian_kernel(sigma)
        assert k.sum() == pytest.approx(1.0, abs=1e-15) and np.allclose(k, k[::-1])
    ones = o.lowpass(np.ones((30, 30, 30)), 1.5)
    r = int(4 * 1.5 + 0.5)
    assert np.abs(ones[r:-r, r:-r, r:-r] - 1.0).max() <= 1e-12


# --------------------------------------------------------------------------
# Sec. 3.2: the per-point components C_alpha(x) = w(x) <tau_x f, T_alpha>,
# which the full-size and sampled GPU tests use as their only checker
# --------------------------------------------------------------------------

@pytest.mark.parametrize("s,shape", [(7, (17, 13, 19)), (8, (16, 21, 14)), (9, (18, 18, 23))])
def test_components_at_matches_whole_interior_and_explicit_loops(s, shape):
    """components_at (one box per point) equals ttm_components (whole-volume
    direct correlation) and local_stats_direct at the same voxels, for odd and
    even s on ragged volumes; at the first and last interior voxel it equals
    the definition written as loops: C_alpha(x) = w(x) sum_u f(x + u - c)
    T_alpha(u) with w = 1 / (sqrt(m_sum) * population std over the ball)."""
    rng = np.random.default_rng(40 + s)
    f = rng.normal(size=shape) + 2.0
    r = synth.default_mask_radius(s)
    m = synth.ball_mask(s, r).astype(np.float64)
    T = rng.normal(size=(3, s, s, s))
    c = s // 2
    Z, Y, X = shape
    lo = (c, c, c)                                        # (x, y, z) of the first interior voxel
    hi = (X - s + c, Y - s + c, Z - s + c)                # and of the last one
    inner = rng.integers(lo, np.array(hi) + 1, size=(6, 3))
    pts = np.array([lo, hi, (lo[0], hi[1], lo[2]), (hi[0], lo[1], hi[2])] + inner.tolist())
    w_p, C_p = o.components_at(f, T, m, pts)
    w_all, C_all = o.ttm_components(f, T, m, use_fft=False)
    _, _, w_ls = o.local_stats_direct(f, m)
    for i, (x, y, z) in enumerate(pts):
        assert w_p[i] == pytest.approx(w_all[z, y, x], rel=1e-12)
        assert w_p[i] == pytest.approx(w_ls[z, y, x], rel=1e-12)
        assert np.allclose(C_p[i], C_all[:, z, y, x], rtol=1e-12, atol=1e-12)
    # the patch is the box whose voxel u sits at x + u - c
    P = o.patches_at(f, pts[:2], s)
    for i, (x, y, z) in enumerate(pts[:2]):
        assert P[i][0] == f[z - c, y - c, x - c]
        assert P[i][-1] == f[z - c + s - 1, y - c + s - 1, x - c + s - 1]
        ball = m.astype(bool)
        win = f[z - c:z - c + s, y - c:y - c + s, x - c:x - c + s]
        w_ref = 1.0 / (math.sqrt(ball.sum()) * np.std(win[ball]))
        assert w_p[i] == pytest.approx(w_ref, rel=1e-12)
        for k in range(T.shape[0]):
            acc = 0.0
            for uz, uy, ux in itertools.product(range(s), repeat=3):
                acc += f[z + uz - c, y + uy - c, x + ux - c] * T[k, uz, uy, ux]
            assert C_p[i, k] == pytest.approx(w_ref * acc, rel=1e-11, abs=1e-12)


def test_components_at_variance_floor_uses_whole_volume_variance():
    """The default var_f of components_at is the whole volume's variance (the
    degenerate-variance rule of the interior maps): a window on a flat patch
    gets w = 0, exactly as in ttm_components."""
    rng = np.random.default_rng(47)
    f = rng.normal(size=(16, 16, 20))
    f[:, :, :9] = 1.5                                     # flat slab in x < 9
    m = synth.ball_mask(5, 2)
    T = rng.normal(size=(2, 5, 5, 5))
    pts = np.array([[3, 7, 7], [14, 8, 9]])
    w_p, _ = o.components_at(f, T, m, pts)
    w_all, _ = o.ttm_components(f, T, m, use_fft=False)
    assert w_p[0] == 0.0 and w_all[7, 7, 3] == 0.0
    assert w_p[1] == pytest.approx(w_all[9, 8, 14], rel=1e-12) and w_p[1] > 0
    # an explicit var_f overrides it (the sampled tests pass the volume's own)
    w_big, _ = o.components_at(f, T, m, pts, var_f=1e9)
    assert np.all(w_big == 0.0)


def test_rotation_angle_closed_forms():
    """rotation_angle_deg against axis-angle closed forms: the quaternion
    (cos(theta/2), sin(theta/2) u) is a turn by theta about u; q and -q are
    the same rotation; and the angle equals acos((tr(R1 R2^T) - 1) / 2)
    computed from the textbook rotation matrices."""
    ident = np.array([1.0, 0.0, 0.0, 0.0])
    rng = np.random.default_rng(48)
    for theta in (0.0, 0.5, 1.0, 13.0, 90.0, 123.4, 179.0, 180.0):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        h = math.radians(theta) / 2
        q = np.concatenate([[math.cos(h)], math.sin(h) * u])
        assert o.rotation_angle_deg(q, ident) == pytest.approx(theta, abs=1e-6)
        assert o.rotation_angle_deg(ident, q) == pytest.approx(theta, abs=1e-6)
        assert o.rotation_angle_deg(-q, ident) == pytest.approx(theta, abs=1e-6)
        assert o.rotation_angle_deg(q, -q) == pytest.approx(0.0, abs=1e-6)
    # quarter turn about z
    qz = np.array([math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)])
    assert o.rotation_angle_deg(qz, ident) == pytest.approx(90.0, abs=1e-9)
    P, Q = _rand_quats(50, 49), _rand_quats(50, 50)
    got = o.rotation_angle_deg(P, Q)
    for i in range(50):
        R = _closed_form_rotation(P[i]) @ _closed_form_rotation(Q[i]).T
        ref = math.degrees(math.acos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)))
        assert got[i] == pytest.approx(ref, abs=1e-5)
