"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: |dC|, |dscore|, |dlambda| <= 1e-4 (the FP32 gate), w to 1e-5
relative, template components to 2e-5 of their largest magnitude; index work
(peaks) bit-exact.  Where several results are correct (two rotations with the
same phi to within 1e-5) the test checks the rotation is a valid maximiser.
"""

import numpy as np
import pytest

import synth
from oracle import ttm_oracle as o

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def ttm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2311_07561_gb300 as ttm
    import os
    if not os.path.exists(ttm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ttm.load_library()
    return ttm


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


PATHS = ["direct", "fft"]


def _opts(ttm, path):
    o_ = ttm.PlanOpts()
    o_.path = {"direct": ttm.TTM_PATH_DIRECT, "fft": ttm.TTM_PATH_FFT}[path]
    return o_


def _run(ttm, wl, comp, desc, opts=None, want_comp=True):
    import torch
    X = wl.volume.shape[2]; Y = wl.volume.shape[1]; Z = wl.volume.shape[0]
    m = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)], opts=opts)
    vol = _cuda(wl.volume)
    comps = [torch.empty((desc.K, Z, Y, X), dtype=torch.float32, device="cuda")] if want_comp else None
    m.run([vol], components_out=comps)
    torch.cuda.synchronize()
    assert ttm.ttm_plan_device_status(m.plan, m.ws) == 0
    out = dict(w=m.w[0].cpu().numpy(), score=m.score[0].cpu().numpy(),
               quat=m.quat[0].cpu().numpy(), lam=m.lam[0].cpu().numpy(),
               comp=comps[0].cpu().numpy() if want_comp else None, matcher=m)
    return out


@pytest.fixture(scope="module")
def c1_oracle(ttm):
    """Config-1 shape: 64^3, 15^3 template (5 blobs), r = 7, 4 copies, SNR 1, n = 4."""
    wl = synth.config_workload("c1", n_rot=1000)
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 4)
    comp, desc = ttm.build_template(wl.template, wl.mask, 4, wl.quadrature)
    w_o, C_o = o.ttm_components(wl.volume, T, wl.mask)
    return dict(wl=wl, T=T, comp=comp, desc=desc, w_o=w_o, C_o=C_o)


@pytest.fixture(scope="module", params=PATHS)
def c1(ttm, c1_oracle, request):
    d = dict(c1_oracle)
    d["res"] = _run(ttm, d["wl"], d["comp"], d["desc"], opts=_opts(ttm, request.param))
    d["path"] = request.param
    assert ttm.ttm_plan_problem_path(d["res"]["matcher"].plan, 0) == _opts(ttm, request.param).path
    return d


def test_tensor_template_matches_oracle(c1):
    g = c1["comp"].cpu().numpy()
    T = c1["T"]
    assert g.shape == T.shape
    err = np.abs(g - T).max()
    assert err <= 2e-5 * np.abs(T).max(), err
    assert c1["desc"].K == 35 and c1["desc"].s == 15 and c1["desc"].centre == 7
    assert c1["desc"].mask_sum == pytest.approx(c1["wl"].mask.sum())


@pytest.mark.parametrize("n,s,r,nrot", [(2, 11, 5, 400), (6, 9, 4, 300)])
def test_tensor_template_other_orders(ttm, n, s, r, nrot):
    t = synth.blob_template(s, 4, seed=n)
    m = synth.ball_mask(s, r)
    q = synth.super_fibonacci_quaternions(nrot).astype(np.float32)
    w = np.full(nrot, 1.0 / nrot)
    comp, desc = ttm.build_template(t, m, n, q)
    T = o.tensor_template(t, m, q.astype(np.float64), w, n)
    err = np.abs(comp.cpu().numpy() - T).max()
    assert err <= 2e-5 * np.abs(T).max(), err
    assert desc.K == len(o.multi_indices(n))


def test_local_stats_match_oracle(c1):
    w = c1["res"]["w"]
    w_o = c1["w_o"]
    assert np.array_equal(w > 0, w_o > 0)
    nz = w_o > 0
    rel = np.abs(w[nz] - w_o[nz]) / w_o[nz]
    assert rel.max() <= 1e-5, rel.max()


def test_components_and_score_match_oracle(c1):
    C = c1["res"]["comp"]
    C_o = c1["C_o"]
    err = np.abs(C - C_o).max()
    assert err <= TOL, err
    score_o = o.frobenius_score(C_o, 4)
    serr = np.abs(c1["res"]["score"] - score_o).max()
    assert serr <= TOL, serr
    # outside the interior everything is zero / identity
    keep = o.interior_mask(c1["wl"].volume.shape, 15)
    assert np.all(c1["res"]["score"][~keep] == 0)
    assert np.all(c1["res"]["quat"][~keep] == np.array([1, 0, 0, 0], dtype=np.float32))
    assert np.all(c1["res"]["lam"][~keep] == 0)


def _rotation_check(C_o_pts, lam, q, n, planted=(), eig_o=None):
    lam_o, q_o = o.dominant_z_eigenpair(C_o_pts, n) if eig_o is None else eig_o
    dl = np.abs(lam - lam_o)
    assert dl.max() <= TOL, (dl.max(), np.argmax(dl))
    # the reported rotation attains the reported value and the maximum
    phi_at_gpu = o.phi_unique(C_o_pts, q.astype(np.float64), n)
    assert np.all(phi_at_gpu >= lam_o - TOL), (lam_o - phi_at_gpu).max()
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-5)
    assert np.all(q[:, 0] >= 0)
    for i in planted:
        ang = o.rotation_angle_deg(q[i], q_o[i])
        assert ang <= 1.0 or phi_at_gpu[i] >= lam_o[i] - 1e-5, (i, ang)
    return lam_o, q_o


def test_rotation_matches_oracle(c1):
    wl = c1["wl"]
    rng = np.random.default_rng(21)
    lo, hi = 7, 64 - 15 + 7
    pts = np.concatenate([wl.positions, rng.integers(lo, hi + 1, size=(300, 3))])
    C_o_pts = c1["C_o"][:, pts[:, 2], pts[:, 1], pts[:, 0]].T
    lam = c1["res"]["lam"][pts[:, 2], pts[:, 1], pts[:, 0]]
    q = c1["res"]["quat"][pts[:, 2], pts[:, 1], pts[:, 0]]
    _rotation_check(C_o_pts, lam, q, 4, planted=range(len(wl.positions)))


def test_peaks_kernel_is_exact_on_given_scores(ttm, c1):
    """Peak extraction on a score map given as input, with many exact ties."""
    import torch
    m = c1["res"]["matcher"]
    rng = np.random.default_rng(3)
    score = np.round(rng.random((64, 64, 64)), 2).astype(np.float32)
    quat = np.zeros((64, 64, 64, 4), dtype=np.float32)
    quat[..., 0] = 1.0
    quat[..., 1] = np.arange(64 ** 3, dtype=np.float32).reshape(64, 64, 64)
    lam = (score * 0.5).astype(np.float32)
    for radius in (0, 1, 3):
        got = ttm.ttm_extract_peaks(m.plan, 0, _cuda(score), _cuda(quat), _cuda(lam), 0.5, radius,
                                    100000, m.ws)
        expect = o.extract_peaks(score.astype(np.float64), 0.5, radius, 100000)
        lin = (got["z"].astype(np.int64) * 64 + got["y"]) * 64 + got["x"]
        assert np.array_equal(lin, expect), radius
        assert np.array_equal(got["score"], score.ravel()[expect])
        assert np.array_equal(got["q"][:, 1], quat[..., 1].ravel()[expect])
        assert np.array_equal(got["lambda"], lam.ravel()[expect])
    few = ttm.ttm_extract_peaks(m.plan, 0, _cuda(score), _cuda(quat), None, 0.5, 3, 7, m.ws)
    assert len(few) == 7 and np.all(few["lambda"] == 0)


def test_peaks_on_planted_volume(ttm, c1):
    m = c1["res"]["matcher"]
    got = m.peaks(0, 0.0, 7, 4)
    score_o = o.frobenius_score(c1["C_o"], 4)
    expect = o.extract_peaks(score_o, 0.0, 7, 4)
    lin = (got["z"].astype(np.int64) * 64 + got["y"]) * 64 + got["x"]
    assert np.array_equal(lin, expect)


@pytest.mark.parametrize("path", PATHS)
def test_ragged_volume_and_order_two(ttm, path):
    wl = synth.make_workload((39, 45, 70), 11, 4, 2, 1.0, 2, 300, radius=5, seeds=(7, 8, 9))
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 2)
    comp, desc = ttm.build_template(wl.template, wl.mask, 2, wl.quadrature)
    res = _run(ttm, wl, comp, desc, opts=_opts(ttm, path))
    w_o, C_o = o.ttm_components(wl.volume, T, wl.mask)
    assert np.abs(res["comp"] - C_o).max() <= TOL
    nz = w_o > 0
    assert np.array_equal(res["w"] > 0, nz)
    assert (np.abs(res["w"][nz] - w_o[nz]) / w_o[nz]).max() <= 1e-5
    pts = np.argwhere(nz)[::97][:200][:, ::-1]
    _rotation_check(C_o[:, pts[:, 2], pts[:, 1], pts[:, 0]].T,
                    res["lam"][pts[:, 2], pts[:, 1], pts[:, 0]],
                    res["quat"][pts[:, 2], pts[:, 1], pts[:, 0]], 2)


@pytest.mark.parametrize("shape_zyx,boxes", [
    ((36, 150, 230), (240, 160, 48)),     # radix 16 x 3 x 5, 16 x 2 x 5, 16 x 3
    ((20, 140, 280), (288, 144, 32)),     # radix 16 x 2 x 3 x 3, 16 x 3 x 3, 16 x 2
])
def test_fft_smooth_lengths(ttm, shape_zyx, boxes):
    """FFT boxes of 2^p 3^a 5^b lengths (radix-3 and radix-5 stages): the
    plan pads each axis to the smallest such length, and the interior
    components, w and score agree with the oracle's FP64 FFT."""
    wl = synth.make_workload(shape_zyx, 9, 3, 3, 1.0, 4, 200, radius=4, seeds=(11, 12, 13))
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 4)
    comp, desc = ttm.build_template(wl.template, wl.mask, 4, wl.quadrature)
    res = _run(ttm, wl, comp, desc, opts=_opts(ttm, "fft"))
    assert tuple(ttm.ttm_plan_problem_fft_box(res["matcher"].plan, 0)) == boxes
    w_o, C_o = o.ttm_components(wl.volume, T, wl.mask)
    assert np.abs(res["comp"] - C_o).max() <= TOL
    nz = w_o > 0
    assert np.array_equal(res["w"] > 0, nz)
    assert (np.abs(res["w"][nz] - w_o[nz]) / w_o[nz]).max() <= 1e-5
    assert np.abs(res["score"] - o.frobenius_score(C_o, 4)).max() <= TOL
    res["matcher"].close()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("shape_zyx,boxes", [
    ((20, 24, 900), (960, 32, 32)),       # x lines of 960 = 32 x 30
    ((20, 900, 24), (32, 960, 32)),       # y lines of 960
    ((470, 24, 20), (32, 32, 480)),       # z lines of 480 = 16 x 30
])
def test_two_level_lengths(ttm, shape_zyx, boxes, precision):
    """The long lines of the 928 x 928 x 464 configuration (960 and 480)
    take the two-level passes (register DFTs of 32 or 16 and 30 points, one
    shared-memory exchange); components, w and score agree with the
    oracle's FP64 FFT on every axis, with FP32 and with bf16 storage."""
    wl = synth.make_workload(shape_zyx, 9, 3, 3, 1.0, 4, 200, radius=4, seeds=(31, 32, 33))
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 4)
    comp, desc = ttm.build_template(wl.template, wl.mask, 4, wl.quadrature)
    opts = _opts(ttm, "fft")
    if precision == "mixed":
        opts.precision = ttm.TTM_PREC_MIXED
    res = _run(ttm, wl, comp, desc, opts=opts)
    assert tuple(ttm.ttm_plan_problem_fft_box(res["matcher"].plan, 0)) == boxes
    tol = TOL if precision == "fp32" else 5e-3
    w_o, C_o = o.ttm_components(wl.volume, T, wl.mask)
    keep = o.interior_mask(wl.volume.shape, 9)
    assert np.abs(res["comp"][:, keep] - C_o[:, keep]).max() <= tol
    nz = w_o > 0
    assert np.array_equal(res["w"] > 0, nz)
    assert (np.abs(res["w"][nz] - w_o[nz]) / w_o[nz]).max() <= 1e-5
    assert np.abs(res["score"] - o.frobenius_score(C_o, 4)).max() <= tol
    res["matcher"].close()


@pytest.mark.parametrize("path", PATHS)
def test_order_six(ttm, path):
    wl = synth.make_workload((30, 28, 26), 9, 3, 1, 1.0, 6, 300, radius=4, seeds=(2, 3, 4))
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 6)
    comp, desc = ttm.build_template(wl.template, wl.mask, 6, wl.quadrature)
    res = _run(ttm, wl, comp, desc, opts=_opts(ttm, path))
    w_o, C_o = o.ttm_components(wl.volume, T, wl.mask)
    assert np.abs(res["comp"] - C_o).max() <= TOL
    assert np.abs(res["score"] - o.frobenius_score(C_o, 6)).max() <= TOL
    pts = np.argwhere(w_o > 0)[::53][:120][:, ::-1]
    _rotation_check(C_o[:, pts[:, 2], pts[:, 1], pts[:, 0]].T,
                    res["lam"][pts[:, 2], pts[:, 1], pts[:, 0]],
                    res["quat"][pts[:, 2], pts[:, 1], pts[:, 0]], 6)


def test_order_six_mixed_precision(ttm):
    """Order 6 with bf16 storage: the plan's default search grid is then 1024
    points (64 regions); components, score and lambda stay within the bf16
    tolerance of the oracle and q is a maximiser of the oracle's phi."""
    wl = synth.make_workload((40, 38, 36), 11, 4, 2, 1.0, 6, 300, radius=5, seeds=(12, 13, 14))
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 6)
    comp, desc = ttm.build_template(wl.template, wl.mask, 6, wl.quadrature)
    opts = _opts(ttm, "fft")
    opts.precision = ttm.TTM_PREC_MIXED
    res = _run(ttm, wl, comp, desc, opts=opts)
    w_o, C_o = o.ttm_components(wl.volume, T, wl.mask)
    tol = 5e-3
    assert np.abs(res["comp"] - C_o).max() <= tol
    assert np.abs(res["score"] - o.frobenius_score(C_o, 6)).max() <= tol
    pts = np.concatenate([wl.positions, np.argwhere(w_o > 0)[::41][:160][:, ::-1]])
    C_pts = C_o[:, pts[:, 2], pts[:, 1], pts[:, 0]].T
    lam_o, _ = o.dominant_z_eigenpair(C_pts, 6)
    lam = res["lam"][pts[:, 2], pts[:, 1], pts[:, 0]]
    q = res["quat"][pts[:, 2], pts[:, 1], pts[:, 0]]
    assert np.abs(lam - lam_o).max() <= tol
    assert np.all(o.phi_unique(C_pts, q.astype(np.float64), 6) >= lam_o - tol)


@pytest.fixture(scope="module")
def order8_oracle():
    """n = 8 (K = 165), the largest supported order: the oracle's maps, and
    its rotation at five sampled voxels (SS-HOPM converges slowly at this
    order, ~7 s per voxel, so both paths share them)."""
    wl = synth.make_workload((26, 24, 22), 7, 3, 1, 1.0, 8, 400, radius=3, seeds=(5, 6, 7))
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 8)
    w_o, C_o = o.ttm_components(wl.volume, T, wl.mask)
    pts = np.argwhere(w_o > 0)[::1151][:5][:, ::-1]
    C_pts = C_o[:, pts[:, 2], pts[:, 1], pts[:, 0]].T
    return dict(wl=wl, C_o=C_o, pts=pts, C_pts=C_pts, eig=o.dominant_z_eigenpair(C_pts, 8))


@pytest.mark.parametrize("path", PATHS)
def test_order_eight(ttm, order8_oracle, path):
    d = order8_oracle
    wl, C_o, pts = d["wl"], d["C_o"], d["pts"]
    comp, desc = ttm.build_template(wl.template, wl.mask, 8, wl.quadrature)
    assert desc.K == 165
    res = _run(ttm, wl, comp, desc, opts=_opts(ttm, path))
    assert np.abs(res["comp"] - C_o).max() <= TOL
    assert np.abs(res["score"] - o.frobenius_score(C_o, 8)).max() <= TOL
    _rotation_check(d["C_pts"], res["lam"][pts[:, 2], pts[:, 1], pts[:, 0]],
                    res["quat"][pts[:, 2], pts[:, 1], pts[:, 0]], 8, eig_o=d["eig"])
    res["matcher"].close()


@pytest.mark.parametrize("path", PATHS)
def test_degenerate_inputs(ttm, path):
    """A volume exactly one box wide (a single interior voxel) and a constant
    volume (zero variance everywhere: w = 0, score 0, identity rotation)."""
    s = 9
    t = synth.blob_template(s, 3, seed=1)
    m = synth.ball_mask(s, 4)
    q = synth.super_fibonacci_quaternions(200).astype(np.float32)
    comp, desc = ttm.build_template(t, m, 4, q)
    T = o.tensor_template(t, m, q.astype(np.float64), np.full(200, 1 / 200), 4)
    rng = np.random.default_rng(0)
    one = synth.Workload("one", rng.normal(size=(s, s, s)).astype(np.float32), t, m, 4, 4, q,
                         np.full(200, 1 / 200), np.zeros((0, 3), int), np.zeros((0, 4)), 0.0, 0.0)
    res = _run(ttm, one, comp, desc, opts=_opts(ttm, path))
    w_o, C_o = o.ttm_components(one.volume, T, m)
    assert np.count_nonzero(res["score"]) == 1
    assert np.abs(res["comp"] - C_o).max() <= TOL
    const = synth.Workload("const", np.full((20, 21, 22), 2.5, np.float32), t, m, 4, 4, q,
                           np.full(200, 1 / 200), np.zeros((0, 3), int), np.zeros((0, 4)), 0.0, 0.0)
    res = _run(ttm, const, comp, desc, opts=_opts(ttm, path))
    assert np.all(res["w"] == 0) and np.all(res["score"] == 0) and np.all(res["lam"] == 0)
    assert np.all(res["quat"] == np.array([1, 0, 0, 0], np.float32))


@pytest.mark.parametrize("path", PATHS)
def test_batched_plan_matches_single_problems(ttm, path):
    import torch
    wa = synth.make_workload((40, 36, 34), 11, 4, 2, 1.0, 4, 200, radius=5, seeds=(1, 2, 3))
    wb = synth.make_workload((33, 47, 29), 9, 3, 1, 1.0, 4, 200, radius=4, seeds=(4, 5, 6))
    ca, da = ttm.build_template(wa.template, wa.mask, 4, wa.quadrature)
    cb, db = ttm.build_template(wb.template, wb.mask, 4, wb.quadrature)
    vols = [wa.volume, wb.volume]
    dims_a = wa.volume.shape[::-1]
    dims_b = wb.volume.shape[::-1]
    probs = [(dims_a, 0), (dims_a, 1), (dims_b, 0), (dims_b, 1)]
    mb = ttm.Matcher([(ca, da, wa.mask), (cb, db, wb.mask)], probs, opts=_opts(ttm, path))
    dv = [_cuda(vols[0]), _cuda(vols[0]), _cuda(vols[1]), _cuda(vols[1])]
    mb.run(dv)
    for p, ((X, Y, Z), k) in enumerate(probs):
        single = ttm.Matcher([((ca, da, wa.mask), (cb, db, wb.mask))[k]], [((X, Y, Z), 0)],
                             opts=_opts(ttm, path))
        single.run([dv[p]])
        torch.cuda.synchronize()
        assert torch.equal(single.score[0], mb.score[p])
        assert torch.equal(single.quat[0], mb.quat[p])
        assert torch.equal(single.w[0], mb.w[p])
        single.close()
    mb.close()


def test_gpu_argument_errors(ttm):
    import torch
    s = 9
    t = synth.blob_template(s, 3, seed=1)
    m = synth.ball_mask(s, 4)
    q = synth.super_fibonacci_quaternions(50).astype(np.float32)
    comp, desc = ttm.build_template(t, m, 4, q)
    # a soft mask runs on the FFT path only; values outside [0, 1] are rejected
    soft = m * 0.5
    with pytest.raises(ttm.TTMError) as e:
        ttm.Matcher([(comp, desc, soft)], [((20, 20, 20), 0)], opts=_opts(ttm, "direct"))
    assert e.value.status == -2
    with pytest.raises(ttm.TTMError) as e:
        ttm.Matcher([(comp, desc, m * 2.0)], [((20, 20, 20), 0)])
    assert e.value.status == -1
    mt = ttm.Matcher([(comp, desc, m)], [((20, 20, 20), 0)])
    vol = _cuda(np.random.default_rng(1).normal(size=(20, 20, 20)))
    small_ws = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(ttm.TTMError) as e:
        ttm.ttm_local_stats(mt.plan, [vol], mt.w, small_ws)
    assert e.value.status == -7
    ttm.ttm_local_stats(mt.plan, [vol], mt.w, mt.ws)
    bad_q = torch.empty(20 * 20 * 20 * 4 + 1, dtype=torch.float32, device="cuda")[1:]
    with pytest.raises(ttm.TTMError) as e:
        ttm.ttm_correlate(mt.plan, [vol], mt.w, mt.score, [bad_q], None, None, mt.ws)
    assert e.value.status == -1
    mt.close()


def test_classical_comparator_matches_oracle(ttm, c1_oracle):
    """Algorithm 1 over a rotation set on the GPU against the oracle's
    classical NCC: the maximum over rotations to 1e-4, and the arg-max either
    equal or a rotation whose NCC reaches the maximum within 1e-4."""
    import torch
    wl = c1_oracle["wl"]
    q = synth.shoemake_quaternions(40, 4).astype(np.float32)
    X = Y = Z = 64
    m = ttm.Matcher([(c1_oracle["comp"], c1_oracle["desc"], wl.mask)], [((X, Y, Z), 0)],
                    opts=_opts(ttm, "fft"))
    vol = _cuda(wl.volume)
    m.run([vol])
    best = torch.empty((Z, Y, X), dtype=torch.float32, device="cuda")
    arg = torch.empty((Z, Y, X), dtype=torch.int32, device="cuda")
    ws = torch.empty(ttm.ttm_classical_workspace_size(m.plan, 0), dtype=torch.uint8, device="cuda")
    ttm.ttm_classical_ncc(m.plan, 0, _cuda(wl.template), _cuda(q), len(q), vol, m.w[0], best, arg, ws)
    torch.cuda.synchronize()
    best, arg = best.cpu().numpy(), arg.cpu().numpy()
    cj = o.classical_ncc(wl.volume, wl.template, wl.mask, q.astype(np.float64))
    keep = o.interior_mask(wl.volume.shape, 15)
    best_o = np.where(keep, cj.max(axis=0), 0.0)
    assert np.abs(best - best_o).max() <= TOL
    assert np.all(arg[~keep] == 0)
    zi, yi, xi = np.nonzero(keep)
    c_at = cj[arg[zi, yi, xi], zi, yi, xi]
    assert np.all(c_at >= best_o[zi, yi, xi] - TOL)
    srt = np.sort(cj[:, zi, yi, xi], axis=0)
    unique = srt[-1] - srt[-2] > 2 * TOL
    assert np.all(arg[zi, yi, xi][unique] == cj[:, zi, yi, xi].argmax(axis=0)[unique])
    m.close()


def test_mixed_precision_within_bf16_tolerance(ttm, c1_oracle):
    """bf16 storage of spectra, products and correlation maps: components,
    score and lambda within 5e-3 of the FP64 oracle; w stays FP32-accurate."""
    o_ = _opts(ttm, "fft")
    o_.precision = ttm.TTM_PREC_MIXED
    res = _run(ttm, c1_oracle["wl"], c1_oracle["comp"], c1_oracle["desc"], opts=o_)
    C_o = c1_oracle["C_o"]
    dC = np.abs(res["comp"] - C_o).max()
    dS = np.abs(res["score"] - o.frobenius_score(C_o, 4)).max()
    assert dC <= 5e-3 and dS <= 5e-3, (dC, dS)
    nz = c1_oracle["w_o"] > 0
    assert (np.abs(res["w"][nz] - c1_oracle["w_o"][nz]) / c1_oracle["w_o"][nz]).max() <= 1e-5
    wl = c1_oracle["wl"]
    rng = np.random.default_rng(22)
    pts = np.concatenate([wl.positions, rng.integers(7, 57, size=(150, 3))])
    Cp = C_o[:, pts[:, 2], pts[:, 1], pts[:, 0]].T
    lam_o, _ = o.dominant_z_eigenpair(Cp, 4)
    dl = np.abs(res["lam"][pts[:, 2], pts[:, 1], pts[:, 0]] - lam_o).max()
    assert dl <= 5e-3, dl
    print(f"mixed precision max errors: C {dC:.2e} score {dS:.2e} lambda {dl:.2e}")


def test_pipelined_rotation_chunks_are_bit_identical(ttm):
    """The search/refinement pipeline over interior chunks (two streams, also
    inside a CUDA graph) gives the same maps as one search + one refinement."""
    import torch
    wl = synth.make_workload((96, 96, 96), 9, 3, 6, 1.0, 4, 200, radius=4, seeds=(5, 6, 7))
    comp, desc = ttm.build_template(wl.template, wl.mask, 4, wl.quadrature)
    vol = _cuda(wl.volume)
    outs = []
    for chunks in (1, 3, 4):
        o_ = _opts(ttm, "fft")
        o_.rotation_chunks = chunks
        m = ttm.Matcher([(comp, desc, wl.mask)], [((96, 96, 96), 0)], opts=o_)
        m.run([vol])
        torch.cuda.synchronize()
        outs.append((m.score[0].clone(), m.quat[0].clone(), m.lam[0].clone()))
        if chunks == 4:
            g = m.capture([vol])
            m.score[0].fill_(-1.0)
            m.lam[0].fill_(-1.0)
            g.replay()
            torch.cuda.synchronize()
            outs.append((m.score[0].clone(), m.quat[0].clone(), m.lam[0].clone()))
        assert ttm.ttm_plan_device_status(m.plan, m.ws) == 0
        m.close()
    for s, q, l in outs[1:]:
        assert torch.equal(s, outs[0][0]) and torch.equal(q, outs[0][1])
        assert torch.equal(l, outs[0][2])


@pytest.mark.parametrize("n,shape,s,r", [(4, (64, 64, 64), 15, 7), (6, (30, 28, 26), 9, 4)])
def test_tensor_core_direct_path(ttm, n, shape, s, r):
    """Direct correlation as an implicit GEMM on the tensor cores (FP16
    operands, FP32 accumulation): components, score and lambda within the
    5e-3 gate of the FP64 oracle (measured errors are printed)."""
    wl = synth.make_workload(shape, s, 5, 3, 1.0, n, 300, radius=r, seeds=(8, 9, 10))
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, n)
    comp, desc = ttm.build_template(wl.template, wl.mask, n, wl.quadrature)
    o_ = _opts(ttm, "direct")
    o_.precision = ttm.TTM_PREC_MIXED
    res = _run(ttm, wl, comp, desc, opts=o_)
    assert ttm.ttm_plan_problem_tensor_direct(res["matcher"].plan, 0)
    w_o, C_o = o.ttm_components(wl.volume, T, wl.mask)
    dC = np.abs(res["comp"] - C_o).max()
    dS = np.abs(res["score"] - o.frobenius_score(C_o, n)).max()
    assert dC <= 5e-3 and dS <= 5e-3, (dC, dS)
    pts = np.argwhere(w_o > 0)[::41][:150][:, ::-1]
    Cp = C_o[:, pts[:, 2], pts[:, 1], pts[:, 0]].T
    lam_o, _ = o.dominant_z_eigenpair(Cp, n)
    dl = np.abs(res["lam"][pts[:, 2], pts[:, 1], pts[:, 0]] - lam_o).max()
    assert dl <= 5e-3, dl
    print(f"tensor-core direct, order {n}: max errors C {dC:.2e} score {dS:.2e} lambda {dl:.2e}")
    res["matcher"].close()


def test_host_pipeline_matches_matcher(ttm):
    """HostPipeline (steps overlapped on two streams, host copies in and out)
    returns exactly the maps Matcher.run computes for each volume."""
    import torch
    wls = [synth.make_workload((40, 44, 48), 9, 3, 3, 1.0, 4, 200, radius=4, seeds=(s, s + 1, s + 2))
           for s in (31, 41)]
    comp, desc = ttm.build_template(wls[0].template, wls[0].mask, 4, wls[0].quadrature)
    prob = [((48, 44, 40), 0)]
    ref = []
    m = ttm.Matcher([(comp, desc, wls[0].mask)], prob, opts=_opts(ttm, "fft"))
    for wl in wls:
        m.run([_cuda(wl.volume)])
        torch.cuda.synchronize()
        ref.append((m.score[0].cpu(), m.quat[0].cpu(), m.lam[0].cpu()))
    m.close()
    pipe = ttm.HostPipeline([(comp, desc, wls[0].mask)], prob, opts=_opts(ttm, "fft"), depth=2)
    order = [0, 1, 0, 1]
    pins = [torch.from_numpy(wl.volume).pin_memory() for wl in wls]
    outs = [[(torch.empty((40, 44, 48)).pin_memory(), torch.empty((40, 44, 48, 4)).pin_memory(),
              torch.empty((40, 44, 48)).pin_memory())] for _ in order]
    for k, v in enumerate(order):
        pipe.submit([pins[v]], outs[k])
    pipe.join()
    torch.cuda.synchronize()
    for k, v in enumerate(order):
        s, q, l = outs[k][0]
        assert torch.equal(s, ref[v][0]) and torch.equal(q, ref[v][1]) and torch.equal(l, ref[v][2])
    pipe.close()
    # one plan, double-buffered volumes and maps: the same maps, step after
    # step, with three volumes cycling through two slots
    order = [0, 1, 1, 0, 1]
    stream = ttm.HostStream([(comp, desc, wls[0].mask)], prob, opts=_opts(ttm, "fft"), depth=2)
    outs = [[(torch.empty((40, 44, 48)).pin_memory(), torch.empty((40, 44, 48, 4)).pin_memory(),
              torch.empty((40, 44, 48)).pin_memory())] for _ in order]
    for k, v in enumerate(order):
        stream.submit([pins[v]], outs[k])
    stream.join()
    torch.cuda.synchronize()
    for k, v in enumerate(order):
        s, q, l = outs[k][0]
        assert torch.equal(s, ref[v][0]) and torch.equal(q, ref[v][1]) and torch.equal(l, ref[v][2])
    stream.close()


@pytest.mark.parametrize("path", PATHS)
def test_match_peaks_equals_dense_maps_at_peaks(ttm, path):
    """Rotations at the score peaks only (ttm_match_peaks) are the dense maps'
    values at those voxels, bit for bit, and the peaks are the same."""
    import torch
    wl = synth.make_workload((48, 52, 56), 11, 4, 6, 2.0, 4, 200, radius=5, seeds=(51, 52, 53))
    comp, desc = ttm.build_template(wl.template, wl.mask, 4, wl.quadrature)
    prob = [((56, 52, 48), 0)]
    vol = _cuda(wl.volume)
    dense = ttm.Matcher([(comp, desc, wl.mask)], prob, opts=_opts(ttm, path))
    dense.run([vol])
    ref = dense.peaks(0, 0.0, 5, 500)
    score_ref = dense.score[0].clone()
    sparse = ttm.Matcher([(comp, desc, wl.mask)], prob, opts=_opts(ttm, path))
    got = sparse.match_peaks([vol], 0, 0.0, 5, 500)
    torch.cuda.synchronize()
    assert len(ref) > 6 and len(got) == len(ref)
    assert torch.equal(sparse.score[0], score_ref)
    for f in ("x", "y", "z", "score", "lambda", "q"):
        assert np.array_equal(got[f], ref[f]), f
    dense.close()
    sparse.close()
    # the records against the oracle: its C at the peak voxels, the score,
    # the dominant Z-eigenvalue, and q a maximiser of the oracle's phi
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 4)
    pts = np.stack([got["x"], got["y"], got["z"]], 1).astype(np.int64)
    _, C_o = o.components_at(wl.volume, T, wl.mask, pts)
    assert np.abs(got["score"] - o.frobenius_score(C_o.T, 4)).max() <= TOL
    _rotation_check(C_o, got["lambda"], got["q"], 4, planted=range(len(pts)))


def test_soft_mask_fft_path(ttm):
    """A raised-cosine (soft) mask: the template build, the FFT window sums
    and the FFT correlations take the mask as weights; w, the components, the
    score and lambda agree with the oracle, which takes any mask."""
    wl = synth.make_workload((40, 44, 48), 13, 4, 3, 1.0, 4, 300, radius=6, seeds=(61, 62, 63))
    m = synth.soft_ball_mask(13, 6, 2.0)
    assert np.any((m > 0) & (m < 1))
    T = o.tensor_template(wl.template, m, wl.quadrature.astype(np.float64), wl.weights, 4)
    comp, desc = ttm.build_template(wl.template, m, 4, wl.quadrature)
    wl_soft = synth.Workload("soft", wl.volume, wl.template, m, wl.radius, 4, wl.quadrature,
                             wl.weights, wl.positions, wl.planted_quats, wl.noise_sigma, wl.snr)
    res = _run(ttm, wl_soft, comp, desc)
    assert ttm.ttm_plan_problem_path(res["matcher"].plan, 0) == ttm.TTM_PATH_FFT
    w_o, C_o = o.ttm_components(wl.volume, T, m)
    nz = w_o > 0
    assert np.array_equal(res["w"] > 0, nz)
    assert (np.abs(res["w"][nz] - w_o[nz]) / w_o[nz]).max() <= 1e-5
    assert np.abs(res["comp"] - C_o).max() <= TOL
    assert np.abs(res["score"] - o.frobenius_score(C_o, 4)).max() <= TOL
    pts = np.argwhere(nz)[::61][:150][:, ::-1]
    _rotation_check(C_o[:, pts[:, 2], pts[:, 1], pts[:, 0]].T,
                    res["lam"][pts[:, 2], pts[:, 1], pts[:, 0]],
                    res["quat"][pts[:, 2], pts[:, 1], pts[:, 0]], 4)
    res["matcher"].close()


@pytest.mark.parametrize("path", PATHS)
def test_gaussian_prefilter(ttm, path):
    """The optional prefilter h (Sec. 2): ttm_lowpass on the template and the
    plan's lowpass_sigma on the volume give the oracle's components of h * f
    against the tensor template of h * t."""
    wl = synth.make_workload((40, 44, 48), 11, 4, 3, 1.0, 4, 300, radius=5, seeds=(71, 72, 73))
    sigma = 1.2
    tf = ttm.ttm_lowpass(_cuda(wl.template), sigma).cpu().numpy()
    t_o = o.lowpass(wl.template, sigma)
    assert np.abs(tf - t_o).max() <= 1e-6 * np.abs(t_o).max()
    comp, desc = ttm.build_template(tf, wl.mask, 4, wl.quadrature)
    o_ = _opts(ttm, path)
    o_.lowpass_sigma = sigma
    res = _run(ttm, wl, comp, desc, opts=o_)
    T = o.tensor_template(t_o, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 4)
    w_o, C_o = o.ttm_components(o.lowpass(wl.volume, sigma), T, wl.mask)
    nz = w_o > 0
    assert np.array_equal(res["w"] > 0, nz)
    assert (np.abs(res["w"][nz] - w_o[nz]) / w_o[nz]).max() <= 1e-5
    assert np.abs(res["comp"] - C_o).max() <= TOL
    assert np.abs(res["score"] - o.frobenius_score(C_o, 4)).max() <= TOL
    res["matcher"].close()
