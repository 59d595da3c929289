"""Host-side arithmetic of bench.py (no GPU): the algorithmic work behind the
roofline fractions, the traffic record's source check, and the angle used by
the order/quadrature sweep."""

import numpy as np
import pytest

import bench

PEAKS = dict(hbm_gbs=6771.0, bf16_tflops=1911.0)


def _one(name, ms=1.0, launches=1):
    return {name: dict(ms=ms, launches=launches)}


def _geo(K=35, nvox=10 ** 6, n_int=10 ** 6, mixed=False, spec=0.0, taps=0):
    return dict(K=K, nvox=nvox, n_interior=n_int, mixed=mixed, spectrum_values=spec, n_taps=taps,
                tc_direct=False)


def test_score_rotation_stage_uses_the_planned_a5_count():
    """Search and refinement form one stage: 400 K FP32 FLOP per interior
    voxel (32 starts x 5 + 30 power iterations x 8 per component) over the sum
    of the two classes' times, against the derived FP32 peak."""
    kern = dict(rotation_search=dict(ms=3.0, launches=8), rotation_polish=dict(ms=1.0, launches=8),
                fft_inverse=dict(ms=2.5, launches=2))
    rf = bench.roofline(kern, 1, _geo(K=35, n_int=2 * 10 ** 6), PEAKS)
    assert rf["kernel"] == "score_rotation" and rf["bound"] == "alu"
    assert bench.a5_flop_per_voxel(35) == 14000 and bench.a5_flop_per_voxel(84) == 33600
    assert rf["achieved"] == pytest.approx(14000 * 2e6 / 4e-3 / 1e12, rel=1e-3)
    assert rf["frac"] == pytest.approx(rf["achieved"] / bench.FP32_ALU_PEAK_TFLOPS, rel=1e-3)
    # the grid contraction alone on the tensor pipe: 2 x 2048 x 48 per voxel
    tp = rf["tensor_pipe"]
    assert tp["achieved"] == pytest.approx(2 * 2048 * 48 * 2e6 / 3e-3 / 1e12, rel=1e-3)
    assert tp["peak"] == PEAKS["bf16_tflops"]
    ref = rf["refinement_alu"]
    assert ref["achieved"] == pytest.approx(bench.refinement_flop_per_voxel(35) * 2e6 / 1e-3 / 1e12,
                                            rel=1e-3)


def test_refinement_work_per_voxel_order_four():
    # 8 candidates x 2 power steps, ranked (3 evaluations of C x^3 over 20
    # cubic monomials x 4 outputs, 2 normalisations) + the 4 best x 3 Newton
    # steps (4 evaluations of C x^2: 10 entries x 10 quadratic monomials, 3
    # solves)
    per_voxel = 8 * (3 * 10 * 20 + 24) + 4 * (4 * (2 * 10 * 10 + 2 * 10 + 40) + 3 * 150)
    assert per_voxel == 10952 == bench.refinement_flop_per_voxel(35, 8, 3, 4)


def test_refinement_work_per_voxel_order_six():
    # 2 candidates, both refined: no ranking evaluation (2 of C x^5 over 56
    # monomials each), then 2 Newton steps (2 evaluations of C x^4 over 35
    # monomials, 2 solves, the last trial one evaluation of C x^5)
    per_voxel = 2 * (2 * 10 * 56 + 24) + 2 * (2 * (2 * 10 * 35 + 2 * 35 + 40) + 10 * 56 + 2 * 150)
    assert per_voxel == bench.refinement_flop_per_voxel(84, 2, 2, 2) == 7248


def test_order_six_search_pads_to_96():
    kern = dict(rotation_search=dict(ms=1.0, launches=1), rotation_polish=dict(ms=1.0, launches=1))
    rf = bench.roofline(kern, 1, _geo(K=84), PEAKS)
    assert rf["tensor_pipe"]["achieved"] == pytest.approx(2 * 2048 * 96 * 1e6 / 1e-3 / 1e12, rel=1e-3)


def test_memory_bound_stages_use_algorithmic_bytes():
    rf = bench.roofline(_one("local_stats"), 1, _geo(nvox=10 ** 8), PEAKS)
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    assert rf["achieved"] == pytest.approx(8 * 10 ** 8 / 1e-3 / 1e9, rel=1e-3)
    spec = 129.0 * 256 * 256
    rf = bench.roofline(_one("fft_spectrum_inverse"), 1, _geo(nvox=256 ** 3, spec=spec), PEAKS)
    # FP32: image spectrum read once, 35 template spectra read, 35 products written
    assert rf["achieved"] == pytest.approx(spec * (8 + 70 * 8) / 1e-3 / 1e9, rel=1e-3)
    # bf16 storage: 4 bytes per stored complex value, 2 per map value
    rf = bench.roofline(_one("fft_inverse"), 1, _geo(K=84, nvox=10 ** 6, mixed=True, spec=spec), PEAKS)
    assert rf["achieved"] == pytest.approx(84 * (3 * spec * 4 + 10 ** 6 * 2) / 1e-3 / 1e9, rel=1e-3)


def test_inverse_passes_count_the_interior_only():
    """With interior fractions kz (z planes) and ky (y rows) of the box, the
    y pass reads kz of every product and writes ky of that, the x pass reads
    it again and writes the interior map; the multiply pass reads the image
    spectrum once per component group and writes kz of every product."""
    spec = 481.0 * 960 * 480
    geo = dict(_geo(K=84, nvox=10 ** 6, n_int=5 * 10 ** 5, mixed=True, spec=spec),
               keep_z_frac=0.8, keep_y_frac=0.9, groups=10)
    rf = bench.roofline(_one("fft_inverse"), 1, geo, PEAKS)
    assert rf["achieved"] == pytest.approx(
        84 * (spec * 4 * 0.8 * (1 + 2 * 0.9) + 5e5 * 2) / 1e-3 / 1e9, rel=1e-6)
    rf = bench.roofline(_one("fft_spectrum_inverse"), 1, geo, PEAKS)
    assert rf["achieved"] == pytest.approx(spec * (8 * 10 + 84 * 4 * 1.8) / 1e-3 / 1e9, rel=1e-6)


def test_traffic_only_while_sources_unchanged(monkeypatch):
    kern = dict(rotation_search=dict(ms=1.0, launches=8), rotation_polish=dict(ms=1.0, launches=8))
    recs = {k: [dict(v[0])] for k, v in bench.NCU_TRAFFIC.items()}
    for k in ("rotation_search", "rotation_polish"):
        recs[k][0]["source_sha"] = bench.source_hash(recs[k][0]["sources"])
    monkeypatch.setattr(bench, "NCU_TRAFFIC", recs)
    rf = bench.roofline(kern, 1, _geo(K=35, n_int=2 * 10 ** 6), PEAKS)
    per = recs["rotation_search"][0]["bytes_per_voxel"] + recs["rotation_polish"][0]["bytes_per_voxel"]
    assert rf["traffic"] == round(per * 2 * 10 ** 6)
    # another kind of launch than the captured one: no figure
    assert bench.roofline(kern, 1, _geo(K=84), PEAKS)["traffic"] is None
    assert bench.roofline(kern, 1, _geo(K=35, mixed=True), PEAKS)["traffic"] is None
    recs["rotation_polish"][0]["source_sha"] = "000000000000"
    assert bench.roofline(kern, 1, _geo(K=35), PEAKS)["traffic"] is None


def test_error_stats_against_the_oracle():
    """The error object: largest score/lambda differences, w relative, the
    rotation angle at the planted voxels, and the validity of q as a maximiser
    of the oracle's phi."""
    from oracle import ttm_oracle as o
    rng = np.random.default_rng(3)
    C = rng.normal(size=(6, 35)) * 0.05
    lam, q = o.dominant_z_eigenpair(C, 4)
    ora = dict(C=C, lam=lam, q=q, score=o.frobenius_score(C.T, 4), w=np.full(6, 2.0))
    got = dict(score=ora["score"] + 2e-5, lam=lam - 3e-5, quat=q.astype(np.float32),
               w=np.full(6, 2.0 + 1e-6))
    st = bench.error_stats(got, ora, 4, 2, 1e-4)
    assert st["max_abs_score"] == pytest.approx(2e-5, rel=1e-6)
    assert st["max_abs_lambda"] == pytest.approx(3e-5, rel=1e-6)
    assert st["max_rel_w"] == pytest.approx(5e-7, rel=1e-6)
    assert st["rotation_deg_planted"]["max"] < 0.01 and st["within_tolerance"]
    got["lam"] = lam - 2e-4
    assert not bench.error_stats(got, ora, 4, 2, 1e-4)["within_tolerance"]


def test_sweep_angle():
    ident = np.array([1.0, 0.0, 0.0, 0.0])
    assert bench._angle_deg(ident, ident) == pytest.approx(0.0, abs=1e-6)
    assert bench._angle_deg(ident, -ident) == pytest.approx(0.0, abs=1e-6)
    for deg in (1.0, 30.0, 90.0, 179.0):
        h = np.radians(deg) / 2
        q = np.array([np.cos(h), 0.0, 0.0, np.sin(h)])    # turn by deg about z
        assert bench._angle_deg(ident, q) == pytest.approx(deg, abs=1e-6)
        p = np.array([np.cos(0.3), np.sin(0.3), 0.0, 0.0])
        # the angle of p^-1 q does not depend on a common left factor
        pq = np.array([p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3],
                       p[0] * q[1] + p[1] * q[0] + p[2] * q[3] - p[3] * q[2],
                       p[0] * q[2] - p[1] * q[3] + p[2] * q[0] + p[3] * q[1],
                       p[0] * q[3] + p[1] * q[2] - p[2] * q[1] + p[3] * q[0]])
        assert bench._angle_deg(p, pq) == pytest.approx(deg, abs=1e-6)
    st = bench._err_stats(np.array([0.5, 2.0, 6.0, 10.0]))
    assert st["within_1deg"] == 0.25 and st["within_5deg"] == 0.5 and st["max_deg"] == 10.0


def test_score_rotation_stage_takes_its_wall_time_span():
    """With the rotation_stage span recorded, the stage's time is the span
    (the two classes overlap on two streams, so their sum overstates it), and
    the span is left out of the per-class shares."""
    kern = dict(rotation_search=dict(ms=3.0, launches=8), rotation_polish=dict(ms=2.0, launches=8),
                rotation_stage=dict(ms=4.0, launches=16), fft_inverse=dict(ms=2.5, launches=2))
    rf = bench.roofline(kern, 1, _geo(K=84, n_int=10 ** 6), PEAKS)
    assert rf["kernel"] == "score_rotation" and rf["ms_per_step"] == pytest.approx(4.0)
    assert rf["achieved"] == pytest.approx(33600 * 1e6 / 4e-3 / 1e12, rel=1e-3)
    assert bench.kernel_ms(kern) == pytest.approx(7.5)
    # the inverse passes win when the span is short enough
    kern["rotation_stage"]["ms"] = 2.0
    assert bench.roofline(kern, 1, _geo(K=84, n_int=10 ** 6), PEAKS)["kernel"] == "fft_inverse"
