"""Host-side arithmetic of bench.py (no GPU): the algorithmic work behind the
roofline fractions, the traffic record's source check, and the angle used by
the order/quadrature sweep."""

import numpy as np
import pytest

import bench

PEAKS = dict(hbm_gbs=6771.0, bf16_tflops=1911.0)


def _one(name, ms=1.0, launches=1):
    return {name: dict(ms=ms, launches=launches)}


def test_refinement_work_per_voxel_order_four():
    # 8 candidates x 2 power steps (3 evaluations of C x^3 over 20 cubic
    # monomials x 4 outputs, 2 normalisations) + the 4 best x 3 Newton steps
    # (4 evaluations of C x^2: 10 entries x 10 quadratic monomials, 3 solves)
    rf = bench.roofline(_one("rotation_polish"), 1, 10 ** 6, 35, 0, 2048, 8, 3, PEAKS,
                        n_interior=10 ** 6)
    per_voxel = 8 * (3 * 10 * 20 + 24) + 4 * (4 * (2 * 10 * 10 + 2 * 10 + 40) + 3 * 150)
    assert per_voxel == 10952
    assert rf["bound"] == "alu" and rf["unit"] == "TFLOP/s"
    assert rf["achieved"] == pytest.approx(per_voxel * 1e6 / 1e-3 / 1e12, rel=1e-3)
    assert rf["frac"] == pytest.approx(rf["achieved"] / bench.FP32_ALU_PEAK_TFLOPS, rel=1e-3)


def test_tensor_core_search_counts_the_mma_only():
    # 2048 grid points x (35 components + constant column, padded to 48)
    rf = bench.roofline(_one("rotation_search", ms=2.0, launches=2), 1, 10 ** 6, 35, 0, 2048, 8, 4,
                        PEAKS, n_interior=10 ** 6)
    assert rf["bound"] == "tensor" and rf["peak"] == PEAKS["bf16_tflops"]
    # two launches per step share the interior voxels; 1 ms each
    assert rf["achieved"] == pytest.approx(2 * 2048 * 48 * 0.5e6 / 1e-3 / 1e12, rel=1e-3)


def test_order_six_search_pads_to_96():
    rf = bench.roofline(_one("rotation_search"), 1, 10 ** 6, 84, 0, 2048, 8, 4, PEAKS,
                        n_interior=10 ** 6)
    assert rf["achieved"] == pytest.approx(2 * 2048 * 96 * 1e6 / 1e-3 / 1e12, rel=1e-3)


def test_memory_bound_stages_use_algorithmic_bytes():
    rf = bench.roofline(_one("local_stats"), 1, 10 ** 8, 35, 0, 2048, 8, 4, PEAKS)
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    assert rf["achieved"] == pytest.approx(8 * 10 ** 8 / 1e-3 / 1e9, rel=1e-3)
    spec = 8.0 * 129 * 256 * 256
    rf = bench.roofline(_one("fft_spectrum_inverse"), 1, 256 ** 3, 35, 0, 2048, 8, 4, PEAKS,
                        spectrum_bytes=spec)
    # image spectrum read once, 35 template spectra read, 35 products written
    assert rf["achieved"] == pytest.approx(spec * 71 / 1e-3 / 1e9, rel=1e-3)


def test_traffic_only_while_sources_unchanged(monkeypatch):
    name = "rotation_polish"
    rec = dict(bench.NCU_TRAFFIC[name])
    src = ["k_rotation.cuh", "k_rotation.cu", "k_rotation_n4.cu"]
    monkeypatch.setitem(bench.NCU_TRAFFIC, name, dict(rec, source_sha=bench.source_hash(src)))
    # 8 launches per step share 2 million interior voxels
    rf = bench.roofline(_one(name, ms=8.0, launches=8), 1, 4 * 10 ** 6, 35, 0, 2048, 8, 4, PEAKS,
                        n_interior=2 * 10 ** 6)
    assert rf["traffic"] == round(rec["bytes_per_voxel"] * 2 * 10 ** 6 / 8)
    # another kind of launch than the captured one: no figure
    rf = bench.roofline(_one(name), 1, 10 ** 6, 84, 0, 2048, 8, 4, PEAKS, n_interior=10 ** 6)
    assert rf["traffic"] is None
    rf = bench.roofline(_one(name), 1, 10 ** 6, 35, 0, 2048, 8, 4, PEAKS, n_interior=10 ** 6,
                        fp32_maps=False)
    assert rf["traffic"] is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, name, dict(rec, source_sha="000000000000"))
    rf = bench.roofline(_one(name), 1, 10 ** 6, 35, 0, 2048, 8, 4, PEAKS, n_interior=10 ** 6)
    assert rf["traffic"] is None


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
