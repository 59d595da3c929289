"""The seeded input generators follow the stated recipe: SNR over the union
of the planted mask balls, planted boxes inside the volume and spaced apart,
unit quaternions (a near-uniform super-Fibonacci quadrature over S^3 and
uniform random planting rotations), the batch's copy counts and smooth shapes, and
reproducibility from the seeds.  CPU only."""

import numpy as np
import pytest

import synth


def _union(shape, s, mask, positions):
    u = np.zeros(shape, dtype=bool)
    c = s // 2
    for p in positions:
        x0, y0, z0 = (int(p[0]) - c, int(p[1]) - c, int(p[2]) - c)
        u[z0:z0 + s, y0:y0 + s, x0:x0 + s] |= mask.astype(bool)
    return u


def test_snr_is_signal_variance_over_the_planted_balls():
    args = ((48, 40, 56), 11, 4, 6, 0.5, 4, 100)
    noisy = synth.make_workload(*args, seeds=(4, 5, 6))
    clean = synth.make_workload(*args, seeds=(4, 5, 6), noise=False)
    assert np.array_equal(noisy.positions, clean.positions)
    u = _union(clean.volume.shape, 11, clean.mask, clean.positions)
    sig_var = np.var(clean.volume[u].astype(np.float64))
    assert sig_var / noisy.noise_sigma ** 2 == pytest.approx(0.5, rel=1e-5)
    noise = noisy.volume.astype(np.float64) - clean.volume
    assert np.std(noise) == pytest.approx(noisy.noise_sigma, rel=0.02)
    assert abs(np.mean(noise)) < 0.02 * noisy.noise_sigma


def test_planted_boxes_inside_and_spaced():
    wl = synth.make_workload((60, 64, 70), 15, 5, 8, 1.0, 4, 100, seeds=(1, 2, 3), noise=False)
    s, r = 15, wl.radius
    assert r == 7
    c = s // 2
    X, Y, Z = 70, 64, 60
    for p in wl.positions:
        assert c <= p[0] <= X - s + c and c <= p[1] <= Y - s + c and c <= p[2] <= Z - s + c
    d = np.linalg.norm(wl.positions[:, None, :] - wl.positions[None, :, :], axis=-1)
    d[np.arange(len(d)), np.arange(len(d))] = np.inf
    assert d.min() >= 2 * r * 0.9 ** 3      # spacing relaxes only when the volume is crowded
    assert np.allclose(np.linalg.norm(wl.planted_quats, axis=1), 1.0, atol=1e-6)


def test_quadrature_and_planting_rotations_are_uniform():
    q = synth.super_fibonacci_quaternions(20000)
    assert q.shape == (20000, 4)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-12)
    # distinct rotations (q and -q are one rotation): no two points that close
    sub = q[::40]
    sim = np.abs(sub @ sub.T) - 2 * np.eye(len(sub))
    assert sim.max() < 0.9999
    # uniform on S^3: E[q q^T] = I / 4
    for pts in (q, synth.shoemake_quaternions(20000, 7)):
        M = pts.T @ pts / len(pts)
        assert np.allclose(M, np.eye(4) / 4, atol=0.01)
    a = synth.shoemake_quaternions(100, 7)
    assert np.array_equal(a, synth.shoemake_quaternions(100, 7))
    assert not np.array_equal(a, synth.shoemake_quaternions(100, 8))


def test_masks_and_templates():
    for s, r in ((15, 7), (32, 15), (40, 19), (64, 31)):
        assert synth.default_mask_radius(s) == r
        m = synth.ball_mask(s, r)
        zz, yy, xx = np.mgrid[:s, :s, :s] - s // 2
        assert np.array_equal(m > 0, xx ** 2 + yy ** 2 + zz ** 2 <= r * r)
    soft = synth.soft_ball_mask(32, 15, 3.0)
    assert soft.min() >= 0.0 and soft.max() <= 1.0
    zz, yy, xx = np.mgrid[:32, :32, :32] - 16
    rad = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2)
    assert np.all(soft[rad > 15] == 0.0)
    assert np.any((soft > 0) & (soft < 1))
    t1 = synth.blob_template(15, 5, 3)
    assert np.array_equal(t1, synth.blob_template(15, 5, 3))
    assert t1.shape == (15, 15, 15) and np.isfinite(t1).all() and t1.max() > 0


def test_batch_copy_counts_and_smooth_shapes():
    cfg = synth.BATCH_CONFIGS["c4"]
    shapes = cfg["shapes_zyx"]
    assert len(shapes) == 16 and len(cfg["sizes"]) == 4

    def smooth(n):
        for f in (2, 3, 5):
            while n % f == 0:
                n //= f
        return n == 1
    assert all(smooth(n) for sh in shapes for n in sh)
    small = synth.make_batch([(24, 28, 32), (20, 24, 26)], (9, 11), 3, 0.5, 4, 50, 2, 4, seed=3)
    vmax = max(np.prod(sh) for sh in ((24, 28, 32), (20, 24, 26)))
    for v, sh in enumerate(((24, 28, 32), (20, 24, 26))):
        want = int(np.clip(round(4 * np.prod(sh) / vmax), 2, 4))
        assert [len(p) for p in small.positions[v]] == [want, want]
        assert small.volumes[v].shape == sh and small.volumes[v].dtype == np.float32
