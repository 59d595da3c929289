"""Parity at the benchmark's full size and launch configuration.

The 256^3 volume with 50 planted copies of a 32^3 template (mask radius 15,
order 4, K = 35) is matched with the same plan options the benchmark uses
(automatic path choice: FFT correlation, tensor-core rotation search).  The
oracle computes w, C, the score and the dominant Z-eigenpair at sampled
voxels (every planted centre plus random interior voxels) by direct sums over
each voxel's own box.  The quadrature has 2000 rotations on both sides.
"""

import numpy as np
import pytest

import synth
from oracle import ttm_oracle as o

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def full(ttm_lib):
    import torch
    ttm = ttm_lib
    wl = synth.config_workload("c2", n_rot=2000)
    Z, Y, X = wl.volume.shape
    comp, desc = ttm.build_template(wl.template, wl.mask, 4, wl.quadrature)
    m = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)])
    assert ttm.ttm_plan_problem_path(m.plan, 0) == ttm.TTM_PATH_FFT
    vol = torch.from_numpy(wl.volume).cuda()
    comps = torch.empty((35, Z, Y, X), dtype=torch.float32, device="cuda")
    m.run([vol], components_out=[comps])
    torch.cuda.synchronize()
    assert ttm.ttm_plan_device_status(m.plan, m.ws) == 0
    rng = np.random.default_rng(7)
    c, s = 16, 32
    pts = np.concatenate([wl.positions,
                          np.stack([rng.integers(c, n - s + c + 1, 250) for n in (X, Y, Z)], 1)])
    zi, yi, xi = (torch.as_tensor(pts[:, k]).cuda() for k in (2, 1, 0))
    got = dict(C=comps[:, zi, yi, xi].T.cpu().numpy(), w=m.w[0][zi, yi, xi].cpu().numpy(),
               score=m.score[0][zi, yi, xi].cpu().numpy(), lam=m.lam[0][zi, yi, xi].cpu().numpy(),
               quat=m.quat[0][zi, yi, xi].cpu().numpy())
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 4)
    w_o, C_o = o.components_at(wl.volume, T, wl.mask, pts)
    peaks = m.peaks(0, 0.0, 10, 200)
    del comps
    return dict(wl=wl, pts=pts, got=got, w_o=w_o, C_o=C_o, peaks=peaks, m=m, T=T)


@pytest.fixture(scope="module")
def ttm_lib():
    import os
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2311_07561_gb300 as ttm
    if not os.path.exists(ttm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ttm.load_library()
    return ttm


def test_full_size_w_components_score(full):
    g = full["got"]
    assert np.all(full["w_o"] > 0)
    assert (np.abs(g["w"] - full["w_o"]) / full["w_o"]).max() <= 1e-5
    assert np.abs(g["C"] - full["C_o"]).max() <= TOL
    assert np.abs(g["score"] - o.frobenius_score(full["C_o"].T, 4)).max() <= TOL


def test_full_size_rotation(full):
    g = full["got"]
    lam_o, q_o = o.dominant_z_eigenpair(full["C_o"], 4)
    assert np.abs(g["lam"] - lam_o).max() <= TOL
    phi_at_gpu = o.phi_unique(full["C_o"], g["quat"].astype(np.float64), 4)
    assert np.all(phi_at_gpu >= lam_o - TOL)
    n_planted = len(full["wl"].positions)
    for i in range(n_planted):
        ang = o.rotation_angle_deg(g["quat"][i], q_o[i])
        assert ang <= 1.0 or phi_at_gpu[i] >= lam_o[i] - 1e-5, (i, ang)


def test_full_size_peaks_find_planted_copies(full):
    """Sanity of the method at SNR 0.5: most planted centres lie within two
    voxels of one of the 200 strongest score peaks."""
    pk = np.stack([full["peaks"]["x"], full["peaks"]["y"], full["peaks"]["z"]], 1)
    d = np.abs(full["wl"].positions[:, None, :] - pk[None, :, :]).max(axis=2).min(axis=1)
    assert np.mean(d <= 2) >= 0.8, np.sort(d)


def test_full_size_peaks_are_the_oracles(full):
    """Sec. 3.4 locates matches at the local maxima of ||C_n(x)||_F.  The
    oracle's score map of the whole 256^3 volume (its own FP64 FFT
    correlations) gives the peaks above a threshold taken from that map (its
    99.5th percentile on the interior) in 21^3 cubes; the GPU returns the same
    voxels for the same threshold and radius.  A voxel in one list and not the
    other is allowed only where it is a near tie: within 2e-4 of the
    threshold, or within 2e-4 of the largest score of its cube in the map that
    did not pick it (scores of the two sides differ by at most 1e-4)."""
    m, wl, T = full["m"], full["wl"], full["T"]
    radius, tie = 10, 2e-4
    _, C_all = o.ttm_components(wl.volume, T, wl.mask, use_fft=True)
    Z = C_all.shape[1]
    score_o = np.empty(C_all.shape[1:])
    for z0 in range(0, Z, 8):
        score_o[z0:z0 + 8] = o.frobenius_score(C_all[:, z0:z0 + 8], 4)
    del C_all
    keep = o.interior_mask(score_o.shape, 32)
    thr = float(np.quantile(score_o[keep], 0.995))
    expect = o.extract_peaks(score_o, thr, radius, 1 << 20)
    got = m.peaks(0, thr, radius, 1 << 20)
    score_g = m.score[0].cpu().numpy().astype(np.float64)
    shape = score_o.shape
    lin_g = (got["z"].astype(np.int64) * shape[1] + got["y"]) * shape[2] + got["x"]
    assert len(expect) > 40

    def near_tie(sc, lin):
        z, rem = divmod(int(lin), shape[1] * shape[2])
        y, x = divmod(rem, shape[2])
        v = sc[z, y, x]
        cube = sc[max(z - radius, 0):z + radius + 1, max(y - radius, 0):y + radius + 1,
                  max(x - radius, 0):x + radius + 1]
        return abs(v - thr) <= tie or cube.max() - v <= tie

    only_g = sorted(set(lin_g.tolist()) - set(expect.tolist()))
    only_o = sorted(set(expect.tolist()) - set(lin_g.tolist()))
    assert all(near_tie(score_o, v) for v in only_g), only_g
    assert all(near_tie(score_g, v) for v in only_o), only_o
    assert len(only_g) + len(only_o) <= 0.05 * len(expect), (len(only_g), len(only_o), len(expect))
    common = np.intersect1d(lin_g, expect)
    assert np.abs(score_g.ravel()[common] - score_o.ravel()[common]).max() <= 1e-4
    m.close()
