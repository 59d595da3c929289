"""FP32 against mixed precision at the 512^3 configuration, both against the
FP64 oracle.

The 512^3 volume with 200 planted copies of a 40^3 template (mask radius 19,
order 4, K = 35, SNR 0.3) is matched twice on the FFT path: with FP32 storage
and with bf16 storage of the template spectra, product spectra and
correlation maps (FP32 arithmetic).  The oracle computes w, C, the score and
the dominant Z-eigenpair at 100 planted centres and 100 random interior voxels
by direct sums over each voxel's own box.  The quadrature has 300 rotations on
both sides (one oracle resampling of the 40^3 box per rotation).  Gates: w to
1e-5 relative; |dC|, |dscore|, |dlambda| <= 1e-4 (FP32) and <= 5e-3 (bf16);
the returned rotation reaches the oracle's maximum to the same gate.
"""

import numpy as np
import pytest

import synth
from oracle import ttm_oracle as o

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "mixed": 5e-3}


@pytest.fixture(scope="module")
def ttm():
    import os
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2311_07561_gb300 as ttm
    if not os.path.exists(ttm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ttm.load_library()
    return ttm


@pytest.fixture(scope="module")
def c3(ttm):
    import torch
    wl = synth.config_workload("c3", n_rot=300)
    Z, Y, X = wl.volume.shape
    comp, desc = ttm.build_template(wl.template, wl.mask, 4, wl.quadrature)
    rng = np.random.default_rng(23)
    s, c = 40, 20
    pts = np.concatenate([wl.positions[:100],
                          np.stack([rng.integers(c, n - s + c + 1, 100) for n in (X, Y, Z)], 1)])
    zi, yi, xi = (torch.as_tensor(pts[:, k]).cuda() for k in (2, 1, 0))
    vol = torch.from_numpy(wl.volume).cuda()
    got = {}
    for prec in ("fp32", "mixed"):
        opts = ttm.PlanOpts()
        opts.path = ttm.TTM_PATH_FFT
        opts.precision = ttm.TTM_PREC_FP32 if prec == "fp32" else ttm.TTM_PREC_MIXED
        m = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)], opts=opts)
        comps = torch.empty((35, Z, Y, X), dtype=torch.float32, device="cuda")
        m.run([vol], components_out=[comps])
        torch.cuda.synchronize()
        assert ttm.ttm_plan_device_status(m.plan, m.ws) == 0
        got[prec] = dict(C=comps[:, zi, yi, xi].T.cpu().numpy(), w=m.w[0][zi, yi, xi].cpu().numpy(),
                         score=m.score[0][zi, yi, xi].cpu().numpy(),
                         lam=m.lam[0][zi, yi, xi].cpu().numpy(),
                         quat=m.quat[0][zi, yi, xi].cpu().numpy())
        del comps
        m.close()
        torch.cuda.empty_cache()
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights, 4)
    w_o, C_o = o.components_at(wl.volume, T, wl.mask, pts)
    lam_o, q_o = o.dominant_z_eigenpair(C_o, 4)
    return dict(got=got, w_o=w_o, C_o=C_o, lam_o=lam_o, q_o=q_o)


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_precision_against_oracle(c3, prec):
    g, tol = c3["got"][prec], TOL[prec]
    assert np.all(c3["w_o"] > 0)
    assert (np.abs(g["w"] - c3["w_o"]) / c3["w_o"]).max() <= 1e-5
    assert np.abs(g["C"] - c3["C_o"]).max() <= tol
    assert np.abs(g["score"] - o.frobenius_score(c3["C_o"].T, 4)).max() <= tol
    assert np.abs(g["lam"] - c3["lam_o"]).max() <= tol
    phi = o.phi_unique(c3["C_o"], g["quat"].astype(np.float64), 4)
    assert np.all(phi >= c3["lam_o"] - tol)
