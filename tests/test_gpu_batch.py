"""Batched plans: uneven volumes x several templates in one plan, the
plan-time path autotuner, and CUDA-graph replay of the whole batch.

Every (volume, template) pair is checked against the FP64 oracle at sampled
interior voxels (w, the K components, score and lambda), so the batch, the
smooth FFT boxes it pads to, and the graph replay are all held to the FP32
gates of the single-problem tests.
"""

import numpy as np
import pytest

import synth
from oracle import ttm_oracle as o

pytestmark = pytest.mark.gpu

TOL = 1e-4
SHAPES = [(40, 48, 64), (36, 60, 50), (30, 45, 72)]     # (z, y, x)
SIZES = (9, 11, 13)


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
def batch(ttm):
    import torch
    bw = synth.make_batch(SHAPES, SIZES, 4, 0.5, 4, 300, 3, 5, seed=21)
    tmpls = []
    for t, m in zip(bw.templates, bw.masks):
        comp, desc = ttm.build_template(t, m, 4, bw.quadrature)
        tmpls.append((comp, desc, m))
    problems, vols = [], []
    dvols = [torch.from_numpy(v).cuda() for v in bw.volumes]
    for v, vol in enumerate(bw.volumes):
        for k in range(len(SIZES)):
            problems.append((vol.shape[::-1], k))
            vols.append(dvols[v])
    opts = ttm.PlanOpts()
    opts.path = ttm.TTM_PATH_TUNE
    m = ttm.Matcher(tmpls, problems, opts=opts)
    yield dict(bw=bw, m=m, vols=vols, problems=problems)
    m.close()


def test_tuner_times_both_paths_and_keeps_the_faster(ttm, batch):
    m = batch["m"]
    for p in range(len(batch["problems"])):
        direct_ms, fft_ms = ttm.ttm_plan_problem_tuning(m.plan, p)
        assert direct_ms > 0 and fft_ms > 0
        path = ttm.ttm_plan_problem_path(m.plan, p)
        assert path == (ttm.TTM_PATH_DIRECT if direct_ms < fft_ms else ttm.TTM_PATH_FFT)


def test_graph_replay_matches_eager_and_oracle(ttm, batch):
    import torch
    bw, m, vols = batch["bw"], batch["m"], batch["vols"]
    m.run(vols)
    torch.cuda.synchronize()
    assert ttm.ttm_plan_device_status(m.plan, m.ws) == 0
    eager = [(s.clone(), q.clone(), l.clone(), w.clone())
             for s, q, l, w in zip(m.score, m.quat, m.lam, m.w)]
    graph = m.capture(vols)
    for x in m.score + m.lam:
        x.fill_(-7.0)
    graph.replay()
    torch.cuda.synchronize()
    for p, (s, q, l, w) in enumerate(eager):
        assert torch.equal(s, m.score[p]) and torch.equal(q, m.quat[p])
        assert torch.equal(l, m.lam[p]) and torch.equal(w, m.w[p])
    rng = np.random.default_rng(3)
    for p, ((X, Y, Z), k) in enumerate(batch["problems"]):
        v = p // len(SIZES)
        s = SIZES[k]
        c = s // 2
        pts = np.concatenate([bw.positions[v][k],
                              np.stack([rng.integers(c, n - s + c + 1, 40) for n in (X, Y, Z)], 1)])
        T = o.tensor_template(bw.templates[k], bw.masks[k], bw.quadrature.astype(np.float64),
                              bw.weights, 4)
        w_o, C_o = o.components_at(bw.volumes[v], T, bw.masks[k], pts)
        zi, yi, xi = pts[:, 2], pts[:, 1], pts[:, 0]
        w_g = m.w[p].cpu().numpy()[zi, yi, xi]
        assert (np.abs(w_g - w_o) / np.maximum(w_o, 1e-30)).max() <= 1e-5, p
        score_g = m.score[p].cpu().numpy()[zi, yi, xi]
        assert np.abs(score_g - o.frobenius_score(C_o.T, 4)).max() <= TOL, p
        lam_o, _ = o.dominant_z_eigenpair(C_o, 4)
        lam_g = m.lam[p].cpu().numpy()[zi, yi, xi]
        assert np.abs(lam_g - lam_o).max() <= TOL, p
