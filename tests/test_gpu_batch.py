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


def test_batch_at_the_configured_sizes(ttm):
    """Two volumes of the 16-volume batch configuration (160x160x128 and
    384x384x192: FFT boxes 160, 128, 384, 192 on the three axes) against its
    four templates (24^3 to 48^3, mask radii 11 to 23; the 24^3 problems sit
    nearest the direct/FFT crossover), all eight problems in one tuned plan
    replayed as one CUDA graph, sampled against the oracle: w to 1e-5
    relative, score and lambda to 1e-4.  The quadrature has 300 rotations on
    both sides."""
    import torch
    from synth import BATCH_CONFIGS
    cfg = BATCH_CONFIGS["c4"]
    shapes = [cfg["shapes_zyx"][1], cfg["shapes_zyx"][15]]
    bw = synth.make_batch(shapes, cfg["sizes"], cfg["n_blobs"], cfg["snr"], 4, 300, 20, 30,
                          lowpass=cfg["lowpass"], seed=5)
    tmpls = []
    for t, m in zip(bw.templates, bw.masks):
        comp, desc = ttm.build_template(t, m, 4, bw.quadrature)
        tmpls.append((comp, desc, m))
    dvols = [torch.from_numpy(v).cuda() for v in bw.volumes]
    problems, vols = [], []
    for v, vol in enumerate(bw.volumes):
        for k in range(len(cfg["sizes"])):
            problems.append((vol.shape[::-1], k))
            vols.append(dvols[v])
    opts = ttm.PlanOpts()
    opts.path = ttm.TTM_PATH_TUNE
    m = ttm.Matcher(tmpls, problems, opts=opts)
    graph = m.capture(vols)
    graph.replay()
    torch.cuda.synchronize()
    assert ttm.ttm_plan_device_status(m.plan, m.ws) == 0
    rng = np.random.default_rng(9)
    Ts = [o.tensor_template(t, mk, bw.quadrature.astype(np.float64), bw.weights, 4)
          for t, mk in zip(bw.templates, bw.masks)]
    for p, ((X, Y, Z), k) in enumerate(problems):
        v = p // len(cfg["sizes"])
        s = cfg["sizes"][k]
        c = s // 2
        pts = np.concatenate([bw.positions[v][k][:12],
                              np.stack([rng.integers(c, n - s + c + 1, 12) for n in (X, Y, Z)], 1)])
        T = Ts[k]
        w_o, C_o = o.components_at(bw.volumes[v], T, bw.masks[k], pts)
        zi, yi, xi = pts[:, 2], pts[:, 1], pts[:, 0]
        w_g = m.w[p].cpu().numpy()[zi, yi, xi]
        assert np.all(w_o > 0)
        assert (np.abs(w_g - w_o) / w_o).max() <= 1e-5, p
        score_g = m.score[p].cpu().numpy()[zi, yi, xi]
        assert np.abs(score_g - o.frobenius_score(C_o.T, 4)).max() <= TOL, p
        lam_o, _ = o.dominant_z_eigenpair(C_o, 4)
        lam_g = m.lam[p].cpu().numpy()[zi, yi, xi]
        assert np.abs(lam_g - lam_o).max() <= TOL, p
    m.close()


def _maps(ttm, m, vols):
    import torch
    m.run(vols)
    torch.cuda.synchronize()
    assert ttm.ttm_plan_device_status(m.plan, m.ws) == 0
    return [t.clone() for t in m.w + m.score + m.quat + m.lam]


@pytest.fixture(scope="module")
def many(ttm):
    """Ten small volumes x three templates (30 problems), templates built once."""
    import torch
    shapes = [(30 + 2 * (v % 3), 32 + v, 36) for v in range(10)]
    sizes = (9, 11, 13)
    bw = synth.make_batch(shapes, sizes, 4, 0.5, 4, 200, 1, 2, seed=17)
    tmpls = []
    for t, mk in zip(bw.templates, bw.masks):
        comp, desc = ttm.build_template(t, mk, 4, bw.quadrature)
        tmpls.append((comp, desc, mk))
    dvols = [torch.from_numpy(v).cuda() for v in bw.volumes]
    problems, vols = [], []
    for v, vol in enumerate(bw.volumes):
        for k in range(len(sizes)):
            problems.append((vol.shape[::-1], k))
            vols.append(dvols[v])
    return dict(tmpls=tmpls, problems=problems, vols=vols)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_resident_waves_match_one_problem_at_a_time(ttm, many, precision):
    """The same 30 problems planned one at a time and in resident waves:
    several waves with the default rotation chunks, one wave of all 30
    problems in a single chunk (two launches per stage: 24 + 6 problems), and
    one wave in two chunks on the two rotation streams.
    Path decisions are the cost model's (no timing), so all plans take the
    same paths; every map agrees bit for bit."""
    prec = ttm.TTM_PREC_FP32 if precision == "fp32" else ttm.TTM_PREC_MIXED

    def opts(batch_mib=0, chunks=0):
        o_ = ttm.PlanOpts()
        o_.precision = prec
        o_.batch_mib = batch_mib
        o_.rotation_chunks = chunks
        return o_

    tm, pb, vols = many["tmpls"], many["problems"], many["vols"]
    base = ttm.Matcher(tm, pb, opts=opts())
    assert ttm.ttm_plan_waves(base.plan) == []
    ref = _maps(ttm, base, vols)
    for batch_mib, chunks, several in ((40, 0, True), (4096, 1, False), (4096, 2, False)):
        m = ttm.Matcher(tm, pb, opts=opts(batch_mib, chunks))
        waves = ttm.ttm_plan_waves(m.plan)
        assert waves[0] == 0 and waves == sorted(waves)
        if several:
            assert len(waves) >= 2, waves
        elif precision == "fp32":
            assert waves == [0]
        got = _maps(ttm, m, vols)
        for p, (a, b) in enumerate(zip(ref, got)):
            assert torch_equal(a, b), (batch_mib, chunks, p)
        m.close()
    base.close()


def torch_equal(a, b) -> bool:
    import torch
    return bool(torch.equal(a, b))


def test_shared_volume_spectra_change_nothing(ttm, many):
    """Consecutive problems of one volume share its moments and spectra (local
    statistics and correlations); giving every problem its own copy of the
    volume turns the sharing off: the maps agree bit for bit."""
    tm, pb, vols = many["tmpls"], many["problems"], many["vols"]
    m = ttm.Matcher(tm, pb)
    shared = _maps(ttm, m, vols)
    copies = [v.clone() for v in vols]
    assert len({c.data_ptr() for c in copies}) == len(copies)
    separate = _maps(ttm, m, copies)
    for p, (a, b) in enumerate(zip(shared, separate)):
        assert torch_equal(a, b), p
    m.close()


def test_host_stream_with_shared_volume_copies(ttm, many):
    """End to end on a batch: HostStream driving an existing plan with one
    device copy per volume (its problems share the volume's spectra) gives
    the maps of Matcher.run, bit for bit, on two consecutive steps."""
    import torch
    tm, pb, vols = many["tmpls"], many["problems"], many["vols"]
    m = ttm.Matcher(tm, pb)
    ref = _maps(ttm, m, vols)
    n_t = 3
    host_vols = [vols[p].cpu().pin_memory() for p in range(0, len(pb), n_t)]
    outs = [[(torch.empty_like(m.score[p], device="cpu").pin_memory(),
              torch.empty_like(m.quat[p], device="cpu").pin_memory(),
              torch.empty_like(m.lam[p], device="cpu").pin_memory()) for p in range(len(pb))]
            for _ in range(2)]
    hs = ttm.HostStream(matcher=m, depth=2, volume_of=[p // n_t for p in range(len(pb))])
    for k in range(2):
        hs.submit(host_vols, outs[k])
    hs.join()
    torch.cuda.synchronize()
    assert ttm.ttm_plan_device_status(m.plan, m.ws) == 0
    n = len(pb)
    for k in range(2):
        for p, (so, qo, lo) in enumerate(outs[k]):
            assert torch.equal(so, ref[n + p].cpu()), (k, p)
            assert torch.equal(qo, ref[2 * n + p].cpu()), (k, p)
            assert torch.equal(lo, ref[3 * n + p].cpu()), (k, p)
    hs.close()
    m.close()
