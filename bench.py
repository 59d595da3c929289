#!/usr/bin/env python
"""Throughput of tensorial template matching on GB300: tomogram voxels/s of
the TTM score + rotation maps.

One step = local statistics + correlation with the K tensor components +
per-voxel Frobenius score and dominant Z-eigenvector rotation, over one
synthetic tomogram.  The default workload is the largest single-GPU
configuration: a 928 x 928 x 464 FP32 volume with 2000 planted copies of a
64^3 lowpassed blob template (SNR 0.2, mask radius 31), tensor order n = 6
(K = 84), bf16 storage of the template spectra, product spectra and
correlation maps (FP32 arithmetic).  The tensor template is built once before
timing (reported separately).  Inputs are resident in HBM when the timed
region starts; L2 is flushed (256 MB write) before every timed step, outside
the step's events.

Beside the timing the line states the error of the maps against the FP64
oracle at sampled voxels, FP32 against bf16 storage at 512^3 (each against the
oracle), the oracle's own rate on all host cores, and the end-to-end rate with
host copies.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs an independent replica (weak scaling); rank 0
prints one JSON line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tomogram voxels/s of TTM score+rotation maps (FP32 vs BF16) at stated NCC error; % roofline"
UNIT = "voxels/s"
WORKLOAD = dict(
    c2="256x256x256 FP32 volume, 50 planted copies of a 32^3 lowpassed 30-blob template, "
       "uniform random rotations, SNR 0.5, ball mask r=15, tensor order n=4 (K=35)",
    c1="64x64x64 FP32 volume, 4 planted copies of a 15^3 5-blob template, SNR 1, "
       "ball mask r=7, tensor order n=4 (K=35)",
    c2s="128x128x128 FP32 volume (profiling size), 8 planted copies of the 32^3 template of c2, "
        "SNR 0.5, ball mask r=15, tensor order n=4 (K=35)",
    c3="512x512x512 FP32 volume, 200 planted copies of a 40^3 lowpassed 30-blob template, "
       "SNR 0.3, ball mask r=19, tensor order n=4 (K=35)",
    c5s="256x256x192 FP32 volume (profiling size), 40 planted copies of the 64^3 template of c5, "
        "SNR 0.2, ball mask r=31, tensor order n=6 (K=84), quadrature of 20000 rotations, "
        "mixed precision",
    c5x="928x96x464 FP32 slab (profiling the length-960 x and length-480 z passes), 10 planted "
        "copies of the 64^3 template of c5, SNR 0.2, ball mask r=31, tensor order n=2 (K=10), "
        "mixed precision",
    c5y="928x928x96 FP32 slab (profiling the length-960 y pass), 20 planted copies of the 64^3 "
        "template of c5, SNR 0.2, ball mask r=31, tensor order n=2 (K=10), mixed precision",
    c5="928x928x464 FP32 volume, 2000 planted copies of a 64^3 lowpassed 30-blob template, "
       "SNR 0.2, ball mask r=31, tensor order n=6 (K=84), quadrature of 20000 rotations; FFT box "
       "960x960x480; mixed precision (bf16 template spectra, products and maps resident in HBM)",
    c4="16 FP32 volumes of uneven 2*3*5-smooth sizes (128^3 to 384x384x192, 216 M voxels) x 4 "
       "lowpassed 30-blob templates (24^3, 32^3, 40^3, 48^3; ball masks r=11,15,19,23): 64 "
       "(volume, template) problems in one plan, 20-100 planted copies of each template per "
       "volume, SNR 0.5, tensor order n=4 (K=35); autotuned FFT-vs-direct, one CUDA graph",
)
BATCH_WORKLOADS = ("c4",)
CPU_SAMPLE_SHAPES = dict(c3=dict(shape_zyx=(160, 160, 160), copies=10),
                         c5=dict(shape_zyx=(192, 192, 192), copies=8))
WORKLOAD_OVERRIDES = dict(c2s=("c2", dict(shape_zyx=(128, 128, 128), copies=8)),
                          c5s=("c5", dict(shape_zyx=(192, 256, 256), copies=40)),
                          c5x=("c5", dict(shape_zyx=(464, 96, 928), copies=10, n_order=2,
                                          n_rot=2000)),
                          c5y=("c5", dict(shape_zyx=(96, 928, 928), copies=20, n_order=2,
                                          n_rot=2000)))


def load_workload(name: str, **extra):
    import synth
    base, over = WORKLOAD_OVERRIDES.get(name, (name, {}))
    return synth.config_workload(base, **dict(over, **extra))
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
# the refinement's defaults (candidates taking two power steps, the best
# points reached taking Newton steps, Newton steps): by tensor order
REFINE_BUDGET = {6: (2, 2, 2)}
DEFAULT_BUDGET = (8, 4, 3)


def budget(K: int):
    n_ord = {10: 2, 35: 4, 84: 6, 165: 8}.get(K, 4)
    return REFINE_BUDGET.get(n_ord, DEFAULT_BUDGET)


def grid_points(K: int, mixed: bool) -> int:
    """The plan's default rotation search grid: 1024 points with bf16
    storage, else 2048."""
    return 1024 if mixed else 2048


def refinement_text(K: int) -> str:
    c, r, nw = budget(K)
    return f"{c} candidates x 2 power steps, the {r} best x {nw} Newton steps"


L2_FLUSH_BYTES = 256 << 20

# Measured DRAM traffic of a kernel class from one ncu capture, per interior
# voxel, for one order (K) and map storage, with the hash of the sources it
# was taken on; reported (times the interior voxels of a step) only while
# those sources are unchanged.
NCU_TRAFFIC: dict = {
    # ncu (dram__bytes_read.sum + dram__bytes_write.sum) of one launch over the
    # whole interior: the 128^3 case (c2s), 912 673 interior voxels, FP32 maps;
    # the 256x256x192 case of the order-6 template (c5s), 4 805 121 interior
    # voxels, bf16 maps.
    "rotation_polish": [dict(bytes_per_voxel=(193203200 + 9803008) / 912673, K=35, storage="f32",
                             source_sha="912e1275591c",
                             sources=["k_rotation.cuh", "k_rotation.cu", "k_rotation_n4.cu"]),
                        dict(bytes_per_voxel=(1193875456 + 90971136) / 4805121, K=84,
                             storage="bf16", source_sha="e2173a68ccde",
                             sources=["k_rotation.cuh", "k_rotation.cu", "k_rotation_n6.cu"])],
    "rotation_search": [dict(bytes_per_voxel=(173863936 + 11920384) / 912673, K=35, storage="f32",
                             source_sha="7ea2aa611a47",
                             sources=["k_search_tc.cu", "k_rotation.cuh"]),
                        dict(bytes_per_voxel=(1094127360 + 91662592) / 4805121, K=84,
                             storage="bf16", source_sha="7ea2aa611a47",
                             sources=["k_search_tc.cu", "k_rotation.cuh"])],
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=["c1", "c2", "c2s", "c3", "c4", "c5", "c5s", "c5x", "c5y"])
    ap.add_argument("--path", default="auto", choices=["auto", "direct", "fft"])
    ap.add_argument("--precision", default=None, choices=["fp32", "mixed"],
                    help="storage of spectra/products/correlation maps on the FFT path "
                         "(default fp32; mixed for c5, whose FP32 maps and spectra exceed HBM)")
    ap.add_argument("--mixed-compare", action=argparse.BooleanOptionalAction, default=True,
                    help="with fp32, also time the mixed-precision plan on the same volume")
    ap.add_argument("--batch-mib", type=int, default=-1,
                    help="batch workloads: resident waves of this many MiB of correlation "
                         "maps (plan option batch_mib); -1 = 32768, 0 = one problem at a time")
    ap.add_argument("--rotation-chunks", type=int, default=0,
                    help="interior chunks of the pipelined search/refinement (0 = library default)")
    ap.add_argument("--peaks-only", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the score map + rotations at its peaks only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-depth", type=int, default=0,
                    help="steps in flight in the end-to-end measurement (0 = 2, or 1 for c5)")
    ap.add_argument("--classical", action=argparse.BooleanOptionalAction, default=True,
                    help="also time classical NCC at 1000 rotations on the same volume")
    ap.add_argument("--oracle-errors", action=argparse.BooleanOptionalAction, default=True,
                    help="state the error of the maps against the FP64 oracle at sampled voxels")
    ap.add_argument("--precision-pair", action=argparse.BooleanOptionalAction, default=True,
                    help="with the 928x928x464 workload, also time FP32 and bf16 storage at "
                         "512^3, each with its error against the oracle")
    ap.add_argument("--order-sweep", action="store_true",
                    help="rotation error at the planted copies of the 256^3 volume against the "
                         "tensor order n and the quadrature size, beside classical NCC at 1000 "
                         "and 7112 sampled rotations; prints its own JSON line")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "mixed" if args.workload.startswith("c5") else "fp32"
    return args


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores: timing (CPU baseline / reference arm) and
# the error of the GPU maps.  Work is spread over spawned worker processes
# (one BLAS thread each); every worker warms the oracle's cached tables before
# anything is timed.
# ---------------------------------------------------------------------------

ORACLE_TEMPLATE_ROTATIONS = 64      # the per-voxel cost does not depend on it
ERROR_ROTATIONS = 300               # quadrature of the error runs, both sides


def oracle_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def _oracle_init(n_order, barrier):
    """Worker start: import the oracle and fill its cached tables (the search
    set and its neighbour lists, the index tables of order n) on a dummy
    voxel, then wait until every worker is ready."""
    import numpy as np
    from oracle import ttm_oracle as o
    K = len(o.multi_indices(n_order))
    o.dominant_z_eigenpair(np.random.default_rng(0).normal(size=(2, K)), n_order)
    o.frobenius_score(np.zeros((K, 1)), n_order)
    if barrier is not None:
        barrier.wait()


def _oracle_voxels(job):
    """Worker: the oracle's per-voxel steps (local statistics, the K
    components by direct sums, score, dominant Z-eigenpair) at the voxels."""
    import numpy as np
    from oracle import ttm_oracle as o
    tdir, pts, n_order, var_f = job
    vol = np.load(os.path.join(tdir, "vol.npy"), mmap_mode="r")
    T = np.load(os.path.join(tdir, "T.npy"), mmap_mode="r")
    m = np.load(os.path.join(tdir, "mask.npy"))
    t0 = time.perf_counter()
    w, C = o.components_at(vol, np.asarray(T), m, pts, var_f=var_f)
    score = o.frobenius_score(C.T, n_order)
    lam, q = o.dominant_z_eigenpair(C, n_order)
    return dict(w=w, C=C, score=score, lam=lam, q=q, seconds=time.perf_counter() - t0)


def _oracle_template_part(job):
    """Worker: the oracle's tensor template over a slice of the quadrature
    (the template is linear in the weights, so the slices add up)."""
    import numpy as np
    from oracle import ttm_oracle as o
    tdir, t, m, quats, weights, n_order, part = job
    T = o.tensor_template(t, m, quats, weights, n_order)
    path = os.path.join(tdir, f"Tpart{part}.npy")
    np.save(path, T)
    return path


class OraclePool:
    """Spawned worker processes running the oracle (one BLAS thread each)."""

    def __init__(self, n_order: int, cores: int | None = None):
        import multiprocessing as mp
        self.cores = cores or oracle_cores()
        self.n_order = n_order
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                "MKL_NUM_THREADS", "CUDA_VISIBLE_DEVICES")}
        os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                          CUDA_VISIBLE_DEVICES="")
        try:
            barrier = ctx.Barrier(self.cores + 1)
            self.pool = ctx.Pool(self.cores, initializer=_oracle_init,
                                 initargs=(n_order, barrier))
            barrier.wait()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.tdir = tempfile.mkdtemp(prefix="ttm_oracle_")

    def tensor_template(self, t, m, quats, weights, name: str):
        """The oracle's tensor template, quadrature slices in parallel."""
        import numpy as np
        n = len(quats)
        parts = min(self.cores, max(1, n // 8))
        bounds = np.linspace(0, n, parts + 1).astype(int)
        jobs = [(self.tdir, t, m, quats[a:b], weights[a:b], self.n_order, f"{name}{i}")
                for i, (a, b) in enumerate(zip(bounds[:-1], bounds[1:])) if b > a]
        T = None
        for path in self.pool.map(_oracle_template_part, jobs, chunksize=1):
            part = np.load(path)
            T = part if T is None else T + part
            os.unlink(path)
        return T

    def stage(self, vol, T, mask) -> None:
        import numpy as np
        np.save(os.path.join(self.tdir, "vol.npy"), np.ascontiguousarray(vol))
        np.save(os.path.join(self.tdir, "T.npy"), np.ascontiguousarray(T))
        np.save(os.path.join(self.tdir, "mask.npy"), np.ascontiguousarray(mask))

    def voxels(self, pts, var_f: float) -> dict:
        """The oracle at the voxels (x, y, z) of the staged volume, split over
        the workers; returns the merged results and the wall seconds."""
        import numpy as np
        chunks = [c for c in np.array_split(np.asarray(pts), 2 * self.cores) if len(c)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_voxels, [(self.tdir, c, self.n_order, var_f) for c in chunks],
                            chunksize=1)
        wall = time.perf_counter() - t0
        out = {k: np.concatenate([r[k] for r in res]) for k in ("w", "C", "score", "lam", "q")}
        out["wall"] = wall
        return out

    def close(self) -> None:
        self.pool.close()
        self.pool.join()
        import shutil
        shutil.rmtree(self.tdir, ignore_errors=True)


def cpu_sample_workload(workload: str):
    """The volume the oracle is timed on: the workload itself, or for the
    large configurations a smaller volume with the same template, mask and
    order (the oracle's cost per voxel is set by those)."""
    import synth
    if workload in BATCH_WORKLOADS:
        cfg = synth.BATCH_CONFIGS[workload]
        bw = synth.batch_workload(workload, shapes_zyx=cfg["shapes_zyx"][:1], sizes=(32,),
                                  n_rot=ORACLE_TEMPLATE_ROTATIONS)
        return synth.Workload("batch-sample", bw.volumes[0], bw.templates[0], bw.masks[0],
                              bw.radii[0], bw.n_order, bw.quadrature, bw.weights,
                              bw.positions[0][0], bw.planted_quats[0][0], 0.0, bw.snr)
    return load_workload(workload, n_rot=ORACLE_TEMPLATE_ROTATIONS,
                         **CPU_SAMPLE_SHAPES.get(workload, {}))


def random_interior(shape_zyx, s: int, n: int, rng):
    import numpy as np
    c = s // 2
    Z, Y, X = shape_zyx
    return np.stack([rng.integers(c, X - s + c + 1, n), rng.integers(c, Y - s + c + 1, n),
                     rng.integers(c, Z - s + c + 1, n)], axis=1)


def oracle_timing(workload: str, n_vox: int, steps: int, cores: int | None = None) -> dict:
    """Wall time of the oracle over `steps` samples of `n_vox` random interior
    voxels each, on all host cores (after every worker has warmed up)."""
    import numpy as np
    wl = cpu_sample_workload(workload)
    pool = OraclePool(wl.n_order, cores)
    try:
        T = pool.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64),
                                 wl.weights, "t")
        pool.stage(wl.volume, T, wl.mask)
        var_f = float(np.var(wl.volume.astype(np.float64)))
        rng = np.random.default_rng(11)
        pool.voxels(random_interior(wl.volume.shape, wl.template.shape[0], pool.cores, rng), var_f)
        times = []
        for _ in range(steps):
            pts = random_interior(wl.volume.shape, wl.template.shape[0], n_vox, rng)
            times.append(pool.voxels(pts, var_f)["wall"])
    finally:
        pool.close()
    return dict(times=times, n_vox=n_vox, cores=pool.cores, shape=wl.volume.shape[::-1])


def cpu_baseline_obj(res: dict, workload: str = "", warmup_steps: int = 1) -> dict:
    tot = sum(res["times"])
    n = res["n_vox"] * len(res["times"])
    where = "the same workload"
    if workload in CPU_SAMPLE_SHAPES:
        where = (f"a {'x'.join(map(str, res['shape']))} volume with the same template, order "
                 "and mask (the oracle's cost per voxel is set by those)")
    elif workload in BATCH_WORKLOADS:
        where = "the batch's first volume with its 32^3 template"
    return dict(value=n / tot, unit=UNIT, cores=res["cores"], kind="oracle",
                sample=f"{len(res['times'])} x {res['n_vox']} random interior voxels of {where}: "
                       "local statistics, K component correlations by direct sums, Frobenius "
                       "score and dominant Z-eigenpair (FP64 numpy oracle), one process per core "
                       f"with one BLAS thread; {tot:.1f} s wall after {warmup_steps} untimed "
                       "warm-up sample per worker; tensor template built beforehand")


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = oracle_cores()
    n_vox = 4 * cores
    res = oracle_timing(args.workload, n_vox, args.warmup + args.steps, cores)
    times = res["times"][args.warmup:]
    total = sum(times)
    value = n_vox * len(times) / total
    cpu = cpu_baseline_obj(dict(res, times=times), args.workload, args.warmup)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
        warmup=args.warmup, ms_per_step=1e3 * total / len(times), higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(workload=WORKLOAD[args.workload], step=f"{n_vox} sampled interior voxels"),
        impl="reference", cpu_baseline=cpu,
        e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0),
    )
    print(json.dumps(line), flush=True)


def gpu_maps_at(matcher, pts) -> dict:
    """w, score, lambda and q of problem 0 at the voxels (x, y, z)."""
    import torch
    zi, yi, xi = (torch.as_tensor(pts[:, k]).cuda() for k in (2, 1, 0))
    return dict(w=matcher.w[0][zi, yi, xi].cpu().numpy(),
                score=matcher.score[0][zi, yi, xi].cpu().numpy(),
                lam=matcher.lam[0][zi, yi, xi].cpu().numpy(),
                quat=matcher.quat[0][zi, yi, xi].cpu().numpy())


def error_stats(got: dict, ora: dict, n_order: int, n_planted: int, tol: float,
                truth=None) -> dict:
    """Errors of the GPU maps against the oracle at the sampled voxels (the
    first n_planted are planted centres; truth: their planted rotations)."""
    import numpy as np
    from oracle import ttm_oracle as o
    dscore = np.abs(got["score"] - ora["score"])
    dlam = np.abs(got["lam"] - ora["lam"])
    relw = np.abs(got["w"] - ora["w"]) / np.where(ora["w"] > 0, ora["w"], 1.0)
    phi = o.phi_unique(ora["C"], got["quat"].astype(np.float64), n_order)
    ang = o.rotation_angle_deg(got["quat"][:n_planted], ora["q"][:n_planted])
    # planted voxels where phi has a unique maximiser to the gate: there the
    # rotation itself is compared (else any maximiser is a valid answer)
    valid = phi >= ora["lam"] - tol
    out = dict(voxels=int(len(dscore)), planted=int(n_planted),
                max_abs_score=float(dscore.max()), max_abs_lambda=float(dlam.max()),
                max_rel_w=float(relw.max()), max_phi_shortfall=float((ora["lam"] - phi).max()),
                rotation_deg_planted=dict(median=float(np.median(ang)), max=float(ang.max()),
                                          within_1deg=float(np.mean(ang <= 1.0))),
                tolerance=tol,
                within_tolerance=bool(dscore.max() <= tol and dlam.max() <= tol and valid.all()
                                      and relw.max() <= 1e-5))
    if truth is not None and n_planted:
        def stats(a):
            return dict(median=float(np.median(a)), max=float(a.max()),
                        within_1deg=float(np.mean(a <= 1.0)), within_5deg=float(np.mean(a <= 5.0)))
        out["rotation_deg_vs_planted_truth"] = dict(
            gpu=stats(o.rotation_angle_deg(got["quat"][:n_planted], truth[:n_planted])),
            oracle=stats(o.rotation_angle_deg(ora["q"][:n_planted], truth[:n_planted])))
    return out


def oracle_error_runs(ttm, wl, plans: dict, pool, n_planted: int = 32, n_random: int = 32,
                      seed: int = 5) -> dict:
    """GPU maps of the volume under each plan option set of `plans` (name ->
    (PlanOpts, tolerance)), with the tensor template of ERROR_ROTATIONS
    quadrature rotations on both sides, against the oracle at the planted
    centres and random interior voxels."""
    import numpy as np
    import synth
    import torch
    quad = synth.super_fibonacci_quaternions(ERROR_ROTATIONS)
    wts = np.full(len(quad), 1.0 / len(quad))
    s = wl.template.shape[0]
    rng = np.random.default_rng(seed)
    pts = np.concatenate([wl.positions[:n_planted],
                          random_interior(wl.volume.shape, s, n_random, rng)]).astype(np.int64)
    n_pl = min(n_planted, len(wl.positions))
    Z, Y, X = wl.volume.shape
    comp, desc = ttm.build_template(wl.template, wl.mask, wl.n_order, quad.astype(np.float32))
    vol = torch.from_numpy(wl.volume).cuda()
    got = {}
    for name, (opts, _) in plans.items():
        m = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)], opts=opts)
        m.run([vol])
        torch.cuda.synchronize()
        if ttm.ttm_plan_device_status(m.plan, m.ws) != 0:
            raise RuntimeError("device status of the error run")
        got[name] = gpu_maps_at(m, pts)
        m.close()
        del m
        torch.cuda.empty_cache()
    del vol, comp
    torch.cuda.empty_cache()
    T = pool.tensor_template(wl.template, wl.mask, quad, wts, "e")
    pool.stage(wl.volume, T, wl.mask)
    ora = pool.voxels(pts, float(np.var(wl.volume.astype(np.float64))))
    truth = np.asarray(wl.planted_quats[:n_pl], dtype=np.float64)
    out = {name: error_stats(got[name], ora, wl.n_order, n_pl, tol, truth)
           for name, (_, tol) in plans.items()}
    for v in out.values():
        v["quadrature_rotations"] = ERROR_ROTATIONS
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        loaded = [r for r in rows if (num(r[4]) or 0) >= 50] or rows
        sm = [num(r[1]) for r in loaded if num(r[1]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in loaded:
            for k, name in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=num(loaded[0][2]), reasons=sorted(reasons),
                    samples=len(rows), samples_under_load=len(loaded))


def source_hash(names) -> str:
    h = hashlib.sha1()
    for n in names:
        p = os.path.join(ROOT, "paper_2311_07561_gb300", "csrc", n)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:12]


def max_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """The largest of every rank's value (a replicated job ends with its
    slowest rank); the value itself on a single process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, steps: int, world: int, t_max_ms: float) -> float:
    """Units all ranks processed per second of the slowest rank's time."""
    return units_per_rank * steps * world / (t_max_ms * 1e-3)


def a5_flop_per_voxel(K: int) -> float:
    """Planned work of the score + rotation step per interior voxel: 32 start
    evaluations of phi (5 FP32 FLOP per component) and ~30 power iterations
    (8 FLOP per component): K x (32 x 5 + 30 x 8) = 400 K (14 k at n = 4,
    33.6 k at n = 6)."""
    return 400.0 * K


def refinement_flop_per_voxel(K: int, n_cand: int | None = None, newton: int | None = None,
                              refined: int | None = None) -> float:
    """FP32 FLOP of this build's refinement per interior voxel: every candidate
    takes 2 normalised power steps, each an evaluation of C x^(n-1) (10 ops
    per term of its 4 sums of KG terms), plus a third evaluation for phi when
    the candidates are ranked (more candidates than refined points); each
    refined point takes 1 + newton evaluations of C x^(n-2) (10 sums of KB
    terms) and newton 4x4 solves, the last of them an evaluation of
    C x^(n-1) instead from order 6 on.  Defaults: the order's budget."""
    c0, r0, nw0 = budget(K)
    n_cand = c0 if n_cand is None else n_cand
    newton = nw0 if newton is None else newton
    refined = r0 if refined is None else refined
    n_ord = {10: 2, 35: 4, 84: 6, 165: 8}.get(K, 4)
    KB = (n_ord + 1) * n_ord * (n_ord - 1) // 6
    KG = (n_ord + 2) * (n_ord + 1) * n_ord // 6
    hess = 2 * 10 * KB + 2 * KB + 40
    power = (3 if n_cand > refined else 2) * 10 * KG + 2 * 12
    # from order 6 on the last trial is an evaluation of C x^(n-1)
    last_grad = n_ord >= 6 and newton > 0
    newton_part = (newton * hess + 10 * KG if last_grad else (1 + newton) * hess) + newton * 150
    return float(n_cand * power + min(refined, n_cand) * newton_part)


def stage_traffic(name: str, K: int, storage: str, n_int: int):
    """ncu DRAM bytes per step of a stage, from the records whose sources are
    unchanged (None when there is no current record)."""
    total = 0.0
    for cls in STAGE_CLASSES.get(name, (name,)):
        rec = next((r for r in NCU_TRAFFIC.get(cls, ())
                    if r["K"] == K and r["storage"] == storage
                    and r["source_sha"] == source_hash(r["sources"])), None)
        if rec is None:
            return None
        total += rec["bytes_per_voxel"] * n_int
    return total


# the score + rotation step runs as two kernel classes (grid search and
# refinement) on two streams; its roofline is taken over both
STAGE_CLASSES = {"score_rotation": ("rotation_search", "rotation_polish")}


def kernel_ms(kern: dict) -> float:
    """Summed event time of the kernel classes (the rotation_stage span, which
    covers other classes' launches, left out)."""
    return sum(v["ms"] for k, v in kern.items() if k != "rotation_stage")


def roofline(kernels: dict, steps: int, geo: dict, peaks: dict) -> dict:
    """Roofline object of the stage with the largest share of the step.

    Work is algorithmic: FLOP for the score + rotation step (the planned a5
    count), bytes for the memory-bound stages (what each pass must read and
    write at the plan's storage precision), never a count of what the kernel
    happens to execute.  The score + rotation stage is timed by its span
    (rotation_stage: the wall time of the stage on the launch stream, its
    search and refinement overlapping on two streams), else as the sum of its
    two kernel classes' CUDA-event times (an upper bound)."""
    K, nvox, n_int = geo["K"], geo["nvox"], geo["n_interior"]
    per_step = {k: v["ms"] / steps for k, v in kernels.items()}
    span = per_step.pop("rotation_stage", None)
    stages = dict(per_step)
    if all(c in per_step for c in STAGE_CLASSES["score_rotation"]):
        stages["score_rotation"] = span if span else sum(per_step[c] for c in
                                                         STAGE_CLASSES["score_rotation"])
        for c in STAGE_CLASSES["score_rotation"]:
            stages.pop(c)
    name = max(stages, key=stages.get)
    ms = stages[name]
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops", 1900.0)
    cs = 4.0 if geo["mixed"] else 8.0           # bytes per stored complex value
    msz = 2.0 if geo["mixed"] else 4.0          # bytes per stored map value
    nh = geo["spectrum_values"]                 # half-spectrum values of the FFT box
    extra = {}
    if name == "score_rotation":
        work, scale, unit = a5_flop_per_voxel(K) * n_int, 1e12, "TFLOP/s"
        bound, peak = "alu", FP32_ALU_PEAK_TFLOPS
        peak_source = "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"
        ks = kernels.get("rotation_search", {}).get("ms", 0.0) / steps
        kp_ = kernels.get("rotation_polish", {}).get("ms", 0.0) / steps
        if ks > 0 and K in (35, 84):
            kp = 48 if K == 35 else 96
            gp = grid_points(K, geo["mixed"])
            mma = 2.0 * gp * kp * n_int / (ks * 1e-3) / 1e12
            extra["tensor_pipe"] = dict(kernel="rotation_search", achieved=round(mma, 2),
                                        peak=round(bf16, 1), unit="TFLOP/s", frac=round(mma / bf16, 4),
                                        work=f"dense FP16 grid contraction 2 x {gp} x KP per voxel")
        if kp_ > 0:
            ref = refinement_flop_per_voxel(K) * n_int / (kp_ * 1e-3) / 1e12
            extra["refinement_alu"] = dict(kernel="rotation_polish", achieved=round(ref, 2),
                                           peak=round(FP32_ALU_PEAK_TFLOPS, 2), unit="TFLOP/s",
                                           frac=round(ref / FP32_ALU_PEAK_TFLOPS, 4),
                                           work=f"{refinement_flop_per_voxel(K):.0f} FLOP per voxel "
                                                f"({refinement_text(K)})")
        work_note = f"{a5_flop_per_voxel(K):.0f} FLOP per interior voxel (400 K)"
    elif name == "direct_corr":
        if geo.get("tc_direct"):
            npad = (K + 15) // 16 * 16
            work, scale, unit = 2.0 * npad * geo["n_taps"] * n_int, 1e12, "TFLOP/s"
            bound, peak = "tensor", bf16
            peak_source = "measured dense bf16 (bf16_tflops); fp16 runs at the bf16 rate"
        else:
            work, scale, unit = 2.0 * K * geo["n_taps"] * nvox, 1e12, "TFLOP/s"
            bound, peak = "alu", FP32_ALU_PEAK_TFLOPS
            peak_source = "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"
        work_note = "2 x K x mask voxels per voxel"
    else:
        kz, ky = geo.get("keep_z_frac", 1.0), geo.get("keep_y_frac", 1.0)
        if name == "fft_inverse":
            # y pass: read the interior z planes of every product spectrum,
            # write their interior rows; x pass: read those rows, write the
            # interior of the real map
            work = K * (nh * cs * kz * (1.0 + 2.0 * ky) + n_int * msz)
            work_note = ("K x (interior planes of the half spectrum read, their interior rows "
                         "written and read again, interior map written)")
        elif name == "fft_spectrum_inverse":
            # image spectrum once per component group, every template spectrum
            # read, the interior z planes of every product written
            work = nh * (8.0 * geo.get("groups", 1) + K * cs * (1.0 + kz))
            work_note = ("image spectrum per component group + K x (template spectrum + "
                         "interior planes of the product)")
        elif name == "fft_forward":
            work = 4.0 * nvox + 40.0 * nh
            work_note = "volume read + three passes over the FP32 half spectrum"
        else:
            work = 8.0 * nvox
            work_note = "one read of the volume, one write of a map"
        scale, unit, bound, peak = 1e9, "GB/s", "hbm", hbm
        peak_source = "measured copy bandwidth (hbm_gbs)"
    achieved = work / (ms * 1e-3) / scale
    traffic = stage_traffic(name, K, "bf16" if geo["mixed"] else "f32", n_int)
    out = dict(kernel=name, bound=bound, achieved=round(achieved, 3), peak=round(peak, 2),
               unit=unit, frac=round(achieved / peak, 4),
               traffic=None if traffic is None else round(traffic),
               ms_per_step=round(ms, 4), work=work_note, peak_source=peak_source)
    out.update(extra)
    return out


def run_ours(args) -> None:
    import numpy as np
    import torch

    import paper_2311_07561_gb300 as ttm
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(ttm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ttm.load_library()

    wl = load_workload(args.workload)
    Z, Y, X = wl.volume.shape
    nvox = X * Y * Z
    # tensor template, once per template (timed separately, after one
    # untimed build that loads the modules and grows the allocator)
    ttm.build_template(wl.template, wl.mask, wl.n_order, wl.quadrature)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    comp, desc = ttm.build_template(wl.template, wl.mask, wl.n_order, wl.quadrature)
    ev1.record()
    torch.cuda.synchronize()
    build_ms = ev0.elapsed_time(ev1)
    opts = ttm.PlanOpts()
    opts.path = {"auto": 0, "direct": 1, "fft": 2}[args.path]
    opts.precision = ttm.TTM_PREC_MIXED if args.precision == "mixed" else ttm.TTM_PREC_FP32
    opts.rotation_chunks = args.rotation_chunks
    matcher = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)], opts=opts)
    path = ttm.ttm_plan_problem_path(matcher.plan, 0)
    vol = torch.from_numpy(wl.volume).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        matcher.run([vol])
    torch.cuda.synchronize()
    ttm.ttm_plan_timing(matcher.plan)            # discard warm-up records
    ttm.ttm_plan_enable_timing(matcher.plan, True)
    launches0 = matcher.launch_count()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("timed_steps")     # the launch list's range
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        matcher.run([vol])
        stops[k].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    status = ttm.ttm_plan_device_status(matcher.plan, matcher.ws)
    if status != 0:
        raise RuntimeError(f"device status {ttm.ttm_status_string(status)}")
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    total_ms = sum(step_ms)
    launches = matcher.launch_count() - launches0
    kern = {name: dict(ms=ms, launches=n) for name, (ms, n) in ttm.ttm_plan_timing(matcher.plan).items()}
    ttm.ttm_plan_enable_timing(matcher.plan, False)
    t_max = max_over_ranks(total_ms, dist, dev)
    value = job_rate(nvox, args.steps, world, t_max)

    # end to end through the public API: pinned host volume in, maps out,
    # every step.  HostStream keeps one plan and double-buffers the volume and
    # the maps, so step k's maps travel to the host and step k+1's volume
    # comes in while step k+1 is matched (depth 1: one step at a time).
    e2e = None
    if not args.no_e2e:
        depth = args.e2e_depth if args.e2e_depth > 0 else 2
        pin_in = torch.from_numpy(wl.volume).pin_memory()

        def pinned_maps():
            return [(torch.empty((Z, Y, X), dtype=torch.float32).pin_memory(),
                     torch.empty((Z, Y, X, 4), dtype=torch.float32).pin_memory(),
                     torch.empty((Z, Y, X), dtype=torch.float32).pin_memory())]
        hs = ttm.HostStream(matcher=matcher, depth=depth)
        outs = [pinned_maps() for _ in range(depth)]
        for k in range(max(args.warmup, depth)):
            hs.submit([pin_in], outs[k % depth])
        hs.join()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(args.steps):
            hs.submit([pin_in], outs[k % depth])
        hs.join()
        b.record(stream)
        b.synchronize()
        e_ms = a.elapsed_time(b)
        st_ = ttm.ttm_plan_device_status(hs.matcher.plan, hs.matcher.ws)
        if st_ != 0:
            raise RuntimeError(f"device status {ttm.ttm_status_string(st_)}")
        matcher = hs.matcher          # the plan stays in use for the rest of the run
        hs.outs, hs.vols = None, None
        del outs
        torch.cuda.empty_cache()
        e_ms = max_over_ranks(e_ms, dist, dev)
        e2e = dict(value=job_rate(nvox, args.steps, world, e_ms), unit=UNIT,
                   h2d_bytes_per_step=nvox * 4, d2h_bytes_per_step=nvox * 4 * 6,
                   pipeline_depth=depth,
                   note="pinned host volume in, score + quaternion + lambda maps out, every step; "
                        "one plan, volume and maps double-buffered (HostStream)")

    # classical template matching (Algorithm 1) at 1000 rotations on the same
    # volume and GPU: the comparator of the paper's speed-up claim
    classical = None
    if args.classical and path == 2 and args.workload in ("c2", "c2s", "c3"):
        import synth as _s
        qc = torch.from_numpy(_s.shoemake_quaternions(1000, 4).astype(np.float32)).to(dev)
        tc = torch.from_numpy(wl.template).to(dev)
        best = torch.empty((Z, Y, X), dtype=torch.float32, device=dev)
        barg = torch.empty((Z, Y, X), dtype=torch.int32, device=dev)
        cws = torch.empty(ttm.ttm_classical_workspace_size(matcher.plan, 0), dtype=torch.uint8,
                          device=dev)
        ttm.ttm_classical_ncc(matcher.plan, 0, tc, qc, 1000, vol, matcher.w[0], best, barg, cws)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        ttm.ttm_local_stats(matcher.plan, [vol], matcher.w, matcher.ws)
        ttm.ttm_classical_ncc(matcher.plan, 0, tc, qc, 1000, vol, matcher.w[0], best, barg, cws)
        b.record(stream)
        b.synchronize()
        c_ms = a.elapsed_time(b)
        classical = dict(rotations=1000, ms_per_volume=round(c_ms, 2),
                         voxels_per_s=nvox / (c_ms * 1e-3),
                         ttm_speedup=round(c_ms / (t_max / args.steps), 2),
                         note="classical NCC per rotation (rotate, normalise, FFT, conjugate "
                              "multiply, inverse FFT, running max) vs TTM score+rotation maps")
        del cws, best, barg

    # the other precision on the same volume (bf16 storage), for the FP32 vs
    # BF16 comparison of the metric
    # the paper's own use of the two outputs (Sec. 3.4): the score map for every
    # voxel, rotations only at its peaks (ttm_match_peaks), same plan and volume
    peaks_only = None
    if args.peaks_only:
        radius = int(wl.radius)
        for _ in range(max(1, args.warmup)):
            recs = matcher.match_peaks([vol], 0, 0.0, radius, 1 << 16)
        torch.cuda.synchronize()
        p_ms = 0.0
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            recs = matcher.match_peaks([vol], 0, 0.0, radius, 1 << 16)
            b.record(stream)
            b.synchronize()
            p_ms += a.elapsed_time(b)
        p_ms = max_over_ranks(p_ms, dist, dev)
        peaks_only = dict(value=job_rate(nvox, args.steps, world, p_ms), unit=UNIT,
                          ms_per_step=p_ms / args.steps, peaks=int(len(recs)),
                          threshold=0.0, nms_radius=radius,
                          note="local statistics, K correlations, score map, peaks "
                               "(ttm_match_peaks), rotation only at the peaks; includes the "
                               "host read of the peak list")

    mixed = None
    if args.mixed_compare and args.precision == "fp32" and path == 2:
        o2 = ttm.PlanOpts()
        o2.path = opts.path
        o2.precision = ttm.TTM_PREC_MIXED
        o2.rotation_chunks = args.rotation_chunks
        m2 = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)], opts=o2)
        for _ in range(args.warmup):
            m2.run([vol])
        torch.cuda.synchronize()
        m_ms = 0.0
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m2.run([vol])
            b.record(stream)
            b.synchronize()
            m_ms += a.elapsed_time(b)
        dscore = float((m2.score[0] - matcher.score[0]).abs().max())
        dlam = float((m2.lam[0] - matcher.lam[0]).abs().max())
        m_ms = max_over_ranks(m_ms, dist, dev)
        mixed = dict(value=job_rate(nvox, args.steps, world, m_ms), unit=UNIT,
                     ms_per_step=m_ms / args.steps, storage="bf16 spectra, products, maps",
                     max_abs_diff_vs_fp32=dict(score=dscore, **{"lambda": dlam}))
        m2.close()

    if rank != 0:
        matcher.close()
        if dist:
            dist.destroy_process_group()
        return
    peaks = load_peaks()
    box = tuple(ttm.ttm_plan_problem_fft_box(matcher.plan, 0)) if path == 2 else (X, Y, Z)
    n_taps = int(wl.mask.sum())
    s_edge = wl.template.shape[0]
    n_interior = max(X - s_edge + 1, 0) * max(Y - s_edge + 1, 0) * max(Z - s_edge + 1, 0)
    geo = dict(K=desc.K, nvox=nvox, n_interior=n_interior, n_taps=n_taps,
               mixed=args.precision == "mixed",
               spectrum_values=float((box[0] // 2 + 1) * box[1] * box[2]),
               keep_z_frac=max(Z - s_edge + 1, 0) / box[2], keep_y_frac=max(Y - s_edge + 1, 0) / box[1],
               groups=kern.get("fft_spectrum_inverse", {}).get("launches", args.steps) / args.steps,
               tc_direct=bool(ttm.ttm_plan_problem_tensor_direct(matcher.plan, 0)))
    rf = roofline(kern, args.steps, geo, peaks)
    matcher.close()
    del matcher, vol, flush
    torch.cuda.empty_cache()

    # the error of the maps against the FP64 oracle, and (for the headline
    # configuration) FP32 against bf16 storage at 512^3, both against the oracle
    errors, pair, cpu = None, None, None
    pool = None
    if world == 1 and (args.oracle_errors or not args.no_cpu_baseline):
        pool = OraclePool(wl.n_order)
    try:
        if pool is not None and args.oracle_errors:
            tol = 5e-3 if args.precision == "mixed" else 1e-4
            errors = oracle_error_runs(ttm, wl, {args.precision: (opts, tol)}, pool)[args.precision]
        if pool is not None and args.precision_pair and args.workload == "c5":
            pool.n_order = 4
            pair = precision_pair(ttm, args, pool, stream)
            pool.n_order = wl.n_order
    finally:
        if pool is not None:
            pool.close()
    if not args.no_cpu_baseline and world == 1:
        cores = oracle_cores()
        res = oracle_timing(args.workload, 8 * cores, 1, cores)
        cpu = cpu_baseline_obj(res, args.workload)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=t_max / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32" if args.precision == "fp32" else "bf16/f32",
        data="synthetic",
        config=dict(workload=WORKLOAD[args.workload], path={1: "direct", 2: "fft"}.get(path, path),
                    precision=("FP32 storage and arithmetic" if args.precision == "fp32" else
                               "bf16 storage of template spectra, product spectra and "
                               "correlation maps; FP32 arithmetic"),
                    fft_box=list(box) if path == 2 else None,
                    voxels=nvox, interior_voxels=n_interior, tensor_order=wl.n_order, K=desc.K,
                    mask_voxels=n_taps, rotation_grid=grid_points(desc.K, args.precision == "mixed"),
                    refinement=refinement_text(desc.K),
                    l2="flushed (256 MB write) before every timed step",
                    parallelism="replicas" if world > 1 else "single GPU",
                    template_build_ms=round(build_ms, 2), quadrature_rotations=desc.n_rot),
        roofline=rf, cpu_baseline=cpu, e2e=e2e, gpu_launches=launches,
        error_vs_oracle=errors, precision_pair=pair, classical=classical,
        mixed_precision=mixed, peaks_only=peaks_only,
        clocks=clk,
        rotation_stage_ms_per_step=(round(kern["rotation_stage"]["ms"] / args.steps, 4)
                                    if "rotation_stage" in kern else None),
        kernels={k: dict(ms_per_step=round(v["ms"] / args.steps, 4),
                         launches_per_step=v["launches"] / args.steps,
                         share=round(v["ms"] / kernel_ms(kern), 4))
                 for k, v in kern.items() if k != "rotation_stage"},
    )
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def load_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def time_steps(matcher, vol, steps: int, warmup: int, stream) -> float:
    """Mean CUDA-event milliseconds of `steps` runs after `warmup` runs, L2
    flushed before each."""
    import torch
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=vol.device)
    for _ in range(warmup):
        matcher.run([vol])
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        matcher.run([vol])
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / steps


def precision_pair(ttm, args, pool, stream) -> dict:
    """The 512^3 configuration (200 copies of a 40^3 template, SNR 0.3, order 4)
    matched with FP32 storage and with bf16 storage on the same GPU: voxels/s
    of each, and each one's error against the oracle (error runs with the
    ERROR_ROTATIONS quadrature on both sides)."""
    import torch
    wl = load_workload("c3")
    Z, Y, X = wl.volume.shape
    comp, desc = ttm.build_template(wl.template, wl.mask, wl.n_order, wl.quadrature)
    vol = torch.from_numpy(wl.volume).cuda()
    plans, out = {}, {}
    for name, prec, tol in (("fp32", ttm.TTM_PREC_FP32, 1e-4), ("bf16", ttm.TTM_PREC_MIXED, 5e-3)):
        o_ = ttm.PlanOpts()
        o_.path = ttm.TTM_PATH_FFT
        o_.precision = prec
        plans[name] = (o_, tol)
        m = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)], opts=o_)
        ms = time_steps(m, vol, 5, 2, stream)
        if ttm.ttm_plan_device_status(m.plan, m.ws) != 0:
            raise RuntimeError("device status of the 512^3 run")
        out[name] = dict(value=X * Y * Z / (ms * 1e-3), unit=UNIT, ms_per_step=round(ms, 3))
        m.close()
        del m
        torch.cuda.empty_cache()
    del vol, comp
    torch.cuda.empty_cache()
    errs = oracle_error_runs(ttm, wl, plans, pool)
    for name in out:
        out[name]["error_vs_oracle"] = errs[name]
    return dict(workload=WORKLOAD["c3"], steps=5, warmup=2, **out)


def run_batch(args) -> None:
    """Batch workload: every volume of the batch against every template, all
    problems in one plan (autotuned paths), each step one CUDA-graph replay."""
    import numpy as np
    import torch

    import paper_2311_07561_gb300 as ttm
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(ttm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ttm.load_library()

    bw = synth.batch_workload(args.workload)
    # one untimed build first (module loading, allocator growth)
    ttm.build_template(bw.templates[0], bw.masks[0], bw.n_order, bw.quadrature)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    tmpls = []
    for t, m in zip(bw.templates, bw.masks):
        comp, desc = ttm.build_template(t, m, bw.n_order, bw.quadrature)
        tmpls.append((comp, desc, m))
    ev1.record()
    torch.cuda.synchronize()
    build_ms = ev0.elapsed_time(ev1)
    opts = ttm.PlanOpts()
    opts.path = {"auto": ttm.TTM_PATH_TUNE, "direct": 1, "fft": 2}[args.path]
    opts.precision = ttm.TTM_PREC_MIXED if args.precision == "mixed" else ttm.TTM_PREC_FP32
    opts.rotation_chunks = args.rotation_chunks
    opts.batch_mib = args.batch_mib if args.batch_mib >= 0 else 32768
    dvols = [torch.from_numpy(v).to(dev) for v in bw.volumes]
    problems, vols = [], []
    for v, vol in enumerate(bw.volumes):
        for k in range(len(bw.templates)):
            problems.append((vol.shape[::-1], k))
            vols.append(dvols[v])
    t0 = time.perf_counter()
    matcher = ttm.Matcher(tmpls, problems, opts=opts)
    plan_s = time.perf_counter() - t0
    paths = [ttm.ttm_plan_problem_path(matcher.plan, p) for p in range(len(problems))]
    tuning = [ttm.ttm_plan_problem_tuning(matcher.plan, p) for p in range(len(problems))]
    waves = ttm.ttm_plan_waves(matcher.plan)
    nvox_total = sum(int(np.prod(d)) for d, _ in problems)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        matcher.run(vols)
    torch.cuda.synchronize()
    l0 = matcher.launch_count()
    graph = matcher.capture(vols)
    launches_per_step = (matcher.launch_count() - l0) // 2      # eager warm-up + capture
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("timed_steps")     # the launch list's range
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        graph.replay()
        stops[k].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    status = ttm.ttm_plan_device_status(matcher.plan, matcher.ws)
    if status != 0:
        raise RuntimeError(f"device status {ttm.ttm_status_string(status)}")
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, stops))
    t_max = max_over_ranks(total_ms, dist, dev)
    value = job_rate(nvox_total, args.steps, world, t_max)

    # per-kernel breakdown from one eager step outside the timed region
    ttm.ttm_plan_timing(matcher.plan)
    ttm.ttm_plan_enable_timing(matcher.plan, True)
    flush.zero_()
    matcher.run(vols)
    torch.cuda.synchronize()
    kern = {name: dict(ms=ms, launches=n) for name, (ms, n) in ttm.ttm_plan_timing(matcher.plan).items()}
    ttm.ttm_plan_enable_timing(matcher.plan, False)

    # end to end: every step copies the 16 pinned host volumes in and the
    # score, quaternion and lambda maps of all 64 problems out, through
    # HostStream on the same plan (one device copy per volume, so its
    # problems still share its spectra; volumes and maps double-buffered)
    e2e = None
    if not args.no_e2e:
        depth = args.e2e_depth if args.e2e_depth > 0 else 2
        n_t = len(bw.templates)
        pin_in = [torch.from_numpy(v).pin_memory() for v in bw.volumes]

        def pinned_maps():
            return [(torch.empty(tuple(d[::-1]), dtype=torch.float32).pin_memory(),
                     torch.empty(tuple(d[::-1]) + (4,), dtype=torch.float32).pin_memory(),
                     torch.empty(tuple(d[::-1]), dtype=torch.float32).pin_memory())
                    for d, _ in problems]
        outs = [pinned_maps() for _ in range(depth)]
        h2d = sum(v.nbytes for v in bw.volumes)
        d2h = sum(int(np.prod(d)) * 24 for d, _ in problems)
        hs = ttm.HostStream(matcher=matcher, depth=depth,
                            volume_of=[p // n_t for p in range(len(problems))])
        for k in range(max(args.warmup, depth)):
            hs.submit(pin_in, outs[k % depth])
        hs.join()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(args.steps):
            hs.submit(pin_in, outs[k % depth])
        hs.join()
        b.record(stream)
        b.synchronize()
        e_ms = max_over_ranks(a.elapsed_time(b), dist, dev)
        st_ = ttm.ttm_plan_device_status(matcher.plan, matcher.ws)
        if st_ != 0:
            raise RuntimeError(f"device status {ttm.ttm_status_string(st_)}")
        hs.outs, hs.vols = None, None
        del outs
        torch.cuda.empty_cache()
        e2e = dict(value=job_rate(nvox_total, args.steps, world, e_ms), unit=UNIT,
                   h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, pipeline_depth=depth,
                   note="pinned host volumes in, score + quaternion + lambda maps of every "
                        "problem out, every step; one plan, volumes and maps double-buffered "
                        "(HostStream, one device copy per volume)")

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = load_peaks()
    n_int = 0
    spec_vals = 0.0
    for p, ((X, Y, Z), k) in enumerate(problems):
        sk = bw.templates[k].shape[0]
        n_int += max(X - sk + 1, 0) * max(Y - sk + 1, 0) * max(Z - sk + 1, 0)
        if paths[p] == ttm.TTM_PATH_FFT:
            bx = ttm.ttm_plan_problem_fft_box(matcher.plan, p)
            spec_vals += float((bx[0] // 2 + 1) * bx[1] * bx[2])
    geo = dict(K=tmpls[0][1].K, nvox=nvox_total, n_interior=n_int, n_taps=0,
               mixed=args.precision == "mixed", spectrum_values=spec_vals, tc_direct=False)
    rf = roofline(kern, 1, geo, peaks)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = oracle_cores()
        cpu = cpu_baseline_obj(oracle_timing(args.workload, 8 * cores, 1, cores), args.workload)
    n_fft = sum(1 for p in paths if p == ttm.TTM_PATH_FFT)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=t_max / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32" if args.precision == "fp32" else "bf16/f32",
        data="synthetic",
        config=dict(workload=WORKLOAD[args.workload], problems=len(problems),
                    voxels=nvox_total, interior_voxels=n_int, tensor_order=bw.n_order,
                    K=tmpls[0][1].K, paths=dict(fft=n_fft, direct=len(paths) - n_fft),
                    tuned_problems=sum(1 for t in tuning if t[0] >= 0 and t[1] >= 0),
                    plan_seconds=round(plan_s, 2), template_build_ms=round(build_ms, 2),
                    graph="one CUDA graph replay per step (all problems)",
                    launches_per_step=launches_per_step,
                    resident_waves=(dict(batch_mib=opts.batch_mib, waves=len(waves),
                                         first_problems=waves,
                                         workspace_gib=round(matcher.ws.numel() / 2**30, 2))
                                    if waves else None),
                    rotation_grid=2048, refinement=refinement_text(tmpls[0][1].K),
                    l2="flushed (256 MB write) before every timed step",
                    parallelism="replicas" if world > 1 else "single GPU",
                    quadrature_rotations=int(len(bw.quadrature))),
        roofline=rf, cpu_baseline=cpu, e2e=e2e, gpu_launches=launches_per_step * args.steps,
        clocks=clk,
        kernels={k: dict(ms_per_step=round(v["ms"], 4), launches_per_step=v["launches"],
                         share=round(v["ms"] / kernel_ms(kern), 4))
                 for k, v in kern.items() if k != "rotation_stage"},
        rotation_stage_ms_per_step=(round(kern["rotation_stage"]["ms"], 4)
                                    if "rotation_stage" in kern else None),
        kernels_note="per-kernel times from one eager (not graph) step outside the timed region",
    )
    print(json.dumps(line), flush=True)
    matcher.close()
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# order / quadrature sweep (Sec. 3: the tensor order n and the quadrature of
# the tensor template set the rotation accuracy; Sec. 5 compares against
# classical matching at 7112 and 45123 sampled rotations)
# ---------------------------------------------------------------------------

SWEEP_TTM = ((2, 10000), (4, 1000), (4, 10000), (4, 20000), (6, 10000), (6, 20000), (8, 10000))
SWEEP_CLASSICAL = (1000, 7112)


def _angle_deg(q1, q2):
    """Angle of the rotation q1^-1 q2 for unit quaternions (q and -q alike)."""
    import numpy as np
    d = np.abs(np.sum(np.asarray(q1, np.float64) * np.asarray(q2, np.float64), axis=-1))
    return np.degrees(2.0 * np.arccos(np.clip(d, 0.0, 1.0)))


def _err_stats(ang):
    import numpy as np
    return dict(median_deg=round(float(np.median(ang)), 3),
                p90_deg=round(float(np.percentile(ang, 90)), 3),
                max_deg=round(float(np.max(ang)), 3),
                within_1deg=round(float(np.mean(ang <= 1.0)), 3),
                within_5deg=round(float(np.mean(ang <= 5.0)), 3))


def run_order_sweep(args) -> None:
    import numpy as np
    import torch

    import paper_2311_07561_gb300 as ttm
    import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    if not os.path.exists(ttm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ttm.load_library()
    wl = load_workload("c2")
    Z, Y, X = wl.volume.shape
    nvox = X * Y * Z
    pos = wl.positions                       # (P, 3) as (x, y, z)
    truth = wl.planted_quats
    vol = torch.from_numpy(wl.volume).to(dev)
    stream = torch.cuda.current_stream()
    steps = max(1, args.steps)
    rows = []
    for n, n_rot in SWEEP_TTM:
        quad = synth.super_fibonacci_quaternions(n_rot).astype(np.float32)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        comp, desc = ttm.build_template(wl.template, wl.mask, n, quad)
        e1.record(stream)
        torch.cuda.synchronize()
        build_ms = e0.elapsed_time(e1)
        m = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)])
        for _ in range(max(1, args.warmup)):
            m.run([vol])
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            m.run([vol])
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        status = ttm.ttm_plan_device_status(m.plan, m.ws)
        if status != 0:
            raise RuntimeError(f"device status {ttm.ttm_status_string(status)}")
        q = m.quat[0].cpu().numpy()[pos[:, 2], pos[:, 1], pos[:, 0]]
        rows.append(dict(n=n, K=desc.K, quadrature_rotations=n_rot, template_build_ms=round(build_ms, 1),
                         ms_per_step=round(ms, 3), voxels_per_s=nvox / (ms * 1e-3),
                         rotation_error=_err_stats(_angle_deg(q, truth))))
        m.close()
        del comp
        torch.cuda.empty_cache()
    # classical matching on the same volume: the best of R sampled rotations
    opts = ttm.PlanOpts()
    opts.path = ttm.TTM_PATH_FFT
    comp, desc = ttm.build_template(wl.template, wl.mask, 4, wl.quadrature)
    m = ttm.Matcher([(comp, desc, wl.mask)], [((X, Y, Z), 0)], opts=opts)
    ttm.ttm_local_stats(m.plan, [vol], m.w, m.ws)
    tc = torch.from_numpy(wl.template).to(dev)
    best = torch.empty((Z, Y, X), dtype=torch.float32, device=dev)
    barg = torch.empty((Z, Y, X), dtype=torch.int32, device=dev)
    cws = torch.empty(ttm.ttm_classical_workspace_size(m.plan, 0), dtype=torch.uint8, device=dev)
    classical = []
    for R in SWEEP_CLASSICAL:
        qs = synth.shoemake_quaternions(R, 4).astype(np.float32)
        qc = torch.from_numpy(qs).to(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ttm.ttm_classical_ncc(m.plan, 0, tc, qc, R, vol, m.w[0], best, barg, cws)
        b.record(stream)
        b.synchronize()
        j = barg.cpu().numpy()[pos[:, 2], pos[:, 1], pos[:, 0]]
        classical.append(dict(rotations=R, ms_per_volume=round(a.elapsed_time(b), 2),
                              rotation_error=_err_stats(_angle_deg(qs[j], truth))))
    m.close()
    line = dict(metric="rotation error at planted copies vs tensor order and quadrature size",
                unit="degrees", data="synthetic",
                config=dict(workload=WORKLOAD["c2"], copies=int(len(pos)), path="auto",
                            rotation_grid=2048, classical_rotations="Shoemake-uniform random"),
                ttm=rows, classical=classical)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.order_sweep:
        run_order_sweep(args)
    elif args.workload in BATCH_WORKLOADS:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
