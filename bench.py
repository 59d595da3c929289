#!/usr/bin/env python
"""Throughput of tensorial template matching on GB300: tomogram voxels/s of
the TTM score + rotation maps.

One step = local statistics + correlation with the K tensor components +
per-voxel Frobenius score and dominant Z-eigenvector rotation, over one
synthetic 256^3 FP32 tomogram (50 planted copies of a 32^3 lowpassed blob
template, SNR 0.5, mask radius 15, order n = 4, K = 35).  The tensor template
is built once before timing (reported separately).  Inputs are resident in
HBM when the timed region starts; L2 is flushed (256 MB write) before every
timed step, outside the step's events.

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
WORKLOAD_OVERRIDES = dict(c2s=("c2", dict(shape_zyx=(128, 128, 128), copies=8)))


def load_workload(name: str, **extra):
    import synth
    base, over = WORKLOAD_OVERRIDES.get(name, (name, {}))
    return synth.config_workload(base, **dict(over, **extra))
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
# the refinement's defaults: 8 candidates take two power steps, the 4 best of
# the points reached take 3 Newton steps
CANDIDATES, REFINED, NEWTON_STEPS = 8, 4, 3
REFINEMENT = (f"{CANDIDATES} candidates x 2 power steps, the {REFINED} best x "
              f"{NEWTON_STEPS} Newton steps")
L2_FLUSH_BYTES = 256 << 20

# Measured DRAM traffic of a kernel class from one ncu capture, per interior
# voxel, with the hash of the sources it was taken on; reported (times the
# interior voxels of one launch) only while those sources are unchanged and
# for the captured kind of launch: order 4 (K = 35) over FP32 maps.
NCU_TRAFFIC: dict = {
    # ncu (dram__bytes_read.sum + dram__bytes_write.sum) of the 128^3 case,
    # 912 673 interior voxels in one launch each
    "rotation_polish": dict(bytes_per_voxel=(193201664 + 9929728) / 912673, K=35,
                            source_sha="9cb54c7dd779"),
    # (the search kernel is unchanged since this capture; the one later edit of
    # k_rotation.cuh is the refinement's candidate count, kRefine)
    "rotation_search": dict(bytes_per_voxel=(173783808 + 12853504) / 912673, K=35,
                            source_sha="047846cd439c"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c2s", "c3", "c4", "c5"])
    ap.add_argument("--path", default="auto", choices=["auto", "direct", "fft"])
    ap.add_argument("--precision", default=None, choices=["fp32", "mixed"],
                    help="storage of spectra/products/correlation maps on the FFT path "
                         "(default fp32; mixed for c5, whose FP32 maps and spectra exceed HBM)")
    ap.add_argument("--mixed-compare", action=argparse.BooleanOptionalAction, default=True,
                    help="with fp32, also time the mixed-precision plan on the same volume")
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
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="internal: run the oracle on this many sampled voxels and print JSON")
    ap.add_argument("--sample-steps", type=int, default=1)
    ap.add_argument("--order-sweep", action="store_true",
                    help="rotation error at the planted copies of the 256^3 volume against the "
                         "tensor order n and the quadrature size, beside classical NCC at 1000 "
                         "and 7112 sampled rotations; prints its own JSON line")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "mixed" if args.workload == "c5" else "fp32"
    return args


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm); runs without touching the GPU
# ---------------------------------------------------------------------------

def cpu_sample(workload: str, n_vox: int, steps: int) -> dict:
    import numpy as np
    import synth
    from oracle import ttm_oracle as o
    if workload in BATCH_WORKLOADS:
        # the batch's first volume with its 32^3 template (cost per voxel is
        # set by the template and the order, not by the data)
        cfg = synth.BATCH_CONFIGS[workload]
        bw = synth.batch_workload(workload, shapes_zyx=cfg["shapes_zyx"][:1], sizes=(32,),
                                  n_rot=300)
        wl = synth.Workload("batch-sample", bw.volumes[0], bw.templates[0], bw.masks[0],
                            bw.radii[0], bw.n_order, bw.quadrature, bw.weights,
                            bw.positions[0][0], bw.planted_quats[0][0], 0.0, bw.snr)
    else:
        # the per-voxel cost of the oracle is set by the template box and the
        # order, so the large configs are sampled from a smaller volume
        wl = load_workload(workload, n_rot=300, **CPU_SAMPLE_SHAPES.get(workload, {}))
    s = wl.template.shape[0]
    c = s // 2
    T = o.tensor_template(wl.template, wl.mask, wl.quadrature.astype(np.float64), wl.weights,
                          wl.n_order)
    var_f = float(np.var(wl.volume.astype(np.float64)))
    rng = np.random.default_rng(11)
    Z, Y, X = wl.volume.shape
    times = []
    for _ in range(steps):
        pts = np.stack([rng.integers(c, X - s + c + 1, n_vox), rng.integers(c, Y - s + c + 1, n_vox),
                        rng.integers(c, Z - s + c + 1, n_vox)], axis=1)
        t0 = time.perf_counter()
        w, C = o.components_at(wl.volume, T, wl.mask, pts, var_f=var_f)
        o.frobenius_score(C.T, wl.n_order)
        o.dominant_z_eigenpair(C, wl.n_order)
        times.append(time.perf_counter() - t0)
    return dict(times=times, n_vox=n_vox)


def run_cpu_sample(workload: str, n_vox: int, steps: int) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", workload,
           "--cpu-sample", str(n_vox), "--sample-steps", str(steps)]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_obj(res: dict, workload: str = "") -> dict:
    tot = sum(res["times"])
    per_vox = tot / (res["n_vox"] * len(res["times"]))
    where = "the same workload"
    if workload in CPU_SAMPLE_SHAPES:
        where = (f"a {'x'.join(map(str, CPU_SAMPLE_SHAPES[workload]['shape_zyx'][::-1]))} volume "
                 "with the same template, order and mask")
    elif workload in BATCH_WORKLOADS:
        where = "the batch's first volume with its 32^3 template"
    return dict(value=1.0 / per_vox, unit=UNIT, cores=1, kind="oracle",
                sample=f"{len(res['times'])} x {res['n_vox']} random interior voxels of {where}: "
                       "local statistics, K component correlations by direct sum, "
                       "Frobenius score and dominant Z-eigenpair (FP64 numpy oracle, one BLAS "
                       f"thread); {tot:.1f} s of CPU work; tensor template built beforehand")


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


def roofline(kernels: dict, steps: int, nvox: int, K: int, n_taps: int, n_grid: int,
             n_cand: int, newton: int, peaks: dict, spectrum_bytes: float = 0.0,
             n_interior: int | None = None, tc_direct: bool = False,
             fp32_maps: bool = True) -> dict:
    """Roofline object for the kernel class with the largest share.  The
    rotation kernels visit only the interior voxels (n_interior)."""
    n_int = nvox if n_interior is None else n_interior
    name = max(kernels, key=lambda k: kernels[k]["ms"])
    ms_launch = kernels[name]["ms"] / max(kernels[name]["launches"], 1)
    launches_per_step = kernels[name]["launches"] / steps
    src = []
    if name == "direct_corr" and tc_direct:
        npad = (K + 15) // 16 * 16
        work = 2.0 * npad * n_taps * n_int / launches_per_step
        bound, peak, unit, scale = "tensor", peaks.get("bf16_tflops", 1900.0), "TFLOP/s", 1e12
        src = ["k_direct_tc.cu"]
        peak_source = "measured dense bf16 (MEASURED_PEAKS.json bf16_tflops); fp16 runs at the bf16 rate"
    elif name == "direct_corr":
        work = 2.0 * K * n_taps * nvox / launches_per_step
        bound, peak, unit, scale = "alu", FP32_ALU_PEAK_TFLOPS, "TFLOP/s", 1e12
        src = ["k_direct.cu"]
        peak_source = "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"
    elif name == "rotation_search" and K in (35, 84) and n_grid == 2048:
        kp = 48 if K == 35 else 96                               # K + constant column, padded
        work = 2.0 * n_grid * kp * n_int / launches_per_step     # FP16 MMA
        bound, peak, unit, scale = "tensor", peaks.get("bf16_tflops", 1900.0), "TFLOP/s", 1e12
        src = ["k_search_tc.cu", "k_rotation.cuh"]
        peak_source = "measured dense bf16 (MEASURED_PEAKS.json bf16_tflops); fp16 runs at the bf16 rate"
    elif name in ("rotation_search", "rotation_polish"):
        # order n from K = C(n+3, 3); H = C x^(n-2) has 10 entries of KB terms
        n_ord = {10: 2, 35: 4, 84: 6, 165: 8}.get(K, 4)
        KB = (n_ord + 1) * n_ord * (n_ord - 1) // 6
        KG = (n_ord + 2) * (n_ord + 1) * n_ord // 6
        # every candidate: 3 evaluations of C x^(n-1) and 2 normalisations; the
        # REFINED best: 1 + newton evaluations of C x^(n-2) and newton Newton solves
        power = 3 * 10 * KG + 2 * 12
        newton_part = (1 + newton) * (2 * 10 * KB + 2 * KB + 40) + newton * 150
        per_vox = n_cand * power + min(REFINED, n_cand) * newton_part
        work = ((2.0 * n_grid * K + 2 * K) if name == "rotation_search" else per_vox) \
            * n_int / launches_per_step
        bound, peak, unit, scale = "alu", FP32_ALU_PEAK_TFLOPS, "TFLOP/s", 1e12
        src = ["k_rotation.cuh", "k_rotation.cu", "k_rotation_n4.cu"]
        peak_source = "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"
    else:
        # memory-bound stage: algorithmic bytes
        if name == "local_stats":
            per = 8.0 * nvox
        elif name == "fft_spectrum_inverse":
            per = spectrum_bytes * (1 + 2 * K)
        elif name == "fft_inverse":
            per = spectrum_bytes * 3 * K + 4.0 * K * nvox
        else:
            per = 8.0 * nvox
        work = per / launches_per_step
        bound, peak, unit, scale = "hbm", peaks.get("hbm_gbs", 6800.0), "GB/s", 1e9
        peak_source = "measured (MEASURED_PEAKS.json hbm_gbs)"
    achieved = work / (ms_launch * 1e-3) / scale
    traffic = None
    rec = NCU_TRAFFIC.get(name)
    if (rec and src and fp32_maps and rec["K"] == K
            and rec.get("source_sha") == source_hash(src)):
        traffic = round(rec["bytes_per_voxel"] * n_int / launches_per_step)
    return dict(kernel=name, bound=bound, achieved=round(achieved, 3), peak=round(peak, 2),
                unit=unit, frac=round(achieved / peak, 4), traffic=traffic,
                ms_per_launch=round(ms_launch, 4), peak_source=peak_source)


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
    # tensor template, once per template (timed separately)
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
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        matcher.run([vol])
        stops[k].record(stream)
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

    # end to end through the public API: pinned host volume in, maps out.
    # With depth > 1 consecutive steps run on HostPipeline's streams, so step
    # k's maps travel to the host while step k+1 is copied in and matched
    # (every step still moves its own input and result); depth 1 repeats
    # Matcher.match_host step after step.
    e2e = None
    if not args.no_e2e:
        depth = args.e2e_depth if args.e2e_depth > 0 else (1 if args.workload == "c5" else 2)
        pin_in = torch.from_numpy(wl.volume).pin_memory()

        def pinned_maps():
            return [(torch.empty((Z, Y, X), dtype=torch.float32).pin_memory(),
                     torch.empty((Z, Y, X, 4), dtype=torch.float32).pin_memory(),
                     torch.empty((Z, Y, X), dtype=torch.float32).pin_memory())]
        if depth == 1:
            pin_out = pinned_maps()
            for _ in range(max(1, args.warmup)):
                matcher.match_host([None], pinned_in=[pin_in], pinned_out=pin_out)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            e_ms = 0.0
            for k in range(args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                matcher.match_host([None], pinned_in=[pin_in], pinned_out=pin_out)
                b.record(stream)
                b.synchronize()
                e_ms += a.elapsed_time(b)
        else:
            pipe = ttm.HostPipeline([(comp, desc, wl.mask)], [((X, Y, Z), 0)], opts=opts,
                                    depth=depth)
            outs = [pinned_maps() for _ in range(depth)]
            for k in range(max(args.warmup, depth)):
                pipe.submit([pin_in], outs[k % depth])
            pipe.join()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for k in range(args.steps):
                pipe.submit([pin_in], outs[k % depth])
            pipe.join()
            b.record(stream)
            b.synchronize()
            e_ms = a.elapsed_time(b)
            for m_ in pipe.matchers:
                st_ = ttm.ttm_plan_device_status(m_.plan, m_.ws)
                if st_ != 0:
                    raise RuntimeError(f"device status {ttm.ttm_status_string(st_)}")
            pipe.close()
            del outs
        e_ms = max_over_ranks(e_ms, dist, dev)
        e2e = dict(value=job_rate(nvox, args.steps, world, e_ms), unit=UNIT,
                   h2d_bytes_per_step=nvox * 4, d2h_bytes_per_step=nvox * 4 * 6,
                   pipeline_depth=depth,
                   note="pinned host volume in, score + quaternion + lambda maps out, every step"
                        + ("; consecutive steps overlap on HostPipeline streams" if depth > 1 else ""))

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
        if dist:
            dist.destroy_process_group()
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    n_taps = int(wl.mask.sum())
    Xh = X // 2 + 1
    spec_bytes = 8.0 * Xh * Y * Z if path == 2 else 0.0
    s_edge = wl.template.shape[0]
    n_interior = max(X - s_edge + 1, 0) * max(Y - s_edge + 1, 0) * max(Z - s_edge + 1, 0)
    rf = roofline(kern, args.steps, nvox, desc.K, n_taps, 2048, CANDIDATES, NEWTON_STEPS, peaks, spec_bytes,
                  n_interior, ttm.ttm_plan_problem_tensor_direct(matcher.plan, 0),
                  fp32_maps=args.precision == "fp32")
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_obj(run_cpu_sample(args.workload, 128, 2), args.workload)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=t_max / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32" if args.precision == "fp32" else "bf16/f32",
        data="synthetic",
        config=dict(workload=WORKLOAD[args.workload], path={1: "direct", 2: "fft"}.get(path, path),
                    voxels=nvox, interior_voxels=n_interior, tensor_order=wl.n_order, K=desc.K, mask_voxels=n_taps,
                    rotation_grid=2048, refinement=REFINEMENT,
                    l2="flushed (256 MB write) before every timed step",
                    parallelism="replicas" if world > 1 else "single GPU",
                    template_build_ms=round(build_ms, 2), quadrature_rotations=desc.n_rot),
        roofline=rf, cpu_baseline=cpu, e2e=e2e, gpu_launches=launches, classical=classical,
        mixed_precision=mixed, peaks_only=peaks_only,
        clocks=clk,
        kernels={k: dict(ms_per_step=round(v["ms"] / args.steps, 4),
                         launches_per_step=v["launches"] / args.steps,
                         share=round(v["ms"] / sum(x["ms"] for x in kern.values()), 4))
                 for k, v in kern.items()},
    )
    print(json.dumps(line), flush=True)
    matcher.close()
    if dist:
        dist.destroy_process_group()


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
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        graph.replay()
        stops[k].record(stream)
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

    e2e = None
    if not args.no_e2e:
        pin_in = [torch.from_numpy(v).pin_memory() for v in bw.volumes]
        pin_out = [(torch.empty(tuple(d[::-1]), dtype=torch.float32).pin_memory(),
                    torch.empty(tuple(d[::-1]) + (4,), dtype=torch.float32).pin_memory(),
                    torch.empty(tuple(d[::-1]), dtype=torch.float32).pin_memory())
                   for d, _ in problems]
        h2d = sum(v.nbytes for v in bw.volumes)
        d2h = sum(int(np.prod(d)) * 24 for d, _ in problems)

        def e2e_step():
            for dv, hv in zip(dvols, pin_in):
                dv.copy_(hv, non_blocking=True)
            graph.replay()
            for p, (so, qo, lo) in enumerate(pin_out):
                so.copy_(matcher.score[p], non_blocking=True)
                qo.copy_(matcher.quat[p], non_blocking=True)
                lo.copy_(matcher.lam[p], non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e_ms = 0.0
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            b.synchronize()
            e_ms += a.elapsed_time(b)
        e_ms = max_over_ranks(e_ms, dist, dev)
        e2e = dict(value=job_rate(nvox_total, args.steps, world, e_ms), unit=UNIT,
                   h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    n_int = 0
    spec_bytes = 0.0
    for (X, Y, Z), k in problems:
        sk = bw.templates[k].shape[0]
        n_int += max(X - sk + 1, 0) * max(Y - sk + 1, 0) * max(Z - sk + 1, 0)
        spec_bytes += 8.0 * (X // 2 + 1) * Y * Z
    rf = roofline(kern, 1, nvox_total, tmpls[0][1].K, 0, 2048, CANDIDATES, NEWTON_STEPS, peaks,
                  spec_bytes / max(1, len(problems)), n_int, fp32_maps=args.precision == "fp32")
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_obj(run_cpu_sample(args.workload, 128, 2), args.workload)
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
                    rotation_grid=2048, refinement=REFINEMENT,
                    l2="flushed (256 MB write) before every timed step",
                    parallelism="replicas" if world > 1 else "single GPU",
                    quadrature_rotations=int(len(bw.quadrature))),
        roofline=rf, cpu_baseline=cpu, e2e=e2e, gpu_launches=launches_per_step * args.steps,
        clocks=clk,
        kernels={k: dict(ms_per_step=round(v["ms"], 4), launches_per_step=v["launches"],
                         share=round(v["ms"] / sum(x["ms"] for x in kern.values()), 4))
                 for k, v in kern.items()},
        kernels_note="per-kernel times from one eager (not graph) step outside the timed region",
    )
    print(json.dumps(line), flush=True)
    matcher.close()
    if dist:
        dist.destroy_process_group()


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_vox = 128
    steps = args.warmup + args.steps
    res = run_cpu_sample(args.workload, n_vox, steps)
    times = res["times"][args.warmup:]
    total = sum(times)
    value = n_vox * len(times) / total
    cpu = cpu_baseline_obj(dict(times=times, n_vox=n_vox), args.workload)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
        warmup=args.warmup, ms_per_step=1e3 * total / len(times), higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(workload=WORKLOAD[args.workload], step=f"{n_vox} sampled voxels"),
        impl="reference", cpu_baseline=cpu,
        e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0),
    )
    print(json.dumps(line), flush=True)


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
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.workload, args.cpu_sample, args.sample_steps)))
        return
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
