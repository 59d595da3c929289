"""Convenience layer over the C ABI: owns torch-allocated buffers and a plan.

A :class:`Matcher` is what a user calls: it builds one plan for a batch of
(volume, template) problems, keeps the output maps and the workspace on the
GPU, and runs local statistics + correlation/score/rotation on a stream.  All
computation happens in libttm.so.
"""

from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _binding as B


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_2311_07561_gb300 needs a CUDA device (sm_103a); none is visible")
    return torch


def build_template(template, mask, n_order: int, quats, weights=None, stream=None):
    """Fold a template into its K tensor components on the GPU (Sec. 3.2).

    template, mask: (s, s, s) float32 arrays (numpy or torch); quats: (n_rot, 4).
    Returns (components (K, s, s, s) cuda tensor, TTDesc).
    """
    torch = _torch()
    dev = torch.device("cuda")
    t = torch.as_tensor(np.asarray(template, dtype=np.float32)).to(dev).contiguous()
    m = torch.as_tensor(np.asarray(mask, dtype=np.float32)).to(dev).contiguous()
    q = torch.as_tensor(np.asarray(quats, dtype=np.float32)).to(dev).contiguous()
    wt = None
    if weights is not None:
        wt = torch.as_tensor(np.asarray(weights, dtype=np.float32)).to(dev).contiguous()
    s = int(t.shape[0])
    n_rot = int(q.shape[0])
    K = (n_order + 1) * (n_order + 2) * (n_order + 3) // 6
    comp = torch.empty((K, s, s, s), dtype=torch.float32, device=dev)
    ws = torch.empty(B.ttm_build_workspace_size(s, n_order, n_rot), dtype=torch.uint8, device=dev)
    desc = B.ttm_build_tensor_template(t, m, s, n_order, q, wt, n_rot, comp, ws, stream)
    return comp, desc


class Matcher:
    """A plan over a batch of problems plus its output buffers.

    templates: list of (components, desc, mask) with components/mask on the GPU
    problems:  list of ((X, Y, Z), template_index)
    """

    def __init__(self, templates: Sequence[Tuple], problems: Sequence[Tuple[Tuple[int, int, int], int]],
                 opts: Optional[B.PlanOpts] = None, want_lambda: bool = True, stream=None):
        torch = _torch()
        dev = torch.device("cuda")
        self._keep = [(c, torch.as_tensor(np.asarray(m, dtype=np.float32)).to(dev).contiguous()
                       if not hasattr(m, "data_ptr") else m) for c, _, m in templates]
        self.descs = [d for _, d, _ in templates]
        self.problems = [(tuple(int(v) for v in dims), int(k)) for dims, k in problems]
        self.plan = B.ttm_plan([p[0] for p in self.problems], [p[1] for p in self.problems],
                               self.descs, [c for c, _ in self._keep], [m for _, m in self._keep],
                               opts, stream)
        self.ws = torch.empty(B.ttm_plan_workspace_size(self.plan), dtype=torch.uint8, device=dev)
        self.w, self.score, self.quat, self.lam = [], [], [], []
        for (X, Y, Z), _ in self.problems:
            shape = (Z, Y, X)
            self.w.append(torch.empty(shape, dtype=torch.float32, device=dev))
            self.score.append(torch.empty(shape, dtype=torch.float32, device=dev))
            self.quat.append(torch.empty(shape + (4,), dtype=torch.float32, device=dev))
            self.lam.append(torch.empty(shape, dtype=torch.float32, device=dev) if want_lambda else None)
        self.want_lambda = want_lambda

    def _check_inputs(self, vols: Sequence, components_out: Optional[Sequence]) -> None:
        if len(vols) != len(self.problems):
            raise ValueError(f"expected {len(self.problems)} volumes, got {len(vols)}")
        for p, ((X, Y, Z), k) in enumerate(self.problems):
            v = vols[p]
            if tuple(v.shape) != (Z, Y, X) or not v.is_cuda or not v.is_contiguous() \
                    or v.dtype != self.w[p].dtype:
                raise ValueError(f"volume {p} must be a contiguous float32 cuda tensor of "
                                 f"shape (Z, Y, X) = {(Z, Y, X)}")
            if components_out is not None:
                c = components_out[p]
                if tuple(c.shape) != (self.descs[k].K, Z, Y, X) or not c.is_contiguous():
                    raise ValueError(f"components_out[{p}] must be (K, Z, Y, X) contiguous")

    def new_outputs(self):
        """A second set of output maps (w, score, quat, lambda lists, one per
        problem) for run(outputs=...)."""
        torch = _torch()
        dev = torch.device("cuda")
        w, score, quat, lam = [], [], [], []
        for (X, Y, Z), _ in self.problems:
            shape = (Z, Y, X)
            w.append(torch.empty(shape, dtype=torch.float32, device=dev))
            score.append(torch.empty(shape, dtype=torch.float32, device=dev))
            quat.append(torch.empty(shape + (4,), dtype=torch.float32, device=dev))
            lam.append(torch.empty(shape, dtype=torch.float32, device=dev) if self.want_lambda else None)
        return w, score, quat, lam

    def run(self, vols: Sequence, components_out: Optional[Sequence] = None, stream=None,
            outputs=None) -> None:
        """Local statistics, correlation, score and rotation for every problem;
        into the matcher's own maps, or into `outputs` (from new_outputs)."""
        self._check_inputs(vols, components_out)
        w, score, quat, lam = outputs if outputs is not None else (self.w, self.score, self.quat,
                                                                    self.lam)
        B.ttm_local_stats(self.plan, vols, w, self.ws, stream)
        B.ttm_correlate(self.plan, vols, w, score, quat, lam if self.want_lambda else None,
                        components_out, self.ws, stream)

    def capture(self, vols: Sequence):
        """Record run(vols) for every problem of the plan into one CUDA graph.

        One eager run on a side stream first (it sets the kernels' shared-memory
        attributes and loads the module), then the capture.  Replaying the
        returned torch.cuda.CUDAGraph recomputes every output map from the
        current contents of vols (same tensors, same addresses)."""
        torch = _torch()
        self._check_inputs(vols, None)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run(vols)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.run(vols)
        return graph

    def match_host(self, host_vols: Sequence[np.ndarray], pinned_in: Optional[List] = None,
                   pinned_out: Optional[List] = None, stream=None) -> Dict[str, List]:
        """End-to-end call from host memory: copy in, run, copy the maps out."""
        torch = _torch()
        dev = torch.device("cuda")
        vols = []
        for i, hv in enumerate(host_vols):
            src = pinned_in[i] if pinned_in is not None else torch.from_numpy(np.ascontiguousarray(hv, dtype=np.float32))
            vols.append(src.to(dev, non_blocking=True))
        self.run(vols, stream=stream)
        outs = {"score": [], "quat": [], "lambda": []}
        for i in range(len(self.problems)):
            if pinned_out is not None:
                so, qo, lo = pinned_out[i]
                so.copy_(self.score[i], non_blocking=True)
                qo.copy_(self.quat[i], non_blocking=True)
                if self.want_lambda and lo is not None:
                    lo.copy_(self.lam[i], non_blocking=True)
                outs["score"].append(so); outs["quat"].append(qo); outs["lambda"].append(lo)
            else:
                outs["score"].append(self.score[i].cpu())
                outs["quat"].append(self.quat[i].cpu())
                outs["lambda"].append(self.lam[i].cpu() if self.want_lambda else None)
        return outs

    def peaks(self, problem: int, threshold: float, radius: int, max_peaks: int, stream=None):
        return B.ttm_extract_peaks(self.plan, problem, self.score[problem], self.quat[problem],
                                   self.lam[problem], threshold, radius, max_peaks, self.ws, stream)

    def match_peaks(self, vols: Sequence, problem: int, threshold: float, radius: int,
                    max_peaks: int, stream=None):
        """Score map and the rotation at its peaks only, for one problem:
        local statistics, correlation, score, peaks, then the search and
        refinement at the peaks (no dense rotation maps).  Returns the peak
        records; self.score[problem] holds the score map."""
        self._check_inputs(vols, None)
        B.ttm_local_stats(self.plan, vols, self.w, self.ws, stream)
        return B.ttm_match_peaks(self.plan, problem, vols[problem], self.w[problem],
                                 self.score[problem], threshold, radius, max_peaks, self.ws,
                                 stream)

    def launch_count(self) -> int:
        return B.ttm_plan_launch_count(self.plan)

    def close(self) -> None:
        if self.plan:
            B.ttm_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipeline:
    """End-to-end matching of a stream of host volumes with the copies hidden.

    ``depth`` independent matchers (each its own plan, workspace and output
    maps) take consecutive steps on their own CUDA streams: while step k's
    maps travel to the host, step k+1's volume is copied in and matched.  Each
    step still copies its inputs from pinned host memory and reads its score,
    rotation and lambda maps back into the pinned host buffers given for it.
    Memory: ``depth`` plans and workspaces (template spectra, K correlation
    maps); use depth 1 where one set barely fits.

    templates, problems, opts: as for :class:`Matcher`.
    """

    def __init__(self, templates, problems, opts=None, depth: int = 2):
        torch = _torch()
        if depth < 1:
            raise ValueError("depth must be at least 1")
        self.matchers = [Matcher(templates, problems, opts=opts) for _ in range(depth)]
        self.streams = [torch.cuda.Stream() for _ in range(depth)]
        dev = torch.device("cuda")
        self.vols = [[torch.empty((Z, Y, X), dtype=torch.float32, device=dev)
                      for (X, Y, Z), _ in m.problems] for m in self.matchers]
        self._next = 0

    def submit(self, host_vols: Sequence, host_out: Sequence) -> None:
        """Queue one step: host_vols[v] (pinned float32 (Z, Y, X), one per
        volume index) in, and (score, quat, lambda) of every problem out into
        host_out[p] (pinned tensors of the map shapes).  Returns at once; the
        step is ordered after everything queued on the current stream before
        the call."""
        torch = _torch()
        i = self._next % len(self.matchers)
        self._next += 1
        m, st, dv = self.matchers[i], self.streams[i], self.vols[i]
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            for d, h in zip(dv, host_vols):
                d.copy_(h, non_blocking=True)
            m.run(dv)
            for p, (so, qo, lo) in enumerate(host_out):
                so.copy_(m.score[p], non_blocking=True)
                qo.copy_(m.quat[p], non_blocking=True)
                if lo is not None and m.lam[p] is not None:
                    lo.copy_(m.lam[p], non_blocking=True)

    def join(self) -> None:
        """Make the current stream wait for every queued step."""
        torch = _torch()
        cur = torch.cuda.current_stream()
        for st in self.streams:
            cur.wait_stream(st)

    def close(self) -> None:
        for m in self.matchers:
            m.close()


class HostStream:
    """End-to-end matching of a stream of host volumes with one plan.

    Where two plans do not fit (large volumes: the template spectra and the K
    correlation maps dominate the memory), one plan serves every step and only
    the inputs and outputs are double-buffered: the volume of step k+1 is
    copied in on a copy stream while step k is matched on the compute stream,
    and the maps of step k travel to the host on another copy stream while
    step k+1 is matched.  Every step still copies its own volume in from
    pinned host memory and its score, rotation and lambda maps out.  Memory
    beyond one Matcher: ``depth - 1`` more volumes and output sets.

    templates, problems, opts: as for :class:`Matcher`; or matcher: an
    existing Matcher to drive (its plan, workspace and maps are then shared
    with its other users).  volume_of: optional problem -> volume index; the
    problems of one volume then read one device copy of it (a batch of
    volumes x templates: one copy in per volume, and the plan shares the
    volume's spectra between its problems), and submit takes one host volume
    per index.
    """

    def __init__(self, templates=None, problems=None, opts=None, depth: int = 2, matcher=None,
                 volume_of: Optional[Sequence[int]] = None):
        if depth < 1:
            raise ValueError("depth must be at least 1")
        self.matcher = matcher if matcher is not None else Matcher(templates, problems, opts=opts)
        self._own = matcher is None
        m = self.matcher
        n_prob = len(m.problems)
        self.volume_of = list(range(n_prob)) if volume_of is None else [int(v) for v in volume_of]
        if len(self.volume_of) != n_prob:
            raise ValueError("volume_of needs one volume index per problem")
        shapes = {}
        for p, v in enumerate(self.volume_of):
            (X, Y, Z), _ = m.problems[p]
            if shapes.setdefault(v, (Z, Y, X)) != (Z, Y, X):
                raise ValueError(f"problems of volume {v} differ in size")
        self.n_vol = max(self.volume_of) + 1
        if sorted(shapes) != list(range(self.n_vol)):
            raise ValueError("volume indices must be 0 .. n-1")
        torch = _torch()
        dev = torch.device("cuda")
        self.outs = [(m.w, m.score, m.quat, m.lam)] + [m.new_outputs() for _ in range(depth - 1)]
        # per slot: one device copy per volume
        self.vols = [[torch.empty(shapes[v], dtype=torch.float32, device=dev)
                      for v in range(self.n_vol)] for _ in range(depth)]
        self.compute = torch.cuda.Stream()
        self.h2d = torch.cuda.Stream()
        self.d2h = torch.cuda.Stream()
        # per slot: inputs copied in, step computed, outputs copied out
        self.ev_in = [torch.cuda.Event() for _ in range(depth)]
        self.ev_done = [torch.cuda.Event() for _ in range(depth)]
        self.ev_out = [torch.cuda.Event() for _ in range(depth)]
        self.used = [False] * depth
        self.depth = depth
        self._next = 0

    def submit(self, host_vols: Sequence, host_out: Sequence) -> None:
        """Queue one step: host_vols[p] (pinned float32 (Z, Y, X)) in, and
        (score, quat, lambda) of every problem out into host_out[p] (pinned
        tensors of the map shapes).  Returns at once; the step is ordered after
        everything queued on the current stream before the call."""
        torch = _torch()
        i = self._next % self.depth
        self._next += 1
        cur = torch.cuda.current_stream()
        for st in (self.h2d, self.compute, self.d2h):
            st.wait_stream(cur)
        with torch.cuda.stream(self.h2d):
            if self.used[i]:
                self.h2d.wait_event(self.ev_done[i])      # the slot's volume is free
            for d, h in zip(self.vols[i], host_vols):
                d.copy_(h, non_blocking=True)
            self.ev_in[i].record(self.h2d)
        with torch.cuda.stream(self.compute):
            self.compute.wait_event(self.ev_in[i])
            if self.used[i]:
                self.compute.wait_event(self.ev_out[i])   # the slot's maps are on the host
            self.matcher.run([self.vols[i][v] for v in self.volume_of], stream=self.compute,
                             outputs=self.outs[i])
            self.ev_done[i].record(self.compute)
        with torch.cuda.stream(self.d2h):
            self.d2h.wait_event(self.ev_done[i])
            _, score, quat, lam = self.outs[i]
            for p, (so, qo, lo) in enumerate(host_out):
                so.copy_(score[p], non_blocking=True)
                qo.copy_(quat[p], non_blocking=True)
                if lo is not None and lam[p] is not None:
                    lo.copy_(lam[p], non_blocking=True)
            self.ev_out[i].record(self.d2h)
        self.used[i] = True

    def join(self) -> None:
        """Make the current stream wait for every queued step."""
        torch = _torch()
        cur = torch.cuda.current_stream()
        for st in (self.h2d, self.compute, self.d2h):
            cur.wait_stream(st)

    def close(self) -> None:
        if self._own:
            self.matcher.close()

