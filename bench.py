#!/usr/bin/env python
"""Benchmark of the LoD Gaussian render path on B300.

One step = one view of the 2M-leaf SH3 scene (70% ground, 30% boxes) on the
32-view aerial-to-street trajectory at 1920x1080: LoD select (upper BFS + SPT
cut), projection with SH colour, tile x depth sort, front-to-back blending,
mean-L1 loss against a seeded target, and the backward to sparse gradient rows
of the selected nodes.  The metric is views per second (fwd+bwd frames/s); the
forward-only rate and the per-stage device times are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lodgs|reference]

N > 1 runs under torchrun, one process per GPU; views are independent, so each
rank takes every N-th view (no collective on the data path).  --impl reference
times the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "frames/s & fwd+bwd step ms at 1080p (LoD splat); serving p50/p99 ms"
WORKLOAD = ("2,097,152-leaf SH3 scene (70% ground plane, 30% in 256 boxes), 32-view aerial-to-street path at "
            "1920x1080, tau 1 px; per view: LoD select + render + mean-L1 loss + backward to sparse node gradients")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=32)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="lodgs", choices=["lodgs", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--leaves", type=int, default=2_097_152)
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-lod-sweep", action="store_true")
    p.add_argument("--no-out-of-core", action="store_true")
    p.add_argument("--serving-leaves", type=int, default=50_000_000)
    p.add_argument("--serving-requests", type=int, default=4000)
    p.add_argument("--ooc-leaves", type=int, default=20_000_000)
    p.add_argument("--ooc-views", type=int, default=200)
    p.add_argument("--train-leaves", type=int, default=150_000_000)
    p.add_argument("--no-train-batch", action="store_true")
    p.add_argument("--no-densify", action="store_true")
    p.add_argument("--no-config1", action="store_true")
    p.add_argument("--streams", type=int, default=3,
                   help="views in flight at once in the timed steps (independent views, one stream each)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class _Nvml:
    """Minimal read-only NVML access through ctypes (libnvidia-ml.so.1)."""
    # clock-event reason bits of the public NVML API
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40, "hw_power_brake": 0x80}

    def __init__(self, index: int):
        import ctypes as C
        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = C.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(self.h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandleByIndex failed")
        self._reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sm_mhz(self) -> float:
        v = self.C.c_uint()
        self.lib.nvmlDeviceGetClockInfo(self.h, self.C.c_int(1), self.C.byref(v))     # NVML_CLOCK_SM
        return float(v.value)

    def max_sm_mhz(self) -> float:
        v = self.C.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.C.c_int(1), self.C.byref(v))
        return float(v.value)

    def reasons(self) -> int:
        v = self.C.c_ulonglong()
        self._reasons(self.h, self.C.byref(v))
        return int(v.value)


class ClockSampler:
    """Samples the SM clock and the clock-event reasons through NVML every 2 ms
    while the timed region runs (reads only; nothing is set)."""

    def __init__(self, index: int):
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self._stop = threading.Event()
        self.ok = False
        self.err = ""
        try:
            self.nv = _Nvml(index)
            self.max_mhz = self.nv.max_sm_mhz()
            self.ok = True
        except Exception as e:  # noqa: BLE001
            self.err = str(e)

    def _poll(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self.nv.sm_mhz())
                mask = self.nv.reasons()
                for name, bit in _Nvml.BITS.items():
                    if mask & bit:
                        self.reasons.add(name)
            except Exception:  # noqa: BLE001
                pass
            time.sleep(0.002)

    def start(self):
        if self.ok:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            while not self.samples and self.t.is_alive():
                time.sleep(0.001)

    def stop(self) -> dict:
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvml unavailable: " + self.err]}
        self._stop.set()
        self.t.join(timeout=1)
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6400.0), "source": "measured"}
    return {"hbm_gbs": 6400.0, "source": "fallback"}


def stage_bytes(stage: str, st: dict, record_bytes: int, n_upper: int, tile_passes: int) -> float:
    """Algorithmic bytes one launch of a stage must move (what the method reads
    and writes at least once), from the frame's counters."""
    ns, nv, npair, scanned = st["n_selected"], st["n_visible"], st["n_pairs"], st["n_spt_scanned"]
    if stage == "select":
        return 32.0 * n_upper + 8.0 * scanned + 4.0 * ns
    if stage == "project":
        return (record_bytes + 56.0) * ns
    if stage == "count":          # area scan (4 B read, 4 B written, twice), rect reads, tile counters
        return 16.0 * ns + 40.0 * nv + 4.0 * npair
    if stage == "emit":           # rect reads again + 8 B written per kept pair
        return 40.0 * nv + 8.0 * npair
    if stage == "tile_sort":      # kept pairs read (key + index) and indices written back
        return 12.0 * npair
    if stage == "project_bwd":
        return (record_bytes + 36.0 + record_bytes) * ns
    return 0.0


# ---------------------------------------------------------------------------
# CUDA arm
# ---------------------------------------------------------------------------
def spread_views(views: list, steps: int) -> list:
    """The views `steps` timed steps take, spread evenly over the path: with
    fewer steps than views, views evenly spaced from the first to the last, so
    a short run still averages aerial and street views alike; with more, the
    path repeated."""
    n = len(views)
    if steps >= n:
        return [views[i % n] for i in range(steps)]
    if steps == 1:
        return [views[0]]
    return [views[(2 * i * (n - 1) + steps - 1) // (2 * (steps - 1))] for i in range(steps)]


def shard_views(n_views: int, rank: int, world: int) -> list:
    """The views rank `rank` of `world` renders: every world-th view from its
    rank on (views are independent units: no exchange between ranks).  With
    more ranks than views a rank repeats one view."""
    return [v for v in range(n_views) if v % world == rank] or [rank % n_views]


def max_over_ranks(x: float, world: int) -> float:
    """The maximum of x over the ranks (the slowest rank's time), through the
    process group's backend (device tensors for NCCL, host tensors for gloo)."""
    if world == 1:
        return x
    import torch
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def run_lodgs(args, rank: int, world: int):
    import torch

    from paper_2507_01110_b300 import _lib, api, build, synth

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    cfg = synth.config2_scene(n=args.leaves)
    cams = cfg["cameras"]
    nv = len(cams)
    scene = api.build_hierarchy(cfg["leaves"], 3, cfg["spt_volume"], cfg["kappa"])
    H, W = cams[0].height, cams[0].width
    # views of this rank (independent units: no exchange between ranks)
    my_views = shard_views(nv, rank, world)
    frames = {v: api.Frame(scene) for v in my_views}     # profiling off: nothing extra in the timed graphs
    gen = torch.Generator().manual_seed(1234)
    # 8-bit RGB targets, the format of training photographs (read as byte / 255 in the backward)
    targets_h = {v: torch.randint(0, 256, (H, W, 3), generator=gen, dtype=torch.uint8).pin_memory()
                 for v in my_views}
    targets_d = {v: t.cuda() for v, t in targets_h.items()}
    # one image and one gradient buffer per view: views in flight at once share nothing
    images = {v: torch.empty((H, W, 3), device="cuda") for v in my_views}
    stream = torch.cuda.current_stream()

    # grow every frame's workspace once (capacity-checked renders), size gradient rows
    max_sel = 1
    fwd_stats = {}
    for v in my_views:
        fr = api.select_lod(scene, cams[v], frames[v])
        api.render(scene, fr, image=images[v], check_capacity=True)
        st = fr.stats()
        fwd_stats[v] = st
        max_sel = max(max_sel, st["n_selected"])
    grads = {v: torch.empty((max(fwd_stats[v]["n_selected"], 1), scene.stride), device="cuda") for v in my_views}
    # one loss slot per view: a view's loss can be read back on the copy stream
    # while the next views compute (no slot is rewritten before its read)
    loss_slots = torch.zeros(nv, device="cuda")

    def step_fwd(v, target, camera):
        fr = api.select_lod(scene, camera, frames[v])                  # camera=None: the frame's view
        api.render(scene, fr, image=images[v], bg=None, check_capacity=False)

    def step_bwd_blend(v):
        # mean-L1 loss against the view's target folded into the blend backward
        api.render_backward_blend_l1(scene, frames[v], targets_d[v], loss_sum=loss_slots[v:v + 1])

    def step_bwd_project(v):
        api.render_backward_project(scene, frames[v], grads[v])

    def step(v, target, camera):
        step_fwd(v, target, camera)
        step_bwd_blend(v)
        step_bwd_project(v)
        return loss_slots[v:v + 1]

    order = spread_views(my_views, args.steps)
    for i in range(args.warmup):
        v = my_views[i % len(my_views)]
        step(v, targets_d[v], cams[v])
    torch.cuda.synchronize()

    # CUDA graphs per frame: [camera upload, select, render], [loss + blend
    # backward], [projection backward]; each training view has a fixed camera,
    # so its upload kernel is captured with the view's graph and runs at every
    # replay.  Events between the graph launches time the blend backward (the
    # dominant kernel) inside the timed region.
    for v in my_views:
        api.set_view(frames[v], cams[v])
    torch.cuda.synchronize()
    cap = torch.cuda.Stream()
    graphs = {}
    with torch.cuda.stream(cap):
        for v in my_views:
            gs = [torch.cuda.CUDAGraph() for _ in range(3)]
            with torch.cuda.graph(gs[0], stream=cap):
                step_fwd(v, targets_d[v], cams[v])
            with torch.cuda.graph(gs[1], stream=cap):
                step_bwd_blend(v)
            with torch.cuda.graph(gs[2], stream=cap):
                step_bwd_project(v)
            graphs[v] = gs
    torch.cuda.synchronize()
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def replay(v, i=None):
        graphs[v][0].replay()
        if i is not None:
            ev_a[i].record(torch.cuda.current_stream())
        graphs[v][1].replay()
        if i is not None:
            ev_b[i].record(torch.cuda.current_stream())
        graphs[v][2].replay()

    # views in flight: step i runs on streams[i % S]; the views are independent
    # (each has its own frame, image, target, gradient rows and loss slot), so a
    # view's latency-bound selection and pair ordering overlap another view's blends
    n_streams = max(1, args.streams)
    streams = [stream] + [torch.cuda.Stream() for _ in range(n_streams - 1)]

    def run_steps(fn):
        """fn(i, v) for every step, step i on streams[i % S], all joined on `stream`."""
        start = torch.cuda.Event()
        start.record(stream)
        for s_ in streams[1:]:
            s_.wait_event(start)
        for i, v in enumerate(order):
            with torch.cuda.stream(streams[i % n_streams]):
                fn(i, v)
        for s_ in streams[1:]:
            stream.wait_stream(s_)

    for v in my_views:                               # one untimed replay each
        replay(v)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs ----
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = _lib.lib().lodgs_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    h0 = time.perf_counter()
    run_steps(lambda i, v: replay(v))
    e1.record(stream)
    host_submit_ms = 1e3 * (time.perf_counter() - h0) / len(order)      # host time to enqueue a step
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    launches_host = _lib.lib().lodgs_kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    # the same steps one view at a time, with events around each blend backward:
    # the dominant kernel's own launch duration (nothing overlaps it here)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for i, v in enumerate(order):
        replay(v, i)
    s1.record(stream)
    torch.cuda.synchronize()
    serial_ms = s0.elapsed_time(s1)
    clk = clocks.stop()
    bwd_ms = [a.elapsed_time(b2) for a, b2 in zip(ev_a, ev_b)]
    stats_ok = all(frames[v].stats()["status"] == 0 for v in set(order))
    # kernels per step: counted on an eager step with the camera upload (graph
    # replays launch the same kernels; launches_host counts any made outside them)
    torch.cuda.synchronize()
    l0 = _lib.lib().lodgs_kernel_launches()
    step(order[0], targets_d[order[0]], cams[order[0]])
    torch.cuda.synchronize()
    per_step = _lib.lib().lodgs_kernel_launches() - l0
    launches = launches_host + per_step * len(order)

    # ---- stage breakdown: the same steps, eager, every stage timed ----
    for fr in frames.values():
        fr.set_profiling(True)
    stage_ms = {s: [] for s in _lib.STAGES}
    for v in order:
        step(v, targets_d[v], cams[v])
    torch.cuda.synchronize()
    work = {}
    for v in set(order):
        t = frames[v].stage_ms()
        for s in _lib.STAGES:
            stage_ms[s].append(t[s])
        work[v] = frames[v].work()          # pixel-Gaussian work, tallied by the profiling launches
    for fr in frames.values():              # no stage events in what follows
        fr.set_profiling(False)
    stage_mean = {s: float(np.mean(x)) for s, x in stage_ms.items()}
    stage_mean_live = dict(stage_mean)
    stage_mean_live["blend_bwd"] = float(np.mean(bwd_ms))

    # ---- forward only (same frames, eager) ----
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for v in order:
        fr = api.select_lod(scene, cams[v], frames[v])
        api.render(scene, fr, image=images[v], check_capacity=False)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1)

    # ---- forward only with K views in flight (graph replays of [camera
    # upload, select, render] round-robin on K streams): how the per-view time
    # of the latency-bound front end falls as views overlap ----
    fwd_inflight = {}
    extra = [torch.cuda.Stream() for _ in range(8)]
    for k in (1, 2, 4, 8):
        sk = [stream] + extra[:k - 1]
        for _ in range(2):
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            for s_ in sk[1:]:
                s_.wait_event(q0)
            for i, v in enumerate(order):
                with torch.cuda.stream(sk[i % k]):
                    graphs[v][0].replay()
            for s_ in sk[1:]:
                stream.wait_stream(s_)
            q1.record(stream)
            torch.cuda.synchronize()
        fwd_inflight[k] = q0.elapsed_time(q1) / len(order)

    # ---- LoD selection of K views (K = 1, 2, 4, 8): K single-view selections
    # one after another against one lodgs_select_lod_batch, each graph-replayed
    # on one stream over the distinct views of this rank, ms per view ----
    select_k = {}
    distinct = list(dict.fromkeys(order)) if len(set(order)) >= 8 else list(my_views)
    with torch.cuda.stream(cap):
        for k in (1, 2, 4, 8):
            groups = [distinct[i:i + k] for i in range(0, len(distinct) - k + 1, k)]
            pair = []
            for g in groups:
                one, many = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
                with torch.cuda.graph(one, stream=cap):
                    for v in g:
                        api.select_lod(scene, cams[v], frames[v])
                with torch.cuda.graph(many, stream=cap):
                    api.select_lod_batch(scene, [cams[v] for v in g], [frames[v] for v in g])
                pair.append((one, many))
            select_k[k] = (pair, sum(len(g) for g in groups))
    torch.cuda.synchronize()
    select_batch_ms = {}
    for k, (pair, nvk) in select_k.items():
        t = {}
        for which in (0, 1):
            for rep in range(3):                 # the last of three passes (the first warms)
                q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                q0.record(stream)
                for p in pair:
                    p[which].replay()
                q1.record(stream)
                torch.cuda.synchronize()
            t[which] = q0.elapsed_time(q1) / nvk
        select_batch_ms[k] = {"one_at_a_time": round(t[0], 4), "batched": round(t[1], 4)}
    del select_k
    for v in my_views:                           # the frames back on their own views (same cuts)
        graphs[v][0].replay()
    torch.cuda.synchronize()

    # ---- training step: the same step followed by a sparse Adam step of the view's
    # cut (device-resident state, 3DGS-style per-column rates on the stored values) ----
    adam = api.AdamState(scene)
    params = scene.rows()
    lr = np.zeros(scene.stride, np.float32)
    lr[0:3], lr[3:6], lr[6:10], lr[10], lr[11:14], lr[14:] = 1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-3 / 20
    adam_graphs = {}
    with torch.cuda.stream(cap):
        for v in my_views:
            rows_p, dn_p = frames[v].selection_device()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                api.adam_step(scene, params, adam, (rows_p, grads[v].shape[0]), grads[v], lr, d_n=dn_p)
            adam_graphs[v] = g
    torch.cuda.synchronize()
    for v in my_views:
        replay(v)
        adam_graphs[v].replay()
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for v in order:
        replay(v)
        adam_graphs[v].replay()
    a1.record(stream)
    torch.cuda.synchronize()
    train_ms = a0.elapsed_time(a1)

    # ---- end to end: targets from pinned host, loss read back every step ----
    # Each step's target goes up on an upload stream ahead of the step (the
    # step's stream waits for it; a target buffer is rewritten only after its
    # last reader, that view's backward, has run), and each step's loss comes
    # back on a read-back stream once the step is done: uploads never queue
    # behind a read-back that waits for a step, and no compute stream waits
    # for a copy engine except for its own input.
    loss_h = torch.empty(len(order), dtype=torch.float32).pin_memory()
    copy_stream = torch.cuda.Stream()
    back_stream = torch.cuda.Stream()

    def e2e_pass():
        """One pass of the K steps end to end: (device ms, wall ms)."""
        used = {v: torch.cuda.Event() for v in set(order)}
        done_ev = [torch.cuda.Event() for _ in order]
        ready = [torch.cuda.Event() for _ in order]

        def upload(i):
            v = order[i]
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(used[v])
                targets_d[v].copy_(targets_h[v], non_blocking=True)
                ready[i].record(copy_stream)

        def read_loss(i):
            v = order[i]
            with torch.cuda.stream(back_stream):
                back_stream.wait_event(done_ev[i])
                loss_h[i:i + 1].copy_(loss_slots[v:v + 1], non_blocking=True)

        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        copy_stream.wait_event(g0)
        upload(0)
        up_issued = [False] * len(order)
        up_issued[0] = True

        def e2e_step(i, v):
            for k in range(i + 1, min(i + 1 + n_streams, len(order))):    # keep the next uploads queued
                if not up_issued[k]:
                    upload(k)
                    up_issued[k] = True
            cs = torch.cuda.current_stream()
            cs.wait_event(ready[i])
            replay(v)
            used[v].record(cs)
            done_ev[i].record(cs)
            read_loss(i)

        run_steps(e2e_step)
        stream.wait_stream(copy_stream)
        stream.wait_stream(back_stream)
        g1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if world > 1:
            torch.distributed.barrier()
        return g0.elapsed_time(g1), wall * 1e3

    # three passes; the pass with the median end-to-end time (the larger of its
    # device and wall times) is reported: one host stall in a ~10 ms pass
    # would otherwise decide the number
    passes = sorted((max(d, w), d, w) for d, w in (e2e_pass() for _ in range(3)))
    _, e2e_ms, e2e_wall_ms = passes[1]
    e2e_wall = e2e_wall_ms / 1e3
    e2e_passes_ms = [round(x[0], 3) for x in passes]

    def maxr(x):
        return max_over_ranks(x, world)

    ms, fwd_ms, e2e_ms, e2e_wall = maxr(ms), maxr(fwd_ms), maxr(e2e_ms), maxr(max(e2e_wall * 1e3, e2e_ms)) / 1e3
    serial_ms = maxr(serial_ms)
    train_ms = maxr(train_ms)
    total_views = args.steps * world
    res = {
        "ms": ms, "fwd_ms": fwd_ms, "e2e_ms": max(e2e_ms, e2e_wall * 1e3), "views": total_views,
        "train_ms": train_ms, "host_submit_ms": host_submit_ms, "serial_ms": serial_ms, "streams": n_streams,
        "fwd_inflight_ms": fwd_inflight, "select_batch_ms": select_batch_ms, "e2e_passes_ms": e2e_passes_ms,
        "stage_ms": stage_mean_live, "stage_ms_eager": stage_mean, "clocks": clk, "launches": launches,
        "stats_ok": stats_ok, "work": work,
        "fwd_stats": fwd_stats, "scene": {"n_nodes": scene.n_nodes, "n_upper": scene.n_upper, "n_spt": scene.n_spt,
                                          "stride": scene.stride},
        "h2d_bytes": H * W * 3 + 64, "d2h_bytes": 4, "order": order,
    }
    return res, cfg


# Algorithmic instructions per (pixel, Gaussian) contribution, counted from the
# method's arithmetic: the support test (2 sub, mul, 2 fma, compare) plus, for
# the forward, exp (2), opacity product, clamp, weight, 3 colour fma, 1 - alpha,
# transmittance product, stop test (11); for the backward, exp (2), opacity
# product, clamp, division (2), 1 - alpha, 3 colour differences, dot product (3),
# T scale, weight, 3 colour-gradient fma, 3 Q updates, clamp test, dL/dp,
# opacity fma, mean (4), conic (6) = 34.  Support tests of pixels a Gaussian does
# not reach and the per-Gaussian warp sums are not counted: they are the
# implementation's, not the method's.  Counts are issue slots: 128 per SM and
# clock is the issue peak for any instruction type.
OPS_EVAL, OPS_BLEND, OPS_BWD_CONTRIB = 6, 11, 34
# DRAM bytes (read + write) per k_blend_bwd launch, mean over the 32 views of
# this workload, from one ncu capture of the launch list with
# dram__bytes_read.sum and dram__bytes_write.sum; a constant of the kernel's
# code at that capture, to be taken again whenever the kernel changes
BLEND_BWD_DRAM_BYTES = 39.26e6
BLEND_BWD_ISSUE_ACTIVE = 0.788    # smsp__issue_active of the same kernel, one view (ncu --set full)
FP32_LANES_PER_SM, N_SM = 128, 148


def alu_ops(stage: str, work: dict) -> float:
    if stage == "blend":
        return (OPS_EVAL + OPS_BLEND) * work["fwd_blend"]
    if stage == "blend_bwd":
        return (OPS_EVAL + OPS_BWD_CONTRIB) * work["bwd_contrib"]
    return 0.0


def roofline(res: dict, peaks: dict) -> dict:
    from paper_2507_01110_b300 import _lib
    st_mean = res["stage_ms"]
    # mean counters over the views of the timed region
    fs = [res["fwd_stats"][v] for v in set(res["order"])]
    mean = {k: float(np.mean([s[k] for s in fs])) for k in ("n_selected", "n_visible", "n_pairs", "n_spt_scanned")}
    rb = 236
    tile_passes = 2
    hbm = {s: stage_bytes(s, mean, rb, res["scene"]["n_upper"], tile_passes) for s in _lib.STAGES}
    dom = max(st_mean, key=lambda s: st_mean[s])
    wk = {k: float(np.mean([w[k] for w in res["work"].values()])) for k in ("fwd_eval", "fwd_blend", "bwd_eval",
                                                                           "bwd_contrib")}
    mhz = res["clocks"].get("sm_mhz") or 2032.0
    alu_peak = N_SM * FP32_LANES_PER_SM * mhz * 1e6 / 1e12      # T thread-instructions / s (issue peak)
    per_stage = {}
    for s in _lib.STAGES:
        t = st_mean[s] * 1e-3
        if hbm[s] > 0 and t > 0:
            per_stage[s] = {"ms": st_mean[s], "gbs": hbm[s] / t / 1e9, "frac_hbm": hbm[s] / t / 1e9 / peaks["hbm_gbs"]}
        elif s in ("blend", "blend_bwd") and t > 0:
            a = alu_ops(s, wk) / t / 1e12
            per_stage[s] = {"ms": st_mean[s], "tinst_s": a, "frac_alu": a / alu_peak}
        else:
            per_stage[s] = {"ms": st_mean[s]}
    return {"dominant": dom, "stages": per_stage, "bytes": hbm, "mean_counts": mean, "work": wk,
            "alu_peak": alu_peak, "mhz": mhz}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_frame_seconds(sc_o, cam, target_seed: int) -> float:
    """One whole view through the oracle, as the CUDA step does it: LoD select,
    projection with SH colour, tile x depth sort, blend, the mean-L1 loss's
    gradient against an 8-bit target, blend backward, projection backward."""
    import oracle
    from paper_2507_01110_b300 import synth
    tb = synth.target_bytes(target_seed, cam.height, cam.width).astype(np.float64) / 255.0
    t0 = time.perf_counter()
    out = oracle.render(sc_o, cam)
    dL = np.sign(out["image"] - tb) / out["image"].size
    oracle.render_backward(sc_o, cam, out, dL)
    return time.perf_counter() - t0


def oracle_forward_seconds(sc_o, cam) -> float:
    import oracle
    t0 = time.perf_counter()
    oracle.render(sc_o, cam)
    return time.perf_counter() - t0


def timed_legs(fn, views) -> dict:
    """The oracle on one thread and on every host core (its OpenMP build):
    seconds per view of fn(view), with the thread counts actually used."""
    import oracle
    out = {}
    for leg, n in (("one_thread", 1), ("all_cores", None)):
        threads = oracle.use_threads(n)
        secs = [fn(v) for v in views]
        out[leg] = {"threads": threads, "s_per_view": [round(x, 3) for x in secs],
                    "frames_per_s": len(secs) / sum(secs)}
    oracle.use_threads(1)
    return out


def cpu_baseline(cfg: dict) -> dict:
    """The oracle timed on whole 1080p frames of the path's two ends, views 0
    (aerial, the largest cut) and 31 (street), forward plus backward: once on
    one thread (the reported value) and once on every host core."""
    import oracle
    sc_o = oracle.build_scene(cfg["leaves"], 3, cfg["spt_volume"], cfg["kappa"])
    cams = cfg["cameras"]
    legs = timed_legs(lambda v: oracle_frame_seconds(sc_o, cams[v], 300 + v), [0, 31])
    one, allc = legs["one_thread"], legs["all_cores"]
    return {"value": one["frames_per_s"], "unit": "frames/s", "cores": one["threads"], "kind": "oracle",
            "sample": "float64 C oracle, whole 1920x1080 frames of views 0 and 31 (select + project + sort + "
                      "blend + mean-L1 gradient + blend backward + projection backward), one thread; "
                      f"seconds per view {one['s_per_view']}",
            "host_cores": os.cpu_count(),
            "all_cores": {"value": allc["frames_per_s"], "unit": "frames/s", "cores": allc["threads"],
                          "s_per_view": allc["s_per_view"],
                          "note": "the same oracle built with OpenMP: pixel rows and Gaussians in parallel"}}


def run_reference(args, rank: int, world: int):
    """The oracle as the reference arm, on one host thread: each timed step one
    whole view of the CUDA arm's view order (forward and backward, as the step
    of that arm); each warm-up step a 16-row band of the street view."""
    import oracle
    from paper_2507_01110_b300 import synth
    if rank != 0:
        return None
    cfg = synth.config2_scene(n=args.leaves)
    sc_o = oracle.build_scene(cfg["leaves"], 3, cfg["spt_volume"], cfg["kappa"])
    cams = cfg["cameras"]
    threads = oracle.use_threads(1)
    for _ in range(args.warmup):
        out = oracle.render(sc_o, cams[31], window=(0, 532, cams[31].width, 548))
        oracle.render_backward(sc_o, cams[31], out, np.zeros_like(out["image"]),
                               window=(0, 532, cams[31].width, 548))
    order = spread_views(list(range(len(cams))), args.steps)
    t0 = time.perf_counter()
    per = [oracle_frame_seconds(sc_o, cams[v], 300 + v) for v in order]
    total = time.perf_counter() - t0
    value = len(order) / total
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "views_timed": order, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads, "kind": "oracle",
                             "sample": "each timed step one whole 1920x1080 view of the CUDA arm's view order "
                                       "(select + project + sort + blend + mean-L1 gradient + backward), "
                                       "one thread, measured wall time",
                             "host_cores": os.cpu_count(), "s_per_view": [round(x, 3) for x in per]},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------
# serving (50M-leaf city, Poisson arrivals) and out-of-core (20M-leaf city)
# ---------------------------------------------------------------------------
SERVING_SPT_VOLUME = 150.0      # ~N/1024 SPT roots on the 50M-leaf city
OOC_SPT_VOLUME = 300.0          # ~N/1024 SPT roots on the 20M-leaf city


def run_serving(args) -> dict:
    """Continuous batching against one request at a time on the 50M-leaf city:
    the config's Poisson 200 requests/s, then 600 and 800 requests/s (past what
    one at a time sustains).  The slots' workspaces are sized within a 16 GiB
    budget from the learned workspace bytes per request class; GPU busy
    fraction from the requests' device intervals."""
    import torch
    from paper_2507_01110_b300 import api, serving, synth
    t0 = time.perf_counter()
    leaves = synth.city_leaves_t(args.serving_leaves, seed=4, degree=3, device="cuda")
    cams = synth.serving_cameras(256, seed=4)
    kappa = min(float(c.fx / c.tau) for c in cams)
    scene = api.build_hierarchy(leaves, 3, SERVING_SPT_VOLUME, kappa)
    del leaves
    torch.cuda.empty_cache()
    t_build = time.perf_counter() - t0
    # workspaces sized and request classes learned before serving, on the pool's
    # most demanding cameras (most pixels per squared LoD threshold) plus a sample
    worst = sorted(cams, key=lambda c: -(c.width * c.height) / (c.tau * c.tau))[:16]
    warm_set = worst + cams[:16]
    mix = serving.RenderServer(scene, n_slots=8, mem_budget_bytes=16 << 30)
    mix.warm(warm_set)
    fifo = serving.RenderServer(scene, n_slots=1, mem_budget_bytes=16 << 30)
    fifo.warm(warm_set)
    mix_pv = serving.RenderServer(scene, n_slots=8, mem_budget_bytes=16 << 30, batch_select=False)
    mix_pv.warm(warm_set)

    def fmt(r):
        return {k: round(v, 4) if isinstance(v, float) else v for k, v in r.items()}

    loads = {}
    for rate, n in ((200.0, args.serving_requests), (600.0, args.serving_requests // 2),
                    (800.0, args.serving_requests // 2)):
        r_mix = mix.run(serving.poisson_requests(cams, rate, n, seed=4))
        r_fifo = fifo.run(serving.poisson_requests(cams, rate, n, seed=4))
        loads[f"{int(rate)}_per_s"] = {"requests": n, "continuous_batching": fmt(r_mix), "one_at_a_time": fmt(r_fifo)}
        if rate >= 800.0:
            r_pv = mix_pv.run(serving.poisson_requests(cams, rate, n, seed=4))
            loads[f"{int(rate)}_per_s"]["continuous_batching_per_view_selection"] = fmt(r_pv)
    return {"workload": f"{args.serving_leaves:,}-leaf SH3 city (2 km), Poisson arrivals, resolution in "
                        "{360p,720p,1080p,2160p}, tau in {0.5,1,2,4} px, half aerial half street; 8 slots, "
                        "16 GiB workspace budget; requests admitted together share one batched LoD selection",
            "nodes": scene.n_nodes, "spt": scene.n_spt, "build_s": round(t_build, 2),
            "request_classes_learned": len(mix.need), **loads["200_per_s"],
            "load_600_per_s": loads["600_per_s"], "load_800_per_s": loads["800_per_s"], "unit": "ms",
            "slot_workspace_gb": [round(sl.held / 1e9, 2) for sl in mix.slots],
            "slot_workspace_after_warm_gb": round(mix.warm_bytes / 1e9, 3),
            "admission": "a request runs on a free slot whose workspace holds the largest bytes its class "
                         "(resolution, tau) needed (lodgs_frame_memory); slots sized within the budget in the "
                         "warm-up"}


def run_config1(args) -> dict:
    """The plain forward render: 65,536-leaf SH0 scene in a 100 m cube, one
    256x256 camera at 60 deg, tau 1 px.  GPU frames/s of select + render as one
    graph replay per frame, back to back (the 4 MB of records stay in L2) and
    with L2 flushed before each frame (a 256 MB write, outside the per-frame
    events); the oracle on whole frames, one thread and every host core."""
    import torch

    import oracle
    from paper_2507_01110_b300 import api, synth
    cfg = synth.config1_scene()
    cam = cfg["cameras"][0]
    scene = api.build_hierarchy(cfg["leaves"], 0, cfg["spt_volume"], cfg["kappa"])
    fr = api.Frame(scene)
    image = torch.empty((cam.height, cam.width, 3), device="cuda")
    api.select_lod(scene, cam, fr)
    api.render(scene, fr, image=image, check_capacity=True)
    n_sel = fr.stats()["n_selected"]
    api.set_view(fr, cam)
    torch.cuda.synchronize()
    cap = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        with torch.cuda.graph(g, stream=cap):
            api.select_lod(scene, None, fr)
            api.render(scene, fr, image=image, bg=None, check_capacity=False)
    for _ in range(20):
        g.replay()
    torch.cuda.synchronize()
    reps = 2000
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    warm_ms = e0.elapsed_time(e1) / reps
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    cold = []
    for _ in range(200):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        cold.append((a, b))
    torch.cuda.synchronize()
    cold_ms = float(np.mean([a.elapsed_time(b) for a, b in cold]))
    sc_o = oracle.build_scene(cfg["leaves"], 0, cfg["spt_volume"], cfg["kappa"])
    legs = timed_legs(lambda _: oracle_forward_seconds(sc_o, cam), [0, 1, 2])
    return {"workload": "65,536-leaf SH0 scene (100 m cube), one 256x256 camera at 60 deg, tau 1 px, forward "
                        "(select + render)", "selected": n_sel,
            "frames_per_s_l2_warm": round(1e3 / warm_ms, 1), "ms_per_frame_l2_warm": round(warm_ms, 4),
            "frames_per_s_l2_flushed": round(1e3 / cold_ms, 1), "ms_per_frame_l2_flushed": round(cold_ms, 4),
            "cpu_oracle": {"one_thread": {"frames_per_s": round(legs["one_thread"]["frames_per_s"], 2),
                                          "cores": legs["one_thread"]["threads"]},
                           "all_cores": {"frames_per_s": round(legs["all_cores"]["frames_per_s"], 2),
                                         "cores": legs["all_cores"]["threads"]},
                           "sample": "three whole frames each"}}


def run_lod_sweep(args) -> dict:
    """LoD effectiveness: forward frames/s against the number of selected nodes over
    50 LoD thresholds tau (log-spaced 0.25..64 px) on the 2M-leaf scene, three views
    of the path (aerial, middle, street); the scene is built for the largest tau."""
    import torch
    from paper_2507_01110_b300 import api, synth
    cfg = synth.config2_scene(n=args.leaves)
    base = [cfg["cameras"][i] for i in (0, 16, 31)]
    taus = np.geomspace(0.25, 64.0, 50)
    scene = api.build_hierarchy(cfg["leaves"], 3, cfg["spt_volume"], float(base[0].fx / taus[-1]))
    frames = [api.Frame(scene) for _ in base]
    image = torch.empty((base[0].height, base[0].width, 3), device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out_tau, out_sel, out_fps = [], [], []
    for tau in taus:
        cams = [dataclasses.replace(c, tau=np.float32(tau)) for c in base]
        for fr, cam in zip(frames, cams):          # size the workspaces for this tau
            api.select_lod(scene, cam, fr)
            api.render(scene, fr, image=image, check_capacity=True)
        sel = float(np.mean([fr.stats()["n_selected"] for fr in frames]))
        reps = 4
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            for fr, cam in zip(frames, cams):
                api.select_lod(scene, cam, fr)
                api.render(scene, fr, image=image, check_capacity=False)
        e1.record()
        torch.cuda.synchronize()
        out_tau.append(round(float(tau), 3))
        out_sel.append(int(sel))
        out_fps.append(round(reps * len(cams) / (e0.elapsed_time(e1) * 1e-3), 1))
    return {"workload": f"{args.leaves:,}-leaf SH3 scene, views 0/16/31 of the path at 1920x1080, forward "
                        "(select + render), tau log-spaced 0.25..64 px", "tau_px": out_tau,
            "selected_mean": out_sel, "frames_per_s": out_fps}


def run_out_of_core(args) -> dict:
    """Out-of-core rendering: records in pinned host memory, a device cache of SPT
    prefixes.  The flythrough with an 8 GiB cache (the headline of this section),
    the same flythrough with smaller caches, and the loads of a training view order
    drawn uniformly against one drawn by the kNN view scheduler."""
    import torch
    from paper_2507_01110_b300 import api, schedule, synth
    leaves = synth.city_leaves_t(args.ooc_leaves, seed=3, degree=3, device="cuda")
    cams = synth.flythrough_path(args.ooc_views)
    kappa = float(cams[0].fx / cams[0].tau)
    scene = api.build_hierarchy(leaves, 3, OOC_SPT_VOLUME, kappa)
    del leaves
    rec_bytes = scene.stride * 4
    fr = api.Frame(scene)
    H, W = cams[0].height, cams[0].width
    image = torch.empty((H, W, 3), device="cuda")
    copy_stream = torch.cuda.Stream()
    keys = ("spt_hits", "spt_resident", "spt_loaded", "bytes_streamed", "evictions")

    def flythrough(cache) -> dict:
        # size the frame's workspace on the path (first pass), then time a fresh cache pass
        for cam in cams[:: max(1, len(cams) // 16)]:
            api.stream_nodes(scene, cache, cam, fr, copy_stream=copy_stream)
            api.render(scene, fr, rows=cache.records, image=image, check_capacity=True)
        cache.flush()                               # timed pass starts from an empty cache
        torch.cuda.synchronize()
        tot = dict.fromkeys(keys, 0)
        t0 = time.perf_counter()
        for cam in cams:
            _, st = api.stream_nodes(scene, cache, cam, fr, copy_stream=copy_stream)
            api.render(scene, fr, rows=cache.records, image=image, check_capacity=False)
            for k in tot:
                tot[k] += st[k]
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        n_spt_views = tot["spt_hits"] + tot["spt_resident"] + tot["spt_loaded"]
        return {"frames_per_s": round(len(cams) / wall, 2), "ms_per_frame": round(1e3 * wall / len(cams), 3),
                "bytes_streamed_per_frame": int(tot["bytes_streamed"] / len(cams)),
                "spt_hit_rate": round(tot["spt_hits"] / max(1, n_spt_views), 4),
                "spt_device_resident_rate": round((tot["spt_hits"] + tot["spt_resident"]) / max(1, n_spt_views), 4),
                "evictions": tot["evictions"]}

    # cache size against frame rate (smaller caches first: they keep the scene's device rows)
    sweep = []
    for gib in (1, 2, 4):
        c = api.Cache(scene, capacity_bytes=gib << 30, d_min=0.9, d_max=1.1, release_scene_rows=False)
        try:
            r = flythrough(c)
            sweep.append({"cache_gib": gib, "frames_per_s": r["frames_per_s"],
                          "bytes_streamed_per_frame": r["bytes_streamed_per_frame"],
                          "spt_hit_rate": r["spt_hit_rate"], "evictions": r["evictions"]})
        except Exception as e:  # noqa: BLE001  (a view whose SPT records exceed the slab)
            torch.cuda.synchronize()
            sweep.append({"cache_gib": gib, "error": f"{type(e).__name__}: {e}"[:160]})
        c.close()
        del c
        torch.cuda.empty_cache()
    # out-of-core training: kNN-scheduled views at 1080p through a 4 GiB training
    # cache (records, Adam moments and step counts streamed together; trained
    # prefixes written back on eviction), select + render + mean-L1 + backward +
    # sparse Adam per iteration, then the write-back of everything still cached
    pool = [synth.camera_look(c.pos, c.R[2], c.R[0], 1920, 1080, tau=1.0)
            for c in synth.serving_cameras(512, seed=33)]

    def train_ooc(gib: int, iters=128) -> dict:
        tc = api.Cache(scene, capacity_bytes=gib << 30, d_min=0.9, d_max=1.1, train=True)
        sched_t = schedule.ViewScheduler(np.array([c.pos for c in pool]), k=10, seed=36)
        order = [sched_t.next() for _ in range(iters + 8)]
        img = torch.empty((1080, 1920, 3), device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(37)
        target = torch.rand((1080, 1920, 3), device="cuda", generator=gen)
        dL = torch.empty_like(img)
        g = torch.empty((scene.n_nodes, scene.stride), device="cuda")   # any cut fits
        lr = np.full(scene.stride, 1.6e-4, np.float32)
        lr[10], lr[3:6] = 5e-2, 5e-3
        ft = api.Frame(scene)

        def it(v):
            _, st = api.stream_nodes(scene, tc, pool[v], ft, copy_stream=copy_stream)
            api.render(scene, ft, rows=tc.records, image=img, check_capacity=True)
            api.render_backward_blend_l1(scene, ft, target)
            api.render_backward_project(scene, ft, g, rows=tc.records)
            tc.adam_step(ft, g, lr)
            return st

        for v in order[:8]:                       # grow the frame's workspace
            it(v)
        torch.cuda.synchronize()
        tot = {"bytes_streamed": 0, "bytes_written_back": 0, "evictions": 0}
        wb0 = tc.written_bytes()
        t0 = time.perf_counter()
        for v in order[8:]:
            st = it(v)
            for k in tot:
                tot[k] += st[k]
        max_cut = max(ft.stats()["n_selected"], 0)
        wb1 = tc.written_bytes()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        t1 = time.perf_counter()
        tc.writeback()
        torch.cuda.synchronize()
        wb = time.perf_counter() - t1
        tc.close()
        return {"iterations": iters, "iters_per_s": round(iters / dt, 1), "ms_per_iter": round(1e3 * dt / iters, 3),
                "bytes_streamed_per_iter": int(tot["bytes_streamed"] / iters),
                "bytes_written_back_per_iter": int((wb1 - wb0) / iters),
                "trained_prefix_bytes_evicted_per_iter": int(tot["bytes_written_back"] / iters),
                "evictions": tot["evictions"], "final_writeback_ms": round(1e3 * wb, 1), "last_cut": max_cut,
                "cache_gib": gib}

    training = {"note": "records, m, v and step counts stream together (3x the record bytes + 4 B); the "
                        "cache size counts the records", "runs": []}
    for gib in (4, 8):
        try:
            training["runs"].append(train_ooc(gib))
        except Exception as e:  # noqa: BLE001  (pinned host memory for the Adam state may be short)
            torch.cuda.synchronize()
            training["runs"].append({"cache_gib": gib, "error": f"{type(e).__name__}: {e}"[:200]})
        torch.cuda.empty_cache()

    cache = api.Cache(scene, capacity_bytes=8 << 30, d_min=0.9, d_max=1.1, release_scene_rows=True)
    torch.cuda.empty_cache()
    main = flythrough(cache)
    sweep.append({"cache_gib": 8, "frames_per_s": main["frames_per_s"],
                  "bytes_streamed_per_frame": main["bytes_streamed_per_frame"],
                  "spt_hit_rate": main["spt_hit_rate"], "evictions": main["evictions"]})

    # training view order: uniform against the kNN scheduler (LoD cut and loads only)
    iters = 256

    def loads(order) -> dict:
        cache.flush()
        tot, cut = dict.fromkeys(keys, 0), 0
        for v in order:
            _, st = api.stream_nodes(scene, cache, pool[v], fr, copy_stream=copy_stream)
            cut += fr.stats()["n_selected"]
            for k in tot:
                tot[k] += st[k]
        n_spt_views = tot["spt_hits"] + tot["spt_resident"] + tot["spt_loaded"]
        return {"nodes_loaded_per_iter": int(tot["bytes_streamed"] / rec_bytes / len(order)),
                "cut_nodes_per_iter": int(cut / len(order)),
                "spt_hit_rate": round(tot["spt_hits"] / max(1, n_spt_views), 4)}

    # the host link: pinned 1 GiB copies each way, the denominator of the streaming stage
    def link_gbs(to_host: bool) -> float:
        h = torch.empty(1 << 28, dtype=torch.float32, pin_memory=True)
        d = torch.empty(1 << 28, dtype=torch.float32, device="cuda")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 0.0
        for _ in range(4):
            ev0.record()
            if to_host:
                h.copy_(d, non_blocking=True)
            else:
                d.copy_(h, non_blocking=True)
            ev1.record()
            ev1.synchronize()
            best = max(best, (1 << 30) / (ev0.elapsed_time(ev1) * 1e-3) / 1e9)
        return best

    link = {"h2d_gbs": round(link_gbs(False), 1), "d2h_gbs": round(link_gbs(True), 1),
            "note": "pinned 1 GiB cudaMemcpyAsync, best of 4"}
    link["flythrough_h2d_frac"] = round(main["bytes_streamed_per_frame"] * main["frames_per_s"] / 1e9
                                        / link["h2d_gbs"], 4)
    for r in training["runs"]:
        if "ms_per_iter" in r:
            # the streaming time alone if both directions ran at the link peak, one after the other
            t_link = r["bytes_streamed_per_iter"] / (link["h2d_gbs"] * 1e9) + \
                r["bytes_written_back_per_iter"] / (link["d2h_gbs"] * 1e9)
            r["link_bound_ms"] = round(1e3 * t_link, 2)
            r["link_frac"] = round(1e3 * t_link / r["ms_per_iter"], 3)

    uniform = loads(np.random.default_rng(34).integers(len(pool), size=iters).tolist())
    sched = schedule.ViewScheduler(np.array([c.pos for c in pool]), k=10, seed=35)
    knn = loads([sched.next() for _ in range(iters)])

    # LoD effectiveness through the cache: frames/s against the selected count
    # over 50 thresholds (log-spaced 0.25..64 px) on three views of the
    # flythrough (first, middle, last); at each threshold every view is rendered
    # once to warm the cache, then four times timed
    sweep_views = [cams[0], cams[len(cams) // 2], cams[-1]]
    taus = np.geomspace(0.25, 64.0, 50)
    sw_tau, sw_sel, sw_fps = [], [], []
    cache.flush()
    for tau in taus:
        vcams = [dataclasses.replace(c, tau=np.float32(tau)) for c in sweep_views]
        sel = []
        for cam in vcams:
            api.stream_nodes(scene, cache, cam, fr, copy_stream=copy_stream)
            api.render(scene, fr, rows=cache.records, image=image, check_capacity=True)
            sel.append(fr.stats()["n_selected"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(4):
            for cam in vcams:
                api.stream_nodes(scene, cache, cam, fr, copy_stream=copy_stream)
                api.render(scene, fr, rows=cache.records, image=image, check_capacity=False)
        torch.cuda.synchronize()
        sw_tau.append(round(float(tau), 3))
        sw_sel.append(int(np.mean(sel)))
        sw_fps.append(round(4 * len(vcams) / (time.perf_counter() - t0), 1))
    lod_sweep = {"workload": "views 0/100/199 of the flythrough through the 8 GiB cache (each rendered once to warm "
                             "the cache per threshold, then 4 timed passes), forward, tau log-spaced 0.25..64 px",
                 "tau_px": sw_tau, "selected_mean": sw_sel, "frames_per_s": sw_fps,
                 "note": "the scene is built for the flythrough's f / (1 px): above 1 px the interval bound no "
                         "longer guarantees f S / d <= tau, so those cuts may be slightly coarser than the exact "
                         "criterion; frames/s includes the cache's host decisions"}
    return {"workload": f"{args.ooc_leaves:,}-leaf SH3 city, records in pinned host memory, 8 GiB device "
                        f"cache, {len(cams)}-view flythrough 300 m -> 20 m at 1920x1080, forward only",
            **main, "host_record_gb": round(scene.n_nodes * scene.stride * 4 / 1e9, 2), "reuse_window": [0.9, 1.1],
            "cache_size_sweep": sweep, "training": training, "host_link": link, "lod_sweep": lod_sweep,
            "view_selection": {"pool_views": len(pool), "iterations": iters,
                               "note": "nodes loaded from host per training iteration; a cache-less run loads "
                                       "the whole cut (cut_nodes_per_iter)",
                               "uniform_views": uniform, "knn_scheduler": knn,
                               "knn": {"k": 10, "W": round(sched.W, 2), "random_every": 128}}}


TRAIN_SPT_VOLUME = 150.0      # per-scene HSPT size for the 150M-leaf city


def run_train_batch(args) -> dict:
    """Training-scale step: 150M-leaf SH3 city, a batch of 8 views (4 aerial, 4
    street) at 1600x1200; LoD select + render + mean-L1 + backward per view on
    its own stream, then the batch gradient summed over the union of the cuts."""
    import torch
    from paper_2507_01110_b300 import api, synth
    t0 = time.perf_counter()
    leaves = synth.city_leaves_t(args.train_leaves, seed=5, degree=3, device="cuda")
    aerial = synth.serving_cameras(64, seed=5)
    views = [c for c in aerial if c.pos[2] > 40.0][:4] + [c for c in aerial if c.pos[2] < 5.0][:4]
    views = [synth.camera_look(c.pos, c.R[2], c.R[0], 1600, 1200, tau=1.0) for c in views]
    kappa = float(views[0].fx)
    scene = api.build_hierarchy(leaves, 3, TRAIN_SPT_VOLUME, kappa)
    del leaves
    torch.cuda.empty_cache()
    t_build = time.perf_counter() - t0
    streams = [torch.cuda.Stream() for _ in views]
    frames = [api.Frame(scene) for _ in views]
    imgs = [torch.empty((1200, 1600, 3), device="cuda") for _ in views]
    gen = torch.Generator(device="cuda").manual_seed(5)
    targets = [torch.rand((1200, 1600, 3), device="cuda", generator=gen) for _ in views]
    for v, cam in enumerate(views):                 # size the workspaces
        api.select_lod(scene, cam, frames[v])
        api.render(scene, frames[v], image=imgs[v], check_capacity=True)
    sizes = [fr.stats()["n_selected"] for fr in frames]
    grads = [torch.empty((max(n, 1), scene.stride), device="cuda") for n in sizes]

    main = torch.cuda.current_stream()

    def step(batched: bool):
        """batched: the 8 cuts in one lodgs_select_lod_batch on the main
        stream, then each view's render and backward on its own stream;
        otherwise each view selects on its own stream."""
        if batched:
            api.select_lod_batch(scene, views, frames, stream=main)
            sel = torch.cuda.Event()
            sel.record(main)
        for v, cam in enumerate(views):
            with torch.cuda.stream(streams[v]):
                if batched:
                    streams[v].wait_event(sel)
                    fr = frames[v]
                else:
                    streams[v].wait_stream(main)
                    fr = api.select_lod(scene, cam, frames[v], stream=streams[v])
                api.render(scene, fr, image=imgs[v], stream=streams[v], check_capacity=False)
                api.render_backward_blend_l1(scene, fr, targets[v], stream=streams[v])
                api.render_backward_project(scene, fr, grads[v], stream=streams[v])
        for s_ in streams:
            main.wait_stream(s_)
        return api.accumulate_grads(scene, frames, grads)

    out = {}
    for batched in (True, False):
        for _ in range(2):
            step(batched)
        torch.cuda.synchronize()
        reps = 5
        t1 = time.perf_counter()
        for _ in range(reps):
            rows, _g = step(batched)
        torch.cuda.synchronize()
        out[batched] = (time.perf_counter() - t1) / reps
    torch.cuda.nvtx.range_push("train_batch_step")       # one more step, for profilers
    step(True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dt = out[True]
    return {"workload": f"{args.train_leaves:,}-leaf SH3 city (2 km), batch of 8 views (4 aerial, 4 street) at "
                        "1600x1200: one batched LoD selection of the 8 views, then render + mean-L1 + backward "
                        "per view on its own stream, batch gradient on the union of the cuts",
            "nodes": scene.n_nodes, "spt": scene.n_spt, "build_s": round(t_build, 2),
            "step_ms": round(dt * 1e3, 3), "views_per_s": round(8 / dt, 1),
            "step_ms_per_view_selection": round(out[False] * 1e3, 3),
            "selected_per_view": sizes, "union_rows": int(rows.numel()),
            "device_gb_peak": round(torch.cuda.max_memory_allocated() / 1e9, 1),
            "note": "wall time per batch step (host enqueue included); step_ms_per_view_selection: the same "
                    "step with each view's selection launched on its own stream"}


def run_densify(args) -> dict:
    """One densification step on the main workload's scene: per-node maximal
    screen-space gradient gathered over 8 training views (fwd + bwd), the plan
    on the device (dead leaves respawned under the candidates with the largest
    gradients, the rest spawned; threshold at the top 5% of the selected
    nodes' gradients, 0.5% of the rows flagged stale by the pruning rule), the
    tree edits and HSPT/SPT rebuild, and the Adam state carried across.  Three
    rounds, each planned on the last."""
    import torch
    from paper_2507_01110_b300 import api, synth
    cfg = synth.config2_scene(n=args.leaves)
    cams = cfg["cameras"][:8]
    scene = api.build_hierarchy(cfg["leaves"], 3, cfg["spt_volume"], cfg["kappa"])
    del cfg
    H, W = cams[0].height, cams[0].width
    image = torch.empty((H, W, 3), device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(77)
    target = torch.rand((H, W, 3), device="cuda", generator=gen)
    adam = api.AdamState(scene)
    rounds = []
    for it in range(3):
        gmax = torch.zeros(scene.n_nodes, device="cuda")
        fr = api.Frame(scene)
        for cam in cams:
            api.select_lod(scene, cam, fr)
            api.render(scene, fr, image=image, check_capacity=True)
            api.render_backward_blend_l1(scene, fr, target)        # the screen-space gradients
            api.screen_grad_max(fr, gmax)
        torch.cuda.synchronize()
        M0, L0 = scene.n_nodes, scene.n_leaves
        # the bench's policy: a threshold at the top 5% of the view-selected nodes' gradients,
        # 0.5% of the rows flagged stale (the pruning rule's output)
        thr = float(torch.quantile(gmax[gmax > 0], 0.95))
        stale = torch.rand(M0, device="cuda", generator=gen) < 0.005
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t1 = t0
        spawn, respawn = scene.plan_densify(gmax, thr, stale=stale)
        t2 = time.perf_counter()
        old = scene.densify(spawn=spawn, respawn=respawn)
        t3 = time.perf_counter()
        adam.remap(old)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        fr = api.Frame(scene)
        api.select_lod(scene, cams[0], fr)
        api.render(scene, fr, image=image, check_capacity=True)
        ok = fr.stats()["status"] == 0
        rounds.append({"nodes_before": M0, "nodes_after": scene.n_nodes, "leaves_after": scene.n_leaves,
                       "spawn": len(spawn), "respawn": len(respawn), "spt_after": scene.n_spt,
                       "plan_ms": round(1e3 * (t2 - t1), 1),
                       "densify_rebuild_ms": round(1e3 * (t3 - t2), 1), "adam_remap_ms": round(1e3 * (t4 - t3), 1),
                       "total_ms": round(1e3 * (t4 - t0), 1), "render_after_ok": ok})
    return {"workload": f"{args.leaves:,}-leaf SH3 scene of the main line; gradient maxima over 8 views at "
                        f"{W}x{H}, threshold at the top 5% of selected-node gradients, 0.5% of rows stale",
            "rounds": rounds}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    res, cfg = run_lodgs(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    peaks = measured_peaks()
    rf = roofline(res, peaks)
    dom = rf["dominant"]
    ds = rf["stages"][dom]
    value = res["views"] / (res["ms"] * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "leaves": args.leaves, "nodes": res["scene"]["n_nodes"],
                   "spt": res["scene"]["n_spt"], "views": 32, "views_timed": res["order"],
                   "resolution": "1920x1080", "tau_px": 1.0,
                   "loss": "mean L1 against 8-bit RGB targets",
                   "l2": "inputs larger than L2 (node records 1.07 GB; per-view reads 100-400 MB)",
                   "parallelism": f"replicas x{world} (views split across ranks); {res['streams']} views in "
                                  "flight per GPU (independent views, one CUDA stream each)"},
        "fwd_bwd_step_ms": res["ms"] / args.steps,
        "views_in_flight": res["streams"],
        "serial": {"ms_per_step": res["serial_ms"] / args.steps,
                   "value": res["views"] / (res["serial_ms"] * 1e-3), "unit": "frames/s",
                   "note": "the same graph-replayed steps one view at a time on one stream"},
        "host_submit_ms_per_step": round(res["host_submit_ms"], 4),
        "train_step": {"value": res["views"] / (res["train_ms"] * 1e-3), "unit": "views/s",
                       "ms_per_step": res["train_ms"] / res["views"] * world,
                       "note": "the fwd+bwd step followed by a sparse Adam step of the view's cut "
                               "(device-resident float32 state, per-column rates)"},
        "fwd_only": {"value": res["views"] / (res["fwd_ms"] * 1e-3), "unit": "frames/s",
                     "ms_per_frame": res["fwd_ms"] / args.steps,
                     "note": "eager, one view at a time",
                     "views_in_flight_ms_per_frame": {str(k): round(v, 4) for k, v in res["fwd_inflight_ms"].items()},
                     "views_in_flight_note": "graph-replayed forward (camera upload, select, render) round-robin "
                                             "on K streams, ms per view"},
        "select_batch": {"ms_per_view": {str(k): v for k, v in res["select_batch_ms"].items()},
                         "note": "LoD selection alone for groups of K distinct views, graph-replayed on one "
                                 "stream: K lodgs_select_lod calls one after another against one "
                                 "lodgs_select_lod_batch (each selection pass launched once for the K views)"},
        "e2e": {"value": res["views"] / (res["e2e_ms"] * 1e-3), "unit": "frames/s",
                "h2d_bytes_per_step": res["h2d_bytes"], "d2h_bytes_per_step": res["d2h_bytes"],
                "note": "each view's 8-bit RGB target (pinned host) uploaded on a copy stream while the "
                        "previous view computes; the loss read back every step; the median of three passes "
                        "over the K steps (each pass's time the larger of its device and wall times)",
                "passes_ms": res["e2e_passes_ms"]},
        "gpu_launches": int(res["launches"]),
        "stages_ms": {k: round(v, 4) for k, v in res["stage_ms_eager"].items()},
        "stages_note": "stages_ms: the timed steps replayed eagerly with every stage timed; the roofline kernel "
                       "(blend_bwd) is timed by events inside the graph-replayed timed region",
        "clocks": res["clocks"],
        "status_ok": res["stats_ok"],
    }
    if "gbs" in ds:
        line["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": ds["gbs"], "peak": peaks["hbm_gbs"],
                            "unit": "GB/s", "frac": ds["frac_hbm"], "traffic": None,
                            "peak_source": peaks["source"] + " (MEASURED_PEAKS hbm_gbs)"}
    else:
        line["roofline"] = {"bound": "alu", "kernel": dom, "achieved": ds.get("tinst_s"), "peak": rf["alu_peak"],
                            "unit": "T inst/s", "frac": ds.get("frac_alu"),
                            "traffic": BLEND_BWD_DRAM_BYTES if dom == "blend_bwd" else None,
                            "peak_source": f"148 SMs x 128 issue lanes x {rf['mhz']:.0f} MHz (median SM clock "
                                           "in the timed region)",
                            "work": f"algorithmic instructions = {OPS_EVAL + OPS_BWD_CONTRIB} per backward "
                                    f"contribution ({OPS_EVAL + OPS_BLEND} per forward blend)",
                            "work_per_view": rf["work"],
                            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                                              "kernel, mean per launch over the 32 views (one capture of "
                                              "the launch list on the current kernel code)",
                            "ncu_issue_active": BLEND_BWD_ISSUE_ACTIVE if dom == "blend_bwd" else None,
                            "ncu_note": "issue slots the kernel used, one 1080p view (ncu "
                                        "smsp__issue_active, --set full capture); frac counts only the "
                                        "method's instructions in those slots"}
    line["roofline_stages"] = {k: {kk: round(vv, 4) for kk, vv in v.items()} for k, v in rf["stages"].items()}
    def section(name, fn):
        try:
            line[name] = fn(args)
        except Exception as e:  # noqa: BLE001  (a failed side workload must not lose the main line)
            line[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        import torch
        torch.cuda.empty_cache()

    if world == 1 and not args.no_config1:
        section("config1", run_config1)
    if world == 1 and not args.no_out_of_core:
        section("out_of_core", run_out_of_core)
    if world == 1 and not args.no_lod_sweep:
        section("lod_sweep", run_lod_sweep)
    if world == 1 and not args.no_serving:
        section("serving", run_serving)
    if world == 1 and not args.no_train_batch:
        section("train_batch", run_train_batch)
    if world == 1 and not args.no_densify:
        section("densify", run_densify)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
