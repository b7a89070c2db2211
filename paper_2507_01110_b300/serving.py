"""Continuous-batching render server over one device-resident scene.

Requests (camera, LoD threshold, resolution, arrival time) are admitted as
soon as a slot and device memory allow, whatever the state of the requests
already on the GPU: each slot owns a frame (LoD cut, splats, sorted pairs,
workspace), an output image and a CUDA stream, so admitted requests run
concurrently and overlap on the device.  Completion is polled with CUDA
events; latency is arrival to completion.  The scene (and the cache, in
out-of-core mode) is shared and read only, so a request's image does not depend
on what else is in flight: every kernel of a view reads only that view's frame.

Admission by memory: the budget bounds the device workspace the slots hold
together (what lodgs_frame_memory reports as held; a frame's workspace only
grows).  warm() learns, per request class (resolution and LoD threshold), the
largest workspace a request of the class needed, then sizes the slots within
the budget: the first slot for the largest class, each next one for the
largest class that still leaves the remaining slots their base size.  A
request is admitted to a free slot whose workspace already holds its class's
need (the one with the least to spare); if none does but the budget has room
to grow a free slot to that need, the largest such slot grows (before the
launch, to the class's largest rendered counts) and takes it; otherwise, if
every slot that could hold it is busy it waits, and up to `lookahead` later
requests that fit a free slot may start before it.  A request whose view
overflows its slot (another camera of its class can need more than the
warm-up saw, or one buffer of a slot can be short while its total is not)
raises its class's need; it is rendered again on the same slot, which grows,
if the budget still holds the grown slot or no slot
it has not yet overflowed could hold it; otherwise the queued growth is
cancelled (lodgs_frame_reserve) and the request goes back to the head of the
queue to wait for one of those slots.  A request therefore goes back to the
queue at most once per slot before it grows one.  A growth that would break
the budget first returns idle slots to a fresh workspace, largest first, if
that makes room; only when the idle slots cannot make room does a growth take
the slots past the budget.  A class not seen in the
warm-up is admitted alone to the largest slot (which grows if it must).  The
server keeps only as many slots as the budget holds at their base size (at
least one).

Requests admitted in the same pass of the loop share one batched LoD
selection (lodgs_select_lod_batch: each selection pass launched once for up
to eight views) on the server's front stream; each one's render then runs on
its own slot's stream after it.  The selection of a view in a batch is the
one it has alone, so a request's image still does not depend on the others.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib, api

GROWTH = 1.25      # a frame buffer that overflows grows to 1.25 x the count that overflowed it
GROWTH_MARGIN = 1.1   # a growth can take more than GROWTH x the needed bytes (buffers grow separately)


@dataclass
class Request:
    rid: int
    arrival_s: float
    camera: object
    t_enqueue: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    retries: int = 0                 # renders again on the same slot after an overflow
    requeues: int = 0                # returns to the queue after an overflow (no growth within the budget)
    status: str = "pending"          # "done", "expired" (deadline passed in the queue), "failed: ..."
    dev_ms: tuple | None = None      # (start, end) on the device, ms from the run's start
    tried: set = field(default_factory=set)   # slots this request overflowed
    ev_start: object = field(default=None, repr=False)
    image: torch.Tensor | None = field(default=None, repr=False)


def request_class(camera) -> tuple:
    """The admission class of a request: its resolution and LoD threshold."""
    return (int(camera.width), int(camera.height), round(float(camera.tau), 6))


def pick_slot(need, tried, free, slots, can_wait: bool, room=None):
    """The free slot a queued request takes, or None (it waits).  need: its
    class's workspace bytes (None: class not seen yet); tried: the slots it has
    overflowed; free: the free slots; slots: all of them; can_wait: whether it
    may wait for a busy slot (the head of the queue may not wait when nothing is
    in flight); room: the bytes the budget has left (None: no slot is grown at
    admission).  When no free slot holds the class but one can grow to it
    within `room`, the request takes the largest such slot (the caller grows
    it) instead of queueing behind a busy slot that holds it.  Slots are
    anything with a `held` byte count."""
    if need is None:                                 # a class not seen yet: alone, on the largest slot
        if can_wait:
            return None
        return max(free, key=lambda s: s.held)
    usable = [s for s in free if id(s) not in tried]
    fits = [s for s in usable if s.held >= GROWTH * need] or [s for s in usable if s.held >= need]
    if fits:
        return min(fits, key=lambda s: s.held)
    if room is not None:
        growable = [s for s in usable if GROWTH * GROWTH_MARGIN * need - s.held <= room]
        if growable:
            return max(growable, key=lambda s: s.held)
    if can_wait and any(s.held >= need and id(s) not in tried for s in slots):
        return None                                  # a slot that holds it is busy: wait for it
    if can_wait:
        return None
    return max(free, key=lambda s: s.held)           # none can: the largest grows


def overflow_action(needed: int, need: int, slot, slots, tried, budget: int) -> str:
    """After a request's view overflowed `slot` (needed: the bytes the view
    needs; need: its class's need, at least `needed`, the threshold pick_slot
    applies), 'retry' on this slot, which grows, or 'requeue' (growth
    cancelled) to wait for another slot.  It requeues only while the grown slot
    would break the budget and some slot it has not overflowed holds `need`;
    pick_slot then gives it such a slot, so every requeue is followed by a
    launch on a slot it has not tried, or by growth: a request requeues at most
    once per slot."""
    grown = sum(s.held for s in slots) - slot.held + int(GROWTH * needed)
    others = [s for s in slots if s is not slot and id(s) not in tried and s.held >= need]
    return "requeue" if grown > budget and others else "retry"


def shrink_plan(grown_total: int, slot, slots, budget: int, base: int) -> list:
    """The idle slots to return to their base workspace (largest first) so
    that `slot`, growing the slots' total to `grown_total`, stays within the
    budget; [] if it already does or if even all of them would not make room
    (the growth then goes past the budget: no slot could hold the view)."""
    if grown_total <= budget:
        return []
    idle = sorted((s for s in slots if s is not slot and s.req is None and s.held > base), key=lambda s: -s.held)
    plan, total = [], grown_total
    for s in idle:
        if total <= budget:
            break
        plan.append(s)
        total -= s.held - base
    return plan if total <= budget else []


class _Slot:
    def __init__(self, scene: api.Scene, max_pixels: int):
        self.frame = api.Frame(scene)
        self.stream = torch.cuda.Stream()
        self.image = torch.empty(max_pixels * 3, dtype=torch.float32, device="cuda")
        self.done = torch.cuda.Event(enable_timing=True)
        self.req: Request | None = None
        self.held = self.frame.memory()[0]


class RenderServer:
    def __init__(self, scene: api.Scene, n_slots: int = 8, mem_budget_bytes: int = 4 << 30,
                 max_pixels: int = 3840 * 2160, rows: torch.Tensor | None = None, keep_images: bool = False,
                 lookahead: int = 8, batch_select: bool = True):
        self.scene = scene
        self.rows = rows
        self.max_pixels = max_pixels
        self.slots = [_Slot(scene, max_pixels) for _ in range(n_slots)]
        self.budget = mem_budget_bytes
        self.keep_images = keep_images
        self.lookahead = lookahead
        self.batch_select = batch_select  # one batched selection for the requests admitted together
        self.front = torch.cuda.Stream()  # where the batched selections run
        self.batches = self.batched_views = self.shrinks = 0
        self.peak = 0                     # the largest workspace the slots held in run(), growths included
        self.need: dict = {}              # request class -> largest workspace bytes it needed
        self.rep: dict = {}               # request class -> the camera of that largest need
        self.counts: dict = {}            # request class -> largest (selected, kept pairs) rendered
        self.grown = 0                    # slots grown at admission (pick_slot with room)
        self._ref = None                  # event at the start of run(): device times are taken from it
        while len(self.slots) > 1 and self.held_bytes() > self.budget:
            self.slots.pop()              # the budget holds fewer slots at their base size (at least one)
        self.warm_bytes = self.held_bytes()   # what the slots hold after warm()
        self.base = min(sl.held for sl in self.slots)   # a fresh frame's workspace

    # ---- memory bookkeeping ----
    def charge(self, camera):
        """The workspace bytes a request's class needs (None: a class not seen yet)."""
        return self.need.get(request_class(camera))

    def held_bytes(self) -> int:
        """Device workspace the slots hold together."""
        return int(sum(s.held for s in self.slots))

    def _learn(self, slot: _Slot, camera, rendered: bool = False) -> int:
        held, needed = slot.frame.memory()
        slot.held = held
        k = request_class(camera)
        if needed > self.need.get(k, -1):
            self.need[k] = needed
            self.rep[k] = camera
        if rendered:                      # a completed view: its counts bound the class's buffers
            st = slot.frame.stats()
            ns, npairs = self.counts.get(k, (0, 0))
            self.counts[k] = (max(ns, int(st["n_selected"])), max(npairs, int(st["n_pairs"])))
        return needed

    def _grow(self, slot: _Slot, camera) -> None:
        """Grow a free slot's workspace for a request's class before its
        launch (admission within the budget's room): GROWTH x the largest
        selection and kept-pair counts the class rendered.  A view that needs
        more (a frame on the global ordering stores every rectangle pair)
        overflows once and grows on the overflow path, as does a class known
        only from an overflow; a failed growth leaves the slot as it was."""
        counts = self.counts.get(request_class(camera))
        if counts is None:
            return
        try:
            slot.frame.reserve(int(GROWTH * counts[0]), int(GROWTH * counts[1]))
            self.grown += 1
        except _lib.LodgsError:
            pass
        slot.held = slot.frame.memory()[0]

    def _render(self, slot: _Slot, cam) -> None:
        img = slot.image[: cam.height * cam.width * 3].view(cam.height, cam.width, 3)
        api.select_lod(self.scene, cam, slot.frame)
        api.render(self.scene, slot.frame, rows=self.rows, image=img, check_capacity=True)

    # ---- one request on one slot ----
    def _launch(self, slot: _Slot, req: Request) -> bool:
        """Enqueue the request on the slot; False (request marked failed, slot
        left free) if the library refused it, e.g. out of device memory."""
        cam = req.camera
        img = slot.image[: cam.height * cam.width * 3].view(cam.height, cam.width, 3)
        try:
            with torch.cuda.stream(slot.stream):
                if req.ev_start is None:             # the device start of the request's first launch
                    req.ev_start = torch.cuda.Event(enable_timing=True)
                    req.ev_start.record(slot.stream)
                api.select_lod(self.scene, cam, slot.frame, stream=slot.stream)
                api.render(self.scene, slot.frame, rows=self.rows, image=img, stream=slot.stream,
                           check_capacity=False)
                slot.done.record(slot.stream)
        except _lib.LodgsError as e:
            req.status = f"failed: {e}"
            return False
        slot.req = req
        return True

    def _launch_together(self, admitted: list) -> list:
        """Enqueue requests admitted in the same pass: one batched LoD
        selection per LODGS_SELECT_BATCH_MAX of them on the front stream, after
        which each render runs on its slot's stream.  A batch the library
        refuses (e.g. one invalid camera) is launched view by view, so only the
        offending request fails.  Returns the pairs that failed (slot left
        free)."""
        failed = []
        nb = _lib.LODGS_SELECT_BATCH_MAX
        for i in range(0, len(admitted), nb):
            chunk = admitted[i:i + nb]
            if len(chunk) == 1 or not self.batch_select:
                failed += [(s, r) for s, r in chunk if not self._launch(s, r)]
                continue
            fs = self.front
            for s, _ in chunk:               # a free slot's stream is idle; the wait keeps the order explicit
                fs.wait_stream(s.stream)
            start = torch.cuda.Event(enable_timing=True)
            start.record(fs)
            try:
                api.select_lod_batch(self.scene, [r.camera for _, r in chunk], [s.frame for s, _ in chunk],
                                     stream=fs)
            except _lib.LodgsError:
                failed += [(s, r) for s, r in chunk if not self._launch(s, r)]
                continue
            selected = torch.cuda.Event()
            selected.record(fs)
            self.batches += 1
            self.batched_views += len(chunk)
            for s, r in chunk:
                cam = r.camera
                img = s.image[: cam.height * cam.width * 3].view(cam.height, cam.width, 3)
                if r.ev_start is None:
                    r.ev_start = start
                s.stream.wait_event(selected)
                try:
                    api.render(self.scene, s.frame, rows=self.rows, image=img, stream=s.stream,
                               check_capacity=False)
                except _lib.LodgsError as e:
                    r.status = f"failed: {e}"
                    failed.append((s, r))
                    continue
                s.done.record(s.stream)
                s.req = r
        return failed

    def _finish(self, slot: _Slot, now: float) -> str:
        """'done', 'retry' (rendered again on this slot, which grows) or
        'requeue' (the slot overflowed and may not grow within the budget)."""
        req = slot.req
        st = slot.frame.stats()                      # the stream is idle: no wait
        if st["status"] == _lib.LODGS_E_CAPACITY:
            needed = self._learn(slot, req.camera)
            req.tried.add(id(slot))
            need = self.charge(req.camera)
            if overflow_action(needed, need, slot, self.slots, req.tried, self.budget) == "retry":
                grown = self.held_bytes() - slot.held + int(GROWTH * GROWTH_MARGIN * needed)
                self._shrink(shrink_plan(grown, slot, self.slots, self.budget, self.base))
                req.retries += 1
                if not self._launch(slot, req):      # growing the workspace failed: give up on it
                    slot.req = None
                    return "done"
                return "retry"
            slot.frame.reserve(0, 0)                 # no growth: wait for a slot that holds it
            req.requeues += 1
            slot.req = None
            return "requeue"
        _lib.check(st["status"])
        cam = req.camera
        img = slot.image[: cam.height * cam.width * 3].view(cam.height, cam.width, 3)
        if self.keep_images:
            req.image = img.clone()
        req.t_done = now
        req.status = "done"
        if self._ref is not None:                    # the request's interval on the device
            req.dev_ms = (self._ref.elapsed_time(req.ev_start), self._ref.elapsed_time(slot.done))
        self._learn(slot, cam, rendered=True)
        self.peak = max(self.peak, self.held_bytes())
        # a growth that took more than its estimate: idle slots make the room back
        self._shrink(shrink_plan(self.held_bytes(), slot, self.slots, self.budget, self.base))
        slot.req = None
        return "done"

    def _shrink(self, idle_slots) -> None:
        """Return slots (idle) to a fresh frame's workspace."""
        for idle in idle_slots:
            idle.frame.close()
            idle.frame = api.Frame(self.scene)
            idle.held = idle.frame.memory()[0]
            self.shrinks += 1

    def warm(self, cameras) -> None:
        """Learn the classes' workspace needs on representative cameras, then
        size the slots within the budget (see the module notes; not timed).
        Slots the budget cannot give their base size are dropped."""
        probe = self.slots[0]
        for cam in cameras:
            self._render(probe, cam)
            self._learn(probe, cam, rendered=True)
        remaining = self.budget - probe.held
        base = min(s.held for s in self.slots[1:]) if len(self.slots) > 1 else 0
        kept = [probe]
        for i, slot in enumerate(self.slots[1:], start=1):
            after = len(self.slots) - i - 1
            room = remaining - after * base
            if slot.held > remaining:
                break
            # a frame grows a quarter beyond what overflowed it: size by 1.25 x the need
            fits = [(n, k) for k, n in self.need.items() if GROWTH * n <= room]
            if fits:
                n, k = max(fits)
                if n > slot.held:
                    self._render(slot, self.rep[k])
                    self._learn(slot, self.rep[k])
                    if slot.held > room:         # grew past its share: a fresh base-size slot instead
                        slot.frame.close()
                        slot = _Slot(self.scene, self.max_pixels)
            kept.append(slot)
            remaining -= slot.held
        self.slots = kept
        torch.cuda.synchronize()
        self.warm_bytes = self.held_bytes()

    def run(self, requests: list[Request], realtime: bool = True, deadline_ms: float | None = None) -> dict:
        """Serve `requests` (sorted by arrival).  realtime: requests arrive on
        the wall clock at their arrival times.  deadline_ms: a request still
        queued that long after it arrived is dropped ("expired").  A request
        the library refuses (e.g. out of device memory) is marked failed and the
        server carries on; latencies are over the completed requests."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        pending = collections.deque()
        nxt = 0
        done = 0
        inflight_max = 0
        held_max = self.held_bytes()
        self.peak = held_max
        self.batches = self.batched_views = self.shrinks = self.grown = 0
        grown_past = 0                    # retries that grew the slots past the budget (no slot could hold the view)
        torch.cuda.synchronize()
        self._ref = torch.cuda.Event(enable_timing=True)
        self._ref.record()
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival_s <= now):
                reqs[nxt].t_enqueue = reqs[nxt].arrival_s if realtime else now
                pending.append(reqs[nxt])
                nxt += 1
            # completions first: they free slots
            for slot in self.slots:
                if slot.req is not None and slot.done.query():
                    req = slot.req
                    out = self._finish(slot, time.perf_counter() - t0)
                    if out == "done":
                        done += 1
                    elif out == "requeue":
                        pending.appendleft(req)
            held = max(self.held_bytes(), self.peak)   # peak: before any shrink that followed a growth
            if held > self.budget and held > held_max:
                grown_past += 1
            held_max = max(held_max, held)
            # admission: the head of the queue, then up to `lookahead` later
            # requests, each to a free slot whose workspace holds its class's need
            free = [s for s in self.slots if s.req is None]
            while deadline_ms is not None and pending and \
                    (time.perf_counter() - t0 - pending[0].t_enqueue) * 1e3 > deadline_ms:
                pending.popleft().status = "expired"     # waited past its deadline: never launched
                done += 1
            q = 0
            admitted = []
            while q < min(len(pending), 1 + self.lookahead) and free:
                req = pending[q]
                busy = len(free) < len(self.slots)
                need = self.charge(req.camera)
                slot = pick_slot(need, req.tried, free, self.slots, can_wait=busy or q > 0,
                                 room=self.budget - self.held_bytes())
                if slot is None:
                    q += 1
                    continue
                if need is not None and slot.held < need:
                    self._grow(slot, req.camera)        # a free slot grown within the budget's room
                del pending[q]
                free.remove(slot)
                req.t_admit = time.perf_counter() - t0
                admitted.append((slot, req))
            done += len(self._launch_together(admitted))
            inflight = sum(s.req is not None for s in self.slots)
            # with nothing in flight every slot is free and pick_slot admits the
            # head (it may not wait): a queue left waiting here would spin forever
            if not inflight and pending and pick_slot(self.charge(pending[0].camera), pending[0].tried,
                                                      self.slots, self.slots, can_wait=False) is None:
                raise RuntimeError("render server: the head of the queue cannot be admitted")
            inflight_max = max(inflight_max, inflight)
            time.sleep(0)
        wall = time.perf_counter() - t0
        # latency from arrival (realtime) or from being queued (batch mode) to completion
        ok = [r for r in reqs if r.status == "done"]
        lat = np.array([(r.t_done - r.t_enqueue) * 1e3 for r in ok]) if ok else np.zeros(1)
        # where the latency goes: the wait before admission (host clock) and the
        # request's interval on the device, first launch to completion (its
        # kernels and whatever ran beside them)
        wait = np.array([(r.t_admit - r.t_enqueue) * 1e3 for r in ok]) if ok else np.zeros(1)
        dev = np.array([r.dev_ms[1] - r.dev_ms[0] for r in ok if r.dev_ms is not None])
        dev = dev if dev.size else np.zeros(1)
        return {"requests": len(reqs), "wall_s": wall, "throughput_rps": len(ok) / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_inflight": inflight_max,
                "admit_wait_p50_ms": float(np.percentile(wait, 50)), "admit_wait_p99_ms": float(np.percentile(wait, 99)),
                "device_p50_ms": float(np.percentile(dev, 50)), "device_p99_ms": float(np.percentile(dev, 99)),
                "gpu_busy": gpu_busy_fraction([r.dev_ms for r in ok if r.dev_ms is not None], wall * 1e3),
                "slots": len(self.slots), "slot_workspace_bytes": self.held_bytes(),
                "peak_slot_workspace_bytes": int(held_max), "budget_bytes": int(self.budget),
                "growths_past_budget": grown_past, "slots_shrunk": self.shrinks,
                "retries": int(sum(r.retries for r in reqs)), "requeues": int(sum(r.requeues for r in reqs)),
                "batched_selections": self.batches, "views_in_batched_selections": self.batched_views,
                "slots_grown_at_admission": self.grown,
                "completed": len(ok), "expired": sum(r.status == "expired" for r in reqs),
                "failed": sum(r.status.startswith("failed") for r in reqs)}


def gpu_busy_fraction(intervals, wall_ms: float) -> float:
    """Fraction of the run's wall time during which at least one request was
    executing on the device: the union of the requests' [start, end] device
    intervals (ms from the run's start) over the wall time."""
    busy, end = 0.0, -np.inf
    for a, b in sorted(intervals):
        if b <= end:
            continue
        busy += b - max(a, end)
        end = b
    return float(busy / wall_ms) if wall_ms > 0 else 0.0


def poisson_requests(cameras, rate_per_s: float, n: int, seed: int) -> list[Request]:
    """Seeded Poisson arrivals over a list of candidate cameras."""
    from . import synth
    idx = np.arange(n, dtype=np.uint64)
    gaps = -np.log(synth.uniform_open(seed, 500, idx)) / rate_per_s
    pick = (synth.uniform(seed, 501, idx) * len(cameras)).astype(np.int64)
    t = np.cumsum(gaps)
    return [Request(rid=i, arrival_s=float(t[i]), camera=cameras[int(pick[i])]) for i in range(n)]
