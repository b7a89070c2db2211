"""Continuous-batching render server over one device-resident scene.

Requests (camera, LoD threshold, resolution, arrival time) are admitted as
soon as a slot and device memory allow, whatever the state of the requests
already on the GPU: each slot owns a frame (LoD cut, splats, sorted pairs,
workspace), an output image and a CUDA stream, so admitted requests run
concurrently and overlap on the device.  Completion is polled with CUDA
events; latency is arrival to completion.  The scene (and the cache, in
out-of-core mode) is shared and read only, so a request's image does not depend
on what else is in flight: every kernel of a view reads only that view's frame.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib, api


@dataclass
class Request:
    rid: int
    arrival_s: float
    camera: object
    t_enqueue: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    retries: int = 0
    status: str = "pending"          # "done", "expired" (deadline passed in the queue), "failed: ..."
    checksum: float | None = None
    image: torch.Tensor | None = field(default=None, repr=False)


def request_bytes(width: int, height: int) -> int:
    """Device memory a request is charged at admission: its image plus the
    per-view workspace that grows with the pixel count ((Gaussian, tile) pairs,
    tile ranges); 64 bytes per pixel covers the workspaces measured on the
    1080p trajectory with margin."""
    return width * height * (12 + 64)


class _Slot:
    def __init__(self, scene: api.Scene, max_pixels: int):
        self.frame = api.Frame(scene)
        self.stream = torch.cuda.Stream()
        self.image = torch.empty(max_pixels * 3, dtype=torch.float32, device="cuda")
        self.done = torch.cuda.Event()
        self.req: Request | None = None
        self.bytes = 0


class RenderServer:
    def __init__(self, scene: api.Scene, n_slots: int = 8, mem_budget_bytes: int = 4 << 30,
                 max_pixels: int = 3840 * 2160, rows: torch.Tensor | None = None, keep_images: bool = False):
        self.scene = scene
        self.rows = rows
        self.slots = [_Slot(scene, max_pixels) for _ in range(n_slots)]
        self.budget = mem_budget_bytes
        self.keep_images = keep_images

    def _launch(self, slot: _Slot, req: Request) -> bool:
        """Enqueue the request on the slot; False (request marked failed, slot
        left free) if the library refused it, e.g. out of device memory."""
        cam = req.camera
        img = slot.image[: cam.height * cam.width * 3].view(cam.height, cam.width, 3)
        try:
            with torch.cuda.stream(slot.stream):
                api.select_lod(self.scene, cam, slot.frame, stream=slot.stream)
                api.render(self.scene, slot.frame, rows=self.rows, image=img, stream=slot.stream,
                           check_capacity=False)
                slot.done.record(slot.stream)
        except _lib.LodgsError as e:
            req.status = f"failed: {e}"
            return False
        slot.req = req
        return True

    def _finish(self, slot: _Slot, now: float) -> bool:
        """True if the request completed; False if its frame had to grow and it
        was launched again."""
        req = slot.req
        st = slot.frame.stats()                      # the stream is idle: no wait
        if st["status"] == _lib.LODGS_E_CAPACITY:
            req.retries += 1
            if not self._launch(slot, req):          # growing the workspace failed: give up on it
                slot.req = None
                return True
            return False
        _lib.check(st["status"])
        cam = req.camera
        img = slot.image[: cam.height * cam.width * 3].view(cam.height, cam.width, 3)
        if self.keep_images:
            req.image = img.clone()
        req.t_done = now
        req.status = "done"
        slot.req = None
        return True

    def warm(self, cameras) -> None:
        """Grow every slot's workspace on representative cameras (not timed)."""
        for slot in self.slots:
            for cam in cameras:
                img = slot.image[: cam.height * cam.width * 3].view(cam.height, cam.width, 3)
                api.select_lod(self.scene, cam, slot.frame)
                api.render(self.scene, slot.frame, rows=self.rows, image=img, check_capacity=True)
        torch.cuda.synchronize()

    def run(self, requests: list[Request], realtime: bool = True, deadline_ms: float | None = None) -> dict:
        """Serve `requests` (sorted by arrival).  realtime: requests arrive on
        the wall clock at their arrival times.  deadline_ms: a request still
        queued that long after it arrived is dropped ("expired").  A request
        the library refuses (e.g. out of device memory) is marked failed and the
        server carries on; latencies are over the completed requests."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        pending = collections.deque()
        nxt = 0
        in_use = 0
        done = 0
        inflight_max = 0
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival_s <= now):
                reqs[nxt].t_enqueue = reqs[nxt].arrival_s if realtime else now
                pending.append(reqs[nxt])
                nxt += 1
            # completions first: they free slots and memory
            for slot in self.slots:
                if slot.req is not None and slot.done.query():
                    if self._finish(slot, time.perf_counter() - t0):
                        in_use -= slot.bytes
                        slot.bytes = 0
                        done += 1
            # admission: any pending request that fits a free slot and the memory budget
            free = [s for s in self.slots if s.req is None]
            while pending and free:
                req = pending[0]
                if deadline_ms is not None and (time.perf_counter() - t0 - req.t_enqueue) * 1e3 > deadline_ms:
                    pending.popleft()                # waited past its deadline: never launched
                    req.status = "expired"
                    done += 1
                    continue
                need = request_bytes(req.camera.width, req.camera.height)
                if in_use + need > self.budget and in_use > 0:
                    break
                pending.popleft()
                slot = free.pop()
                req.t_admit = time.perf_counter() - t0
                if not self._launch(slot, req):
                    free.append(slot)
                    done += 1
                    continue
                slot.bytes = need
                in_use += need
            inflight_max = max(inflight_max, sum(s.req is not None for s in self.slots))
            time.sleep(0)
        wall = time.perf_counter() - t0
        # latency from arrival (realtime) or from being queued (batch mode) to completion
        ok = [r for r in reqs if r.status == "done"]
        lat = np.array([(r.t_done - r.t_enqueue) * 1e3 for r in ok]) if ok else np.zeros(1)
        return {"requests": len(reqs), "wall_s": wall, "throughput_rps": len(ok) / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_inflight": inflight_max,
                "retries": int(sum(r.retries for r in reqs)),
                "completed": len(ok), "expired": sum(r.status == "expired" for r in reqs),
                "failed": sum(r.status.startswith("failed") for r in reqs)}


def poisson_requests(cameras, rate_per_s: float, n: int, seed: int) -> list[Request]:
    """Seeded Poisson arrivals over a list of candidate cameras."""
    from . import synth
    idx = np.arange(n, dtype=np.uint64)
    gaps = -np.log(synth.uniform_open(seed, 500, idx)) / rate_per_s
    pick = (synth.uniform(seed, 501, idx) * len(cameras)).astype(np.int64)
    t = np.cumsum(gaps)
    return [Request(rid=i, arrival_s=float(t[i]), camera=cameras[int(pick[i])]) for i in range(n)]
