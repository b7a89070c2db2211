"""The out-of-core node cache as a per-view decision model (test infrastructure
only: tests/ use it; the product library never imports it).

What it follows (Sec. 4.4 "Caching on the GPU", Eq. 7, Algorithm 3):
  * the cache holds SPT cuts, each with the distance it was cut at;
  * per view, Algorithm 1 cuts the upper hierarchy and reaches SPT roots j,
    each at the focal-normalised distance x_j = tau d_j / f (times the LoD
    noise factor);
  * a cached SPT with D_min <= x_j / xbar_j <= D_max (Eq. 7) is reused: its cut
    is the one at xbar_j;
  * any other SPT is cut at x_j (Eq. 4), and the cache then holds that cut,
    xbar_j = x_j;
  * when the cache is full, least-recently-used SPTs are written back (Algorithm 3).

Readings of what the paper leaves open (both sides follow them):
  * the ratio of Eq. 7 is taken unsquared, on the float32 x values, as
    x_j / xbar_j compared with float32 D_min, D_max (Algorithm 3 squares the
    distances, Eq. 7 does not);
  * what the cache keeps of an SPT is the prefix [0, high(x)) of its entries in
    descending-hi order, which holds every node a cut at x can select; a non-hit
    whose cached prefix already covers high(x_j) is cut at x_j from it without a
    transfer, and one whose prefix is too short grows it to high(x_j);
  * the memory threshold is a slab of `capacity_records` record slots; each
    cached prefix occupies one contiguous range of it.  A new prefix takes the
    shortest free range that holds it (lowest offset among equals).  A prefix
    that grows takes the free range right after it if that range is long
    enough, else it moves to a new range, and its old range is freed once all
    of the view's SPT roots are decided.  While no free range fits, the least
    recently used SPT is evicted, but never one that this view already used:
    that is a capacity error.  Freed ranges merge with free neighbours.

The statistics use the same names as the CUDA cache's: spt_hits, spt_resident
(non-hits cut from the cached prefix), spt_loaded (new or grown prefixes),
records_streamed, evictions, cached_spts, cached_records.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np


class CacheCapacityError(RuntimeError):
    pass


class NodeCache:
    def __init__(self, scene: dict, capacity_records: int, d_min: float = 0.9, d_max: float = 1.1):
        self.sc = scene
        self.capacity = int(capacity_records)
        self.d_min, self.d_max = np.float32(d_min), np.float32(d_max)
        self.base = np.asarray(scene["spt_base"], np.int64)
        self.lo, self.hi = scene["lo_row"], scene["hi_row"]
        self.flush()

    def flush(self) -> None:
        """Drop every cached SPT (Algorithm 3's periodic flush)."""
        self.entries = {}                 # j -> dict(x, h, off, used)
        self.lru = OrderedDict()          # least recently used first
        self.free = {0: self.capacity}    # offset -> length
        self.view_id = 0
        self.cached_records = 0
        self.evicted = []                 # (view, j, the view that last used j)

    # ---- the slab (reading above) ----
    def _take_best_fit(self, n: int):
        fits = [(ln, off) for off, ln in self.free.items() if ln >= n]
        if not fits:
            return None
        ln, off = min(fits)
        del self.free[off]
        if ln > n:
            self.free[off + n] = ln - n
        return off

    def _take_at(self, at: int, n: int) -> bool:
        ln = self.free.get(at)
        if ln is None or ln < n:
            return False
        del self.free[at]
        if ln > n:
            self.free[at + n] = ln - n
        return True

    def _release(self, off: int, n: int) -> None:
        prev = [o for o, ln in self.free.items() if o + ln == off]
        if prev:
            off, n = prev[0], n + self.free.pop(prev[0])
        if off + n in self.free:
            n += self.free.pop(off + n)
        self.free[off] = n

    def _evict(self, j: int) -> None:
        e = self.entries.pop(j)
        self.evicted.append((self.view_id, j, e["used"]))
        del self.lru[j]
        self._release(e["off"], e["h"])
        self.cached_records -= e["h"]

    def _alloc(self, n: int, st: dict) -> int:
        while True:
            off = self._take_best_fit(n)
            if off is not None:
                return off
            j_old = next(iter(self.lru), None)
            if j_old is None or self.entries[j_old]["used"] == self.view_id:
                raise CacheCapacityError("the view's SPT prefixes exceed the cache")
            self._evict(j_old)
            st["evictions"] += 1

    def _touch(self, j: int) -> None:
        self.lru.move_to_end(j)
        self.entries[j]["used"] = self.view_id

    # ---- the SPT cut (Eq. 4) ----
    def _high(self, j: int, x: np.float32) -> int:
        b, e = self.base[j], self.base[j + 1]
        return int(np.count_nonzero(self.hi[b:e] > x))

    def _cut(self, j: int, x: np.float32) -> np.ndarray:
        b = self.base[j]
        h = self._high(j, x)
        return b + np.nonzero(self.lo[b:b + h] <= x)[0]

    # ---- one view ----
    def view(self, cam, cull: bool = True):
        from . import select_upper
        upper_rows, spt_j, spt_x = select_upper(self.sc, cam, cull)
        self.view_id += 1
        st = dict.fromkeys(("spt_hits", "spt_resident", "spt_loaded", "records_streamed", "evictions"), 0)
        moved_from = []
        parts = [upper_rows]
        for j, x in zip(spt_j.tolist(), spt_x):
            x = np.float32(x)
            need = self._high(j, x)
            e = self.entries.get(j)
            x_used = x
            if e is not None:
                ratio = np.float32(x / e["x"])
                if self.d_min <= ratio <= self.d_max:                     # Eq. 7: reuse the cached cut
                    self._touch(j)
                    st["spt_hits"] += 1
                    parts.append(self._cut(j, e["x"]))
                    continue
                if e["h"] >= need:                                        # cut at x_j from the cached prefix
                    self._touch(j)
                    e["x"] = x
                    st["spt_resident"] += 1
                    parts.append(self._cut(j, x))
                    continue
                self._touch(j)                                            # grow the cached prefix
                grow = need - e["h"]
                if not self._take_at(e["off"] + e["h"], grow):
                    off = self._alloc(need, st)
                    moved_from.append((e["off"], e["h"]))
                    e["off"] = off
                e["h"], e["x"] = need, x
                self.cached_records += grow
                st["records_streamed"] += grow
            else:                                                         # load the prefix
                off = self._alloc(need, st)
                self.entries[j] = {"x": x, "h": need, "off": off, "used": self.view_id}
                self.lru[j] = None
                self.cached_records += need
                st["records_streamed"] += need
            st["spt_loaded"] += 1
            parts.append(self._cut(j, x_used))
        for off, n in moved_from:
            self._release(off, n)
        st["cached_spts"] = len(self.entries)
        st["cached_records"] = self.cached_records
        return np.sort(np.concatenate(parts)).astype(np.int64), st
