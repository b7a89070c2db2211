"""Pins of the oracle's out-of-core cache model (Sec. 4.4 "Caching on the GPU",
Eq. 7, Algorithm 3) against facts that do not come from the model itself: the
cache-free cut, a brute-force descent inside each SPT at the distance its
cached cut was taken at, proper cuts, the streamed prefix sizes, and the slab
and LRU invariants."""
import numpy as np
import pytest

import oracle
from oracle import cache as oc
from paper_2507_01110_b300 import synth


@pytest.fixture(scope="module")
def world(oracle_lib):
    leaves = synth.leaves_ground_and_boxes(20000, seed=43, degree=0, extent=300.0, n_boxes=40)
    cams = synth.flyover_path()
    sc = oracle.build_scene(leaves, 0, 50.0, float(cams[0].fx))
    needs = [oracle.select(sc, c)[1]["spt_scanned"] for c in cams]
    return sc, cams + cams[::-1], int(1.3 * max(needs)), sum(needs)


def _descend(sc, j, x):
    """Brute force inside SPT j: the first node on every root-to-leaf path whose
    own unclamped bound lo_raw <= x (leaves always), as render rows."""
    left, right, lo_raw, row = sc["left"], sc["right"], sc["lo_raw"], sc["row_of_node"]
    out, stack = [], [int(sc["spt_root"][j])]
    while stack:
        v = stack.pop()
        if left[v] < 0 or lo_raw[v] <= x:
            out.append(row[v])
        else:
            stack += [right[v], left[v]]
    return out


def _covered_leaves_ok(sc, rows):
    left, right = sc["left"], sc["right"]
    cover = np.zeros(len(left), dtype=np.int32)
    for v in sc["node_of_row"][rows]:
        st = [v]
        while st:
            w = st.pop()
            if left[w] < 0:
                cover[w] += 1
            else:
                st += [left[w], right[w]]
    return cover.max() <= 1


def test_window_of_one_gives_the_cache_free_cut_under_eviction(world):
    """D_min = D_max = 1 reuses a cached cut only at the distance it was taken,
    so every view's cut is the plain LoD cut, whatever the cache evicted."""
    sc, cams, cap, total = world
    assert cap < total
    m = oc.NodeCache(sc, cap, 1.0, 1.0)
    ev = 0
    for i, cam in enumerate(cams):
        rows, st = m.view(cam)
        sel, st_o = oracle.select(sc, cam)
        assert np.array_equal(rows, sel)
        if i == 0:
            assert st["records_streamed"] == st_o["spt_scanned"] and st["spt_hits"] == 0
        ev += st["evictions"]
    assert ev > 0


def test_wide_window_reuses_the_first_cut_of_each_spt(world):
    """With a window wide enough to accept any distance and room for every SPT,
    each SPT keeps the cut taken the first time a view reached it: the view's
    cut is the upper cut plus, per SPT, the brute-force descent at that first
    distance."""
    sc, cams, _, _ = world
    m = oc.NodeCache(sc, int(sc["node_rec"].shape[0]), 1e-3, 1e3)
    first = {}
    for cam in cams[:12]:
        rows, st = m.view(cam)
        up, js, xs = oracle.select_upper(sc, cam)
        expect = list(up)
        for j, x in zip(js.tolist(), xs):
            first.setdefault(j, np.float32(x))
            expect += _descend(sc, j, first[j])
        assert np.array_equal(rows, np.sort(np.array(expect, dtype=np.int64)))
        assert st["evictions"] == 0
    assert st["spt_hits"] > 0


def test_cuts_proper_slab_tiled_and_evictions_least_recent(world):
    """Eq. 7 window [0.9, 1.1] under eviction: every view's cut is proper (no
    node together with an ancestor); after every view the cached prefixes and
    the free ranges tile the slab exactly, with no two free ranges adjacent;
    and every SPT evicted was, at its eviction, no more recently used than any
    SPT that stayed cached without being used by that view."""
    sc, cams, cap, _ = world
    m = oc.NodeCache(sc, cap, 0.9, 1.1)
    kinds = dict.fromkeys(("spt_hits", "spt_resident", "spt_loaded", "evictions"), 0)
    for v, cam in enumerate(cams, start=1):
        rows, st = m.view(cam)
        for k in kinds:
            kinds[k] += st[k]
        assert _covered_leaves_ok(sc, rows)
        spans = sorted([(e["off"], e["h"]) for e in m.entries.values()] + sorted(m.free.items()))
        at = 0
        for off, n in spans:
            assert off == at and n > 0
            at += n
        assert at == cap
        fr = sorted(m.free.items())
        assert all(a + n < b for (a, n), (b, _) in zip(fr, fr[1:]))
        assert st["cached_records"] == sum(e["h"] for e in m.entries.values()) <= cap
        stayed = [e["used"] for e in m.entries.values() if e["used"] < v]
        for (ve, _, used) in m.evicted:
            if ve == v:
                assert all(u >= used for u in stayed)
    assert all(n > 0 for n in kinds.values()), kinds


def test_capacity_smaller_than_one_view_is_an_error(world):
    sc, cams, cap, _ = world
    m = oc.NodeCache(sc, 64, 0.9, 1.1)
    with pytest.raises(oc.CacheCapacityError):
        m.view(cams[0])
