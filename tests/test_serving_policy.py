"""The render server's admission and overflow decisions (pick_slot, with and
without growth of a free slot at admission, and overflow_action) on the CPU:
a simulation with the server loop's structure
over fake slots whose selection and pair buffers overflow separately, as the
library's do.  Every request completes (no request goes back to the queue
forever), each one returns to the queue at most once per slot, and the slots
grow past the budget only when no slot could hold a view and the idle slots,
returned to their base size, could not make room (shrink_plan)."""
import collections
import random
from types import SimpleNamespace

import pytest

from paper_2507_01110_b300 import serving

FIXED, PER_SEL, PER_PAIR = 1000, 128, 24


def _bytes(ns, npairs):
    return FIXED + ns * PER_SEL + npairs * PER_PAIR


def _slot(cap_sel, cap_pairs):
    s = SimpleNamespace(cap_sel=cap_sel, cap_pairs=cap_pairs, req=None, age=0)
    s.held = _bytes(cap_sel, cap_pairs)
    return s


def _simulate(rng, n_slots, budget, views, lookahead, sizes=None, grow=False):
    """The server loop: completions (overflow -> retry or requeue), then
    admission of the head and up to `lookahead` later requests.  sizes: the
    slots' (selection, pair) capacities after a warm-up (default: base).
    grow: admission may grow a free slot within the budget's room to GROWTH x
    the largest counts its class completed with (the server's reserve)."""
    base = _bytes(64, 256)
    slots = [_slot(*(sizes[i] if sizes else (64, 256))) for i in range(n_slots)]
    while len(slots) > 1 and sum(s.held for s in slots) > budget:
        slots.pop()
    need = {}
    counts = {}                                          # class -> largest completed (selection, pairs)
    _simulate.max_inflight = 0
    reqs = [SimpleNamespace(rid=i, cls=c, ns=ns, np=npairs, tried=set(), requeues=0, done=False)
            for i, (c, ns, npairs) in enumerate(views)]
    pending = collections.deque(reqs)
    forced = 0
    shrinks = [0]
    done = 0
    for tick in range(20_000):
        if done == len(reqs):
            break
        for s in slots:                                  # every launched view finishes in one tick
            r = s.req
            if r is None:
                continue
            s.req = None
            vb = _bytes(r.ns, r.np)
            if r.ns > s.cap_sel or r.np > s.cap_pairs:   # overflow: the class's need rises
                need[r.cls] = max(need.get(r.cls, 0), vb)
                r.tried.add(id(s))
                act = serving.overflow_action(vb, need[r.cls], s, slots, r.tried, budget)
                if act == "retry":                       # grows the short buffer, launches again
                    grown = sum(x.held for x in slots) - s.held + int(serving.GROWTH * vb)
                    for idle in serving.shrink_plan(grown, s, slots, budget, base):
                        idle.cap_sel, idle.cap_pairs, idle.held = 64, 256, base
                        shrinks[0] += 1
                    before = sum(x.held for x in slots)
                    if r.ns > s.cap_sel:
                        s.cap_sel = int(serving.GROWTH * r.ns)
                    else:
                        s.cap_pairs = int(serving.GROWTH * r.np)
                    s.held = _bytes(s.cap_sel, s.cap_pairs)
                    if sum(x.held for x in slots) > budget >= before:
                        forced += 1
                    s.req = r
                else:
                    r.requeues += 1
                    pending.appendleft(r)
                continue
            need[r.cls] = max(need.get(r.cls, 0), vb)
            c = counts.get(r.cls, (0, 0))
            counts[r.cls] = (max(c[0], r.ns), max(c[1], r.np))
            r.done = True
            done += 1
            for idle in serving.shrink_plan(sum(x.held for x in slots), s, slots, budget, base):
                idle.cap_sel, idle.cap_pairs, idle.held = 64, 256, base    # a growth past its estimate
                shrinks[0] += 1
        free = [s for s in slots if s.req is None]
        q = 0
        while q < min(len(pending), 1 + lookahead) and free:
            r = pending[q]
            busy = len(free) < len(slots)
            room = budget - sum(x.held for x in slots) if grow else None
            s = serving.pick_slot(need.get(r.cls), r.tried, free, slots, can_wait=busy or q > 0, room=room)
            if s is None:
                q += 1
                continue
            if grow and need.get(r.cls) is not None and s.held < need[r.cls] and r.cls in counts:
                ns, npairs = counts[r.cls]                # the server's reserve: grow, never shrink
                s.cap_sel = max(s.cap_sel, int(serving.GROWTH * ns))
                s.cap_pairs = max(s.cap_pairs, int(serving.GROWTH * npairs))
                s.held = _bytes(s.cap_sel, s.cap_pairs)
            del pending[q]
            free.remove(s)
            s.req = r
        _simulate.max_inflight = max(_simulate.max_inflight, sum(x.req is not None for x in slots))
    _simulate.shrinks = shrinks[0]
    return reqs, slots, forced, tick, base


@pytest.mark.parametrize("seed", range(200))
def test_every_request_completes_and_requeues_at_most_once_per_slot(seed):
    rng = random.Random(seed)
    grow = seed % 2 == 1                                  # half the cases grow free slots at admission
    n_slots = rng.randint(1, 6)
    budget = rng.choice([1, 50_000, 200_000, 2_000_000])
    classes = [(rng.randint(10, 3000), rng.randint(10, 20000)) for _ in range(rng.randint(1, 5))]
    views = []
    for _ in range(rng.randint(1, 40)):
        c = rng.randrange(len(classes))
        ns, npairs = classes[c]
        views.append((c, max(1, int(ns * rng.uniform(0.3, 1.6))), max(1, int(npairs * rng.uniform(0.3, 1.6)))))
    reqs, slots, forced, ticks, _ = _simulate(rng, n_slots, budget, views, lookahead=rng.choice([0, 1, 8]),
                                              grow=grow)
    assert all(r.done for r in reqs), (seed, ticks)
    assert all(r.requeues <= len(slots) for r in reqs)


def test_the_budget_holds_when_a_large_enough_slot_exists():
    """Two large slots and four small ones within the budget; heavy views of a
    class learned on light ones overflow the small slots and wait for the large
    ones instead of growing the small ones."""
    rng = random.Random(7)
    views = [(0, 50, 200)] * 4 + [(0, 2000, 9000)] * 6 + [(0, 50, 200)] * 6
    big = _bytes(2500, 11000)
    budget = 2 * big + 4 * _bytes(64, 256) + 10
    slots_ref = None

    def run():
        reqs, slots, forced, _, _ = _simulate(rng, 6, budget, views, lookahead=8)
        return reqs, slots, forced

    # pre-size two slots as the warm-up would
    orig = _slot

    def sized(cap_sel, cap_pairs, made=[0]):
        made[0] += 1
        return orig(2500, 11000) if made[0] <= 2 else orig(cap_sel, cap_pairs)

    globals()["_slot"] = sized
    try:
        reqs, slots, forced = run()
    finally:
        globals()["_slot"] = orig
    assert all(r.done for r in reqs) and forced == 0
    assert sum(s.held for s in slots) <= budget
    assert any(r.requeues for r in reqs)


def test_shrink_plan_returns_the_largest_idle_slots_until_the_growth_fits():
    base = 100
    mk = lambda held, busy=False: SimpleNamespace(held=held, req=object() if busy else None)
    grower, a, b, c, busy = mk(300), mk(900), mk(400), mk(100), mk(2000, busy=True)
    slots = [grower, a, b, c, busy]
    total = sum(x.held for x in slots)                               # 3700
    assert serving.shrink_plan(total, grower, slots, 4000, base) == []          # fits already
    assert serving.shrink_plan(total + 500, grower, slots, 4000, base) == [a]   # 4200 - 800 <= 4000
    assert serving.shrink_plan(total + 1200, grower, slots, 4000, base) == [a, b]   # 4900 - 800 - 300
    assert serving.shrink_plan(total + 3000, grower, slots, 4000, base) == []   # idle slots cannot make room


def test_a_view_larger_than_every_slot_grows_within_the_budget_by_shrinking_idle_slots():
    """Light requests spread over all slots, then heavy ones of the same class
    that no slot holds: the slot that grows takes its room from idle slots
    returned to their base size, and the slots stay within the budget."""
    rng = random.Random(11)
    light, heavy = (0, 200, 800), (0, 3000, 12000)
    views = [light] * 12 + [heavy] * 3 + [light] * 6
    g = serving.GROWTH
    lcap = (int(g * 200), int(g * 800))
    light_slot = _bytes(*lcap)
    heavy_slot = _bytes(int(g * 3000), int(g * 12000))
    budget = 4 * light_slot + heavy_slot          # six light slots fit; a heavy one needs two of them back
    reqs, slots, forced, _, _ = _simulate(rng, 6, budget, views, lookahead=8, sizes=[lcap] * 6)
    assert all(r.done for r in reqs)
    assert forced == 0 and _simulate.shrinks > 0
    assert sum(s.held for s in slots) <= budget


def test_admission_grows_free_base_slots_instead_of_queueing_behind_the_one_large_slot():
    """Slots returned to their base size (after shrinks) hold no mid-size
    class; one large slot does.  Without growth at admission every request of
    the class waits for the large slot (one in flight); with it, free base
    slots grow within the budget's room and the requests overlap, and the
    growth at admission never takes the slots past the budget."""
    g = serving.GROWTH
    mid = (0, 1000, 4000)
    views = [mid] * 30
    mid_slot = _bytes(int(g * 1000), int(g * 4000))
    big = (4 * int(g * 1000), 4 * int(g * 4000))
    budget = _bytes(*big) + 3 * mid_slot + 2 * _bytes(64, 256)
    sizes = [big] + [(64, 256)] * 5
    inflight = {}
    for grow in (False, True):
        reqs, slots, forced, _, _ = _simulate(random.Random(5), 6, budget, views, lookahead=8, sizes=sizes,
                                              grow=grow)
        assert all(r.done for r in reqs)
        assert forced == 0 and sum(x.held for x in slots) <= budget
        inflight[grow] = _simulate.max_inflight
    # the room's check charges GROWTH x the 10% margin: two of the three mid-size slots it could hold
    assert inflight[False] == 1 and inflight[True] == 3, inflight
