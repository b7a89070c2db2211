"""The render server's admission and overflow decisions (pick_slot,
overflow_action) on the CPU: a simulation with the server loop's structure
over fake slots whose selection and pair buffers overflow separately, as the
library's do.  Every request completes (no request goes back to the queue
forever), each one returns to the queue at most once per slot, and the slots
grow past the budget only when no slot could hold a view."""
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


def _simulate(rng, n_slots, budget, views, lookahead):
    """The server loop: completions (overflow -> retry or requeue), then
    admission of the head and up to `lookahead` later requests."""
    base = _bytes(64, 256)
    slots = [_slot(64, 256) for _ in range(n_slots)]
    while len(slots) > 1 and sum(s.held for s in slots) > budget:
        slots.pop()
    need = {}
    reqs = [SimpleNamespace(rid=i, cls=c, ns=ns, np=npairs, tried=set(), requeues=0, done=False)
            for i, (c, ns, npairs) in enumerate(views)]
    pending = collections.deque(reqs)
    forced = 0
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
            r.done = True
            done += 1
        free = [s for s in slots if s.req is None]
        q = 0
        while q < min(len(pending), 1 + lookahead) and free:
            r = pending[q]
            busy = len(free) < len(slots)
            s = serving.pick_slot(need.get(r.cls), r.tried, free, slots, can_wait=busy or q > 0)
            if s is None:
                q += 1
                continue
            del pending[q]
            free.remove(s)
            s.req = r
    return reqs, slots, forced, tick, base


@pytest.mark.parametrize("seed", range(200))
def test_every_request_completes_and_requeues_at_most_once_per_slot(seed):
    rng = random.Random(seed)
    n_slots = rng.randint(1, 6)
    budget = rng.choice([1, 50_000, 200_000, 2_000_000])
    classes = [(rng.randint(10, 3000), rng.randint(10, 20000)) for _ in range(rng.randint(1, 5))]
    views = []
    for _ in range(rng.randint(1, 40)):
        c = rng.randrange(len(classes))
        ns, npairs = classes[c]
        views.append((c, max(1, int(ns * rng.uniform(0.3, 1.6))), max(1, int(npairs * rng.uniform(0.3, 1.6)))))
    reqs, slots, forced, ticks, _ = _simulate(rng, n_slots, budget, views, lookahead=rng.choice([0, 1, 8]))
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
