"""Continuous-batching server: overlapping requests of mixed resolution and
LoD threshold, admitted together and sharing batched LoD selections, give
exactly the images they give alone."""
import pytest
import torch

from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    from paper_2507_01110_b300 import api, build
    build.build()
    leaves = synth.city_leaves_t(400_000, seed=51, degree=1, extent=600.0, block=60.0, device="cuda")
    cams = synth.serving_cameras(8, seed=51, extent=600.0)
    kappa = min(float(c.fx / c.tau) for c in cams)
    sc = api.build_hierarchy(leaves, 1, 1.0, kappa)
    return sc


def _requests(seed, n=24):
    from paper_2507_01110_b300 import serving
    cams = synth.serving_cameras(12, seed=seed, extent=600.0)
    cams = [c for c in cams if c.width <= 1920]          # keep the test quick
    return serving.poisson_requests(cams, rate_per_s=2000.0, n=n, seed=seed)


def test_results_identical_alone_and_in_the_mix(scene):
    from paper_2507_01110_b300 import serving
    alone = serving.RenderServer(scene, n_slots=1, keep_images=True, max_pixels=1920 * 1080)
    r_alone = _requests(52)
    st_alone = alone.run(r_alone, realtime=False)
    mix = serving.RenderServer(scene, n_slots=6, keep_images=True, max_pixels=1920 * 1080)
    mix.warm([r.camera for r in r_alone[:4]])          # some classes known, the others admitted alone first
    r_mix = _requests(52)
    st_mix = mix.run(r_mix, realtime=False)
    assert st_alone["max_inflight"] == 1 and st_mix["max_inflight"] > 1
    assert st_alone["batched_selections"] == 0 and st_mix["batched_selections"] > 0   # shared selections
    by_id = {r.rid: r for r in r_alone}
    for r in r_mix:
        assert torch.equal(r.image, by_id[r.rid].image), r.rid
    for st in (st_alone, st_mix):
        assert st["p99_ms"] >= st["p50_ms"] > 0


def test_memory_admission_limits_concurrency(scene):
    from paper_2507_01110_b300 import serving
    srv = serving.RenderServer(scene, n_slots=6, mem_budget_bytes=1, max_pixels=1920 * 1080)
    st = srv.run(_requests(53, n=10), realtime=False)
    assert st["max_inflight"] == 1 and st["requests"] == 10


def test_frame_memory_reports_what_the_workspace_holds_and_needs(scene):
    """lodgs_frame_memory: a larger view needs more; after a render that fit,
    the workspace holds at least what the view needed; it never shrinks; and a
    frame grown on the largest view takes about the reported bytes of device
    memory (within 10% and 32 MB: the driver rounds allocations to pages and
    packs small ones into pages it already holds)."""
    from paper_2507_01110_b300 import api
    cams = synth.serving_cameras(12, seed=54, extent=600.0)
    small = min(cams, key=lambda c: c.width * c.height)
    large = synth.camera_look([5.0, 3.0, 2.0], [1.0, 0.2, -0.05], [0.2, -1.0, 0.0], 3840, 2160, tau=0.5)
    img = torch.empty(large.height * large.width * 3, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    fr = api.Frame(scene)
    api.select_lod(scene, large, fr)
    api.render(scene, fr, image=img.view(large.height, large.width, 3), check_capacity=True)
    held_l, need_l = fr.memory()
    torch.cuda.synchronize()
    drop = free0 - torch.cuda.mem_get_info()[0]
    assert held_l > (32 << 20) and abs(drop - held_l) <= 0.1 * held_l + (32 << 20), (drop, held_l)
    held_prev = held_l
    for cam in (small, large):
        api.select_lod(scene, cam, fr)
        api.render(scene, fr, image=img[: cam.height * cam.width * 3].view(cam.height, cam.width, 3),
                   check_capacity=True)
        held, needed = fr.memory()
        assert needed <= held and held >= held_prev
        held_prev = held
        if cam is small:
            assert needed < need_l
    assert needed == need_l


def test_admission_by_learned_workspace_bytes(scene):
    """The budget bounds the workspace the slots hold.  With room for one slot
    sized for a heavy 4K street view beside five base-size slots, heavy
    requests run one at a time while light ones share the other slots; with
    room for two, two heavy ones at a time.  The slots never hold more than the
    budget, and the GPU busy fraction lies in (0, 1]."""
    from paper_2507_01110_b300 import serving
    big = synth.camera_look([5.0, 3.0, 2.0], [1.0, 0.2, -0.05], [0.2, -1.0, 0.0], 3840, 2160, tau=0.5)
    small = synth.camera_look([0.0, 0.0, 300.0], [0.0, 0.01, -1.0], [1.0, 0.0, 0.0], 160, 90, tau=4.0)
    probe = serving.RenderServer(scene, n_slots=2, max_pixels=3840 * 2160)
    base = probe.slots[1].held
    probe.warm([big, small])
    big_held = probe.slots[0].held
    assert probe.charge(big) > 3 * base and probe.charge(small) <= base
    for n_big in (1, 2):
        budget = n_big * big_held + (6 - n_big) * base + base // 2      # no room for one more large slot
        srv = serving.RenderServer(scene, n_slots=6, mem_budget_bytes=budget, max_pixels=3840 * 2160)
        srv.warm([big, small])
        need = srv.charge(big)
        assert len(srv.slots) == 6 and srv.held_bytes() <= budget
        assert sum(sl.held >= need for sl in srv.slots) == n_big
        st = srv.run([serving.Request(rid=i, arrival_s=0.0, camera=big) for i in range(10)], realtime=False)
        assert st["completed"] == 10 and st["max_inflight"] == n_big
        assert st["peak_slot_workspace_bytes"] <= budget and 0.0 < st["gpu_busy"] <= 1.0
        mixed = [serving.Request(rid=i, arrival_s=0.0, camera=big if i % 4 == 0 else small) for i in range(16)]
        st = srv.run(mixed, realtime=False)
        assert st["completed"] == 16 and st["max_inflight"] > n_big
        assert st["peak_slot_workspace_bytes"] <= budget


def test_an_overflow_waits_for_a_larger_slot_instead_of_growing_past_the_budget(scene):
    """A class learned on a light camera, then asked for with a heavy camera of
    the same resolution and threshold: the request overflows a slot sized for
    the light view; with the budget full it is not grown there but goes back
    to the queue and runs on the one slot large enough; the slots stay within
    the budget."""
    from paper_2507_01110_b300 import serving
    heavy = synth.camera_look([5.0, 3.0, 2.0], [1.0, 0.2, -0.05], [0.2, -1.0, 0.0], 3840, 2160, tau=0.5)
    light = synth.camera_look([0.0, 0.0, 50.0], [0.0, 0.01, 1.0], [1.0, 0.0, 0.0], 3840, 2160, tau=0.5)   # sky
    srv = serving.RenderServer(scene, n_slots=4, mem_budget_bytes=1 << 40, max_pixels=3840 * 2160)
    srv.warm([light])                                  # the class's need learned on the light view
    srv._render(srv.slots[0], heavy)                   # one slot large enough for the heavy view
    srv.slots[0].held = srv.slots[0].frame.memory()[0]
    base = min(sl.held for sl in srv.slots)
    assert srv.slots[0].held > 2 * base
    srv.budget = srv.held_bytes() + base // 2          # full: no other slot may grow to the heavy size
    reqs = [serving.Request(rid=i, arrival_s=0.0, camera=heavy if i == 1 else light) for i in range(4)]
    st = srv.run(reqs, realtime=False)
    assert st["completed"] == 4 and st["peak_slot_workspace_bytes"] <= srv.budget
    assert reqs[1].requeues >= 1 and reqs[1].retries == 0
