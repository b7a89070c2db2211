"""Failure paths, driven by host-side fault injection (nothing faults, traps or
hangs on the device): a failed streaming copy, device memory running out when
a workspace grows, a request refused in the middle of serving, and requests
dropped at their deadline.  After each failure the library keeps working and
its results are unchanged."""
import pytest
import torch

from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world():
    from paper_2507_01110_b300 import _lib, api, build
    build.build()
    leaves = synth.leaves_ground_and_boxes(60_000, seed=61, degree=1, extent=200.0, n_boxes=20)
    cams = synth.aerial_to_street_path(n_views=6, width=256, height=144, alt_hi=100.0, alt_lo=3.0, travel=80.0)
    kappa = float(cams[0].fx / cams[0].tau)
    return api, _lib, api.build_hierarchy(leaves, 1, 20.0, kappa), cams


def test_failed_stream_copy_leaves_the_cache_consistent(world):
    api, _lib, scene, cams = world
    cache = api.Cache(scene, capacity_bytes=64 << 20, d_min=1.0, d_max=1.0)
    fr, ref = api.Frame(scene), api.Frame(scene)
    api.stream_nodes(scene, cache, cams[0], fr)
    api.inject_fault(_lib.FAULT_STREAM, 0)
    with pytest.raises(RuntimeError, match="injected"):
        api.stream_nodes(scene, cache, cams[1], fr)
    for cam in cams[1:]:
        api.stream_nodes(scene, cache, cam, fr)
        img = api.render(scene, fr, rows=cache.records)
        api.select_lod(scene, cam, ref)
        assert torch.equal(img, api.render(scene, ref))


def test_out_of_memory_in_a_workspace_is_reported_and_recoverable(world):
    api, _lib, scene, cams = world
    api.inject_fault(_lib.FAULT_ALLOC, 0)            # the frame's first workspace allocation
    with pytest.raises(RuntimeError, match="injected allocation failure"):
        api.Frame(scene)
    fr = api.Frame(scene)
    img = api.render(scene, api.select_lod(scene, cams[-1], fr))
    ref = api.render(scene, api.select_lod(scene, cams[-1], api.Frame(scene)))
    assert torch.equal(img, ref)
    api.inject_fault(_lib.FAULT_RENDER, 0)
    with pytest.raises(RuntimeError, match="injected out of device memory"):
        api.render(scene, api.select_lod(scene, cams[-1], fr))
    assert torch.equal(api.render(scene, api.select_lod(scene, cams[-1], fr)), ref)


def test_server_carries_on_when_a_request_is_refused(world):
    from paper_2507_01110_b300 import serving
    api, _lib, scene, cams = world
    reqs = serving.poisson_requests(cams, rate_per_s=2000.0, n=12, seed=62)
    srv = serving.RenderServer(scene, n_slots=3, keep_images=True, max_pixels=256 * 144)
    api.inject_fault(_lib.FAULT_RENDER, 3)           # the fourth render is refused
    st = srv.run(reqs, realtime=False)
    api.inject_fault(_lib.FAULT_RENDER, -1)
    assert st["failed"] == 1 and st["completed"] == 11 and st["expired"] == 0
    alone = serving.RenderServer(scene, n_slots=1, keep_images=True, max_pixels=256 * 144)
    again = serving.poisson_requests(cams, rate_per_s=2000.0, n=12, seed=62)
    alone.run(again, realtime=False)
    by_id = {r.rid: r for r in again}
    for r in reqs:
        if r.status == "done":
            assert torch.equal(r.image, by_id[r.rid].image)


def test_requests_expire_at_their_deadline(world):
    from paper_2507_01110_b300 import serving
    api, _lib, scene, cams = world
    srv = serving.RenderServer(scene, n_slots=1, max_pixels=256 * 144)
    srv.warm(cams)
    reqs = serving.poisson_requests(cams, rate_per_s=2000.0, n=40, seed=63)
    st = srv.run(reqs, realtime=False, deadline_ms=2.0)
    assert st["completed"] >= 1 and st["expired"] >= 1
    assert st["completed"] + st["expired"] == 40 and st["failed"] == 0
    assert all(r.status in ("done", "expired") for r in reqs)
