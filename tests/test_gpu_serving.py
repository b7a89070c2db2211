"""Continuous-batching server: overlapping requests of mixed resolution and
LoD threshold give exactly the images they give alone."""
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
    r_mix = _requests(52)
    st_mix = mix.run(r_mix, realtime=False)
    assert st_alone["max_inflight"] == 1 and st_mix["max_inflight"] > 1
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
