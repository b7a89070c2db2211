"""Out-of-core training (Algorithm 3 with the optimiser step): sparse Adam on the
cache's device slabs, write-back of trained prefixes on LRU eviction, on flush
and on request.  The trained records and Adam state that come back to host
memory must equal, bit for bit, those of the same Adam steps on a
device-resident copy of the scene (same cuts, same per-row gradients)."""
import numpy as np
import pytest
import torch

from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world():
    from paper_2507_01110_b300 import api, build
    build.build()
    leaves = synth.leaves_ground_and_boxes(120_000, seed=43, degree=1, extent=250.0, n_boxes=30)
    cams = synth.aerial_to_street_path(n_views=10, width=320, height=180, alt_hi=120.0, alt_lo=3.0, travel=150.0)
    kappa = float(cams[0].fx / cams[0].tau)
    return api, leaves, cams, kappa


def test_cache_training_matches_device_resident_adam(world):
    api, leaves, cams, kappa = world
    sc_d = api.build_hierarchy(leaves, 1, 40.0, kappa)
    sc_c = api.build_hierarchy(leaves, 1, 40.0, kappa)
    M, st = sc_d.n_nodes, sc_d.stride
    gen = torch.Generator(device="cuda").manual_seed(17)
    G = (torch.rand((M, st), device="cuda", generator=gen) - 0.5) * 1e-2      # fixed per-row gradients
    lr = np.full(st, 1e-3, np.float32)
    lr[10] = 5e-2
    adam = api.AdamState(sc_d)
    fr_d, fr_c = api.Frame(sc_d), api.Frame(sc_c)
    need = []
    for cam in cams:
        api.select_lod(sc_d, cam, fr_d)
        need.append(fr_d.stats()["n_spt_scanned"])
    cap = int(1.3 * max(need))
    assert cap < sum(need)
    cache = api.Cache(sc_c, capacity_bytes=cap * st * 4, d_min=1.0, d_max=1.0, train=True)
    copy_stream = torch.cuda.Stream()
    dL = torch.zeros((cams[0].height, cams[0].width, 3), device="cuda")
    written = evictions = 0
    path = cams + cams[::-1] + cams[::2]
    for i, cam in enumerate(path):
        api.select_lod(sc_d, cam, fr_d)
        sel = fr_d.selection()
        api.adam_step(sc_d, sc_d.rows(), adam, sel, G[sel].contiguous(), lr)
        _, s = api.stream_nodes(sc_c, cache, cam, fr_c, copy_stream=copy_stream)
        assert torch.equal(fr_c.selection(), sel)
        api.render(sc_c, fr_c, rows=cache.records)
        api.render_backward(sc_c, fr_c, dL, rows=cache.records)
        cache.adam_step(fr_c, G[sel].contiguous(), lr)
        written += s["bytes_written_back"]
        evictions += s["evictions"]
        if i == len(cams):
            cache.flush()                         # the periodic flush writes back and empties the cache
    assert evictions > 0 and written > 0
    cache.writeback()
    torch.cuda.synchronize()
    hs = cache.host_state()
    assert np.array_equal(hs["rows"].view(np.uint32), sc_d.rows().cpu().numpy().view(np.uint32))
    assert np.array_equal(hs["m"].view(np.uint32), adam.m.cpu().numpy().view(np.uint32))
    assert np.array_equal(hs["v"].view(np.uint32), adam.v.cpu().numpy().view(np.uint32))
    assert np.array_equal(hs["t"].astype(np.int64), adam.t.cpu().numpy().astype(np.int64))
    assert int(adam.t.max()) >= 3


def test_cache_adam_step_preconditions(world):
    api, leaves, cams, kappa = world
    sc = api.build_hierarchy(leaves, 1, 40.0, kappa)
    lr = np.full(sc.stride, 1e-3, np.float32)
    plain = api.Cache(sc, capacity_bytes=64 << 20, d_min=1.0, d_max=1.0)
    fr = api.Frame(sc)
    api.stream_nodes(sc, plain, cams[0], fr)
    api.render(sc, fr, rows=plain.records)
    g = api.render_backward(sc, fr, torch.zeros((cams[0].height, cams[0].width, 3), device="cuda"),
                            rows=plain.records)
    with pytest.raises(RuntimeError, match="not created for training"):
        plain.adam_step(fr, g, lr)
    train = api.Cache(sc, capacity_bytes=64 << 20, d_min=1.0, d_max=1.0, train=True)
    fr2 = api.Frame(sc)
    with pytest.raises(RuntimeError, match="latest view"):
        train.adam_step(fr2, g, lr)               # nothing streamed through this cache yet
    api.stream_nodes(sc, train, cams[0], fr2)
    with pytest.raises(RuntimeError, match="latest view"):
        train.adam_step(fr2, g, lr)               # not rendered and back-propagated
    torch.cuda.synchronize()
