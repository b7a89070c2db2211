"""Out-of-core node cache (a3): records in pinned host memory, a device slab of
SPT record prefixes, Eq. 7 reuse window, LRU eviction."""
import numpy as np
import pytest
import torch

from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world():
    from paper_2507_01110_b300 import api, build
    build.build()
    leaves = synth.leaves_ground_and_boxes(200_000, seed=41, degree=1, extent=300.0, n_boxes=40)
    cams = synth.aerial_to_street_path(n_views=12, width=480, height=270, alt_hi=150.0, alt_lo=3.0, travel=200.0)
    kappa = float(cams[0].fx / cams[0].tau)
    scene = api.build_hierarchy(leaves, 1, 60.0, kappa)
    return api, scene, cams


def _proper_cut(ex, sel):
    left, right = ex["left"], ex["right"]
    n = ex["n_leaves"]
    cover = np.zeros(n, dtype=np.int32)
    for node in ex["node_of_row"][sel]:
        st = [node]
        while st:
            v = st.pop()
            if left[v] < 0:
                cover[v] += 1
            else:
                st += [left[v], right[v]]
    return cover.max() <= 1


def test_exact_window_matches_resident_render_under_eviction(world):
    api, scene, cams = world
    rec_bytes = scene.stride * 4
    fr_c, fr_r = api.Frame(scene), api.Frame(scene)
    need = []
    for cam in cams:
        api.select_lod(scene, cam, fr_r)
        need.append(fr_r.stats()["n_spt_scanned"])
    # a slab that holds any one view but not the whole trajectory forces LRU evictions
    cap = int(1.3 * max(need))
    assert cap < sum(need)
    cache = api.Cache(scene, capacity_bytes=cap * rec_bytes, d_min=1.0, d_max=1.0)
    copy_stream = torch.cuda.Stream()
    total_evict = 0
    for i, cam in enumerate(cams + cams[::-1]):
        _, st = api.stream_nodes(scene, cache, cam, fr_c, copy_stream=copy_stream)
        img_c = api.render(scene, fr_c, rows=cache.records).cpu().numpy()
        api.select_lod(scene, cam, fr_r)
        img_r = api.render(scene, fr_r).cpu().numpy()
        assert np.array_equal(fr_c.selection().cpu().numpy(), fr_r.selection().cpu().numpy())
        assert np.array_equal(img_c, img_r)
        total_evict += st["evictions"]
        if i == 0:
            # empty cache: every emitted SPT streams exactly its needed prefix
            assert st["spt_hits"] == 0 and st["spt_resident"] == 0
            assert st["bytes_streamed"] == fr_r.stats()["n_spt_scanned"] * rec_bytes
        assert st["bytes_streamed"] % rec_bytes == 0
    assert total_evict > 0


def test_reuse_window_gives_hits_and_proper_cuts(world):
    api, scene, cams = world
    ex = scene.export()
    cache = api.Cache(scene, capacity_bytes=400_000 * scene.stride * 4, d_min=0.9, d_max=1.1)
    fr = api.Frame(scene)
    hits = loaded_bytes = 0
    # a slow, coherent path: consecutive views within a few percent in distance
    base = synth.aerial_to_street_path(n_views=40, width=320, height=180, alt_hi=60.0, alt_lo=40.0, travel=20.0)
    for cam in base:
        _, st = api.stream_nodes(scene, cache, cam, fr)
        img = api.render(scene, fr, rows=cache.records)
        assert torch.isfinite(img).all()
        hits += st["spt_hits"]
        loaded_bytes += st["bytes_streamed"]
        assert _proper_cut(ex, fr.selection().cpu().numpy())
    assert hits > 0 and loaded_bytes > 0


def test_stream_nodes_matches_the_oracle_cache_model():
    """lodgs_stream_nodes against the oracle's cache model (Eq. 7 window
    [0.9, 1.1], LRU eviction, Algorithm 3) on an 80-view out-and-back flyover
    of a 20K-leaf scene through a slab of 1.3 times the largest view's prefix
    records: per view the cut (render rows) bit for bit and every counter
    (hits, re-cuts, loads, streamed bytes, evictions, cached SPTs and
    records); every tenth view's image against the oracle's render of the
    model's cut."""
    import oracle
    from oracle import cache as oc
    from paper_2507_01110_b300 import api
    leaves = synth.leaves_ground_and_boxes(20000, seed=43, degree=0, extent=300.0, n_boxes=40)
    path = synth.flyover_path()
    sc_o = oracle.build_scene(leaves, 0, 50.0, float(path[0].fx))
    sc_g = api.build_hierarchy(leaves, 0, 50.0, float(path[0].fx))
    cap = int(1.3 * max(oracle.select(sc_o, c)[1]["spt_scanned"] for c in path))
    rec_bytes = sc_g.stride * 4
    model = oc.NodeCache(sc_o, cap, 0.9, 1.1)
    cache = api.Cache(sc_g, capacity_bytes=cap * rec_bytes, d_min=0.9, d_max=1.1)
    fr = api.Frame(sc_g)
    tot = dict.fromkeys(("spt_hits", "spt_resident", "spt_loaded", "evictions"), 0)
    for i, cam in enumerate(path + path[::-1]):
        _, st = api.stream_nodes(sc_g, cache, cam, fr)
        rows_o, st_o = model.view(cam)
        assert np.array_equal(fr.selection().cpu().numpy(), rows_o), i
        for k in ("spt_hits", "spt_resident", "spt_loaded", "evictions", "cached_spts", "cached_records"):
            assert st[k] == st_o[k], (i, k, st[k], st_o[k])
        assert st["bytes_streamed"] == st_o["records_streamed"] * rec_bytes
        for k in tot:
            tot[k] += st[k]
        if i % 10 == 0:
            img = api.render(sc_g, fr, rows=cache.records).cpu().numpy()
            ref = oracle.render(sc_o, cam, sel=rows_o)["image"]
            assert np.abs(img - ref).max() <= 2e-4
    assert all(v > 0 for v in tot.values()), tot


def test_released_scene_rows_need_cache_records(world):
    from paper_2507_01110_b300 import _lib
    api, _, cams = world
    leaves = synth.leaves_uniform_cube(5000, seed=42, half_extent=10.0)
    scene = api.build_hierarchy(leaves, 0, 1.0, 100.0)
    cache = api.Cache(scene, capacity_bytes=1 << 24, release_scene_rows=True)
    cam = synth.camera_look([0.0, 0.0, -40.0], [0, 0, 1], [1, 0, 0], 64, 64)
    fr, _ = api.stream_nodes(scene, cache, cam)
    img = api.render(scene, fr, rows=cache.records)
    assert torch.isfinite(img).all()
    with pytest.raises(_lib.LodgsError):
        api.render(scene, api.select_lod(scene, cam))
