"""Densification on the device (spawn / respawn tree edits, the split of the
target's record, the HSPT and SPT layout rebuilt) against the oracle: the new
layout bit-exact, the row map exact, and renders of the densified scene within
the image bar.  Per-row state carried across by the row gather."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_01110_b300 import synth
from oracle import densify_plan as dplan
from test_gpu_parity import _assert_scene_equal, _compare_render

pytestmark = pytest.mark.gpu

REC_OP = 10


@pytest.fixture(scope="module")
def api():
    from paper_2507_01110_b300 import build
    build.build()
    from paper_2507_01110_b300 import api as a
    return a


def _plan(sc_o, rng, thr, max_extra):
    M = sc_o["node_rec"].shape[0]
    opac = sc_o["row_rec"][:, REC_OP].copy()
    opac[rng.random(M) < 0.04] = 0.0
    grad = rng.random(M).astype(np.float32)
    topo = {"left": sc_o["left"], "right": sc_o["right"], "node_of_row": sc_o["node_of_row"]}
    return dplan.plan(topo, opac, grad, thr, max_nodes=M + max_extra)


def _ops(spawn, respawn):
    return [(oracle.DENSIFY_SPAWN, t, -1) for t in spawn] + [(oracle.DENSIFY_RESPAWN, t, d) for t, d in respawn]


@pytest.mark.parametrize("n,deg,vol", [(4099, 1, 0.05), (20000, 0, 0.5)])
def test_densify_matches_oracle(api, n, deg, vol):
    rng = np.random.default_rng(n)
    leaves = synth.leaves_uniform_cube(n, seed=300 + n, half_extent=20.0, degree=deg)
    kappa = 150.0
    sc_o = oracle.build_scene(leaves, deg, vol, kappa)
    sc_g = api.build_hierarchy(leaves, deg, vol, kappa)
    cam = synth.camera_look([3.0, -2.0, -60.0], [0.0, 0.03, 1.0], [1.0, 0.0, 0.0], 150, 90, tau=1.0)
    cam2 = synth.camera_look([0.0, 0.0, 0.0], [0.3, 0.2, 1.0], [1.0, 0.0, 0.0], 161, 97, tau=0.5)
    stale_frame = api.Frame(sc_g)
    for it in range(3):
        spawn, respawn = _plan(sc_o, rng, 0.8, 400)
        assert spawn and respawn
        # the planner sees the same topology on both sides
        topo = sc_g.topology()
        assert np.array_equal(topo["node_of_row"], sc_o["node_of_row"]) and topo["root"] == sc_o["root"]
        sc_o, old_o = oracle.densify(sc_o, _ops(spawn, respawn))
        old_g = sc_g.densify(spawn=spawn, respawn=respawn)
        assert sc_g.layout_version == it + 1 and sc_g.root == sc_o["root"]
        assert np.array_equal(old_g.cpu().numpy(), old_o)
        _assert_scene_equal(sc_o, sc_g)
        fr = api.Frame(sc_g)
        for c in (cam, cam2):
            _compare_render(api, sc_o, sc_g, c, bg=(0.1, 0.0, 0.25), fr=fr)
    # frames made before a densification are refused (host check, nothing launched)
    with pytest.raises(RuntimeError, match="densified"):
        api.select_lod(sc_g, cam, stale_frame)


def test_respawn_moves_the_root_on_the_device(api):
    """With 2^k + 1 leaves the level-wise merge leaves the last Morton leaf as
    a child of the root; respawning it hands the root's place to its sibling
    subtree."""
    leaves = synth.leaves_uniform_cube(65, seed=9, half_extent=5.0, degree=0)
    sc_o = oracle.build_scene(leaves, 0, 0.5, 150.0)
    sc_g = api.build_hierarchy(leaves, 0, 0.5, 150.0)
    root = sc_o["root"]
    dead = int(sc_o["right"][root])
    assert sc_o["left"][dead] < 0
    d_row = int(sc_o["row_of_node"][dead])
    t_row = int(sc_o["row_of_node"][0])
    sc_o, old_o = oracle.densify(sc_o, [(oracle.DENSIFY_RESPAWN, t_row, d_row)])
    assert sc_o["root"] != root
    assert np.array_equal(sc_g.densify(respawn=[(t_row, d_row)]).cpu().numpy(), old_o)
    assert sc_g.root == sc_o["root"]
    _assert_scene_equal(sc_o, sc_g)
    cam = synth.camera_look([0.0, 0.0, -20.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0], 64, 48, tau=1.0)
    _compare_render(api, sc_o, sc_g, cam)


def test_invalid_densify_leaves_the_scene_unchanged(api):
    leaves = synth.leaves_uniform_cube(100, seed=4, half_extent=5.0, degree=0)
    sc_o = oracle.build_scene(leaves, 0, 0.5, 150.0)
    sc_g = api.build_hierarchy(leaves, 0, 0.5, 150.0)
    internal_row = int(sc_o["row_of_node"][sc_o["root"]])
    leaf_row = int(sc_o["row_of_node"][0])
    for spawn, respawn in (([internal_row], []), ([], [(leaf_row, leaf_row)]), ([leaf_row, leaf_row], []),
                           ([10 ** 6], [])):
        with pytest.raises(RuntimeError):
            sc_g.densify(spawn=spawn, respawn=respawn)
        assert sc_g.layout_version == 0
    _assert_scene_equal(sc_o, sc_g)


def test_gather_rows_carries_adam_state(api):
    leaves = synth.leaves_uniform_cube(2000, seed=7, half_extent=10.0, degree=1)
    sc_o = oracle.build_scene(leaves, 1, 0.05, 150.0)
    sc_g = api.build_hierarchy(leaves, 1, 0.05, 150.0)
    st = api.AdamState(sc_g)
    gen = torch.Generator(device="cuda").manual_seed(3)
    st.m.copy_(torch.randn(st.m.shape, generator=gen, device="cuda"))
    st.v.copy_(torch.rand(st.v.shape, generator=gen, device="cuda"))
    st.t.copy_(torch.randint(0, 1000, st.t.shape, generator=gen, device="cuda", dtype=torch.int32))
    m0, v0, t0 = st.m.cpu().numpy(), st.v.cpu().numpy(), st.t.cpu().numpy()
    spawn, respawn = _plan(sc_o, np.random.default_rng(1), 0.7, 200)
    old = sc_g.densify(spawn=spawn, respawn=respawn)
    st.remap(old)
    old = old.cpu().numpy()
    ok = old >= 0
    for new, ref in ((st.m, m0), (st.v, v0), (st.t, t0)):
        a = new.cpu().numpy()
        assert a.shape[0] == sc_g.n_nodes
        assert np.array_equal(a[ok].view(np.uint32), ref[old[ok]].view(np.uint32))
        assert not np.any(a[~ok])


@pytest.mark.parametrize("n,deg,budget", [(4099, 1, 300), (20000, 0, None)])
def test_device_plan_matches_host_planner(api, n, deg, budget):
    """lodgs_densify_plan (classification, sibling rule, compaction and the
    gradient sort on the device) gives exactly the operations of the host
    planner for the same opacities, gradients and stale flags."""
    rng = np.random.default_rng(n + 1)
    leaves = synth.leaves_uniform_cube(n, seed=400 + n, half_extent=20.0, degree=deg)
    sc_o = oracle.build_scene(leaves, deg, 0.05, 150.0)
    sc_g = api.build_hierarchy(leaves, deg, 0.05, 150.0)
    M = sc_o["node_rec"].shape[0]
    for it in range(3):
        rows = sc_g.rows().clone()
        opac = rows[:, REC_OP].cpu().numpy()
        opac[rng.random(M) < 0.05] = 0.0
        opac[rng.random(M) < 0.01] = 0.004                      # just under the threshold
        rows[:, REC_OP] = torch.from_numpy(opac).cuda()
        grad = rng.random(M).astype(np.float32)
        grad[rng.random(M) < 0.2] = 0.5                          # ties at the threshold: ordered by row
        stale = rng.random(M) < 0.01
        topo = {"left": sc_o["left"], "right": sc_o["right"], "node_of_row": sc_o["node_of_row"]}
        max_nodes = None if budget is None else M + budget
        sp_h, rs_h = dplan.plan(topo, opac, grad, 0.5, max_nodes=max_nodes, stale=stale)
        sp_d, rs_d = sc_g.plan_densify(torch.from_numpy(grad).cuda(), 0.5, max_nodes=max_nodes,
                                       stale=torch.from_numpy(stale), rows=rows)
        assert sp_d == sp_h and rs_d == rs_h
        assert len(rs_h) > 0 and len(sp_h) > 0
        # apply, so the next round plans on a densified tree
        sc_o, old_o = oracle.densify(sc_o, _ops(sp_h, rs_h))
        assert np.array_equal(sc_g.densify(spawn=sp_d, respawn=rs_d).cpu().numpy(), old_o)
        M = sc_o["node_rec"].shape[0]


def test_checkpoint_round_trip_after_densification(api, tmp_path):
    """A densified scene (spawned nodes, a moved root) saved and loaded: the
    loaded layout (tree, records, upper hierarchy, SPT layout, intervals, row
    order) and its renders equal the saved scene's bit for bit; damaged files
    are refused."""
    leaves = synth.leaves_uniform_cube(65, seed=9, half_extent=5.0, degree=1)
    sc_o = oracle.build_scene(leaves, 1, 0.5, 150.0)
    sc_g = api.build_hierarchy(leaves, 1, 0.5, 150.0)
    dead_row = int(sc_o["row_of_node"][sc_o["right"][sc_o["root"]]])
    t_row = int(sc_o["row_of_node"][0])
    sc_g.densify(spawn=[int(sc_o["row_of_node"][1])], respawn=[(t_row, dead_row)])
    assert sc_g.root != sc_g.n_nodes - 1
    path = tmp_path / "scene.lodgs"
    sc_g.save(path)
    sc_l = api.load_scene(path)
    a, b = sc_g.export(), sc_l.export()
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k
        else:
            assert a[k] == b[k], k
    assert torch.equal(sc_g.rows(), sc_l.rows())
    cam = synth.camera_look([0.0, 0.0, -20.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0], 96, 64, tau=1.0)
    img_a = api.render(sc_g, api.select_lod(sc_g, cam))
    img_b = api.render(sc_l, api.select_lod(sc_l, cam))
    assert torch.equal(img_a, img_b)
    raw = path.read_bytes()
    bad = bytearray(raw)
    bad[len(bad) // 2] ^= 0x40
    (tmp_path / "bad.lodgs").write_bytes(bytes(bad))
    with pytest.raises(RuntimeError, match="checksum"):
        api.load_scene(tmp_path / "bad.lodgs")
    (tmp_path / "short.lodgs").write_bytes(raw[: len(raw) // 3])
    with pytest.raises(RuntimeError, match="truncated"):
        api.load_scene(tmp_path / "short.lodgs")
    with pytest.raises(RuntimeError, match="cannot open"):
        api.load_scene(tmp_path / "missing.lodgs")
