"""Densification (Sec. 3 "Densification"; appendix "Respawning, Densifying, and
Pruning Gaussians"): pins of the oracle's split and tree edits, and checks of
the host-side planner.  CPU only."""
import numpy as np
import pytest

from paper_2507_01110_b300 import synth
from oracle import densify_plan as dplan

REC_S, REC_OP = 3, 10


def _rec(stride, s, op):
    r = np.zeros(stride, np.float32)
    r[0:3] = (1.0, -2.0, 3.0)
    r[3:6] = s
    r[6:10] = (1.0, 0.0, 0.0, 0.0)
    r[10] = op
    r[11:14] = (0.2, 0.4, 0.6)
    return r


@pytest.mark.parametrize("op", [0.02, 0.3, 0.7, 0.95, 1.0])
def test_split_keeps_centre_and_line_integral_of_opacity(oracle_lib, op):
    """The two children composited front to back: at the centre the opacity is
    the parent's, 1 - (1 - o')^2 = o; along any line through the centre the
    composited opacity integrates to the parent's o * integral(g) (numerical
    quadrature of o' g_f + o' g_f (1 - o' g_f), the matching 3DGS-MCMC's split
    rule makes).  The same factor scales all three axes; the rest of the record
    is the parent's."""
    parent = _rec(16, (0.7, 0.3, 0.5), op)
    child = oracle_lib.split_record(parent)
    sp = float(child[REC_OP])
    ratio = child[REC_S:REC_S + 3].astype(np.float64) / parent[REC_S:REC_S + 3]
    assert np.allclose(ratio, ratio[0], rtol=1e-6)
    f = float(ratio[0])
    assert abs((1 - (1 - sp) ** 2) - op) < 2e-6
    for s in (0.7, 0.3, 0.5):               # a line along each principal axis
        h = s * 1e-3
        x = np.arange(-12 * s, 12 * s, h)
        g = np.exp(-0.5 * (x / s) ** 2)
        gf = np.exp(-0.5 * (x / (s * f)) ** 2)
        parent_int = op * g.sum() * h
        pair = sp * gf + sp * gf * (1 - sp * gf)
        assert abs(pair.sum() * h - parent_int) < 2e-6 * parent_int
        # not the image-plane (2D) matching: that would need f^2 = o / (2 o' - o'^2 / 2)
    if op > 0.1:
        assert abs(f * f - op / (2 * sp - sp * sp / 2)) > 1e-3
    keep = np.ones(16, bool)
    keep[REC_OP] = False
    keep[REC_S:REC_S + 3] = False
    assert np.array_equal(child[keep], parent[keep])


def test_split_of_zero_opacity_is_a_copy(oracle_lib):
    parent = _rec(16, (0.7, 0.3, 0.5), 0.0)
    assert np.array_equal(oracle_lib.split_record(parent), parent)


def _tiny_scene(oracle_lib):
    """Three leaves on a line; Morton order pairs leaves 0 and 1 (node 3), then
    node 3 with leaf 2 (root 4)."""
    st = oracle_lib.stride(0)
    leaves = np.stack([_rec(st, (0.1, 0.1, 0.1), 0.5) for _ in range(3)])
    leaves[:, 0] = (0.0, 0.1, 9.0)
    sc = oracle_lib.build_scene(leaves, 0, 1e-9, 150.0)
    assert list(sc["left"]) == [-1, -1, -1, 0, 3] and list(sc["right"]) == [-1, -1, -1, 1, 2]
    return sc


def test_spawn_on_a_tiny_tree_by_hand(oracle_lib):
    sc = _tiny_scene(oracle_lib)
    row = sc["row_of_node"]
    new, old = oracle_lib.densify(sc, [(oracle_lib.DENSIFY_SPAWN, row[2], -1)])
    # leaf 2 gets children 5, 6
    assert list(new["left"]) == [-1, -1, 5, 0, 3, -1, -1]
    assert list(new["right"]) == [-1, -1, 6, 1, 2, -1, -1]
    assert new["root"] == 4 and new["n_leaves"] == 4
    child = oracle_lib.split_record(sc["node_rec"][2])
    assert np.array_equal(new["node_rec"][5], child) and np.array_equal(new["node_rec"][6], child)
    assert np.array_equal(new["node_rec"][:5], sc["node_rec"])
    nor = new["node_of_row"]
    for r in range(7):
        if nor[r] >= 5:
            assert old[r] == -1
        else:
            assert old[r] == row[nor[r]]


def test_respawn_on_a_tiny_tree_by_hand(oracle_lib):
    """Dead leaf 0 (parent 3, sibling 1) respawned under leaf 2: leaf 1 takes
    node 3's place under the root, and 3 and 0 become the children of 2."""
    sc = _tiny_scene(oracle_lib)
    row = sc["row_of_node"]
    new, old = oracle_lib.densify(sc, [(oracle_lib.DENSIFY_RESPAWN, row[2], row[0])])
    assert list(new["left"]) == [-1, -1, 3, -1, 1]
    assert list(new["right"]) == [-1, -1, 0, -1, 2]
    assert new["root"] == 4
    child = oracle_lib.split_record(sc["node_rec"][2])
    assert np.array_equal(new["node_rec"][3], child) and np.array_equal(new["node_rec"][0], child)
    # a dead child of the root: its sibling becomes the root
    new2, _ = oracle_lib.densify(sc, [(oracle_lib.DENSIFY_RESPAWN, row[0], row[2])])
    assert new2["root"] == 3
    assert list(new2["left"]) == [4, -1, -1, 0, -1] and list(new2["right"]) == [2, -1, -1, 1, -1]


def _check_tree(sc):
    left, right, root = sc["left"], sc["right"], int(sc["root"])
    M = left.shape[0]
    seen = np.zeros(M, int)
    st = [root]
    while st:
        v = st.pop()
        seen[v] += 1
        if left[v] >= 0:
            assert right[v] >= 0
            st += [int(left[v]), int(right[v])]
        else:
            assert right[v] < 0
    assert np.all(seen == 1)                         # a tree over all nodes
    assert (left < 0).sum() == (M + 1) // 2          # full binary


def _covered(sc, sel):
    left, right = sc["left"], sc["right"]
    cover = np.zeros(left.shape[0], int)
    for v in sc["node_of_row"][sel]:
        st = [int(v)]
        while st:
            w = st.pop()
            if left[w] < 0:
                cover[w] += 1
            else:
                st += [int(left[w]), int(right[w])]
    return cover[left < 0]


def test_random_batches_keep_a_valid_hspt_and_proper_cuts(oracle_lib):
    """Three rounds of planned spawns and respawns on a 3000-leaf scene: the
    result is a full binary tree, every record of an old row moves with its
    node, each child is the split of its parent, and the rebuilt HSPT gives
    proper cuts equal to the brute-force descent (a root other than the last
    node included)."""
    rng = np.random.default_rng(5)
    leaves = synth.leaves_uniform_cube(3000, seed=21, half_extent=20.0, degree=1)
    sc = oracle_lib.build_scene(leaves, 1, 0.05, 150.0)
    cams = [synth.camera_look([3.0, -2.0, -60.0], [0.0, 0.03, 1.0], [1.0, 0.0, 0.0], 150, 90, tau=1.0),
            synth.camera_look([0.0, 0.0, 0.0], [0.3, 0.2, 1.0], [1.0, 0.0, 0.0], 120, 120, tau=3.0)]
    for it in range(3):
        M = sc["node_rec"].shape[0]
        opac = sc["row_rec"][:, REC_OP].copy()
        opac[rng.random(M) < 0.05] = 0.001
        grad = rng.random(M).astype(np.float32)
        topo = {"left": sc["left"], "right": sc["right"], "node_of_row": sc["node_of_row"]}
        spawn, respawn = dplan.plan(topo, opac, grad, 0.9, max_nodes=M + 60)
        assert len(respawn) > 0 and len(spawn) > 0
        ops = [(oracle_lib.DENSIFY_SPAWN, t, -1) for t in spawn] + \
              [(oracle_lib.DENSIFY_RESPAWN, t, d) for t, d in respawn]
        new, old = oracle_lib.densify(sc, ops)
        _check_tree(new)
        assert new["node_rec"].shape[0] == M + 2 * len(spawn)
        assert (old < 0).sum() == 2 * len(ops)
        ok = old >= 0
        assert np.array_equal(new["row_rec"][ok], sc["row_rec"][old[ok]])
        for t, _ in [(t, None) for t in spawn] + respawn:
            T = sc["node_of_row"][t]
            c = oracle_lib.split_record(sc["node_rec"][T])
            assert np.array_equal(new["node_rec"][new["left"][T]], c)
            assert np.array_equal(new["node_rec"][new["right"][T]], c)
        for cam in cams:
            sel, _ = oracle_lib.select(new, cam, False)
            assert np.array_equal(sel, oracle_lib.select_bruteforce(new, cam, False))
            assert np.all(_covered(new, sel) == 1)
        sc = new


def test_densify_rejects_invalid_operations(oracle_lib):
    sc = _tiny_scene(oracle_lib)
    row = sc["row_of_node"]
    S, R = oracle_lib.DENSIFY_SPAWN, oracle_lib.DENSIFY_RESPAWN
    with pytest.raises(ValueError):
        oracle_lib.densify(sc, [(S, row[3], -1)])                     # internal target
    with pytest.raises(ValueError):
        oracle_lib.densify(sc, [(R, row[1], row[1])])                 # dead == target
    with pytest.raises(ValueError):
        oracle_lib.densify(sc, [(S, row[2], -1), (S, row[2], -1)])    # target split twice
    with pytest.raises(ValueError):
        oracle_lib.densify(sc, [(R, row[2], row[0]), (S, row[0], -1)])  # a moved node as target


# ---------------------------------------------------------------------------
# planner
# ---------------------------------------------------------------------------

def _topo_balanced(depth):
    """Complete binary tree, canonical ids in heap order, rows = ids."""
    M = 2 ** (depth + 1) - 1
    left = np.full(M, -1, np.int64)
    right = np.full(M, -1, np.int64)
    for u in range(M):
        if 2 * u + 2 < M:
            left[u], right[u] = 2 * u + 1, 2 * u + 2
    return {"left": left, "right": right, "node_of_row": np.arange(M)}


def test_plan_sibling_rule_and_order():
    topo = _topo_balanced(3)                       # leaves 7..14; siblings (7,8), (9,10), ...
    M = 15
    opac = np.full(M, 0.5, np.float32)
    grad = np.zeros(M, np.float32)
    opac[[7, 8, 11]] = 0.0                         # 7 and 8 both dead: only 8 (right) respawns
    grad[[9, 10, 12, 13, 14]] = [0.5, 0.9, 0.7, 0.9, 0.1]
    spawn, respawn = dplan.plan(topo, opac, grad, 0.4)
    # candidates by gradient, ties by row: 10, 13, 12, 9
    assert respawn == [(10, 8), (13, 11)]
    assert spawn == [12, 9]
    spawn_b, _ = dplan.plan(topo, opac, grad, 0.4, max_nodes=M + 2)
    assert spawn_b == [12]
    # stale leaves count as dead; a dead leaf is never a candidate
    stale = np.zeros(M, bool)
    stale[10] = True
    spawn_c, respawn_c = dplan.plan(topo, opac, grad, 0.4, stale=stale)
    assert respawn_c == [(13, 8), (12, 10), (9, 11)] and spawn_c == []


def test_plan_against_brute_force():
    rng = np.random.default_rng(2)
    topo = _topo_balanced(6)
    M = topo["left"].shape[0]
    for _ in range(20):
        opac = rng.random(M).astype(np.float32)
        opac[rng.random(M) < 0.3] = 0.001
        grad = rng.random(M).astype(np.float32)
        spawn, respawn = dplan.plan(topo, opac, grad, 0.6, max_nodes=M + 10)
        leaves = [u for u in range(M) if topo["left"][u] < 0]
        par = {int(c): u for u in range(M) for c in (topo["left"][u], topo["right"][u]) if c >= 0}
        dead = []
        for u in leaves:
            if opac[u] < 0.005 and u in par:
                p = par[u]
                sib = topo["right"][p] if topo["left"][p] == u else topo["left"][p]
                if topo["left"][p] == u and topo["left"][sib] < 0 and opac[sib] < 0.005:
                    continue
                dead.append(u)
        cand = sorted([u for u in leaves if opac[u] >= 0.005 and grad[u] >= 0.6], key=lambda u: (-grad[u], u))
        k = min(len(dead), len(cand))
        assert respawn == list(zip(cand[:k], dead[:k]))
        assert spawn == cand[k:k + 5]
