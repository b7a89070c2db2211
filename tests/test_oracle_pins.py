"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed
form, an invariant the paper states, a library routine (LAPACK eigh, scipy
rotations and spherical harmonics, numpy lexsort), brute force on small
inputs, or finite differences.  None of them needs a GPU.
"""
import math

import numpy as np
import torch
import pytest

from paper_2507_01110_b300 import synth

REC_MU, REC_S, REC_Q, REC_OP, REC_B, REC_F = 0, 3, 6, 10, 11, 14


def _rec(stride, mu, s, q=(1, 0, 0, 0), op=0.5, b=(0.5, 0.5, 0.5)):
    r = np.zeros(stride, dtype=np.float32)
    r[0:3], r[3:6], r[6:10], r[10], r[11:14] = mu, s, q, op, b
    return r


def _rot_from_quat(q):
    from scipy.spatial.transform import Rotation
    w, x, y, z = q
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def _cov(rec):
    R = _rot_from_quat(rec[6:10].astype(np.float64))
    s = rec[3:6].astype(np.float64)
    return R @ np.diag(s * s) @ R.T


# ---------------------------------------------------------------------------
# hierarchy: Morton order, eigen-decomposition, merges, topology
# ---------------------------------------------------------------------------

def test_morton_order_is_bitplane_lexicographic(oracle_lib):
    """Z-order on a 4x4x4 grid = lexicographic order of (x_hi, y_hi, z_hi, x_lo, y_lo, z_lo)."""
    g = np.array([(x, y, z) for x in range(4) for y in range(4) for z in range(4)], dtype=np.float32)
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(g))
    g = g[perm]
    recs = np.zeros((len(g), 16), dtype=np.float32)
    recs[:, 0:3] = g
    order = oracle_lib.morton_order(recs)
    xi, yi, zi = (g[:, a].astype(int) for a in range(3))
    expect = np.lexsort((zi & 1, yi & 1, xi & 1, zi >> 1, yi >> 1, xi >> 1))
    assert np.array_equal(order, expect)


def test_morton_ties_broken_by_index(oracle_lib):
    recs = np.zeros((5, 16), dtype=np.float32)
    recs[:, 0] = [1.0, 0.0, 1.0, 0.0, 1.0]
    assert list(oracle_lib.morton_order(recs)) == [1, 3, 0, 2, 4]


def test_eigendecomposition_matches_lapack(oracle_lib):
    rng = np.random.default_rng(1)
    for trial in range(200):
        A = rng.normal(size=(3, 3)) * rng.uniform(0.01, 100)
        C = A @ A.T
        if trial % 7 == 0:
            C = np.diag(rng.uniform(0.1, 10, 3))                  # already diagonal
        if trial % 11 == 0:
            v = rng.normal(size=3)
            C = np.outer(v, v) + 1e-6 * np.eye(3)                   # nearly rank one
        s, q = oracle_lib.cov_to_scale_rot(C)
        lam = np.linalg.eigh(C)[0][::-1]
        assert np.allclose(s * s, lam, rtol=1e-10, atol=1e-12 * lam.max())
        assert s[0] >= s[1] >= s[2]
        assert abs(np.linalg.norm(q) - 1) < 1e-12 and q[0] >= 0
        R = _rot_from_quat(q)
        assert np.allclose(R @ np.diag(s * s) @ R.T, C, rtol=0, atol=1e-10 * np.abs(C).max())


def test_merge_identical_children_returns_them(oracle_lib):
    st = synth.record_stride(0)
    q = np.array([0.9, 0.1, -0.3, 0.2]); q /= np.linalg.norm(q)
    a = _rec(st, (1, 2, 3), (0.5, 0.2, 0.1), q, op=0.3, b=(0.1, 0.6, 0.9))
    p = oracle_lib.merge_pair(a, a, 0)
    assert np.allclose(p[0:3], a[0:3], atol=1e-6)
    assert np.allclose(_cov(p), _cov(a), rtol=1e-5, atol=1e-7)
    assert p[REC_OP] == pytest.approx(min(1.0, 2 * 0.3), rel=1e-6)
    assert np.allclose(p[11:14], a[11:14], atol=1e-7)


def test_merge_zero_weight_child_is_ignored(oracle_lib):
    st = synth.record_stride(1)
    q = np.array([0.5, 0.5, -0.5, 0.5])
    a = _rec(st, (1, 2, 3), (0.5, 0.2, 0.1), q, op=0.7, b=(0.1, 0.6, 0.9))
    a[14:23] = np.linspace(-0.3, 0.3, 9)
    b = _rec(st, (9, -4, 7), (2.0, 1.0, 3.0), (1, 0, 0, 0), op=0.0, b=(1, 1, 1))
    p = oracle_lib.merge_pair(a, b, 1)
    assert np.allclose(p[0:3], a[0:3], atol=1e-6)
    assert np.allclose(_cov(p), _cov(a), rtol=1e-5, atol=1e-7)
    assert p[REC_OP] == pytest.approx(0.7, rel=1e-5)
    assert np.allclose(p[11:23], a[11:23], atol=1e-7)


def test_merge_point_like_children_closed_form(oracle_lib):
    """Two equal, tiny, equal-opacity children at mu +- (d,0,0): the moment-matched
    parent has mean mu and covariance diag(d^2, ~0, ~0) (+ the children's own)."""
    st = synth.record_stride(0)
    d, eps = 3.0, 1e-3
    a = _rec(st, (10 + d, 5, -2), (eps, eps, eps), op=0.5)
    b = _rec(st, (10 - d, 5, -2), (eps, eps, eps), op=0.5)
    p = oracle_lib.merge_pair(a, b, 0)
    assert np.allclose(p[0:3], (10, 5, -2), atol=1e-6)
    assert p[3] == pytest.approx(math.sqrt(d * d + eps * eps), rel=1e-6)
    assert p[4] == pytest.approx(eps, rel=1e-4) and p[5] == pytest.approx(eps, rel=1e-4)
    R = _rot_from_quat(p[6:10].astype(np.float64))
    assert abs(abs(R[0, 0]) - 1) < 1e-6                          # major axis along x
    # opacity keeps sigma * area: 2 * 0.5 * 3 eps^2 / (2 d eps + eps^2)
    assert p[REC_OP] == pytest.approx(3 * eps * eps / (2 * math.sqrt(d * d + eps * eps) * eps + eps * eps), rel=1e-4)


def test_merge_weighted_mean(oracle_lib):
    st = synth.record_stride(0)
    a = _rec(st, (0, 0, 0), (1, 1, 1), op=0.2)
    b = _rec(st, (4, 0, 0), (2, 2, 2), op=0.4)
    wa, wb = 0.2 * 3, 0.4 * 12
    p = oracle_lib.merge_pair(a, b, 0)
    assert p[0] == pytest.approx(4 * wb / (wa + wb), rel=1e-6)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 64])
def test_hierarchy_topology(oracle_lib, n):
    leaves = synth.leaves_uniform_cube(n, seed=5)
    h = oracle_lib.merge_hierarchy(leaves, 0)
    M = 2 * n - 1
    left, right, parent = h["left"], h["right"], h["parent"]
    assert h["root"] == M - 1 and parent[M - 1] == -1
    assert np.all(left[:n] == -1) and np.all(right[:n] == -1)
    assert np.all(left[n:] >= 0) and np.all(right[n:] >= 0)
    seen = np.zeros(M, dtype=int)
    stack = [M - 1]
    while stack:
        v = stack.pop()
        seen[v] += 1
        if left[v] >= 0:
            assert parent[left[v]] == v and parent[right[v]] == v and left[v] < v and right[v] < v
            stack += [left[v], right[v]]
    assert np.all(seen == 1)


def test_hierarchy_pairs_consecutive_morton_leaves(oracle_lib):
    """Leaves sorted along x: level 1 pairs (0,1),(2,3); an odd last node is carried up."""
    recs = np.zeros((5, 16), dtype=np.float32)
    recs[:, 0] = [0, 1, 2, 3, 4]
    recs[:, 3:6] = 0.1
    recs[:, 6] = 1
    recs[:, 10] = 0.5
    h = oracle_lib.merge_hierarchy(recs, 0)
    L, R = h["left"], h["right"]
    assert (L[5], R[5]) == (0, 1) and (L[6], R[6]) == (2, 3)
    assert (L[7], R[7]) == (5, 6) and (L[8], R[8]) == (7, 4)


# ---------------------------------------------------------------------------
# HSPT and SPT intervals
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def scene1(oracle_lib):
    cfg = synth.config1_scene()
    return cfg, oracle_lib.build_scene(cfg["leaves"], 0, cfg["spt_volume"], cfg["kappa"])


def _subtree(left, right, r):
    out, st = [], [r]
    while st:
        v = st.pop()
        out.append(v)
        if left[v] >= 0:
            st += [left[v], right[v]]
    return out


def test_hspt_partitions_the_hierarchy(scene1):
    cfg, sc = scene1
    M = sc["node_rec"].shape[0]
    rec, left, right = sc["node_rec"], sc["left"], sc["right"]
    vol = (rec[:, 3] * rec[:, 4]) * rec[:, 5]
    owner = np.full(M, -1)
    for u in range(sc["n_upper"]):
        node, kind = sc["up_node"][u], sc["up_kind"][u]
        if kind == 2:
            assert vol[node] < np.float32(cfg["spt_volume"])
            for v in _subtree(left, right, node):
                assert owner[v] == -1
                owner[v] = 1
        else:
            assert vol[node] >= np.float32(cfg["spt_volume"])
            assert owner[node] == -1
            owner[node] = 0
    assert np.all(owner >= 0)
    assert np.array_equal(np.sort(sc["node_of_row"]), np.arange(M))
    assert np.array_equal(sc["row_of_node"][sc["node_of_row"]], np.arange(M))
    # SPT entries sorted by hi descending, root first with hi = +inf
    for j in range(sc["n_spt"]):
        b, c = sc["spt_base"][j], sc["spt_count"][j]
        hi = sc["hi_row"][b:b + c]
        assert np.isinf(hi[0]) and sc["node_of_row"][b] == sc["spt_root"][j]
        assert np.all(np.diff(hi) <= 0)


def _paths(left, right, r):
    """All root-to-leaf paths of the subtree at r."""
    out, st = [], [(r, [r])]
    while st:
        v, p = st.pop()
        if left[v] < 0:
            out.append(p)
        else:
            st += [(left[v], p + [left[v]]), (right[v], p + [right[v]])]
    return out


def test_spt_intervals_cut_every_path_exactly_once(scene1):
    """Eq. 4 with clamped intervals: for any x >= 0 exactly one node per
    root-to-leaf path satisfies lo <= x < hi, and it is the node the unclamped
    top-down descent picks."""
    _, sc = scene1
    left, right = sc["left"], sc["right"]
    rng = np.random.default_rng(3)
    for j in rng.choice(sc["n_spt"], 6, replace=False):
        b, c = sc["spt_base"][j], sc["spt_count"][j]
        rows = np.arange(b, b + c)
        nodes = sc["node_of_row"][rows]
        lo = dict(zip(nodes, sc["lo_row"][rows]))
        hi = dict(zip(nodes, sc["hi_row"][rows]))
        paths = _paths(left, right, sc["spt_root"][j])
        xs = np.concatenate([[0.0], rng.uniform(0, 1.5 * lo[sc["spt_root"][j]], 20),
                             sc["lo_row"][rows][:10], [1e30]]).astype(np.float32)
        for x in xs:
            chosen = {v for v in nodes if lo[v] <= x < hi[v]}
            for p in paths:
                assert sum(v in chosen for v in p) == 1
            # brute force: first node on the path with lo_raw <= x (leaves qualify)
            bf = set()
            for p in paths:
                for v in p:
                    if left[v] < 0 or sc["lo_raw"][v] <= x:
                        bf.add(v)
                        break
            assert bf == chosen
            if x == 0:
                assert all(left[v] < 0 for v in chosen)
            if x >= lo[sc["spt_root"][j]]:
                assert chosen == {sc["spt_root"][j]}


def test_unreachable_nodes_never_selected(scene1):
    """Nodes whose own size term exceeds their parent's clamped bound get an
    empty interval (lo == hi) and are never selected (appendix, Unreachable
    Gaussians)."""
    _, sc = scene1
    M = sc["node_rec"].shape[0]
    rows = np.arange(sc["n_upper_rows"], M)
    empty = rows[sc["lo_row"][rows] >= sc["hi_row"][rows]]
    assert empty.size > 0
    lo, hi = sc["lo_row"], sc["hi_row"]
    for x in np.linspace(0, 200, 101, dtype=np.float32):
        assert not np.any((lo[empty] <= x) & (x < hi[empty]))


def test_spt_conservative_distance(scene1):
    """Sec. 4.1: selecting with M_d guarantees m_d(i) <= |mu_i - p| for every
    selected SPT node (k = f/tau = kappa, triangle inequality)."""
    cfg, sc = scene1
    cam = cfg["cameras"][0]
    sel, _ = __import__("oracle").select(sc, cam, cull=False)
    rec = sc["row_rec"][sel].astype(np.float64)
    in_spt = sel >= sc["n_upper_rows"]
    s = rec[:, 3:6]
    S = np.sqrt((s[:, 0] * s[:, 1] + s[:, 0] * s[:, 2] + s[:, 1] * s[:, 2]) / 3)
    d = np.linalg.norm(rec[:, 0:3] - cam.pos.astype(np.float64), axis=1)
    k = cam.fx / cam.tau
    leaf = sc["left"][sc["node_of_row"][sel]] < 0
    chk = in_spt & ~leaf
    assert chk.sum() > 0
    assert np.all(k * S[chk] <= d[chk] * (1 + 1e-5))


def _covered_leaves(sc, sel):
    left, right = sc["left"], sc["right"]
    nodes = sc["node_of_row"][sel]
    cover = np.zeros(sc["n_leaves"], dtype=int)
    for v in nodes:
        for w in _subtree(left, right, v):
            if left[w] < 0:
                cover[w] += 1
    return cover


def test_select_is_proper_cut_and_matches_bruteforce(oracle_lib, scene1):
    cfg, sc = scene1
    cams = [cfg["cameras"][0],
            synth.camera_look([80.0, -60.0, 40.0], [-1.0, 0.7, -0.3], [0.0, 0.0, 1.0], 200, 120, tau=2.0),
            synth.camera_look([0.0, 0.0, 0.0], [0.3, 0.2, 1.0], [1.0, 0.0, 0.0], 160, 160, tau=0.5)]
    for cam in cams:
        for cull in (True, False):
            sel, st = oracle_lib.select(sc, cam, cull)
            bf = oracle_lib.select_bruteforce(sc, cam, cull)
            assert np.array_equal(sel, bf)
            assert np.all(np.diff(sel) > 0)
            cover = _covered_leaves(sc, sel)
            assert cover.max() <= 1                       # proper: no node with its ancestor
            if not cull:
                assert np.all(cover == 1)                 # every root-to-leaf path crossed once
        sel_c, _ = oracle_lib.select(sc, cam, True)
        sel_n, _ = oracle_lib.select(sc, cam, False)
        cov_c, cov_n = _covered_leaves(sc, sel_c), _covered_leaves(sc, sel_n)
        assert np.all(cov_c <= cov_n)                     # culling only removes coverage


def _corner_ray_planes(cam):
    """The view frustum's four side planes rebuilt in float64 from the pinhole
    model alone: each plane holds the camera centre and two adjacent image
    corner rays ((x - cx)/fx, (y - cy)/fy, 1); its unit normal points to the
    side of the image centre's ray."""
    W, H = float(cam.width), float(cam.height)
    fx, fy, cx, cy = (float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy))
    ray = lambda x, y: np.array([(x - cx) / fx, (y - cy) / fy, 1.0])
    corners = [ray(0, 0), ray(W, 0), ray(W, H), ray(0, H)]
    inside = ray(0.5 * W, 0.5 * H)
    planes = []
    for a, b in zip(corners, corners[1:] + corners[:1]):
        n = np.cross(a, b)
        n /= np.linalg.norm(n)
        planes.append(n if n @ inside > 0 else -n)
    return planes


def test_frustum_culling_matches_corner_ray_planes(oracle_lib):
    """Sec. 4.3 "Frustum Culling": a sphere is dropped iff it lies wholly behind
    the near plane or wholly outside one side plane.  Against side planes built
    independently from the image corner rays (float64), on cameras with an
    off-centre principal point, fx != fy and W != H, the oracle culls exactly
    the spheres the rebuilt planes cull, wherever the float64 margin exceeds
    float32 rounding.  A plane tilted inwards, or cx and W - cx swapped, fails."""
    import dataclasses
    rng = np.random.default_rng(51)
    n_cull = n_keep = n_side = 0
    for it in range(24):
        W, H = int(rng.integers(64, 400)), int(rng.integers(48, 300))
        cam = synth.camera_look(rng.normal(0, 20, 3), rng.normal(size=3), rng.normal(size=3), W, H,
                                fovx_deg=float(rng.uniform(30, 100)), znear=float(rng.uniform(0.05, 2.0)))
        cam = dataclasses.replace(cam, fy=np.float32(cam.fx * rng.uniform(0.7, 1.4)),
                                  cx=np.float32(W * rng.uniform(0.2, 0.8)), cy=np.float32(H * rng.uniform(0.2, 0.8)))
        planes = _corner_ray_planes(cam)
        R, pos = cam.R.astype(np.float64), cam.pos.astype(np.float64)
        for _ in range(400):
            # points around the frustum's boundary: a direction through the image
            # (or just beyond it) at a random depth, pushed sideways
            x, y = rng.uniform(-0.4 * W, 1.4 * W), rng.uniform(-0.4 * H, 1.4 * H)
            z = rng.uniform(-5.0, 60.0)
            t = np.array([(x - float(cam.cx)) / float(cam.fx) * z, (y - float(cam.cy)) / float(cam.fy) * z, z])
            rad = float(np.float32(rng.choice([0.01, 0.3, 2.0, 8.0])))
            mu = (R.T @ t + pos).astype(np.float32)
            t64 = R @ (mu.astype(np.float64) - pos)          # the float32 centre, exactly
            ms = np.float32(rad / 3.0)
            r64 = 3.0 * float(ms)
            margins = [n @ t64 + r64 for n in planes] + [t64[2] + r64 - float(cam.znear)]
            tol = 1e-4 * (np.linalg.norm(t64) + r64 + 1.0)
            if min(abs(m) for m in margins) < tol:
                continue                                      # within float32 rounding of a plane
            expect = min(margins) < 0
            got = oracle_lib.cull_sphere(cam, mu, float(ms))
            assert got == expect, (it, margins)
            n_cull += expect
            n_keep += not expect
            n_side += expect and min(margins[:4]) < 0 and margins[4] > 0
    assert n_cull > 2000 and n_keep > 2000 and n_side > 1000


def test_culling_drops_only_what_cannot_be_seen_up_to_the_subtree_proxy(oracle_lib, scene1):
    """Culling on against culling off, image by image.  Sec. 4.3 culls a whole
    subtree by its root's sphere (radius 3 max s) and says that this proxy for
    the subtree's extent is not exact.  So, of the nodes a cull-off cut adds
    (E), those whose own sphere is outside the frustum must change no pixel,
    bit for bit, and every pixel that does change must come from the rest:
    descendants of a culled node whose own sphere reaches the frustum, a small
    fraction of E."""
    cfg, sc = scene1
    bg = (0.2, 0.1, 0.3)
    cams = [synth.camera_look([5.0, -3.0, -20.0], [0.2, 0.1, 1.0], [1.0, 0.0, 0.0], 160, 120, tau=1.0),
            synth.camera_look([30.0, 20.0, -90.0], [-0.2, -0.1, 1.0], [1.0, 0.0, 0.0], 256, 200, tau=1.0),
            synth.camera_look([0.0, 0.0, 0.0], [0.3, 0.2, 1.0], [1.0, 0.0, 0.0], 160, 160, tau=0.5)]
    n_e = n_leak = 0
    for cam in cams:
        on = oracle_lib.render(sc, cam, bg=bg, cull=True)
        off = oracle_lib.render(sc, cam, bg=bg, cull=False)
        E = np.setdiff1d(off["sel"], on["sel"])
        assert len(np.setdiff1d(on["sel"], off["sel"])) == 0
        rec = sc["row_rec"][E]
        own = np.array([oracle_lib.cull_sphere(cam, r[:3], float(r[3:6].max())) for r in rec], dtype=bool)
        with_out = oracle_lib.render(sc, cam, bg=bg, sel=np.union1d(on["sel"], E[own]))
        with_leak = oracle_lib.render(sc, cam, bg=bg, sel=np.union1d(on["sel"], E[~own]))
        assert np.array_equal(with_out["image"], on["image"])
        assert np.array_equal(with_leak["image"], off["image"])
        n_e += len(E)
        n_leak += int((~own).sum())
    assert n_e > 10_000 and n_leak <= n_e // 1000


def test_upper_bfs_matches_recursive_dfs(scene1):
    """Algorithm 1 (queue) against a textbook recursion with the same predicates."""
    import oracle
    cfg, sc = scene1
    cam = synth.camera_look([30.0, 20.0, -90.0], [-0.2, -0.1, 1.0], [1.0, 0.0, 0.0], 256, 200, tau=1.0)
    sel, _ = oracle.select(sc, cam, True)
    # recursion in float32 numpy with the documented expressions
    f32 = np.float32
    R, pos = cam.R.astype(f32), cam.pos.astype(f32)
    fx, fy, cx, cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
    W, H = f32(cam.width), f32(cam.height)
    planes = []
    for (a, b_, c_) in ((fx, f32(0), cx), (-fx, f32(0), W - cx)):
        l_ = np.sqrt(a * a + c_ * c_, dtype=f32)
        planes.append((a / l_, f32(0), c_ / l_))
    for (a, c_) in ((fy, cy), (-fy, H - cy)):
        l_ = np.sqrt(a * a + c_ * c_, dtype=f32)
        planes.append((f32(0), a / l_, c_ / l_))
    inv_k = f32(cam.tau) / fx
    rec = sc["node_rec"]
    out = []

    def view(v):
        d = rec[v, 0:3] - pos
        dist = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2], dtype=f32)
        t = [(R[a, 0] * d[0] + R[a, 1] * d[1]) + R[a, 2] * d[2] for a in range(3)]
        return t, dist

    def rec_dfs(u):
        v = sc["up_node"][u]
        t, dist = view(v)
        r = f32(3) * max(rec[v, 3], rec[v, 4], rec[v, 5])
        if t[2] + r < f32(cam.znear) or any((p[0] * t[0] + p[1] * t[1]) + p[2] * t[2] < -r for p in planes):
            return
        x = dist * inv_k
        kind = sc["up_kind"][u]
        s = rec[v, 3:6]
        S = np.sqrt(((s[0] * s[1] + s[0] * s[2]) + s[1] * s[2]) / f32(3), dtype=f32)
        if kind == 2:
            j = sc["up_ref"][u]
            b, c = sc["spt_base"][j], sc["spt_count"][j]
            for e in range(b, b + c):
                if sc["lo_row"][e] <= x < sc["hi_row"][e]:
                    out.append(e)
        elif kind == 1 or S <= x:
            out.append(sc["up_ref"][u])
        else:
            rec_dfs(sc["up_child"][u][0])
            rec_dfs(sc["up_child"][u][1])

    rec_dfs(0)
    assert np.array_equal(np.sort(np.array(out)), sel)


# ---------------------------------------------------------------------------
# projection and colour
# ---------------------------------------------------------------------------

def _one_gaussian_scene(recs, degree=0):
    import oracle
    recs = np.ascontiguousarray(np.atleast_2d(recs), dtype=np.float32)
    st = recs.shape[1]
    n = recs.shape[0]
    return {"stride": st, "degree": degree, "row_rec": recs}, np.arange(n, dtype=np.int64)


def test_projection_isotropic_on_axis_closed_form(oracle_lib):
    """Sigma' = (f s / z)^2 I + 0.3 I for an isotropic Gaussian on the optical axis."""
    st = synth.record_stride(0)
    rng = np.random.default_rng(4)
    for z, s in ((10.0, 0.5), (50.0, 2.0), (3.0, 0.05)):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        cam = synth.camera_look([0.0, 0.0, -z], [0, 0, 1], [1, 0, 0], 128, 96)
        scene, sel = _one_gaussian_scene(_rec(st, (0, 0, 0), (s, s, s), q))
        pr = oracle_lib.project(scene, sel, cam)
        f, s32 = float(cam.fx), float(np.float32(s))
        var = (f * s32 / z) ** 2 + 0.3
        u, v, A, B, Cc = pr["f64"][0, 0:5]
        assert pr["vis"][0] == 1
        assert u == pytest.approx(64.0) and v == pytest.approx(48.0)
        assert A == pytest.approx(1 / var, rel=1e-9) and Cc == pytest.approx(1 / var, rel=1e-9)
        assert abs(B) < 1e-12 / var
        assert np.allclose(pr["f32"][0, 2:5], [1 / var, 0, 1 / var], rtol=1e-5, atol=1e-6 / var)
        assert pr["key"][0] == np.float32(z).view(np.uint32)


def test_projection_jacobian_matches_finite_differences(oracle_lib):
    """EWA (Sec. 3): Sigma' = J W Sigma W^T J^T + 0.3 I with J the derivative of
    the perspective map, here taken by central differences."""
    st = synth.record_stride(0)
    rng = np.random.default_rng(5)
    cam = synth.camera_look([1.0, -2.0, -20.0], [0.05, 0.1, 1.0], [1, 0, 0], 320, 240)
    R = cam.R.astype(np.float64)
    for _ in range(10):
        mu = rng.uniform(-3, 3, 3)
        s = rng.uniform(0.1, 1.5, 3)
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        rec = _rec(st, mu, s, q)
        scene, sel = _one_gaussian_scene(rec)
        pr = oracle_lib.project(scene, sel, cam)
        t = R @ (rec[0:3].astype(np.float64) - cam.pos.astype(np.float64))

        def pi(t):
            return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])
        J = np.zeros((2, 3))
        for a in range(3):
            e = np.zeros(3); e[a] = 1e-5 * max(1.0, abs(t[a]))
            J[:, a] = (pi(t + e) - pi(t - e)) / (2 * e[a])
        S2 = J @ R @ _cov(rec) @ R.T @ J.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S2)
        A, B, Cc = pr["f64"][0, 2:5]
        assert np.allclose([A, B, Cc], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-6, atol=1e-9)
        assert np.allclose(pr["f64"][0, 0:2], pi(t), rtol=1e-12)


def test_projection_rotation_invariant_for_isotropic(oracle_lib):
    st = synth.record_stride(0)
    cam = synth.camera_look([2.0, 1.0, -15.0], [0.1, 0, 1], [1, 0, 0], 200, 200)
    rng = np.random.default_rng(6)
    ref = None
    for _ in range(5):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        scene, sel = _one_gaussian_scene(_rec(st, (0.5, -0.3, 1.0), (0.7, 0.7, 0.7), q))
        v = oracle_lib.project(scene, sel, cam)["f64"][0, :5]
        ref = v if ref is None else ref
        assert np.allclose(v, ref, rtol=1e-6)


def _real_sh_scipy(l, m, v):
    from scipy.special import sph_harm_y
    x, y, z = v
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    Y = sph_harm_y(l, abs(m), theta, phi)
    sgn = (-1) ** abs(m)
    return math.sqrt(2) * sgn * (Y.real if m > 0 else Y.imag)


def test_sh_matches_scipy_and_derivative(oracle_lib):
    rng = np.random.default_rng(7)
    for _ in range(20):
        v = rng.normal(size=3); v /= np.linalg.norm(v)
        Y, dY = oracle_lib.sh_eval(3, v)
        k = 0
        for l in range(1, 4):
            for m in range(-l, l + 1):
                assert Y[k] == pytest.approx(_real_sh_scipy(l, m, v), abs=1e-12)
                k += 1
        # derivative of the polynomial form vs central differences, tangential part
        for a in range(3):
            e = np.zeros(3); e[a] = 1e-6
            num = (oracle_lib.sh_eval(3, v + e)[0] - oracle_lib.sh_eval(3, v - e)[0]) / 2e-6
            assert np.allclose(dY[:, a], num, atol=1e-7)


def test_sh_orthonormal_by_quadrature(oracle_lib):
    xg, wg = np.polynomial.legendre.leggauss(24)
    nphi = 48
    K = 15
    G = np.zeros((K, K))
    for z, w in zip(xg, wg):
        for i in range(nphi):
            phi = 2 * math.pi * i / nphi
            r = math.sqrt(1 - z * z)
            Y, _ = oracle_lib.sh_eval(3, np.array([r * math.cos(phi), r * math.sin(phi), z]))
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    assert np.allclose(G, np.eye(K), atol=1e-12)


def test_colour_degree0_is_base_colour(oracle_lib):
    st = synth.record_stride(0)
    cam = synth.camera_look([0, 0, -10.0], [0, 0, 1], [1, 0, 0], 64, 64)
    scene, sel = _one_gaussian_scene(_rec(st, (0.3, 0.2, 0), (0.2, 0.3, 0.4), b=(0.25, 0.5, 0.75)))
    pr = oracle_lib.project(scene, sel, cam)
    assert np.allclose(pr["f64"][0, 6:9], [0.25, 0.5, 0.75], rtol=0, atol=1e-7)


# ---------------------------------------------------------------------------
# sort and blend
# ---------------------------------------------------------------------------

def _rect_pairs(pr, TX):
    tiles, keys, idx = [], [], []
    for i in np.nonzero(pr["vis"])[0]:
        x0, y0, x1, y1 = pr["rect"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                tiles.append(ty * TX + tx); keys.append(pr["key"][i]); idx.append(i)
    return map(np.array, (tiles, keys, idx))


def test_sort_matches_lexsort_of_kept_pairs(oracle_lib, scene1):
    """The pair list is the (tile, depth, index) lexsort of the rectangle pairs
    that pass the tile support test D9."""
    cfg, sc = scene1
    cam = cfg["cameras"][0]
    sel, _ = oracle_lib.select(sc, cam)
    pr = oracle_lib.project(sc, sel, cam)
    pairs = oracle_lib.sort_pairs(pr, cam.width, cam.height)
    TX = pairs["TX"]
    tiles, keys, idx = _rect_pairs(pr, TX)
    f = pr["f32"]
    keep = np.array([oracle_lib.tile_keep(*f[i][:5], t % TX, t // TX) for t, i in zip(tiles, idx)])
    assert 0 < keep.sum() < len(keep)
    tiles, keys, idx = tiles[keep], keys[keep], idx[keep]
    o = np.lexsort((idx, keys, tiles))
    assert np.array_equal(pairs["pair_i"], idx[o])
    assert np.array_equal(np.diff(pairs["tile_start"]), np.bincount(tiles, minlength=len(pairs["tile_start"]) - 1))


def _support_f32(u, v, A, B, C, px, py):
    f32 = np.float32
    dx = f32(u) - (f32(px) + f32(0.5))
    dy = f32(v) - (f32(py) + f32(0.5))
    nha, nhc, nb = f32(-0.5) * f32(A), f32(-0.5) * f32(C), -f32(B)
    # fmaf(nb*dx, dy, fmaf(nhc*dy, dy, (nha*dx)*dx)) with exact fused steps in float64
    inner = f32(np.float64(nhc * dy) * np.float64(dy) + np.float64((nha * dx) * dx))
    return f32(np.float64(nb * dx) * np.float64(dy) + np.float64(inner))


def test_tile_support_test_is_conservative(oracle_lib):
    """Brute force over every pixel centre: a tile that D9 drops has no pixel
    passing the float32 support test D8, for random anisotropic Gaussians."""
    rng = np.random.default_rng(21)
    kept = dropped = 0
    for _ in range(300):
        ang = rng.uniform(0, np.pi)
        s1, s2 = rng.uniform(0.5, 40.0), rng.uniform(0.5, 6.0)
        Rm = np.array([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]])
        S = Rm @ np.diag([s1 * s1, s2 * s2]) @ Rm.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S)
        A, B, C = (np.float32(Q[0, 0]), np.float32(Q[0, 1]), np.float32(Q[1, 1]))
        u, v = np.float32(rng.uniform(-40, 104)), np.float32(rng.uniform(-40, 104))
        for tx in range(4):
            for ty in range(4):
                k = oracle_lib.tile_keep(u, v, A, B, C, tx, ty)
                kept += k
                if not k:
                    dropped += 1
                    for py in range(16 * ty, 16 * ty + 16):
                        for px in range(16 * tx, 16 * tx + 16):
                            assert _support_f32(u, v, A, B, C, px, py) < np.float32(-4.5)
    assert kept > 100 and dropped > 100


def _support_f32_grid(u, v, A, B, C, px, py):
    """_support_f32 over integer pixel arrays (numpy float32 steps, fused steps in float64)."""
    f32 = np.float32
    dx = f32(u) - (px.astype(f32) + f32(0.5))
    dy = f32(v) - (py.astype(f32) + f32(0.5))
    nha, nhc, nb = f32(-0.5) * f32(A), f32(-0.5) * f32(C), -f32(B)
    inner = ((nhc * dy).astype(np.float64) * dy.astype(np.float64) + ((nha * dx) * dx).astype(np.float64)).astype(f32)
    return ((nb * dx).astype(np.float64) * dy.astype(np.float64) + inner.astype(np.float64)).astype(f32)


def test_block_support_test_is_conservative(oracle_lib):
    """Brute force over every pixel centre near the Gaussian: an 8x8 block that
    D10 skips has no pixel passing the float32 support test D8, for random
    anisotropic covariances up to condition numbers past the cut-off (1e5)."""
    rng = np.random.default_rng(22)
    f32 = np.float32
    kept = skipped = 0
    kaps = []
    for it in range(160):
        ang = rng.uniform(0, np.pi)
        s1 = rng.choice([rng.uniform(0.3, 5.0), rng.uniform(5.0, 60.0), rng.uniform(60.0, 400.0)])
        s2 = rng.uniform(0.05, 3.0)
        c_, s_ = f32(np.cos(ang)), f32(np.sin(ang))
        # covariance in float32 as the projection forms it: entries + 0.3 dilation
        l1, l2 = f32(s1 * s1), f32(s2 * s2)
        a = (c_ * c_) * l1 + (s_ * s_) * l2 + f32(0.3)
        b = (c_ * s_) * l1 - (c_ * s_) * l2
        c = (s_ * s_) * l1 + (c_ * c_) * l2 + f32(0.3)
        det = a * c - b * b
        if not det > 0:
            continue
        A, B, C = c / det, -b / det, a / det
        rx, ry = oracle_lib.support_extents(a, c, det)
        kaps.append(float((a + c) * (a + c) / det))
        u, v = f32(rng.uniform(100, 108)), f32(rng.uniform(100, 108))
        g = np.array([u, v, A, B, C, rx, ry], np.float32)
        R = int(min(3.2 * s1 + 12, 700))
        ys, xs = np.mgrid[max(0, 104 - R) & ~7:(104 + R) | 7, max(0, 104 - R) & ~7:(104 + R) | 7]
        p = _support_f32_grid(u, v, A, B, C, xs, ys)
        inside = p >= f32(-4.5)
        assert inside.any()
        for by in range(ys[0, 0], ys[-1, 0] + 1, 8):
            for bx in range(xs[0, 0], xs[0, -1] + 1, 8):
                k = oracle_lib.block_keep(g, bx, by)
                kept += k
                if not k:
                    skipped += 1
                    blk = inside[by - ys[0, 0]:by - ys[0, 0] + 8, bx - xs[0, 0]:bx - xs[0, 0] + 8]
                    assert not blk.any(), (it, bx, by, s1, s2)
    assert kept > 500 and skipped > 5000
    assert max(kaps) > 1e5 and sum(1e3 < k < 1e5 for k in kaps) > 20


def test_block_test_skips_no_supported_pixel_on_a_real_view(oracle_lib, scene1):
    """On a config-1 view, for every listed (tile, Gaussian) pair of the first
    three tile rows and every 8x8 block of the tile that D10 skips, no pixel
    centre of the block passes the float32 support test D8 (brute force); and
    the test does skip blocks there, so it is not vacuous.  The oracle's own
    blend and backward never call D10."""
    cfg, sc = scene1
    cam = cfg["cameras"][0]
    sel, _ = oracle_lib.select(sc, cam)
    pr = oracle_lib.project(sc, sel, cam)
    pairs = oracle_lib.sort_pairs(pr, cam.width, cam.height)
    f = pr["f32"]
    ts = pairs["tile_start"]
    TX = pairs["TX"]
    skips = checked = 0
    for t in range(0, min(len(ts) - 1, 3 * TX)):
        x0, y0 = (t % TX) * 16, (t // TX) * 16
        for e in range(ts[t], ts[t + 1]):
            gi = f[pairs["pair_i"][e]]
            for j in range(2):
                for i in range(2):
                    bx, by = x0 + 8 * i, y0 + 8 * j
                    if oracle_lib.block_keep(gi, bx, by):
                        continue
                    skips += 1
                    ys, xs = np.mgrid[by:by + 8, bx:bx + 8]
                    p = _support_f32_grid(gi[0], gi[1], gi[2], gi[3], gi[4], xs, ys)
                    assert not (p >= np.float32(-4.5)).any(), (t, e, i, j)
                    checked += 64
    assert skips > 0 and checked > 0


def test_tile_culling_leaves_the_image_unchanged(oracle_lib, scene1):
    """Blending the full rectangle pair list gives the same image, bit for bit."""
    cfg, sc = scene1
    cam = cfg["cameras"][0]
    sel, _ = oracle_lib.select(sc, cam)
    pr = oracle_lib.project(sc, sel, cam)
    culled = oracle_lib.sort_pairs(pr, cam.width, cam.height)
    TX = culled["TX"]
    tiles, keys, idx = _rect_pairs(pr, TX)
    o = np.lexsort((idx, keys, tiles))
    full = {"pair_i": idx[o].astype(np.int64), "TX": TX, "TY": culled["TY"],
            "tile_start": np.concatenate([[0], np.cumsum(np.bincount(tiles, minlength=TX * culled["TY"]))]).astype(np.int64)}
    assert len(full["pair_i"]) > len(culled["pair_i"])
    a = oracle_lib.blend(pr, culled, cam.width, cam.height)
    b = oracle_lib.blend(pr, full, cam.width, cam.height)
    assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["T_final"], b["T_final"])


def test_lone_gaussian_analytic_image(oracle_lib):
    """Eq. 1-2 for one isotropic on-axis Gaussian: c * min(0.99, sigma exp(-r^2 / (2 var)))
    inside the 3-sigma support, background outside."""
    st = synth.record_stride(0)
    z, s, op = 20.0, 0.4, 0.8
    col = np.array([0.9, 0.4, 0.2])
    cam = synth.camera_look([0, 0, -z], [0, 0, 1], [1, 0, 0], 64, 48)
    scene, sel = _one_gaussian_scene(_rec(st, (0, 0, 0), (s, s, s), op=op, b=col))
    out = oracle_lib.render(scene, cam, bg=(0.1, 0.2, 0.3), sel=sel)
    s, op = float(np.float32(s)), float(np.float32(op))
    col = col.astype(np.float32).astype(np.float64)
    var = (float(cam.fx) * s / z) ** 2 + 0.3
    py, px = np.mgrid[0:48, 0:64]
    r2 = (px + 0.5 - 32.0) ** 2 + (py + 0.5 - 24.0) ** 2
    p = -0.5 * r2 / var
    alpha = np.minimum(0.99, op * np.exp(p)) * (p >= -4.5)
    expect = col[None, None, :] * alpha[..., None] + (1 - alpha[..., None]) * np.array([0.1, 0.2, 0.3])
    inner = np.abs(p + 4.5) > 1e-4                               # away from the float32 support edge
    assert np.allclose(out["image"][inner], expect[inner], atol=1e-12)


def test_two_gaussians_composite_front_to_back(oracle_lib):
    st = synth.record_stride(0)
    cam = synth.camera_look([0, 0, -10.0], [0, 0, 1], [1, 0, 0], 32, 32)
    g1 = _rec(st, (0, 0, 0), (0.5, 0.5, 0.5), op=0.6, b=(1, 0, 0))
    g2 = _rec(st, (0, 0, 5), (0.75, 0.75, 0.75), op=0.7, b=(0, 1, 0))
    scene, sel = _one_gaussian_scene(np.stack([g2, g1]))         # order in input must not matter
    out = oracle_lib.render(scene, cam, sel=sel)
    f, f32 = float(cam.fx), lambda x: float(np.float32(x))
    c = out["image"][16, 16]                                      # pixel centre (16.5, 16.5)
    r2 = 0.5
    a1 = f32(0.6) * math.exp(-0.5 * r2 / ((f * 0.5 / 10) ** 2 + 0.3))
    a2 = f32(0.7) * math.exp(-0.5 * r2 / ((f * 0.75 / 15) ** 2 + 0.3))
    assert c[0] == pytest.approx(a1, rel=1e-12)
    assert c[1] == pytest.approx(a2 * (1 - a1), rel=1e-12)


def test_blend_transmittance_and_transparent_scene(oracle_lib, scene1):
    cfg, sc = scene1
    cam = cfg["cameras"][0]
    out = oracle_lib.render(sc, cam)
    # transmittance stops falling at the first value below 1e-4; alpha <= 0.99
    assert np.all(out["T_final"] <= 1.0) and np.all(out["T_final"] >= (1 - 0.99) * 1e-4)
    assert np.all(out["image"] >= 0) and np.all(out["image"] <= 1.0 + 1e-12)
    clear = dict(sc)
    clear["row_rec"] = sc["row_rec"].copy()
    clear["row_rec"][:, REC_OP] = 0.0
    o2 = oracle_lib.render(clear, cam, bg=(0.2, 0.4, 0.6), sel=out["sel"])
    assert np.allclose(o2["image"], np.array([0.2, 0.4, 0.6]), atol=0)


def _untruncated_eq1(proj, pairs, W, H, bg):
    """Eq. 1 without truncation, per tile in numpy: every listed Gaussian that
    passes the float32 support test D8 at a pixel is composited, however small
    the transmittance in front of it."""
    img = np.zeros((H, W, 3))
    f32, f64 = proj["f32"], proj["f64"]
    ts, TX = pairs["tile_start"], pairs["TX"]
    for t in range(len(ts) - 1):
        x0, y0 = (t % TX) * 16, (t // TX) * 16
        ys, xs = np.mgrid[y0:min(y0 + 16, H), x0:min(x0 + 16, W)]
        ids = pairs["pair_i"][ts[t]:ts[t + 1]]
        if len(ids) == 0:
            img[ys, xs] = bg
            continue
        g, q = f32[ids], f64[ids]
        sup = _support_f32_grid(g[:, 0, None, None], g[:, 1, None, None], g[:, 2, None, None],
                                g[:, 3, None, None], g[:, 4, None, None], xs[None], ys[None]) >= np.float32(-4.5)
        dx, dy = q[:, 0, None, None] - (xs[None] + 0.5), q[:, 1, None, None] - (ys[None] + 0.5)
        p = -0.5 * (q[:, 2, None, None] * dx * dx + q[:, 4, None, None] * dy * dy) - q[:, 3, None, None] * dx * dy
        alpha = np.where(sup, np.minimum(0.99, q[:, 5, None, None] * np.exp(p)), 0.0)
        T = np.cumprod(np.concatenate([np.ones((1,) + alpha.shape[1:]), 1.0 - alpha]), axis=0)
        img[ys, xs] = np.einsum("kyx,kc->yxc", alpha * T[:-1], q[:, 6:9]) + T[-1][..., None] * np.asarray(bg)
    return img


def test_transmittance_truncation_bound_against_untruncated_eq1(oracle_lib, scene1):
    """Eq. 1 truncated at T < 1e-4 (the Gaussian that takes T below the bound
    is still composited, then the pixel stops) differs from the untruncated sum
    by at most 1e-4 times the largest colour or background value: what is
    dropped is composited behind a transmittance already below 1e-4.  The 3DGS
    rule, which skips that Gaussian, drops alpha T c with T up to 1e-2 and
    fails.  On a config-1 view with over a thousand truncated pixels."""
    cfg, sc = scene1
    cam = cfg["cameras"][0]
    bg = (0.3, 0.6, 0.9)
    out = oracle_lib.render(sc, cam, bg=bg)
    stopped = out["T_final"] < 1e-4
    assert stopped.sum() > 1000
    full = _untruncated_eq1(out["proj"], out["pairs"], cam.width, cam.height, bg)
    cmax = max(out["proj"]["f64"][:, 6:9].max(), max(bg))
    d = np.abs(out["image"] - full).max(axis=2)
    assert d.max() <= 1e-4 * cmax, d.max() / cmax
    assert d[~stopped].max() <= 1e-12 and d[stopped].max() > 0


def test_the_gaussian_crossing_the_transmittance_bound_is_composited(oracle_lib):
    """A stack of equal on-axis Gaussians in front of the pixel (16, 12):
    with alpha ~ 0.6 each, T falls below 1e-4 at the eleventh.  The eleventh
    (red) must appear in the pixel with weight alpha T_10, the twelfth (blue)
    must not, and the first ten (green) are composited in full."""
    st = synth.record_stride(0)
    cam = synth.camera_look([0, 0, -10.0], [0, 0, 1], [1, 0, 0], 32, 24)
    recs = []
    for k in range(14):
        col = (1, 0, 0) if k == 10 else ((0, 0, 1) if k == 11 else (0, 1, 0))
        recs.append(_rec(st, (0, 0, 0.5 * k), (2.0, 2.0, 2.0), op=0.6, b=col))
    scene, sel = _one_gaussian_scene(np.stack(recs))
    out = oracle_lib.render(scene, cam, sel=sel)
    f = out["proj"]["f64"]
    order = np.argsort(f[:, 9], kind="stable")
    assert np.array_equal(order, np.arange(14))                  # depth order = index order
    dx, dy = f[:, 0] - 16.5, f[:, 1] - 12.5
    alpha = np.minimum(0.99, f[:, 5] * np.exp(-0.5 * (f[:, 2] * dx * dx + f[:, 4] * dy * dy) - f[:, 3] * dx * dy))
    T = np.cumprod(np.concatenate([[1.0], 1.0 - alpha]))
    assert T[10] >= 1e-4 > T[11]                                  # the eleventh crosses the bound
    px = out["image"][12, 16]
    assert px[0] == pytest.approx(alpha[10] * T[10], rel=1e-12) and px[0] > 0
    assert px[2] == 0.0
    assert px[1] == pytest.approx(float(np.sum(alpha[:10] * T[:10])), rel=1e-12)
    assert out["T_final"][12, 16] == pytest.approx(T[11], rel=1e-12)


# ---------------------------------------------------------------------------
# backward: finite differences on the oracle's own forward
# ---------------------------------------------------------------------------

def _fd_scene(degree, rng, n=6, case=None):
    """Six overlapping Gaussians in front of a 32x24 camera.  case:
    "jacobian": Gaussian 0 centred off-screen (clamped Jacobian);
    "alpha":    Gaussian 0 narrow, opacity 0.999, centred on pixel (16, 12), so
                alpha = min(0.99, sigma exp(p)) is clamped at that pixel;
    "negative": Gaussian 1's raw red channel b + sum Y f is -0.3 (clamped at 0)."""
    st = synth.record_stride(degree)
    cam = synth.camera_look([0.1, -0.05, -6.0], [0.02, 0.01, 1.0], [1, 0, 0], 32, 24)
    recs = []
    for i in range(n):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        mu = (rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(-0.5, 2.0))
        scales = rng.uniform(3.0, 4.5, 3)
        op = rng.uniform(0.1, 0.45)
        if case == "jacobian" and i == 0:
            mu = (9.0, 0.2, 1.0)                                  # centre off-screen: clamped Jacobian
            scales = np.array([8.0, 7.0, 9.0])
        if case == "alpha" and i == 0:
            z = 7.0                                               # depth of the pixel-centre ray point
            t = np.array([(16.5 - float(cam.cx)) / float(cam.fx) * z, (12.5 - float(cam.cy)) / float(cam.fy) * z, z])
            mu = cam.R.astype(np.float64).T @ t + cam.pos.astype(np.float64)
            scales, op = np.array([0.5, 0.7, 0.6]), 0.999
        r = _rec(st, mu, scales, q, op=op, b=rng.uniform(0.3, 0.7, 3))
        if degree:
            r[14:14 + 3 * ((degree + 1) ** 2 - 1)] = rng.normal(0, 0.05, 3 * ((degree + 1) ** 2 - 1))
        if case == "negative" and i == 1:
            import oracle
            d = r[0:3].astype(np.float64) - cam.pos.astype(np.float64)
            Y, _ = oracle.sh_eval(degree, d / np.linalg.norm(d))
            r[REC_B] = 0.1
            r[14 + 0:14 + 3 * len(Y):3] = ((-0.3 - 0.1) * Y / (Y @ Y)).astype(np.float32)
        recs.append(r)
    return np.stack(recs), cam


@pytest.mark.parametrize("degree,case", [(0, None), (3, None), (1, "jacobian"), (0, "alpha"), (3, "negative")])
def test_backward_matches_finite_differences(oracle_lib, degree, case):
    """The oracle's hand-derived gradients against central differences of its own
    forward, including the three clamped branches: the Jacobian clamp, the
    alpha clamp at 0.99 (zero gradient through alpha where it binds) and the
    colour clamp at 0 (zero gradient through a negative raw channel)."""
    rng = np.random.default_rng(10 + degree)
    recs, cam = _fd_scene(degree, rng, case=case)
    scene, sel = _one_gaussian_scene(recs, degree)
    bg = (0.05, 0.1, 0.15)
    fwd = oracle_lib.render(scene, cam, bg=bg, sel=sel)
    assert fwd["proj"]["vis"].all()
    assert np.all(fwd["proj"]["rect"] == [0, 0, 2, 2])
    py, px = np.mgrid[0:cam.height, 0:cam.width]

    def masks(proj, i):
        """Gaussian i's pixel decisions: the float32 support test D8 and the alpha clamp."""
        f32, f64 = proj["f32"][i], proj["f64"][i]
        sup = _support_f32_grid(f32[0], f32[1], f32[2], f32[3], f32[4], px, py) >= np.float32(-4.5)
        dx, dy = f64[0] - (px + 0.5), f64[1] - (py + 0.5)
        p = -0.5 * (f64[2] * dx * dx + f64[4] * dy * dy) - f64[3] * dx * dy
        return sup, f64[5] * np.exp(p) > 0.99

    base_masks = [masks(fwd["proj"], i) for i in range(recs.shape[0])]
    f = fwd["proj"]["f64"]
    if case == "alpha":
        assert base_masks[0][1].sum() == 1 and base_masks[0][0].sum() < 0.8 * px.size
        assert sum(m[1].sum() for m in base_masks[1:]) == 0    # clamped at one pixel, by Gaussian 0
    if case == "jacobian":
        assert f[0, 0] > cam.width                                # centre off-screen
    if case == "negative":
        assert f[1, 6] == 0.0 and f[1, 7] > 0 and f[1, 8] > 0    # red clamped at 0
    wimg = np.random.default_rng(99).uniform(-1, 1, fwd["image"].shape)
    g = oracle_lib.render_backward(scene, cam, fwd, wimg, bg=bg)["g_rec"]
    if case == "negative":
        K = (degree + 1) ** 2 - 1
        assert g[1, REC_B] == 0.0 and not np.any(g[1, 14:14 + 3 * K:3])
    K = (degree + 1) ** 2 - 1
    cols = list(range(0, 14 + 3 * K))
    for i in range(recs.shape[0]):
        for c in cols:
            base = recs[i, c]
            h = np.float32(2e-3 * max(1.0, abs(float(base))))
            vals = []
            for sgn in (1, -1):
                rr = recs.copy()
                rr[i, c] = np.float32(base + sgn * h)
                sc2, _ = _one_gaussian_scene(rr, degree)
                out2 = oracle_lib.render(sc2, cam, bg=bg, sel=sel)
                m2 = masks(out2["proj"], i)                   # the step flips no decision
                assert np.array_equal(m2[0], base_masks[i][0]) and np.array_equal(m2[1], base_masks[i][1]), (i, c)
                vals.append((out2["image"] * wimg).sum())
            hp = float(np.float32(base + h)) - float(np.float32(base - h))
            num = (vals[0] - vals[1]) / hp
            assert g[i, c] == pytest.approx(num, rel=2e-3, abs=2e-4 * (1 + abs(num))), (i, c)


# ---------------------------------------------------------------------------
# sparse Adam over the cut set
# ---------------------------------------------------------------------------

def test_adam_every_row_every_step_equals_torch(oracle_lib):
    """With every row selected at every step the sparse Adam is torch.optim.Adam."""
    rng = np.random.default_rng(40)
    n, stride, lr = 6, 8, 3e-3
    p0 = rng.standard_normal((n, stride))
    params, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    t = np.zeros(n, np.uint32)
    tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    for _ in range(7):
        g = rng.standard_normal((n, stride))
        oracle_lib.adam_sparse(params, m, v, t, np.arange(n), g, lr, eps=1e-8)
        tp.grad = torch.tensor(g)
        opt.step()
    assert np.allclose(params, tp.detach().numpy(), rtol=1e-12, atol=1e-14)
    assert np.all(t == 7)


def test_adam_rows_count_their_own_steps(oracle_lib):
    """A row selected at some steps only moves then, with the bias correction of
    its own step count: it matches a torch Adam that steps only at those steps;
    rows never selected are untouched, bit for bit."""
    rng = np.random.default_rng(41)
    n, stride, lr = 5, 4, 1e-2
    p0 = rng.standard_normal((n, stride))
    params, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    t = np.zeros(n, np.uint32)
    sel_by_step = [[0, 2], [2], [0, 1, 2], [1], [0, 2]]
    ref = {}
    for r in range(n):
        tp = torch.tensor(p0[r].copy(), dtype=torch.float64, requires_grad=True)
        ref[r] = (tp, torch.optim.Adam([tp], lr=lr, eps=1e-15))
    for sel in sel_by_step:
        g = rng.standard_normal((len(sel), stride))
        oracle_lib.adam_sparse(params, m, v, t, sel, g, lr)
        for i, r in enumerate(sel):
            tp, opt = ref[r]
            tp.grad = torch.tensor(g[i])
            opt.step()
    for r in range(n):
        assert np.allclose(params[r], ref[r][0].detach().numpy(), rtol=1e-12, atol=1e-14)
    assert list(t) == [3, 2, 4, 0, 0]
    assert np.array_equal(params[3:], p0[3:])


def test_adam_constant_gradient_closed_form(oracle_lib):
    """A constant gradient makes both bias-corrected moments exact (m = g, v = g^2),
    so every step moves a column by lr_c g / (|g| + eps)."""
    stride, steps, eps = 6, 9, 1e-8
    lr = np.array([1e-3, 2e-3, 5e-4, 1e-2, 3e-3, 0.0])
    g = np.array([[0.5, -2.0, 1e-3, 4.0, -0.25, 1.0]])
    params = np.ones((1, stride))
    m, v, t = np.zeros_like(params), np.zeros_like(params), np.zeros(1, np.uint32)
    for _ in range(steps):
        oracle_lib.adam_sparse(params, m, v, t, [0], g, lr, eps=eps)
    assert np.allclose(params[0], 1.0 - steps * lr * g[0] / (np.abs(g[0]) + eps), rtol=1e-12, atol=1e-15)


def test_lod_noise_keeps_proper_cuts_and_coarsens(oracle_lib, scene1):
    """Training LoD noise multiplies the distances to the SPT roots by 1 + 5 r^4:
    every scaled cut is still proper (each root-to-leaf path crossed once), equals
    the brute-force descent at the scaled distances, and coarsens as the factor grows;
    a factor of 1 is the plain cut."""
    import dataclasses
    cfg, sc = scene1
    cam = cfg["cameras"][0]
    plain, _ = oracle_lib.select(sc, cam, False)
    counts = []
    for r in (0.0, 0.3, 0.7, 1.0):
        s = synth.lod_noise_factor(r)
        cam_s = dataclasses.replace(cam, spt_scale=s)
        sel, _ = oracle_lib.select(sc, cam_s, False)
        assert np.array_equal(sel, oracle_lib.select_bruteforce(sc, cam_s, False))
        assert np.all(_covered_leaves(sc, sel) == 1)
        counts.append(len(sel))
        if r == 0.0:
            assert np.array_equal(sel, plain)
    assert counts == sorted(counts, reverse=True) and counts[-1] < counts[0]


def _torch_render_fp64(recs, cam, bg):
    """Projection (EWA, Sec. 3 Eq. 2) and front-to-back blending (Eq. 1) of SH0
    records, restated densely in float64 PyTorch: every pixel against every
    Gaussian in depth order, no tiles, no support test, no early stop (the
    scenes below keep every pixel inside every support and T above T_min)."""
    f64 = torch.float64
    R = torch.tensor(np.asarray(cam.R, np.float64).reshape(3, 3), dtype=f64)
    pos = torch.tensor(np.asarray(cam.pos, np.float64), dtype=f64)
    mu, s, q, op, b = recs[:, 0:3], recs[:, 3:6], recs[:, 6:10], recs[:, 10], recs[:, 11:14]
    t = (mu - pos) @ R.T
    qn = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = qn.unbind(1)
    Rq = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)], 1)
    Sig = Rq @ torch.diag_embed(s * s) @ Rq.transpose(1, 2)
    tx, ty, tz = t.unbind(1)
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([cam.fx / tz, zero, -cam.fx * tx / (tz * tz)], 1),
                     torch.stack([zero, cam.fy / tz, -cam.fy * ty / (tz * tz)], 1)], 1)
    M = J @ R
    S2 = M @ Sig @ M.transpose(1, 2) + 0.3 * torch.eye(2, dtype=f64)
    det = S2[:, 0, 0] * S2[:, 1, 1] - S2[:, 0, 1] * S2[:, 1, 0]
    A, B, Cc = S2[:, 1, 1] / det, -S2[:, 0, 1] / det, S2[:, 0, 0] / det
    u = cam.fx * tx / tz + cam.cx
    v = cam.fy * ty / tz + cam.cy
    col = torch.clamp_min(b, 0.0)
    py, px = torch.meshgrid(torch.arange(cam.height, dtype=f64) + 0.5, torch.arange(cam.width, dtype=f64) + 0.5,
                            indexing="ij")
    T = torch.ones_like(px)
    img = torch.zeros((cam.height, cam.width, 3), dtype=f64)
    for i in np.argsort(tz.detach().numpy(), kind="stable"):
        dx, dy = u[i] - px, v[i] - py
        p = -0.5 * (A[i] * dx * dx + Cc[i] * dy * dy) - B[i] * dx * dy
        alpha = op[i] * torch.exp(p)
        img = img + (T * alpha)[..., None] * col[i]
        T = T * (1 - alpha)
    return img + T[..., None] * torch.tensor(bg, dtype=f64)


def test_backward_matches_autograd_of_a_dense_restatement(oracle_lib):
    """The oracle's hand-derived backward (Eq. 1-2 and the EWA projection,
    differentiated) against torch autograd of the dense float64 restatement
    above, on six overlapping Gaussians and a 32x24 image: image and every
    record gradient (mean, scales, raw quaternion, opacity, base colour)."""
    rng = np.random.default_rng(21)
    recs, cam = _fd_scene(0, rng)
    scene, sel = _one_gaussian_scene(recs, 0)
    bg = (0.05, 0.1, 0.15)
    fwd = oracle_lib.render(scene, cam, bg=bg, sel=sel)
    f = fwd["proj"]["f64"]
    py, px = np.mgrid[0:cam.height, 0:cam.width]
    for i in range(recs.shape[0]):                                # every pixel inside every support
        dx, dy = f[i, 0] - (px + 0.5), f[i, 1] - (py + 0.5)
        assert (-0.5 * (f[i, 2] * dx * dx + f[i, 4] * dy * dy) - f[i, 3] * dx * dy).min() > -4.3
    assert fwd["T_final"].min() > 1e-3                            # no early stop
    rt = torch.tensor(recs.astype(np.float64), requires_grad=True)
    img_t = _torch_render_fp64(rt, cam, bg)
    assert np.allclose(img_t.detach().numpy(), fwd["image"], rtol=1e-10, atol=1e-12)
    wimg = np.random.default_rng(98).uniform(-1, 1, fwd["image"].shape)
    (img_t * torch.tensor(wimg)).sum().backward()
    g = oracle_lib.render_backward(scene, cam, fwd, wimg, bg=bg)["g_rec"][:, :14]
    ga = rt.grad.numpy()[:, :14]
    scale = np.abs(ga).max(axis=0) + 1e-30
    assert np.all(np.abs(g - ga) <= 1e-8 * scale + 1e-12), np.abs(g - ga).max(axis=0) / scale
