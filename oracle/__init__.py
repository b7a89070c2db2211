"""CPU oracle for the LoD Gaussian render path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may import
this package.  The product library never calls it.  The arithmetic lives in
`lodgs_oracle.c` (plain C, float64 values, float32 decisions); this module
compiles it with gcc and marshals numpy arrays.

Functions and the paper passage they follow:
  build_scene      hierarchy merge (Sec. 3 "Gaussian Hierarchies"), HSPT
                   construction (Sec. 4.3) and SPT layout (Sec. 4.1, Eq. 4, Eq. 6)
  select           Algorithm 1 (upper BFS with frustum culling) + Algorithm 2
  select_bruteforce  top-down descent inside each SPT (independent check)
  select_upper     Algorithm 1 alone (selected upper rows, SPT roots with x_j)
  cache.NodeCache  the out-of-core cache's decisions per view (Sec. 4.4 Eq. 7,
                   Algorithm 3): hit, re-cut or load per SPT root, LRU
                   eviction, and the cut that results
  project          EWA projection and SH colour (Sec. 3, Eq. 2)
  sort_pairs       tile x depth ordering (3DGS sort reused by the paper)
  blend            Eq. 1 front-to-back compositing
  render_backward  exact derivative of blend + projection
  split_record, densify
                   densification by moving Gaussians (Sec. 3 "Densification",
                   the 3DGS-MCMC split) and the HSPT rebuild after it
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lodgs_oracle.c")
_LIB = os.path.join(_HERE, "liblodgs_oracle.so")
_LIB_OMP = os.path.join(_HERE, "liblodgs_oracle_omp.so")
_libs = {}
_use_omp = False

KIND_INTERNAL, KIND_LEAF, KIND_SPT = 0, 1, 2
TILE = 16


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle shared library with gcc (no fused multiply-add).
    omp=True builds the OpenMP variant the benchmark times on all host cores."""
    out = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC"] + (["-fopenmp"] if omp else []) + ["-o", out + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)
    return out


def lib():
    key = "omp" if _use_omp else "serial"
    if key not in _libs:
        path = build(omp=_use_omp)
        lb = C.CDLL(path)
        lb.or_morton_code.restype = C.c_uint64
        _libs[key] = lb
    return _libs[key]


def use_threads(n: int | None) -> int:
    """Route the oracle's calls to its OpenMP build with n threads (None or 0:
    the OpenMP default, every host core), or back to the single-threaded build
    (n = 1).  Returns the thread count the calls will use."""
    global _use_omp
    _use_omp = n != 1
    if _use_omp:
        lib().or_set_threads(C.c_int(int(n or 0)))
    return int(lib().or_threads())


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
    return C.c_void_p(a.ctypes.data)


def stride(degree: int) -> int:
    return int(lib().or_stride(C.c_int(degree)))


def pack_camera(cam) -> np.ndarray:
    """R[9], pos[3], fx, fy, cx, cy, W, H, tau, znear, spt_scale as float32."""
    v = np.zeros(21, dtype=np.float32)
    v[0:9] = np.asarray(cam.R, dtype=np.float32).reshape(9)
    v[9:12] = np.asarray(cam.pos, dtype=np.float32)
    v[12:20] = [cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.tau, cam.znear]
    v[20] = getattr(cam, "spt_scale", 1.0)
    return v


# ---------------------------------------------------------------------------
# hierarchy
# ---------------------------------------------------------------------------

def morton_order(leaves: np.ndarray) -> np.ndarray:
    leaves = np.ascontiguousarray(leaves, dtype=np.float32)
    n = leaves.shape[0]
    order = np.zeros(n, dtype=np.int64)
    rc = lib().or_morton_order(C.c_int64(n), C.c_int(leaves.shape[1]), _p(leaves), _p(order))
    assert rc == 0
    return order


def merge_hierarchy(leaves: np.ndarray, degree: int, order: np.ndarray | None = None) -> dict:
    leaves = np.ascontiguousarray(leaves, dtype=np.float32)
    n, st = leaves.shape
    if order is None:
        order = morton_order(leaves)
    order = np.ascontiguousarray(order, dtype=np.int64)
    M = 2 * n - 1
    node = np.zeros((M, st), dtype=np.float32)
    left = np.zeros(M, dtype=np.int64)
    right = np.zeros(M, dtype=np.int64)
    parent = np.zeros(M, dtype=np.int64)
    rc = lib().or_merge(C.c_int64(n), C.c_int(st), C.c_int(degree), _p(leaves), _p(order), _p(node),
                        _p(left), _p(right), _p(parent))
    assert rc == 0
    return {"n_leaves": n, "degree": degree, "stride": st, "node_rec": node, "left": left,
            "right": right, "parent": parent, "root": M - 1, "order": order}


def merge_pair(ra: np.ndarray, rb: np.ndarray, degree: int) -> np.ndarray:
    ra = np.ascontiguousarray(ra, dtype=np.float32)
    rb = np.ascontiguousarray(rb, dtype=np.float32)
    out = np.zeros_like(ra)
    lib().or_merge_pair(C.c_int(ra.shape[0]), C.c_int(degree), _p(ra), _p(rb), _p(out))
    return out


def cov_to_scale_rot(cov: np.ndarray):
    A = np.ascontiguousarray(cov, dtype=np.float64).reshape(3, 3)
    s = np.zeros(3)
    q = np.zeros(4)
    lib().or_cov_to_scale_rot(_p(A), _p(s), _p(q))
    return s, q


def hspt(h: dict, spt_volume: float, kappa: float) -> dict:
    node = h["node_rec"]
    M, st = node.shape
    counts = np.zeros(3, dtype=np.int64)
    up_node = np.zeros(M, dtype=np.int64)
    up_kind = np.zeros(M, dtype=np.int32)
    up_parent = np.zeros(M, dtype=np.int64)
    up_child = np.zeros(2 * M, dtype=np.int64)
    up_ref = np.zeros(M, dtype=np.int64)
    spt_root = np.zeros(M, dtype=np.int64)
    spt_base = np.zeros(M + 1, dtype=np.int64)
    spt_count = np.zeros(M, dtype=np.int64)
    node_of_row = np.zeros(M, dtype=np.int64)
    row_of_node = np.zeros(M, dtype=np.int64)
    lo_row = np.zeros(M, dtype=np.float32)
    hi_row = np.zeros(M, dtype=np.float32)
    lo_raw = np.zeros(M, dtype=np.float32)
    rc = lib().or_hspt(C.c_int64(M), C.c_int(st), _p(node), _p(h["left"]), _p(h["right"]),
                       C.c_int64(h["root"]), C.c_float(spt_volume), C.c_float(kappa), _p(counts),
                       _p(up_node), _p(up_kind), _p(up_parent), _p(up_child), _p(up_ref),
                       _p(spt_root), _p(spt_base), _p(spt_count), _p(node_of_row), _p(row_of_node),
                       _p(lo_row), _p(hi_row), _p(lo_raw))
    assert rc == 0, rc
    nu, ns, nr = (int(x) for x in counts)
    spt_base[ns] = M
    out = dict(h)
    out.update({
        "spt_volume": float(np.float32(spt_volume)), "kappa": float(np.float32(kappa)),
        "n_upper": nu, "n_spt": ns, "n_upper_rows": nr,
        "up_node": up_node[:nu].copy(), "up_kind": up_kind[:nu].copy(), "up_parent": up_parent[:nu].copy(),
        "up_child": up_child[:2 * nu].reshape(nu, 2).copy(), "up_ref": up_ref[:nu].copy(),
        "spt_root": spt_root[:ns].copy(), "spt_base": spt_base[:ns + 1].copy(),
        "spt_count": spt_count[:ns].copy(), "node_of_row": node_of_row, "row_of_node": row_of_node,
        "lo_row": lo_row, "hi_row": hi_row, "lo_raw": lo_raw,
        "row_rec": np.ascontiguousarray(node[node_of_row]),
    })
    return out


def build_scene(leaves: np.ndarray, degree: int, spt_volume: float, kappa: float) -> dict:
    """Leaves -> binary hierarchy -> HSPT with SPT layout (render-row order)."""
    return hspt(merge_hierarchy(leaves, degree), spt_volume, kappa)


# ---------------------------------------------------------------------------
# densification (Sec. 3 "Densification")
# ---------------------------------------------------------------------------
DENSIFY_SPAWN, DENSIFY_RESPAWN = 0, 1
REC_S, REC_OP = 3, 10


def split_record(rec: np.ndarray) -> np.ndarray:
    """The record each of the two children of a split leaf carries (Sec. 3
    "Densification", the split of 3DGS-MCMC with N = 2 copies): the same mean,
    rotation and colour; opacity o' = 1 - (1 - o)^(1/2), so the centre's
    composited opacity is kept; scales times o / (2 o' - o'^2 / sqrt 2), the
    MCMC factor for N = 2 (sum over the copies i and the terms k of
    C(i-1, k) (-1)^k o'^(k+1) / sqrt(k+1)).  Records are float32 and both sides
    evaluate these operations in float32, in this order (sqrt 2 as the float32
    constant), because the HSPT volume test and the SPT bounds are float32
    decisions on the result."""
    f32 = np.float32
    out = np.array(rec, dtype=np.float32, copy=True)
    sg = f32(rec[REC_OP])
    if not sg > 0:
        return out
    sp = f32(1) - np.sqrt(f32(1) - sg)
    den = f32(2) * sp - (sp * sp) / f32(np.sqrt(2.0))
    f = sg / den
    out[REC_OP] = sp
    out[REC_S:REC_S + 3] = (np.asarray(rec[REC_S:REC_S + 3], np.float32) * f).astype(np.float32)
    return out


def densify(scene: dict, ops) -> tuple[dict, np.ndarray]:
    """Apply spawn / respawn operations (kind, target row, dead row) given in
    the scene's render rows, in order, then rebuild the HSPT and SPT layout with
    the scene's own spt_volume and kappa.

    spawn:   leaf T gets two new leaf children with the next free canonical ids.
    respawn: dead leaf D and its parent P leave; D's sibling takes P's place
             (the root's place if P was the root); P and D become T's children.
    Both children carry split_record(T); T keeps its record and is their parent.
    Returns the new scene and, per new render row, the row the node had before
    (-1 for a node whose record is new)."""
    node = scene["node_rec"]
    M0, st = node.shape
    nor0 = np.asarray(scene["node_of_row"], np.int64)
    row_of_node0 = np.empty(M0, np.int64)
    row_of_node0[nor0] = np.arange(M0)
    n_spawn = sum(1 for k, _, _ in ops if k == DENSIFY_SPAWN)
    M = M0 + 2 * n_spawn
    left = np.full(M, -1, np.int64)
    right = np.full(M, -1, np.int64)
    left[:M0], right[:M0] = scene["left"], scene["right"]
    parent = np.full(M, -1, np.int64)
    for u in range(M0):
        for c in (left[u], right[u]):
            if c >= 0:
                parent[c] = u
    root = int(scene["root"])
    rec = np.zeros((M, st), np.float32)
    rec[:M0] = node
    fresh = np.zeros(M, bool)
    nxt = M0
    for kind, t_row, d_row in ops:
        T = int(nor0[t_row])
        if left[T] >= 0 or fresh[T]:
            raise ValueError("densify: the target is not an original leaf")
        if kind == DENSIFY_SPAWN:
            a, b = nxt, nxt + 1
            nxt += 2
        elif kind == DENSIFY_RESPAWN:
            D = int(nor0[d_row])
            P = int(parent[D])
            if left[D] >= 0 or fresh[D] or D == T or P < 0:
                raise ValueError("densify: the dead node must be an original leaf with a parent, not the target")
            S = int(right[P]) if left[P] == D else int(left[P])
            G = int(parent[P])
            if G >= 0:
                if left[G] == P:
                    left[G] = S
                else:
                    right[G] = S
            else:
                root = S
            parent[S] = G
            a, b = P, D
        else:
            raise ValueError("densify: unknown operation")
        child = split_record(rec[T])
        left[T], right[T] = a, b
        parent[a] = parent[b] = T
        left[a] = right[a] = left[b] = right[b] = -1
        rec[a] = rec[b] = child
        fresh[a] = fresh[b] = True
    h = {"n_leaves": (M + 1) // 2, "degree": scene["degree"], "stride": st, "node_rec": rec, "left": left,
         "right": right, "parent": parent, "root": root}
    out = hspt(h, scene["spt_volume"], scene["kappa"])
    nor = out["node_of_row"]
    old = np.where((nor < M0) & ~fresh[nor], row_of_node0[np.minimum(nor, M0 - 1)], -1)
    return out, old


# ---------------------------------------------------------------------------
# selection
# ---------------------------------------------------------------------------

def select(scene: dict, cam, cull: bool = True):
    M = scene["node_rec"].shape[0]
    sel = np.zeros(M, dtype=np.int64)
    n = np.zeros(1, dtype=np.int64)
    stats = np.zeros(5, dtype=np.int64)
    up_child = np.ascontiguousarray(scene["up_child"].reshape(-1))
    camv = pack_camera(cam)
    rc = lib().or_select(C.c_int64(scene["n_upper"]), _p(scene["up_node"]), _p(scene["up_kind"]), _p(up_child),
                         _p(scene["up_ref"]), _p(scene["spt_base"]), _p(scene["lo_row"]), _p(scene["hi_row"]),
                         C.c_int(scene["stride"]), _p(scene["node_rec"]), _p(camv), C.c_int(int(cull)),
                         _p(sel), _p(n), _p(stats))
    assert rc == 0
    return sel[: int(n[0])].copy(), {"upper_visited": int(stats[0]), "upper_culled": int(stats[1]),
                                     "spt_cut": int(stats[2]), "spt_scanned": int(stats[3]),
                                     "selected": int(stats[4])}


def select_upper(scene: dict, cam, cull: bool = True):
    """Algorithm 1 alone: the upper rows it selects (ascending) and the SPT roots
    it reaches in BFS order, as (spt ids, float32 query distances x_j)."""
    n_up = scene["n_upper"]
    sel = np.zeros(max(n_up, 1), dtype=np.int64)
    sj = np.zeros(max(n_up, 1), dtype=np.int64)
    sx = np.zeros(max(n_up, 1), dtype=np.float32)
    n, m = np.zeros(1, dtype=np.int64), np.zeros(1, dtype=np.int64)
    up_child = np.ascontiguousarray(scene["up_child"].reshape(-1))
    camv = pack_camera(cam)
    rc = lib().or_select_upper(C.c_int64(n_up), _p(scene["up_node"]), _p(scene["up_kind"]), _p(up_child),
                               _p(scene["up_ref"]), C.c_int(scene["stride"]), _p(scene["node_rec"]), _p(camv),
                               C.c_int(int(cull)), _p(sel), _p(n), _p(sj), _p(sx), _p(m))
    assert rc == 0
    return np.sort(sel[: int(n[0])]), sj[: int(m[0])].copy(), sx[: int(m[0])].copy()


def cull_sphere(cam, mu, max_scale: float) -> bool:
    """Frustum culling (Sec. 4.3) of one sphere: centre mu, radius 3 * max_scale."""
    camv = pack_camera(cam)
    m = np.ascontiguousarray(mu, dtype=np.float32)
    return bool(lib().or_cull_sphere(_p(camv), _p(m), C.c_float(max_scale)))


def select_bruteforce(scene: dict, cam, cull: bool = True) -> np.ndarray:
    M = scene["node_rec"].shape[0]
    sel = np.zeros(M, dtype=np.int64)
    n = np.zeros(1, dtype=np.int64)
    up_child = np.ascontiguousarray(scene["up_child"].reshape(-1))
    camv = pack_camera(cam)
    rc = lib().or_select_bruteforce(C.c_int64(scene["n_upper"]), _p(scene["up_node"]), _p(scene["up_kind"]),
                                    _p(up_child), _p(scene["up_ref"]), _p(scene["spt_root"]), _p(scene["left"]),
                                    _p(scene["right"]), _p(scene["lo_raw"]), _p(scene["row_of_node"]),
                                    C.c_int(scene["stride"]), _p(scene["node_rec"]), _p(camv),
                                    C.c_int(int(cull)), _p(sel), _p(n))
    assert rc == 0
    return sel[: int(n[0])].copy()


# ---------------------------------------------------------------------------
# projection, sort, blend, backward
# ---------------------------------------------------------------------------

def project(scene: dict, sel: np.ndarray, cam) -> dict:
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    n = sel.shape[0]
    vis = np.zeros(n, dtype=np.int32)
    rect = np.zeros((n, 4), dtype=np.int32)
    key = np.zeros(n, dtype=np.uint32)
    f32 = np.zeros((n, 7), dtype=np.float32)       # u, v, A, B, C, rx, ry
    f64 = np.zeros((n, 12), dtype=np.float64)
    camv = pack_camera(cam)
    lib().or_project(C.c_int64(n), _p(sel), C.c_int(scene["stride"]), C.c_int(scene["degree"]),
                     _p(scene["row_rec"]), _p(camv), _p(vis), _p(rect), _p(key), _p(f32), _p(f64))
    return {"vis": vis, "rect": rect, "key": key, "f32": f32, "f64": f64, "n": n}


def sort_pairs(proj: dict, width: int, height: int) -> dict:
    TX, TY = (width + TILE - 1) // TILE, (height + TILE - 1) // TILE
    r = proj["rect"].astype(np.int64)
    cap = int(((r[:, 2] - r[:, 0]) * (r[:, 3] - r[:, 1]) * (proj["vis"] != 0)).sum())
    pair_i = np.zeros(max(cap, 1), dtype=np.int64)
    tile_start = np.zeros(TX * TY + 1, dtype=np.int64)
    npairs = np.zeros(1, dtype=np.int64)
    rc = lib().or_sort_pairs(C.c_int64(proj["n"]), _p(proj["vis"]), _p(proj["rect"]), _p(proj["key"]),
                             _p(proj["f32"]), C.c_int(TX), C.c_int(TY), C.c_int64(cap), _p(npairs), _p(pair_i),
                             _p(tile_start))
    assert rc == 0
    return {"pair_i": pair_i[: int(npairs[0])].copy(), "tile_start": tile_start, "TX": TX, "TY": TY}


def _win(window):
    if window is None:
        return None
    w = np.ascontiguousarray(window, dtype=np.int32)
    return w


def tile_keep(u, v, ca, cb, cc, tx, ty) -> bool:
    """Tile support test D9 for one (Gaussian, tile); (ca, cb, cc) is the conic."""
    f = C.c_float
    return bool(lib().or_tile_keep(f(u), f(v), f(ca), f(cb), f(cc), C.c_int(int(tx)), C.c_int(int(ty))))


def block_keep(g, px: int, py: int) -> bool:
    """Block support test D10 for one (Gaussian, pixel); g = (u, v, A, B, C, rx, ry).
    The predicate the CUDA blend skips whole 8x8 blocks by; blend() and
    blend_backward() here do not use it (they test D8 on every listed pair)."""
    gv = np.ascontiguousarray(g, dtype=np.float32)
    return bool(lib().or_block_keep(_p(gv), C.c_int(int(px)), C.c_int(int(py))))


def support_extents(a: float, c: float, det: float) -> tuple:
    """Float32 support half extents (rx, ry) of D10 from a 2D covariance (a, c) and its determinant."""
    rx, ry = C.c_float(), C.c_float()
    lib().or_support_extents(C.c_float(a), C.c_float(c), C.c_float(det), C.byref(rx), C.byref(ry))
    return rx.value, ry.value


def blend(proj: dict, pairs: dict, width: int, height: int, bg=(0.0, 0.0, 0.0), window=None) -> dict:
    img = np.zeros((height, width, 3), dtype=np.float64)
    ncon = np.zeros((height, width), dtype=np.int32)
    tfin = np.zeros((height, width), dtype=np.float64)
    bgv = np.asarray(bg, dtype=np.float64)
    pair_i = pairs["pair_i"] if pairs["pair_i"].size else np.zeros(1, dtype=np.int64)
    w = _win(window)
    lib().or_blend(C.c_int(width), C.c_int(height), _p(bgv), _p(pairs["tile_start"]), _p(pair_i),
                   _p(proj["f32"]), _p(proj["f64"]), _p(img), _p(ncon), _p(tfin), _p(w) if w is not None else None)
    return {"image": img, "n_contrib": ncon, "T_final": tfin}


def blend_backward(proj: dict, pairs: dict, width: int, height: int, dL_dimg: np.ndarray,
                   bg=(0.0, 0.0, 0.0), window=None) -> np.ndarray:
    g = np.zeros((proj["n"], 9), dtype=np.float64)
    bgv = np.asarray(bg, dtype=np.float64)
    dL = np.ascontiguousarray(dL_dimg, dtype=np.float64)
    pair_i = pairs["pair_i"] if pairs["pair_i"].size else np.zeros(1, dtype=np.int64)
    w = _win(window)
    lib().or_blend_backward(C.c_int(width), C.c_int(height), _p(bgv), _p(pairs["tile_start"]), _p(pair_i),
                            _p(proj["f32"]), _p(proj["f64"]), _p(dL), C.c_int64(proj["n"]), _p(g),
                            _p(w) if w is not None else None)
    return g


def project_backward(scene: dict, sel: np.ndarray, cam, proj: dict, g2d: np.ndarray) -> np.ndarray:
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    n = sel.shape[0]
    out = np.zeros((n, scene["stride"]), dtype=np.float64)
    camv = pack_camera(cam)
    lib().or_project_backward(C.c_int64(n), _p(sel), C.c_int(scene["stride"]), C.c_int(scene["degree"]),
                              _p(scene["row_rec"]), _p(camv), _p(proj["vis"]),
                              _p(np.ascontiguousarray(g2d, dtype=np.float64)), _p(out))
    return out


def sh_eval(degree: int, v: np.ndarray):
    v = np.ascontiguousarray(v, dtype=np.float64)
    K = (degree + 1) ** 2 - 1
    Y = np.zeros(max(K, 1))
    dY = np.zeros(max(3 * K, 1))
    lib().or_sh_eval(C.c_int(degree), _p(v), _p(Y), _p(dY))
    return Y[:K], dY[: 3 * K].reshape(K, 3)


def render(scene: dict, cam, bg=(0.0, 0.0, 0.0), cull: bool = True, sel: np.ndarray | None = None,
           window=None) -> dict:
    """Full forward: select -> project -> sort -> blend (blend limited to `window` if given)."""
    stats = None
    if sel is None:
        sel, stats = select(scene, cam, cull)
    proj = project(scene, sel, cam)
    pairs = sort_pairs(proj, cam.width, cam.height)
    out = blend(proj, pairs, cam.width, cam.height, bg, window)
    out.update({"sel": sel, "proj": proj, "pairs": pairs, "select_stats": stats})
    return out


def adam_sparse(params: np.ndarray, m: np.ndarray, v: np.ndarray, t: np.ndarray, rows, grads: np.ndarray,
                lr, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15, used: int | None = None) -> None:
    """Sparse Adam step in place (float64 params/m/v of shape n x stride, uint32 t):
    only `rows` move, each with its own step count; lr is per column."""
    assert params.dtype == m.dtype == v.dtype == np.float64 and t.dtype == np.uint32
    stride = params.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    g = np.ascontiguousarray(grads, dtype=np.float64).reshape(len(rows), -1)
    if g.shape[1] != stride:
        g = np.ascontiguousarray(np.pad(g, ((0, 0), (0, stride - g.shape[1]))))
    lrv = np.ascontiguousarray(np.broadcast_to(np.asarray(lr, dtype=np.float64), (stride,)))
    lib().or_adam_sparse(C.c_int64(len(rows)), _p(rows), _p(g), C.c_int(stride), C.c_int(used or stride), _p(lrv),
                         C.c_double(b1), C.c_double(b2), C.c_double(eps), _p(params), _p(m), _p(v), _p(t))


def screen_grad_max(n_nodes: int, views) -> np.ndarray:
    """Per node, the largest norm of the screen-space mean gradient dL/d(u, v) over
    the views (the densification criterion); views = [(selected rows, g2d)]."""
    out = np.zeros(n_nodes, dtype=np.float64)
    for sel, g2d in views:
        np.maximum.at(out, np.asarray(sel, dtype=np.int64), np.hypot(g2d[:, 0], g2d[:, 1]))
    return out


def render_backward(scene: dict, cam, fwd: dict, dL_dimg: np.ndarray, bg=(0.0, 0.0, 0.0), window=None) -> dict:
    g2d = blend_backward(fwd["proj"], fwd["pairs"], cam.width, cam.height, dL_dimg, bg, window)
    grec = project_backward(scene, fwd["sel"], cam, fwd["proj"], g2d)
    return {"g2d": g2d, "g_rec": grec}
