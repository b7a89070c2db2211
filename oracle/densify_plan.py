"""Densification planning (Sec. 3 "Densification"; appendix "Respawning,
Densifying, and Pruning Gaussians"), restated on the host as the checker of
the library's device planner (lodgs_densify_plan).  Test infrastructure, like
the rest of this package: only tests/ use it.

It turns per-row statistics into the operations of `Scene.densify`:

* dead leaves: opacity below `min_opacity`, or flagged stale (the pruning
  rule zeroes the opacity of Gaussians that have not contributed for a number
  of iterations, so that the next densification respawns them);
* candidates: leaves whose maximal screen-space gradient reaches
  `grad_threshold` (the selection of hierarchical 3DGS), largest first;
* each dead leaf is respawned under one candidate, in candidate order; the
  remaining candidates spawn two children while the node budget allows.

Edge cases the appendix fixes: when both children of a node are dead leaves
only the right one is respawned (the left one becomes a dead leaf with a new
sibling and is respawned by a later densification); a dead leaf whose sibling
is an internal node hands the whole subtree of that sibling its parent's
place, which `Scene.densify` does by construction.
"""
from __future__ import annotations

import numpy as np


def plan(topology: dict, opacity: np.ndarray, grad_max: np.ndarray, grad_threshold: float,
         min_opacity: float = 0.005, max_nodes: int | None = None, stale: np.ndarray | None = None):
    """Operations for one densification step.

    topology: `Scene.topology()` (left, right in canonical ids; node_of_row).
    opacity, grad_max, stale: per render row (n_nodes).
    Returns (spawn_rows, respawn_pairs): render rows of leaves that get two new
    children, and (target row, dead row) pairs, in the order they are applied.
    """
    left = np.asarray(topology["left"], np.int64)
    right = np.asarray(topology["right"], np.int64)
    nor = np.asarray(topology["node_of_row"], np.int64)
    M = left.shape[0]
    row_of = np.empty(M, np.int64)
    row_of[nor] = np.arange(M)
    opacity = np.asarray(opacity, np.float32)
    grad_max = np.asarray(grad_max, np.float32)
    # per row: leaf flag, parent row, and whether it is a left child
    leaf_n = left < 0
    parent_n = np.full(M, -1, np.int64)
    is_left_n = np.zeros(M, bool)
    internal = np.nonzero(~leaf_n)[0]
    parent_n[left[internal]] = internal
    parent_n[right[internal]] = internal
    is_left_n[left[internal]] = True
    leaf = leaf_n[nor]
    has_parent = parent_n[nor] >= 0
    is_left = is_left_n[nor]

    low = leaf & (opacity < np.float32(min_opacity))
    if stale is not None:
        low |= leaf & np.asarray(stale, bool)
    dead = low & has_parent
    # both children dead: respawn only the right one
    sib_n = np.where(is_left_n, right[np.maximum(parent_n, 0)], left[np.maximum(parent_n, 0)])
    sib_row = row_of[sib_n[nor]]
    dead &= ~(is_left & dead[sib_row])
    dead_rows = np.nonzero(dead)[0]

    # a dead (or transparent) leaf is never split
    cand = leaf & ~low & (grad_max >= np.float32(grad_threshold))
    cand_rows = np.nonzero(cand)[0]
    cand_rows = cand_rows[np.lexsort((cand_rows, -grad_max[cand_rows].astype(np.float64)))]

    n_resp = min(dead_rows.size, cand_rows.size)
    respawn = [(int(cand_rows[i]), int(dead_rows[i])) for i in range(n_resp)]
    rest = cand_rows[n_resp:]
    if max_nodes is not None:
        room = max(0, (int(max_nodes) - M) // 2)
        rest = rest[:room]
    spawn = [int(r) for r in rest]
    return spawn, respawn
