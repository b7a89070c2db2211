"""Training view selection (Sec. 4.4, "View Selection").

Successive training views are drawn near the current one so that the device
cache is reused: a k-nearest-neighbour graph over the training camera
positions (edge weight w_ij = Euclidean distance) is built once, and the next
view j is drawn among the k neighbours of the current view i with probability
proportional to 1 / (w_ij + W); W controls how far the walk explores.  Every
`random_every` iterations a uniformly random view is injected instead, which
keeps the view distribution from drifting.  Host-side logic; the random
numbers come from a seeded numpy generator.
"""
from __future__ import annotations

import numpy as np


def knn_graph(positions: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """(neighbours, distances): for every view its k nearest other views, nearest
    first (ties by index), and their Euclidean distances.  Brute force, in blocks."""
    p = np.asarray(positions, dtype=np.float64)
    n = p.shape[0]
    if not 1 <= k < n:
        raise ValueError("need 1 <= k < number of views")
    nbr = np.empty((n, k), dtype=np.int64)
    dist = np.empty((n, k), dtype=np.float64)
    for s in range(0, n, 1024):
        d = np.sqrt(((p[s:s + 1024, None, :] - p[None, :, :]) ** 2).sum(-1))
        d[np.arange(d.shape[0]), np.arange(s, s + d.shape[0])] = np.inf      # not its own neighbour
        idx = np.argsort(d, axis=1, kind="stable")[:, :k]
        nbr[s:s + d.shape[0]] = idx
        dist[s:s + d.shape[0]] = np.take_along_axis(d, idx, axis=1)
    return nbr, dist


class ViewScheduler:
    """Yields training view indices: a walk on the kNN graph with
    P(j | i) proportional to 1 / (w_ij + W), and a uniform view every
    `random_every` iterations (the first iteration is uniform too)."""

    def __init__(self, positions: np.ndarray, k: int = 10, W: float | None = None, random_every: int = 128,
                 seed: int = 0):
        self.nbr, self.dist = knn_graph(positions, k)
        self.W = float(np.median(self.dist)) if W is None else float(W)
        if not self.W >= 0.0:
            raise ValueError("W must be >= 0")
        self.random_every = int(random_every)
        self.rng = np.random.default_rng(seed)
        self.n = self.nbr.shape[0]
        self.it = 0
        self.cur = -1

    def probabilities(self, i: int) -> np.ndarray:
        """P(j | i) over the k neighbours of view i (in knn_graph order)."""
        w = 1.0 / (self.dist[i] + self.W)
        return w / w.sum()

    def next(self) -> int:
        if self.cur < 0 or (self.random_every > 0 and self.it % self.random_every == 0):
            self.cur = int(self.rng.integers(self.n))
        else:
            self.cur = int(self.nbr[self.cur, self.rng.choice(self.nbr.shape[1], p=self.probabilities(self.cur))])
        self.it += 1
        return self.cur
