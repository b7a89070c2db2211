"""Training view selection: kNN graph, transition probabilities, random injection."""
import numpy as np

from paper_2507_01110_b300 import schedule


def test_knn_graph_is_the_brute_force_nearest_neighbours():
    rng = np.random.default_rng(1)
    p = rng.uniform(-100, 100, (300, 3))
    nbr, dist = schedule.knn_graph(p, 7)
    for i in range(0, 300, 17):
        d = np.linalg.norm(p - p[i], axis=1)
        d[i] = np.inf
        ref = np.argsort(d, kind="stable")[:7]
        assert np.array_equal(nbr[i], ref) and np.allclose(dist[i], d[ref])
    assert not np.any(nbr == np.arange(300)[:, None])          # never its own neighbour


def test_transition_frequencies_follow_inverse_distance_weights():
    """Empirical P(j | i) over many draws against 1 / (w_ij + W), normalised."""
    p = np.array([[0.0, 0, 0], [1.0, 0, 0], [3.0, 0, 0], [7.0, 0, 0], [0.0, 2.0, 0]])
    s = schedule.ViewScheduler(p, k=4, W=0.5, random_every=0, seed=3)
    w = 1.0 / (np.array([1.0, 2.0, 3.0, 7.0]) + 0.5)                # neighbours of view 0 by distance
    assert np.array_equal(s.nbr[0], [1, 4, 2, 3])
    assert np.allclose(s.probabilities(0), w / w.sum())
    counts = np.zeros(5)
    for _ in range(20000):
        s.cur = 0
        counts[s.next()] += 1
    freq = counts[[1, 4, 2, 3]] / counts.sum()
    assert np.allclose(freq, w / w.sum(), atol=0.01)


def test_random_view_every_n_iterations_and_seeded():
    rng = np.random.default_rng(2)
    p = rng.uniform(0, 1000, (500, 3))
    a = schedule.ViewScheduler(p, k=5, random_every=128, seed=9)
    b = schedule.ViewScheduler(p, k=5, random_every=128, seed=9)
    seq = [a.next() for _ in range(600)]
    assert seq == [b.next() for _ in range(600)]                   # reproducible
    nbr = a.nbr
    for t in range(1, 600):
        if t % 128:                                                 # a walk step: a kNN neighbour
            assert seq[t] in nbr[seq[t - 1]]
    # the walk stays local: steps are much shorter than uniform jumps
    steps = [np.linalg.norm(p[seq[t]] - p[seq[t - 1]]) for t in range(1, 600) if t % 128]
    jumps = np.linalg.norm(p[rng.integers(500, size=500)] - p[rng.integers(500, size=500)], axis=1)
    assert np.median(steps) < 0.3 * np.median(jumps)
