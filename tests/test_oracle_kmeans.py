"""Pins of the oracle's K-means (Alg. 1 "Apply K-means clustering") against
scikit-learn's Lloyd iteration, and of the population seeding rule."""
import numpy as np
import pytest

from paper_2511_20511_gb300 import inputs


def test_features_relative_to_own_bs(oracle):
    inst = inputs.instance(7, 4, seed=1)
    fx, fy = oracle.features(inst["user_xy_mm"], inst["bs_xy_mm"])
    u = inst["user_xy_mm"].astype(np.int64)
    b = inst["bs_xy_mm"].astype(np.int64)
    assert (fx.reshape(7, 4) == u[:, :, 0] - b[:, None, 0]).all()
    assert (fy.reshape(7, 4) == u[:, :, 1] - b[:, None, 1]).all()


def _blobs(seed, k, per, spread=2000, sep=100000):
    rng = np.random.default_rng(seed)
    centres = rng.integers(-sep * 3, sep * 3, size=(k, 2))
    pts = np.concatenate([c + rng.integers(-spread, spread, size=(per, 2)) for c in centres])
    return pts[:, 0].astype(np.int64), pts[:, 1].astype(np.int64)


@pytest.mark.parametrize("seed,k", [(0, 4), (1, 10), (4, 16), (6, 16)])
def test_kmeans_matches_sklearn_lloyd(oracle, seed, k):
    """Same initial centroids, same Lloyd iteration.  Only runs where no
    cluster empties: scikit-learn relocates an empty cluster, while the
    reading used here keeps its centroid (checked separately below)."""
    sk = pytest.importorskip("sklearn.cluster")
    fx, fy = _blobs(seed, k, 30)
    # one assignment pass leaves the initial centroids untouched
    _, cx0, cy0, passes = oracle.kmeans(fx, fy, k, max_iter=1, seed=seed)
    assert passes == 1
    lab, cx, cy, passes = oracle.kmeans(fx, fy, k, max_iter=100, seed=seed)
    assert (np.bincount(lab, minlength=k) > 0).all()
    X = np.stack([fx, fy], axis=1).astype(np.float64)
    km = sk.KMeans(n_clusters=k, init=np.stack([cx0, cy0], axis=1), n_init=1, max_iter=100,
                   tol=0.0, algorithm="lloyd").fit(X)
    assert (km.labels_ == lab).all()
    assert np.allclose(km.cluster_centers_, np.stack([cx, cy], axis=1), rtol=0, atol=1e-6)


def test_kmeans_fixed_point_properties(oracle):
    inst = inputs.instance(19, 10, seed=0)
    fx, fy = oracle.features(inst["user_xy_mm"], inst["bs_xy_mm"])
    lab, cx, cy, passes = oracle.kmeans(fx, fy, 10, max_iter=100, seed=0)
    assert 1 <= passes <= 100
    d = (fx[:, None] - cx[None, :]) ** 2 + (fy[:, None] - cy[None, :]) ** 2
    assert (lab == np.argmin(d, axis=1)).all()
    if passes < 100:  # converged: centroids are the means of their members
        for c in range(10):
            m = lab == c
            if m.any():
                assert cx[c] == pytest.approx(fx[m].mean(), abs=1e-6)
                assert cy[c] == pytest.approx(fy[m].mean(), abs=1e-6)


def test_kmeans_init_distinct_points(oracle):
    fx = np.arange(50, dtype=np.int64) * 1000
    fy = np.zeros(50, dtype=np.int64)
    for seed in range(20):
        _, cx0, _, _ = oracle.kmeans(fx, fy, 12, max_iter=1, seed=seed)
        assert len(set(cx0.tolist())) == 12


def test_seed_rule_hand_case(oracle):
    """One cell, K = 3.  Labels (0, 0, 2); user 1 is closer to centroid 0
    than user 0, so user 1 keeps pilot 0, user 0 is deferred to the lowest
    free pilot (1), user 2 keeps pilot 2."""
    L, K = 1, 3
    label = np.array([0, 0, 2], dtype=np.int32)
    fx = np.array([10, 1, 50], dtype=np.int64)
    fy = np.zeros(3, dtype=np.int64)
    cx = np.array([0.0, 100.0, 50.0])
    cy = np.zeros(3)
    pop = oracle.seed_population(L, K, 1, 1, 0, label, fx, fy, cx, cy)
    assert pop[0, 0].tolist() == [1, 0, 2]


def test_seed_population_structure(oracle):
    inst = inputs.instance(19, 10, seed=2)
    fx, fy = oracle.features(inst["user_xy_mm"], inst["bs_xy_mm"])
    lab, cx, cy, _ = oracle.kmeans(fx, fy, 10, seed=2)
    N, ns = 64, 32
    pop = oracle.seed_population(19, 10, N, ns, 2, lab, fx, fy, cx, cy)
    assert (np.sort(pop, axis=-1) == np.arange(10)).all()
    astar = pop[0]
    for n in range(1, ns):
        diff = (pop[n] != astar).sum(axis=1)
        assert set(np.unique(diff)) <= {0, 2}
    # where a cell's labels already form a permutation, A* is exactly the labels
    L3 = lab.reshape(19, 10)
    for l in range(19):
        if sorted(L3[l].tolist()) == list(range(10)):
            assert (astar[l] == L3[l]).all()
    # random part: rows spread over many permutations
    rnd = {pop[n, l].tobytes() for n in range(ns, N) for l in range(19)}
    assert len(rnd) > 0.95 * (N - ns) * 19
    # without positions every member is random
    pop0 = oracle.seed_population(19, 10, N, 0, 2)
    assert (np.sort(pop0, axis=-1) == np.arange(10)).all()
    assert (pop0[ns:] == pop[ns:]).all()  # same random stream per slot


def test_kmeans_empty_cluster_keeps_centroid(oracle):
    """Blob data where a cluster empties during the iteration (two initial
    centroids in one blob): its centroid stays where it was and every point
    still goes to its nearest centroid."""
    fx, fy = _blobs(2, 16, 30)
    lab, cx, cy, _ = oracle.kmeans(fx, fy, 16, max_iter=100, seed=2)
    empty = np.flatnonzero(np.bincount(lab, minlength=16) == 0)
    assert len(empty) == 1
    _, cx0, cy0, _ = oracle.kmeans(fx, fy, 16, max_iter=1, seed=2)
    d = (fx[:, None] - cx[None, :]) ** 2 + (fy[:, None] - cy[None, :]) ** 2
    assert (lab == np.argmin(d, axis=1)).all()
    # an emptied cluster's centroid is one of the means it held earlier, never NaN
    assert np.isfinite(cx[empty]).all() and np.isfinite(cy[empty]).all()


def _chi2_pvalue(counts, expect):
    from scipy import stats

    counts = np.asarray(counts, dtype=np.float64)
    expect = np.asarray(expect, dtype=np.float64)
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    return float(stats.chi2.sf(chi2, df=len(counts) - 1))


@pytest.mark.parametrize("K", [3, 4])
def test_random_row_uniform_over_all_permutations(oracle, K):
    """Random rows (Fisher-Yates from the top, j uniform on 0..i): every one
    of the K! permutations equally likely.  Sattolo's variant (j < i) makes
    only cyclic permutations and a shortened loop misses permutations, so
    both fail here."""
    import itertools

    L, N = 10, 2400  # 24,000 rows
    pop = oracle.seed_population(L, K, N, 0, seed=123)
    perms = {p: i for i, p in enumerate(itertools.permutations(range(K)))}
    counts = np.zeros(len(perms))
    for row in pop.reshape(-1, K):
        counts[perms[tuple(int(v) for v in row)]] += 1
    assert counts.sum() == N * L
    assert (counts > 0).all()
    assert _chi2_pvalue(counts, np.full(len(perms), N * L / len(perms))) > 1e-4


def test_kmeans_initial_centroids_uniform_ordered_pairs(oracle):
    """The partial Fisher-Yates draw of k = 2 initial centroids among U = 6
    points: every ordered pair of distinct points has probability 1/30.  A
    draw that never reaches the last index, or allows a repeat, fails."""
    U, k = 6, 2
    fx = np.arange(U, dtype=np.int64) * 1000
    fy = np.zeros(U, dtype=np.int64)
    counts = np.zeros((U, U))
    seeds = range(6000)
    for seed in seeds:
        # one assignment pass: the returned centroids are the initial ones
        _, cx0, _, _ = oracle.kmeans(fx, fy, k, max_iter=1, seed=seed)
        a, b = int(round(cx0[0] / 1000)), int(round(cx0[1] / 1000))
        counts[a, b] += 1
    assert np.trace(counts) == 0  # distinct points
    off = counts[~np.eye(U, dtype=bool)]
    assert (off > 0).all()
    assert _chi2_pvalue(off, np.full(U * (U - 1), len(seeds) / (U * (U - 1)))) > 1e-4
