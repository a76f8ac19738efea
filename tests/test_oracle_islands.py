"""Pins of the oracle's PK-means GA (Sec. 4.3, Alg. 2: the population is
partitioned by K-means and every cluster evolves on its own; K-means
re-applied every three generations, Sec. 6.1).

What fixes each piece, independently of the oracle's own code:
  * one island holding the whole population is exactly the plain generation
    and solve of Alg. 1 (pinned elsewhere), bit for bit;
  * the population K-means agrees with scikit-learn's Lloyd iteration on the
    chromosomes' one-hot encodings from the same initial centroids, and its
    result is a fixed point of the definition (every member nearest, by the
    exact squared distance to its cluster's mean, ties to the lower index);
  * the initial centroid draw is uniform over ordered pairs (chi-square);
  * structure of an island generation: per-island elites in the island's
    first slots, parents only from the child's own island;
  * invariants of the whole run (monotone global and per-island best) and
    the exhaustive optimum on tiny instances.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from paper_2511_20511_gb300 import inputs

FULL = 1 << 32


def _onehot(pop):
    N, L, K = pop.shape
    return (pop.reshape(N, L * K)[:, :, None] == np.arange(K)[None, None, :]).reshape(N, -1)


def _chi2_pvalue(counts, expect):
    from scipy import stats

    counts = np.asarray(counts, dtype=np.float64)
    expect = np.asarray(expect, dtype=np.float64)
    return float(stats.chi2.sf(np.sum((counts - expect) ** 2 / expect), df=len(counts) - 1))


def _ga(oracle, N, E=2, tour=3, pc=0.9, pm=0.05, seed=0):
    return oracle.ga_params(N, E, tour, oracle.prob_thresh(pc), oracle.prob_thresh(pm), seed=seed)


@pytest.mark.parametrize("L,K,N,E,mode", [(7, 4, 32, 2, 1), (19, 10, 48, 5, 0), (7, 8, 20, 0, 1)])
def test_one_island_is_the_plain_ga(oracle, L, K, N, E, mode):
    inst = inputs.instance(L, K, seed=L + K)
    sp = oracle.sinr_params(mode, K, 128.0, inst["rho"], 1.0)
    gp = _ga(oracle, N, E=E, seed=7)
    pop = inputs.random_population(N, L, K, seed=1)
    fit = oracle.fitness_batch(inst["beta"], pop, sp)
    zero = np.zeros(N, dtype=np.int32)
    assert (oracle.island_step(pop, fit, gp, 5, zero, 1) == oracle.ga_step(pop, fit, gp, 5)).all()
    G = 12
    a = oracle.solve(inst["beta"], sp, gp, G, inst["user_xy_mm"], inst["bs_xy_mm"])
    b = oracle.solve_islands(inst["beta"], sp, gp, G, 1, 3, 100, inst["user_xy_mm"],
                             inst["bs_xy_mm"])
    assert (a["pop"] == b["pop"]).all() and (a["fit"] == b["fit"]).all()
    assert (a["hist_best"] == b["hist_best"]).all() and a["best_fit"] == b["best_fit"]
    assert (b["label"] == 0).all()


def _grouped_population(rng, sizes, L, K, swaps, shared_rows):
    """Groups of members around base chromosomes that share their first
    shared_rows rows (so groups overlap); member i of group g is its base with
    swaps[g] random transpositions."""
    common = np.array([rng.permutation(K) for _ in range(L)], dtype=np.uint8)
    out, truth = [], []
    for g, (n, s) in enumerate(zip(sizes, swaps)):
        base = common.copy()
        for l in range(shared_rows, L):
            base[l] = rng.permutation(K)
        for _ in range(n):
            X = base.copy()
            for _ in range(s):
                l = rng.integers(L)
                i, j = rng.choice(K, 2, replace=False)
                X[l, i], X[l, j] = X[l, j], X[l, i]
            out.append(X)
            truth.append(g)
    order = rng.permutation(len(out))
    return np.array(out)[order], np.array(truth)[order]


def _exact_nearest(E, lab, C):
    """Per member: the exact scaled squared distances to its final clusters'
    means, and whether the nearest one is unique (no tie)."""
    sizes = np.bincount(lab, minlength=C)
    cnt = np.stack([E[lab == c].sum(axis=0) for c in range(C)])
    tie_free = True
    for n in range(len(E)):
        vals = sorted(Fraction(int(((sizes[c] * E[n] - cnt[c]) ** 2).sum()), int(sizes[c]) ** 2)
                      for c in range(C))
        tie_free &= vals[0] != vals[1]
    return tie_free


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_pop_kmeans_matches_sklearn_lloyd(oracle, seed):
    """Same initial centroids, same Lloyd iteration (scikit-learn centres the
    data first, so exact ties may break either way there: the run is taken at
    the first generation key whose initial centroids fall in distinct groups
    and whose first and last assignments have no tie and no empty cluster)."""
    sk = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(seed)
    C, L, K = 4, 8, 6
    pop, truth = _grouped_population(rng, [20, 12, 9, 5], L, K, swaps=[2, 4, 7, 10],
                                     shared_rows=4)
    E = _onehot(pop).astype(np.int64)
    for gen in range(200):
        lab, passes, init = oracle.pop_kmeans(pop, C, max_iter=100, seed=seed, gen=gen,
                                              with_init=True)
        if len(set(truth[init].tolist())) < C or (np.bincount(lab, minlength=C) == 0).any():
            continue
        d0 = np.sort(((E[:, None, :] - E[init][None]) ** 2).sum(-1), axis=1)
        if (d0[:, 0] == d0[:, 1]).any():  # a tie in the first assignment pass
            continue
        if _exact_nearest(E, lab, C):
            break
    else:
        pytest.fail("no tie-free run")
    assert len(set(init.tolist())) == C
    km = sk.KMeans(n_clusters=C, init=E[init].astype(np.float64), n_init=1, max_iter=100,
                   tol=0.0, algorithm="lloyd").fit(E.astype(np.float64))
    assert (km.labels_ == lab).all()


@pytest.mark.parametrize("N,C,L,K,seed", [(40, 3, 7, 4, 0), (64, 5, 19, 10, 1), (33, 4, 5, 6, 2),
                                          (24, 6, 7, 3, 3)])
def test_pop_kmeans_fixed_point_of_the_definition(oracle, N, C, L, K, seed):
    """Unstructured populations: after convergence every member's label is the
    nearest cluster mean by the exact squared distance sum (m e - cnt)^2 / m^2
    (integers, compared by cross-multiplication), ties to the lower index."""
    pop = inputs.random_population(N, L, K, seed=seed)
    lab, passes = oracle.pop_kmeans(pop, C, max_iter=200, seed=seed, gen=0)
    assert passes < 200
    E = _onehot(pop).astype(np.int64)
    sizes = np.bincount(lab, minlength=C)
    if (sizes == 0).any():
        pytest.skip("an emptied cluster keeps a centroid this check cannot rebuild")
    cnt = np.stack([E[lab == c].sum(axis=0) for c in range(C)])
    for n in range(N):
        d = [int(((sizes[c] * E[n] - cnt[c]) ** 2).sum()) for c in range(C)]
        best = 0
        for c in range(1, C):
            if d[c] * int(sizes[best]) ** 2 < d[best] * int(sizes[c]) ** 2:
                best = c
        assert lab[n] == best, n


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pop_kmeans_first_pass_is_nearest_member_ties_low(oracle, seed):
    """One assignment pass: each initial centroid is one member, so a
    member's squared distance to centroid c is twice the number of users whose
    pilots differ from that member's (Hamming distance).  Short rows make ties
    common; every tie goes to the lower cluster index."""
    N, C, L, K = 60, 6, 3, 3
    pop = inputs.random_population(N, L, K, seed=seed)
    lab, passes, init = oracle.pop_kmeans(pop, C, max_iter=1, seed=seed, gen=2, with_init=True)
    assert passes == 1
    ham = (pop[:, None] != pop[init][None]).reshape(N, C, -1).sum(-1)
    ties = 0
    for n in range(N):
        best = int(np.argmin(ham[n]))  # first minimum: the lower index
        ties += int((ham[n] == ham[n].min()).sum() > 1)
        assert lab[n] == best
    assert ties >= 10


def test_pop_kmeans_initial_centroids_uniform(oracle):
    """C = 2 initial centroids among N = 6 members: every ordered pair of
    distinct members equally likely (draws keyed by the generation)."""
    N, C = 6, 2
    pop = inputs.random_population(N, 3, 4, seed=9)
    counts = np.zeros((N, N))
    for g in range(6000):
        _, _, init = oracle.pop_kmeans(pop, C, max_iter=1, seed=11, gen=g, with_init=True)
        counts[init[0], init[1]] += 1
    assert np.trace(counts) == 0
    off = counts[~np.eye(N, dtype=bool)]
    assert (off > 0).all()
    assert _chi2_pvalue(off, np.full(N * (N - 1), 6000 / (N * (N - 1)))) > 1e-4


def _unique_rows(N, L, K, seed):
    perms = np.array(list(itertools.permutations(range(K))), dtype=np.uint8)
    pick = np.random.default_rng(seed).choice(len(perms), N * L, replace=False)
    return perms[pick].reshape(N, L, K)


@pytest.mark.parametrize("E", [0, 1, 3])
def test_island_step_structure(oracle, E):
    """Always crossover, no mutation, rows unique across the population: the
    child's row 0 names parent a and its row L-1 parent b; both come from the
    child's island.  Island c's min(E, m_c) best members (fitness desc, index
    asc) fill its first slots in that order."""
    N, L, K, C = 40, 6, 6, 4
    pop = _unique_rows(N, L, K, seed=E)
    where = {pop[n, l].tobytes(): n for n in range(N) for l in range(L)}
    rng = np.random.default_rng(E)
    fit = rng.integers(0, 8, size=N).astype(np.float64)  # many ties
    label = rng.integers(0, C, size=N).astype(np.int32)
    label[label == 2] = 1  # an empty island
    gp = oracle.ga_params(N, E, 3, FULL, 0, seed=3)
    for g in range(20):
        nxt = oracle.island_step(pop, fit, gp, g, label, C)
        for c in range(C):
            mem = np.flatnonzero(label == c)
            m = len(mem)
            Ec = min(E, m)
            order = mem[np.lexsort((mem, -fit[mem]))]
            for e in range(Ec):
                assert (nxt[mem[e]] == pop[order[e]]).all()
            for n in mem[Ec:]:
                a = where[nxt[n, 0].tobytes()]
                b = where[nxt[n, L - 1].tobytes()]
                assert label[a] == c and label[b] == c


def test_island_solve_invariants(oracle):
    inst = inputs.instance(19, 10, seed=4)
    sp = oracle.sinr_params(1, 10, 256.0, inst["rho"], 1.0)
    gp = _ga(oracle, 64, E=2, seed=5)
    G, C, R = 24, 5, 3
    r = oracle.solve_islands(inst["beta"], sp, gp, G, C, R, 100, inst["user_xy_mm"],
                             inst["bs_xy_mm"])
    h = r["hist_best"]
    assert (np.diff(h) >= 0).all()
    assert r["best_fit"] == h[-1] == r["fit"].max()
    assert (np.sort(r["pop"], axis=-1) == np.arange(10)).all()
    assert (oracle.fitness_batch(inst["beta"], r["pop"], sp) == r["fit"]).all()
    assert set(np.unique(r["label"])) <= set(range(C))
    # the same run step by step: within an epoch (labels fixed) the best member
    # of every island never gets worse
    a = oracle.solve(inst["beta"], sp, gp, 0, inst["user_xy_mm"], inst["bs_xy_mm"])
    pop = a["pop"]
    for g in range(G):
        fit = oracle.fitness_batch(inst["beta"], pop, sp)
        assert fit.max() == h[g]
        if g % R == 0:
            label, _ = oracle.pop_kmeans(pop, C, 100, gp.seed, g)
        elif g > 0:
            for c in range(C):
                if (label == c).any():
                    assert fit[label == c].max() >= prev_best[c]
        prev_best = {c: fit[label == c].max() for c in range(C) if (label == c).any()}
        pop = oracle.island_step(pop, fit, gp, g, label, C)
    assert (pop == r["pop"]).all()


@pytest.mark.parametrize("L,K,seed", [(3, 3, 0), (3, 4, 1), (4, 3, 2)])
def test_island_ga_reaches_exhaustive_optimum(oracle, L, K, seed):
    inst = inputs.instance(7, K, seed=seed)
    beta = np.ascontiguousarray(inst["beta"][:L, :L, :])
    sp = oracle.sinr_params(0, K, 0.0, 1.0, 1.0)
    gp = _ga(oracle, 32, E=1, pm=0.2, seed=seed)
    r = oracle.solve_islands(beta, sp, gp, 60, 3, 3, 100)
    opt, _, _ = oracle.exhaustive(beta, sp)
    assert r["best_fit"] <= opt
    assert r["best_fit"] == pytest.approx(opt, rel=1e-12)
