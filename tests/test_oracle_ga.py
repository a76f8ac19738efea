"""Pins of the oracle's GA generation (Alg. 1 selection / crossover / mutation,
elitism of Sec. 1) and of the whole solve: invariants, closed-form selection
probabilities, and exhaustive search on tiny instances."""
import math

import numpy as np
import pytest

from paper_2511_20511_gb300 import inputs

FULL = 1 << 32


def _is_perm_rows(pop):
    K = pop.shape[-1]
    return (np.sort(pop, axis=-1) == np.arange(K)).all()


def _distinct_pop(N, L, K, seed):
    pop = inputs.random_population(N, L, K, seed=seed)
    # make every (chromosome, row) distinguishable: rows are compared whole
    return pop


def test_children_are_permutations_and_elites_copied(oracle):
    L, K, N, E = 7, 6, 40, 3
    pop = inputs.random_population(N, L, K, seed=1)
    fit = np.random.default_rng(0).random(N)
    fit[5] = fit[9] = fit.max() + 1.0  # tie at the top: lower index first
    gp = oracle.ga_params(N, E, 3, oracle.prob_thresh(0.9), oracle.prob_thresh(0.05), seed=11)
    nxt = oracle.ga_step(pop, fit, gp, gen=4)
    assert _is_perm_rows(nxt)
    order = np.lexsort((np.arange(N), -fit))  # fitness desc, index asc
    for e in range(E):
        assert (nxt[e] == pop[order[e]]).all()
    assert (nxt[0] == pop[5]).all() and (nxt[1] == pop[9]).all()


def test_tournament_winner_distribution(oracle):
    """No crossover, no mutation: each child is a copy of the first
    tournament's winner.  With distinct fitness, the winner has rank r
    (0 = best) with probability ((N-r)^t - (N-r-1)^t) / N^t (t draws with
    replacement, best one wins)."""
    L, K, N, t = 3, 5, 24, 3
    pop = inputs.random_population(N, L, K, seed=2)
    flat = {pop[i].tobytes(): i for i in range(N)}
    assert len(flat) == N
    fit = np.linspace(1.0, 2.0, N)[np.random.default_rng(3).permutation(N)]
    rank_of = np.empty(N, dtype=int)
    rank_of[np.argsort(-fit)] = np.arange(N)
    gp = oracle.ga_params(N, 0, t, 0, 0, seed=5)
    counts = np.zeros(N)
    G = 600
    for g in range(G):
        nxt = oracle.ga_step(pop, fit, gp, gen=g)
        for c in nxt:
            counts[rank_of[flat[c.tobytes()]]] += 1
    total = counts.sum()
    assert total == G * N
    r = np.arange(N)
    p = ((N - r) ** t - (N - r - 1) ** t) / N ** t
    expect = p * total
    sd = np.sqrt(total * p * (1 - p))
    assert (np.abs(counts - expect) <= 5 * sd + 1).all()
    chi2 = np.sum((counts - expect) ** 2 / expect)
    assert chi2 < 2.5 * N


def test_crossover_is_one_cut_of_two_winners(oracle):
    """Always crossover, no mutation: child rows [0, c) come from one member,
    rows [c, L) from another, with c uniform on 1..L-1."""
    L, K, N = 8, 5, 30
    pop = inputs.random_population(N, L, K, seed=4)
    fit = np.random.default_rng(1).random(N)
    gp = oracle.ga_params(N, 0, 3, FULL, 0, seed=6)
    cuts = np.zeros(L + 1)
    for g in range(200):
        nxt = oracle.ga_step(pop, fit, gp, gen=g)
        for ch in nxt:
            found = False
            for a in range(N):
                c = 0
                while c < L and (ch[c] == pop[a][c]).all():
                    c += 1
                if c == 0:
                    continue
                tails = [b for b in range(N) if (ch[c:] == pop[b][c:]).all()]
                if tails:
                    found = True
                    break
            assert found
            # the first row where the child leaves parent a is the cut (or a later
            # row when b agrees with a there); count the upper bound c
            cuts[c] += 1
    assert cuts[0] == 0
    # most cuts are observed exactly; all positions 1..L-1 and L (b == a rows) occur
    assert (cuts[1:L] > 0).all()


def test_mutation_rate_per_row(oracle):
    """No crossover: a child row differs from its parent row by exactly one
    transposition with probability p_m (swap of two distinct positions)."""
    L, K, N, pm = 10, 6, 40, 0.3
    pop = inputs.random_population(N, L, K, seed=7)
    fit = np.arange(N, dtype=float)
    gp = oracle.ga_params(N, 0, 1, 0, oracle.prob_thresh(pm), seed=8)
    changed = 0
    rows = 0
    for g in range(100):
        nxt = oracle.ga_step(pop, fit, gp, gen=g)
        assert _is_perm_rows(nxt)
        for ch in nxt:
            # tour = 1: the parent is the single drawn candidate; find it by
            # majority of equal rows
            best = max(range(N), key=lambda a: int((ch == pop[a]).all(axis=1).sum()))
            diff = (ch != pop[best]).sum(axis=1)
            assert set(np.unique(diff)) <= {0, 2}
            changed += int((diff == 2).sum())
            rows += L
    p_hat = changed / rows
    sd = math.sqrt(pm * (1 - pm) / rows)
    assert abs(p_hat - pm) < 5 * sd


def test_ga_step_deterministic_and_keyed(oracle):
    L, K, N = 7, 4, 32
    pop = inputs.random_population(N, L, K, seed=9)
    fit = np.random.default_rng(2).random(N)
    gp = oracle.ga_params(N, 2, 3, oracle.prob_thresh(0.9), oracle.prob_thresh(0.05), seed=0)
    a = oracle.ga_step(pop, fit, gp, gen=3)
    b = oracle.ga_step(pop, fit, gp, gen=3)
    c = oracle.ga_step(pop, fit, gp, gen=4)
    gp2 = oracle.ga_params(N, 2, 3, oracle.prob_thresh(0.9), oracle.prob_thresh(0.05), seed=1)
    d = oracle.ga_step(pop, fit, gp2, gen=3)
    assert (a == b).all()
    assert not (a == c).all()
    assert not (a == d).all()


def _solve_cfg(oracle, inst, N, seed=0):
    L, _, K = inst["beta"].shape
    sp = oracle.sinr_params(oracle.ASYMPTOTIC, K, 128.0, inst["rho"], 1.0)
    gp = oracle.ga_params(N, 2, 3, oracle.prob_thresh(0.9), oracle.prob_thresh(0.05), seed=seed)
    return sp, gp


def test_solve_elite_monotone_and_consistent(oracle):
    inst = inputs.instance(7, 4, seed=0)
    sp, gp = _solve_cfg(oracle, inst, 32)
    r = oracle.solve(inst["beta"], sp, gp, 50, inst["user_xy_mm"], inst["bs_xy_mm"])
    h = r["hist_best"]
    assert (np.diff(h) >= 0).all()
    assert r["best_fit"] == h[-1]
    assert oracle.fitness(inst["beta"], r["best"], sp) == r["best_fit"]
    assert _is_perm_rows(r["pop"])
    assert (oracle.fitness_batch(inst["beta"], r["pop"], sp) == r["fit"]).all()


@pytest.mark.parametrize("L,K,seed", [(3, 3, 0), (3, 4, 1), (4, 3, 2), (2, 4, 3)])
def test_solve_reaches_exhaustive_optimum_on_tiny_instances(oracle, L, K, seed):
    """Quality check against EX-PA: on instances with at most a few thousand
    assignments the GA finds the global optimum (never exceeds it)."""
    inst = inputs.instance(7, K, seed=seed)
    beta = np.ascontiguousarray(inst["beta"][:L, :L, :])
    sp = oracle.sinr_params(oracle.ASYMPTOTIC, K, 0.0, 1.0, 1.0)
    gp = oracle.ga_params(32, 2, 3, oracle.prob_thresh(0.9), oracle.prob_thresh(0.2), seed=seed)
    r = oracle.solve(beta, sp, gp, 60)
    opt, _, _ = oracle.exhaustive(beta, sp)
    assert r["best_fit"] <= opt
    assert r["best_fit"] == pytest.approx(opt, rel=1e-12)


def _chi2_pvalue(counts, expect):
    from scipy import stats

    counts = np.asarray(counts, dtype=np.float64)
    expect = np.asarray(expect, dtype=np.float64)
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    return float(stats.chi2.sf(chi2, df=len(counts) - 1))


def _unique_row_population(N, L, K, seed):
    """A population in which no row occurs twice anywhere (so that a child's
    rows name their parents): N*L distinct permutations drawn without
    replacement."""
    import itertools

    perms = np.array(list(itertools.permutations(range(K))), dtype=np.uint8)
    pick = np.random.default_rng(seed).choice(len(perms), N * L, replace=False)
    return perms[pick].reshape(N, L, K)


def test_crossover_cut_uniform(oracle):
    """Always crossover, no mutation, tournament of one: the cut c is uniform
    on 1..L-1 (Sec. 6.1 single-point crossover, at a row boundary).  The
    child's row 0 names parent a, its row L-1 parent b; with a != b the first
    row taken from b is the cut.  A cut drawn from 0..L-2 or 1..L-2 fails."""
    L, K, N = 8, 6, 30
    pop = _unique_row_population(N, L, K, seed=40)
    where = {pop[n, l].tobytes(): n for n in range(N) for l in range(L)}
    fit = np.random.default_rng(2).random(N)
    gp = oracle.ga_params(N, 0, 1, FULL, 0, seed=12)
    counts = np.zeros(L - 1)
    for g in range(300):
        nxt = oracle.ga_step(pop, fit, gp, gen=g)
        for ch in nxt:
            a = where[ch[0].tobytes()]
            b = where[ch[L - 1].tobytes()]
            if a == b:
                assert (ch == pop[a]).all()
                continue
            c = next(l for l in range(L) if (ch[l] == pop[b][l]).all())
            assert (ch[:c] == pop[a][:c]).all() and (ch[c:] == pop[b][c:]).all()
            counts[c - 1] += 1
    assert (counts > 0).all()
    assert _chi2_pvalue(counts, np.full(L - 1, counts.sum() / (L - 1))) > 1e-4


def test_swap_positions_uniform_pairs(oracle):
    """Every row mutated, no crossover, identical members: each child row is
    the base row with one transposition, and the unordered position pair is
    uniform over the K(K-1)/2 pairs (first position uniform on 0..K-1, the
    second uniform on the other K-1).  A second position that can equal the
    first, or never reaches K-1, fails."""
    L, K, N = 10, 5, 64
    base = inputs.random_population(1, L, K, seed=3)[0]
    pop = np.repeat(base[None], N, axis=0)
    fit = np.zeros(N)
    gp = oracle.ga_params(N, 0, 2, 0, FULL, seed=21)
    pairs = {(i, j): t for t, (i, j) in enumerate((i, j) for i in range(K) for j in range(i + 1, K))}
    counts = np.zeros(len(pairs))
    for g in range(50):
        nxt = oracle.ga_step(pop, fit, gp, gen=g)
        for ch in nxt:
            for l in range(L):
                diff = np.flatnonzero(ch[l] != base[l])
                assert len(diff) == 2
                i, j = int(diff[0]), int(diff[1])
                assert ch[l][i] == base[l][j] and ch[l][j] == base[l][i]
                counts[pairs[(i, j)]] += 1
    assert counts.sum() == 50 * N * L
    assert _chi2_pvalue(counts, np.full(len(pairs), counts.sum() / len(pairs))) > 1e-4
