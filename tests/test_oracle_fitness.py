"""Pins of the oracle's fitness (paper Sec. 3, Eq. 3-7) against values that do
not come from the oracle: a hand-computed instance, closed forms, brute force
and invariants."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2511_20511_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_2cell_2user.json")


def _gold():
    with open(GOLD) as f:
        return json.load(f)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def test_hand_instance_asymptotic(oracle):
    g = _gold()
    beta = np.array(g["beta"])
    for case in g["cases"]:
        X = np.array(case["X"], dtype=np.uint8)
        fit, sinr, se = oracle.user_sinr_se(beta, X)
        expect_fit = 0.0
        for j in range(2):
            for k in range(2):
                num, den = (Fraction(v) for v in case["asymptotic_sinr_num_den"][j][k])
                s = float(num / den)
                assert _rel(sinr[j, k], s) < 4e-16
                assert _rel(se[j, k], math.log2(1.0 + s)) < 4e-15
                expect_fit += math.log2(1.0 + s)
        assert _rel(fit, expect_fit) < 4e-15
        assert _rel(fit, case["asymptotic_fitness"]) < 4e-15


@pytest.mark.parametrize("M", [64.0, 128.0, 256.0, 512.0])
def test_hand_instance_finite_m(oracle, M):
    g = _gold()
    beta = np.array(g["beta"])
    for case in g["cases"]:
        fm = case["finite_M"]
        sp = oracle.sinr_params(oracle.FINITE_M, fm["tau_p"], M, fm["rho"], fm["sigma2"])
        X = np.array(case["X"], dtype=np.uint8)
        fit, sinr, _ = oracle.user_sinr_se(beta, X, sp)
        expect = 0.0
        for j in range(2):
            for k in range(2):
                a, b, c = (Fraction(v) for v in fm["abc"][j][k])
                s = float(a * Fraction(M) / (b * Fraction(M) + c))
                assert _rel(sinr[j, k], s) < 1e-14
                expect += math.log2(1.0 + s)
        assert _rel(fit, expect) < 1e-14


def test_hand_instance_optimum(oracle):
    g = _gold()
    beta = np.array(g["beta"])
    best, X, n = oracle.exhaustive(beta)
    opt = [c for c in g["cases"] if c.get("is_optimum")][0]
    assert n == 2
    assert best == oracle.fitness(beta, np.array(opt["X"]))
    assert (X == np.array(opt["X"])).all()


def _closed_form_beta(L, K, a, b):
    beta = np.full((L, L, K), b)
    for j in range(L):
        beta[j, j, :] = a
    return beta


@pytest.mark.parametrize("L,K,a,b", [(2, 3, 1.0, 0.25), (7, 4, 3e-7, 2e-9), (19, 10, 0.5, 0.01),
                                     (5, 1, 2.0, 1.0)])
def test_closed_form_uniform_cross_gain(oracle, L, K, a, b):
    """beta = a on the own cell, b elsewhere: every user sees L-1 equal
    co-pilot interferers whatever the assignment, so the sum SE is
    L K log2(1 + a^2 / ((L-1) b^2)) (Eq. 5-6)."""
    beta = _closed_form_beta(L, K, a, b)
    expect = L * K * math.log2(1.0 + a * a / ((L - 1) * b * b))
    for seed in range(3):
        X = inputs.random_population(1, L, K, seed=seed)[0]
        assert _rel(oracle.fitness(beta, X), expect) < 1e-13


def test_closed_form_finite_m(oracle):
    """Same uniform instance in the finite-M mode: S2 = (L-1) b^2,
    S1 = a + (L-1) b, B_j = K (a + (L-1) b) for every user."""
    L, K, a, b, M, rho, s2, tau = 7, 5, 1.0, 0.1, 100.0, 4.0, 2.0, 5
    beta = _closed_form_beta(L, K, a, b)
    S2 = (L - 1) * b * b
    S1 = a + (L - 1) * b
    B = K * (a + (L - 1) * b)
    sinr = M * a * a / (M * S2 + (B + s2 / rho) * (S1 + s2 / (tau * rho)))
    expect = L * K * math.log2(1.0 + sinr)
    sp = oracle.sinr_params(oracle.FINITE_M, tau, M, rho, s2)
    X = inputs.random_population(1, L, K, seed=5)[0]
    assert _rel(oracle.fitness(beta, X, sp), expect) < 1e-13


def test_k1_fixed(oracle):
    """K = 1: one pilot, every assignment is the same (K!^(L-1) = 1)."""
    inst = inputs.instance(7, 1, seed=3)
    X = np.zeros((7, 1), dtype=np.uint8)
    f = oracle.fitness(inst["beta"], X)
    b = inst["beta"][:, :, 0]
    expect = sum(math.log2(1 + b[j, j] ** 2 / sum(b[j, l] ** 2 for l in range(7) if l != j))
                 for j in range(7))
    assert _rel(f, expect) < 1e-14


def test_global_relabel_invariance_bitwise(oracle):
    """Applying one pilot relabelling to every cell leaves the set of users
    sharing each pilot unchanged, so the fitness is bit-identical."""
    inst = inputs.instance(19, 10, seed=1)
    pop = inputs.random_population(8, 19, 10, seed=2)
    rng = np.random.default_rng(0)
    for mode in (oracle.ASYMPTOTIC, oracle.FINITE_M):
        sp = oracle.sinr_params(mode, 10, 256.0, inst["rho"], 1.0)
        for X in pop:
            sigma = rng.permutation(10).astype(np.uint8)
            assert oracle.fitness(inst["beta"], sigma[X], sp) == oracle.fitness(inst["beta"], X, sp)


def test_power_of_two_scaling_bitwise(oracle):
    """Asymptotic SINR is a ratio of squares: beta * 2^s changes nothing."""
    inst = inputs.instance(7, 4, seed=4)
    pop = inputs.random_population(16, 7, 4, seed=1)
    for s in (-40, -3, 5, 60):
        f0 = oracle.fitness_batch(inst["beta"], pop)
        f1 = oracle.fitness_batch(inst["beta"] * 2.0 ** s, pop)
        assert (f0 == f1).all()


def test_cell_relabel_invariance(oracle):
    """Renumbering the cells consistently permutes the terms of Eq. 6."""
    inst = inputs.instance(19, 6, seed=7)
    beta = inst["beta"]
    pop = inputs.random_population(4, 19, 6, seed=3)
    pi = np.random.default_rng(1).permutation(19)
    beta_p = np.empty_like(beta)
    beta_p[np.ix_(pi, pi)] = beta  # beta_p[pi[j], pi[l]] = beta[j, l]
    for X in pop:
        Xp = np.empty_like(X)
        Xp[pi] = X
        assert _rel(oracle.fitness(beta_p, Xp), oracle.fitness(beta, X)) < 1e-13


def test_transposed_beta_is_different(oracle):
    """Guard on the index reading: BS index first.  Swapping the roles of j
    and l must change the value on an asymmetric instance."""
    inst = inputs.instance(7, 3, seed=9)
    X = inputs.random_population(1, 7, 3, seed=9)[0]
    bt = np.ascontiguousarray(inst["beta"].transpose(1, 0, 2))
    assert oracle.fitness(bt, X) != oracle.fitness(inst["beta"], X)


def test_finite_m_limit_is_asymptotic(oracle):
    """Eq. 4: the finite-M SINR tends to the asymptotic one as M grows."""
    inst = inputs.instance(7, 4, seed=2)
    pop = inputs.random_population(8, 7, 4, seed=8)
    fa = oracle.fitness_batch(inst["beta"], pop)
    prev = None
    for M in (1e2, 1e5, 1e8, 1e11, 1e14, 1e17, 1e20):
        sp = oracle.sinr_params(oracle.FINITE_M, 4, M, inst["rho"], 1.0)
        fm = oracle.fitness_batch(inst["beta"], pop, sp)
        err = np.max(np.abs(fm - fa) / fa)
        assert (fm < fa + 1e-12 * fa).all()  # noise and estimation error only cost
        if prev is not None:
            assert err <= prev
        prev = err
    assert prev < 1e-9


def _brute_force_max(oracle, beta, all_rows):
    L, _, K = beta.shape
    perms = [np.array(p, dtype=np.uint8) for p in itertools.permutations(range(K))]
    ident = np.arange(K, dtype=np.uint8)
    best = -math.inf
    count = 0
    rows = [perms if (l > 0 or all_rows) else [ident] for l in range(L)]
    for combo in itertools.product(*rows):
        f = oracle.fitness(beta, np.stack(combo))
        count += 1
        best = max(best, f)
    return best, count


@pytest.mark.parametrize("L,K", [(2, 2), (3, 3), (2, 4), (4, 3), (3, 4)])
def test_exhaustive_matches_brute_force(oracle, L, K):
    """EX-PA (Table 3, K!^(L-1) assignments): the oracle's enumeration visits
    every assignment with row 0 fixed, and fixing row 0 loses nothing."""
    inst = inputs.instance(7, K, seed=L * 10 + K)
    beta = np.ascontiguousarray(inst["beta"][:L, :L, :])
    f_fixed, X, n = oracle.exhaustive(beta)
    assert n == math.factorial(K) ** (L - 1)
    assert oracle.fitness(beta, X) == f_fixed
    bf, cnt = _brute_force_max(oracle, beta, all_rows=False)
    assert cnt == n and bf == f_fixed
    if math.factorial(K) ** L <= 20000:
        f_all, _, n_all = oracle.exhaustive(beta, all_rows=True)
        assert n_all == math.factorial(K) ** L
        assert f_all == f_fixed
