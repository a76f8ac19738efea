"""Pins of the oracle's max-min objective (Sec. 2: the GA maximises the
smallest per-user SIR) against values that do not come from the oracle: the
hand-computed 2-cell/2-user instance, closed forms, invariants and the
exhaustive optimum."""
import json
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
    return abs(a - b) / abs(b)


def _sp(oracle, mode=0, tau_p=1, M=0.0, rho=1.0, sigma2=1.0):
    return oracle.sinr_params(mode, tau_p, M, rho, sigma2, objective=oracle.OBJ_MIN_SINR)


def test_hand_instance_min_sinr_asymptotic(oracle):
    """The smallest of the four hand SINRs (exact fractions), e.g. 25/4 for
    X = [[0,1],[0,1]] and 16/9 for X = [[0,1],[1,0]]."""
    g = _gold()
    beta = np.array(g["beta"])
    for case in g["cases"]:
        X = np.array(case["X"], dtype=np.uint8)
        want = min(Fraction(n) / Fraction(d) for row in case["asymptotic_sinr_num_den"]
                   for n, d in row)
        assert _rel(oracle.fitness(beta, X, _sp(oracle)), float(want)) < 4e-16
    assert _rel(oracle.fitness(beta, np.array([[0, 1], [0, 1]], np.uint8), _sp(oracle)),
                25 / 4) < 4e-16
    assert _rel(oracle.fitness(beta, np.array([[0, 1], [1, 0]], np.uint8), _sp(oracle)),
                16 / 9) < 4e-16


@pytest.mark.parametrize("M", [64.0, 256.0])
def test_hand_instance_min_sinr_finite_m(oracle, M):
    g = _gold()
    beta = np.array(g["beta"])
    for case in g["cases"]:
        fm = case["finite_M"]
        X = np.array(case["X"], dtype=np.uint8)
        want = min(Fraction(a) * Fraction(M) / (Fraction(b) * Fraction(M) + Fraction(c))
                   for row in fm["abc"] for a, b, c in row)
        got = oracle.fitness(beta, X, _sp(oracle, 1, fm["tau_p"], M, fm["rho"], fm["sigma2"]))
        assert abs(got - float(want)) <= 1e-14 * float(want)


def test_hand_instance_max_min_optimum_differs_from_sum_se(oracle):
    """Max-min prefers [[0,1],[0,1]] (min SINR 25/4) where the sum SE of Eq. 7
    prefers [[0,1],[1,0]] (min SINR 16/9): the objectives disagree here."""
    beta = np.array(_gold()["beta"])
    best, X, n = oracle.exhaustive(beta, _sp(oracle))
    assert n == 2 and _rel(best, 6.25) < 4e-16
    assert (X == np.array([[0, 1], [0, 1]])).all()
    _, Xs, _ = oracle.exhaustive(beta)
    assert (Xs == np.array([[0, 1], [1, 0]])).all()


def test_closed_form_uniform_cross_gains(oracle):
    """Own gains a_k, every cross gain b: user k of every cell has SINR
    a_k^2 / ((L-1) b^2) whatever the assignment, so the objective is
    min_k a_k^2 / ((L-1) b^2) for every chromosome."""
    L, K, b = 5, 4, 0.01
    a = np.array([0.9, 0.3, 0.6, 0.45])
    beta = np.full((L, L, K), b)
    for j in range(L):
        beta[j, j, :] = a
    want = min(float(Fraction(x) ** 2 / ((L - 1) * Fraction(b) ** 2)) for x in a)
    for X in inputs.random_population(6, L, K, seed=3):
        got = oracle.fitness(beta, X, _sp(oracle))
        assert abs(got - want) <= 4e-16 * want


def test_min_sinr_is_min_of_the_per_user_sinrs(oracle):
    inst = inputs.instance(7, 4, seed=2)
    sp = _sp(oracle, 1, 4, 128.0, inst["rho"], 1.0)
    for X in inputs.random_population(8, 7, 4, seed=4):
        f, sinr, _ = oracle.user_sinr_se(inst["beta"], X, sp)
        assert f == sinr.min()


def test_invariances(oracle):
    """Global pilot relabelling and beta * 2^s (asymptotic) leave the objective
    bit-identical; a different assignment generally changes it."""
    inst = inputs.instance(19, 10, seed=5)
    beta = inst["beta"]
    sp = _sp(oracle)
    pop = inputs.random_population(10, 19, 10, seed=6)
    perm = np.random.default_rng(0).permutation(10).astype(np.uint8)
    vals = set()
    for X in pop:
        f = oracle.fitness(beta, X, sp)
        assert oracle.fitness(beta, perm[X], sp) == f
        assert oracle.fitness(beta * 2.0 ** 40, X, sp) == f
        vals.add(f)
    assert len(vals) > 1


def test_ga_reaches_max_min_optimum_on_tiny_instances(oracle):
    for L, K, seed in [(3, 3, 0), (3, 4, 1), (4, 3, 2)]:
        inst = inputs.instance(7, K, seed=seed)
        beta = np.ascontiguousarray(inst["beta"][:L, :L, :])
        sp = _sp(oracle)
        gp = oracle.ga_params(32, 2, 3, oracle.prob_thresh(0.9), oracle.prob_thresh(0.2),
                              seed=seed)
        r = oracle.solve(beta, sp, gp, 60)
        opt, _, _ = oracle.exhaustive(beta, sp)
        assert r["best_fit"] == opt
        assert (np.diff(r["hist_best"]) >= 0).all()
