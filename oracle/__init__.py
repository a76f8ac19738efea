"""ctypes binding of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it.

Every function follows the paper (arXiv 2511.20511) step by step; see the
comments in ``oracle.c`` for the equation each one implements.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

ASYMPTOTIC = 0
FINITE_M = 1
OBJ_SUM_SE = 0
OBJ_MIN_SINR = 1


class SinrParams(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tau_p", C.c_int32), ("M", C.c_double),
                ("rho", C.c_double), ("sigma2", C.c_double), ("objective", C.c_int32),
                ("pad0", C.c_int32)]


class GaParams(C.Structure):
    _fields_ = [("N", C.c_int32), ("E", C.c_int32), ("tour", C.c_int32), ("pad0", C.c_int32),
                ("pc_thresh", C.c_uint64), ("pm_thresh", C.c_uint64), ("seed", C.c_uint64)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


def _p(t):
    return C.POINTER(t)


def _declare(L):
    L.or_philox4x64_10.argtypes = [_p(C.c_uint64), _p(C.c_uint64), _p(C.c_uint64)]
    L.or_draw32.argtypes = [C.c_uint64] * 4 + [C.c_uint32]
    L.or_draw32.restype = C.c_uint32
    L.or_log2_det.argtypes = [C.c_double]
    L.or_log2_det.restype = C.c_double
    L.or_fitness.argtypes = [_p(C.c_double), C.c_int32, C.c_int32, _p(C.c_uint8),
                             _p(SinrParams), _p(C.c_double), _p(C.c_double)]
    L.or_fitness.restype = C.c_double
    L.or_fitness_batch.argtypes = [_p(C.c_double), C.c_int32, C.c_int32, _p(C.c_uint8),
                                   C.c_int64, _p(SinrParams), _p(C.c_double)]
    L.or_ga_step.argtypes = [_p(C.c_uint8), _p(C.c_double), C.c_int32, C.c_int32,
                             _p(GaParams), C.c_int32, _p(C.c_uint8)]
    L.or_features.argtypes = [C.c_int32, C.c_int32, _p(C.c_int32), _p(C.c_int32),
                              _p(C.c_int64), _p(C.c_int64)]
    L.or_kmeans.argtypes = [C.c_int32, _p(C.c_int64), _p(C.c_int64), C.c_int32, C.c_int32,
                            C.c_uint64, _p(C.c_int32), _p(C.c_double), _p(C.c_double)]
    L.or_kmeans.restype = C.c_int32
    L.or_dist2.argtypes = [C.c_int64, C.c_int64, C.c_double, C.c_double]
    L.or_dist2.restype = C.c_double
    L.or_seed_population.argtypes = [C.c_int32, C.c_int32, _p(C.c_int32), _p(C.c_int64),
                                     _p(C.c_int64), _p(C.c_double), _p(C.c_double), C.c_int32,
                                     C.c_int32, C.c_uint64, _p(C.c_uint8)]
    L.or_solve.argtypes = [_p(C.c_double), C.c_int32, C.c_int32, _p(SinrParams), _p(GaParams),
                           _p(C.c_int32), _p(C.c_int32), C.c_int32, C.c_int32, C.c_int32,
                           C.c_int32, _p(C.c_uint8), _p(C.c_double), _p(C.c_uint8),
                           _p(C.c_double), _p(C.c_double)]
    L.or_pop_kmeans.argtypes = [_p(C.c_uint8), C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                C.c_int32, C.c_uint64, C.c_int32, _p(C.c_int32),
                                _p(C.c_int32)]
    L.or_pop_kmeans.restype = C.c_int32
    L.or_island_step.argtypes = [_p(C.c_uint8), _p(C.c_double), C.c_int32, C.c_int32,
                                 _p(GaParams), C.c_int32, _p(C.c_int32), C.c_int32,
                                 _p(C.c_uint8)]
    L.or_solve_islands.argtypes = [_p(C.c_double), C.c_int32, C.c_int32, _p(SinrParams),
                                   _p(GaParams), _p(C.c_int32), _p(C.c_int32), C.c_int32,
                                   C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   C.c_int32, _p(C.c_uint8), _p(C.c_double), _p(C.c_uint8),
                                   _p(C.c_double), _p(C.c_double), _p(C.c_int32)]
    L.or_exhaustive.argtypes = [_p(C.c_double), C.c_int32, C.c_int32, _p(SinrParams),
                                C.c_int32, _p(C.c_uint8), _p(C.c_int64)]
    L.or_exhaustive.restype = C.c_double


def _ptr(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(_p(t))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def sinr_params(mode=ASYMPTOTIC, tau_p=1, M=0.0, rho=1.0, sigma2=1.0, objective=OBJ_SUM_SE):
    return SinrParams(int(mode), int(tau_p), float(M), float(rho), float(sigma2),
                      int(objective), 0)


def ga_params(N, E=2, tour=3, pc_thresh=0, pm_thresh=0, seed=0):
    return GaParams(int(N), int(E), int(tour), 0, int(pc_thresh), int(pm_thresh), int(seed))


def prob_thresh(p):
    """Bernoulli(p) threshold on a 32-bit draw: floor(p * 2^32), in [0, 2^32]."""
    return int(np.floor(float(p) * 4294967296.0))


# ---------------------------------------------------------------- primitives
def philox4x64_10(ctr, key):
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(_ptr(c, C.c_uint64), _ptr(k, C.c_uint64), _ptr(out, C.c_uint64))
    return out


def draw32(seed, slot, gen, tag, d):
    return int(lib().or_draw32(seed, slot, gen, tag, d))


def log2_det(x):
    return float(lib().or_log2_det(float(x)))


# ---------------------------------------------------------------- fitness
def fitness(beta, X, sp=None):
    beta = _f64(beta)
    X = _u8(X)
    L, K = X.shape
    assert beta.shape == (L, L, K)
    sp = sp or sinr_params()
    return float(lib().or_fitness(_ptr(beta, C.c_double), L, K, _ptr(X, C.c_uint8),
                                  C.byref(sp), None, None))


def user_sinr_se(beta, X, sp=None):
    beta = _f64(beta)
    X = _u8(X)
    L, K = X.shape
    sp = sp or sinr_params()
    sinr = np.zeros((L, K))
    se = np.zeros((L, K))
    f = lib().or_fitness(_ptr(beta, C.c_double), L, K, _ptr(X, C.c_uint8), C.byref(sp),
                         _ptr(sinr, C.c_double), _ptr(se, C.c_double))
    return float(f), sinr, se


def fitness_batch(beta, pop, sp=None):
    beta = _f64(beta)
    pop = _u8(pop)
    n, L, K = pop.shape
    sp = sp or sinr_params()
    fit = np.zeros(n)
    lib().or_fitness_batch(_ptr(beta, C.c_double), L, K, _ptr(pop, C.c_uint8), n,
                           C.byref(sp), _ptr(fit, C.c_double))
    return fit


# ---------------------------------------------------------------- GA
def ga_step(pop, fit, gp, gen):
    pop = _u8(pop)
    fit = _f64(fit)
    n, L, K = pop.shape
    assert gp.N == n
    nxt = np.zeros_like(pop)
    lib().or_ga_step(_ptr(pop, C.c_uint8), _ptr(fit, C.c_double), L, K, C.byref(gp),
                     int(gen), _ptr(nxt, C.c_uint8))
    return nxt


def features(user_xy_mm, bs_xy_mm):
    u = _i32(user_xy_mm)
    b = _i32(bs_xy_mm)
    L, K, _ = u.shape
    fx = np.zeros(L * K, dtype=np.int64)
    fy = np.zeros(L * K, dtype=np.int64)
    lib().or_features(L, K, _ptr(u, C.c_int32), _ptr(b, C.c_int32), _ptr(fx, C.c_int64),
                      _ptr(fy, C.c_int64))
    return fx, fy


def kmeans(fx, fy, k, max_iter=100, seed=0):
    fx = _i64(fx)
    fy = _i64(fy)
    U = fx.shape[0]
    label = np.zeros(U, dtype=np.int32)
    cx = np.zeros(k)
    cy = np.zeros(k)
    passes = lib().or_kmeans(U, _ptr(fx, C.c_int64), _ptr(fy, C.c_int64), k, max_iter, seed,
                             _ptr(label, C.c_int32), _ptr(cx, C.c_double), _ptr(cy, C.c_double))
    return label, cx, cy, int(passes)


def dist2(fx, fy, cx, cy):
    return float(lib().or_dist2(int(fx), int(fy), float(cx), float(cy)))


def seed_population(L, K, N, n_seeded, seed, label=None, fx=None, fy=None, cx=None, cy=None):
    pop = np.zeros((N, L, K), dtype=np.uint8)
    if label is None:
        lib().or_seed_population(L, K, None, None, None, None, None, N, 0, seed,
                                 _ptr(pop, C.c_uint8))
    else:
        label = _i32(label)
        fx, fy, cx, cy = _i64(fx), _i64(fy), _f64(cx), _f64(cy)
        lib().or_seed_population(L, K, _ptr(label, C.c_int32), _ptr(fx, C.c_int64),
                                 _ptr(fy, C.c_int64), _ptr(cx, C.c_double),
                                 _ptr(cy, C.c_double), N, n_seeded, seed, _ptr(pop, C.c_uint8))
    return pop


def solve(beta, sp, gp, G, user_xy_mm=None, bs_xy_mm=None, kmeans_k=None, kmeans_max_iter=100,
          n_seeded=None):
    beta = _f64(beta)
    L, _, K = beta.shape
    N = gp.N
    kmeans_k = K if kmeans_k is None else kmeans_k
    n_seeded = (N + 1) // 2 if n_seeded is None else n_seeded
    u = None if user_xy_mm is None else _i32(user_xy_mm)
    b = None if bs_xy_mm is None else _i32(bs_xy_mm)
    pop = np.zeros((N, L, K), dtype=np.uint8)
    fit = np.zeros(N)
    best = np.zeros((L, K), dtype=np.uint8)
    best_fit = C.c_double(0.0)
    hist = np.zeros(G + 1)
    lib().or_solve(_ptr(beta, C.c_double), L, K, C.byref(sp), C.byref(gp), _ptr(u, C.c_int32),
                   _ptr(b, C.c_int32), kmeans_k, kmeans_max_iter, n_seeded, G,
                   _ptr(pop, C.c_uint8), _ptr(fit, C.c_double), _ptr(best, C.c_uint8),
                   C.byref(best_fit), _ptr(hist, C.c_double))
    return dict(pop=pop, fit=fit, best=best, best_fit=best_fit.value, hist_best=hist)


# ---------------------------------------------------------------- islands (Alg. 2)
def pop_kmeans(pop, C_islands, max_iter=100, seed=0, gen=0, with_init=False):
    """K-means of the population's chromosomes into C islands: (labels,
    passes), plus the initial centroid members with with_init."""
    pop = _u8(pop)
    N, L, K = pop.shape
    label = np.zeros(N, dtype=np.int32)
    init = np.zeros(int(C_islands), dtype=np.int32)
    passes = lib().or_pop_kmeans(_ptr(pop, C.c_uint8), N, L, K, int(C_islands), int(max_iter),
                                 int(seed), int(gen), _ptr(label, C.c_int32),
                                 _ptr(init, C.c_int32))
    if with_init:
        return label, int(passes), init
    return label, int(passes)


def island_step(pop, fit, gp, gen, label, C_islands):
    pop = _u8(pop)
    fit = _f64(fit)
    label = _i32(label)
    n, L, K = pop.shape
    assert gp.N == n and label.shape == (n,)
    nxt = np.zeros_like(pop)
    lib().or_island_step(_ptr(pop, C.c_uint8), _ptr(fit, C.c_double), L, K, C.byref(gp),
                         int(gen), _ptr(label, C.c_int32), int(C_islands), _ptr(nxt, C.c_uint8))
    return nxt


def solve_islands(beta, sp, gp, G, C_islands, R=3, iters=100, user_xy_mm=None, bs_xy_mm=None,
                  kmeans_k=None, kmeans_max_iter=100, n_seeded=None):
    beta = _f64(beta)
    L, _, K = beta.shape
    N = gp.N
    kmeans_k = K if kmeans_k is None else kmeans_k
    n_seeded = (N + 1) // 2 if n_seeded is None else n_seeded
    u = None if user_xy_mm is None else _i32(user_xy_mm)
    b = None if bs_xy_mm is None else _i32(bs_xy_mm)
    pop = np.zeros((N, L, K), dtype=np.uint8)
    fit = np.zeros(N)
    best = np.zeros((L, K), dtype=np.uint8)
    best_fit = C.c_double(0.0)
    hist = np.zeros(G + 1)
    label = np.zeros(N, dtype=np.int32)
    lib().or_solve_islands(_ptr(beta, C.c_double), L, K, C.byref(sp), C.byref(gp),
                           _ptr(u, C.c_int32), _ptr(b, C.c_int32), kmeans_k, kmeans_max_iter,
                           n_seeded, G, int(C_islands), int(R), int(iters), _ptr(pop, C.c_uint8),
                           _ptr(fit, C.c_double), _ptr(best, C.c_uint8), C.byref(best_fit),
                           _ptr(hist, C.c_double), _ptr(label, C.c_int32))
    return dict(pop=pop, fit=fit, best=best, best_fit=best_fit.value, hist_best=hist,
                label=label)


def exhaustive(beta, sp=None, all_rows=False):
    beta = _f64(beta)
    L, _, K = beta.shape
    sp = sp or sinr_params()
    best = np.zeros((L, K), dtype=np.uint8)
    n = C.c_int64(0)
    f = lib().or_exhaustive(_ptr(beta, C.c_double), L, K, C.byref(sp), int(bool(all_rows)),
                            _ptr(best, C.c_uint8), C.byref(n))
    return float(f), best, int(n.value)
