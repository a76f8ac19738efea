"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every entry point that include/pa.h declares, and rejects
invalid arguments before any GPU work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2511_20511_gb300 import binding, build

    build.build()
    binding.lib()
    return binding


def _declared():
    src = open(os.path.join(ROOT, "include", "pa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(B):
    names = _declared()
    assert "pa_eval_population" in names and "pa_solve" in names
    lib = C.CDLL(B.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.exported_symbols())


def test_config_defaults(B):
    c = B.pa_config_default(19, 10)
    assert (c.L, c.K, c.tau_p, c.N, c.E, c.tour) == (19, 10, 10, 256, 2, 3)
    assert c.mode == B.PA_SINR_ASYMPTOTIC and c.prec == B.PA_FP32
    assert c.pc_thresh == int(np.floor(0.9 * 2**32))
    assert c.pm_thresh == int(np.floor(0.05 * 2**32))
    assert c.kmeans_k == 10 and c.kmeans_max_iter == 100 and c.n_seeded == 128
    assert c.objective == B.PA_OBJ_SUM_SE and c.islands == 0
    assert c.recluster == 3 and c.island_iter == 100
    assert c.rho == pytest.approx(10.0 / 500.0 ** -3.8)


def test_prob_to_thresh(B):
    assert B.pa_prob_to_thresh(0.0) == 0
    assert B.pa_prob_to_thresh(-1.0) == 0
    assert B.pa_prob_to_thresh(1.0) == 2**32
    assert B.pa_prob_to_thresh(0.5) == 2**31
    assert B.pa_prob_to_thresh(0.9) == 3865470566


def _create_status(B, cfg, beta, u=None, b=None):
    out = C.c_void_p()
    bp = beta.ctypes.data_as(C.c_void_p) if beta is not None else None
    up = u.ctypes.data_as(C.c_void_p) if u is not None else None
    bsp = b.ctypes.data_as(C.c_void_p) if b is not None else None
    return B.lib().pa_create(C.byref(cfg), bp, up, bsp, None, C.byref(out))


@pytest.mark.parametrize("field,value", [("L", 1), ("K", 0), ("K", 65), ("N", 1), ("E", 256),
                                         ("tour", 0), ("kmeans_k", 11), ("kmeans_max_iter", 0),
                                         ("n_seeded", 300), ("flags", 2), ("prec", 7),
                                         ("mode", 3), ("pc_thresh", 2**32 + 1), ("objective", 2),
                                         ("islands", 65), ("islands", -1), ("island_iter", -1),
                                         ("recluster", -2)])
def test_create_rejects_bad_config(B, field, value):
    cfg = B.pa_config_default(19, 10)
    setattr(cfg, field, value)
    L, K = max(cfg.L, 1), max(cfg.K, 1)
    beta = np.ones((L, L, K))
    assert _create_status(B, cfg, beta) == B.PA_EINVAL


def test_create_rejects_bad_beta_and_positions(B):
    cfg = B.pa_config_default(7, 4)
    beta = np.ones((7, 7, 4))
    bad = beta.copy()
    bad[1, 2, 3] = 0.0
    assert _create_status(B, cfg, bad) == B.PA_EINVAL
    bad[1, 2, 3] = np.nan
    assert _create_status(B, cfg, bad) == B.PA_EINVAL
    u = np.zeros((7, 4, 2), dtype=np.int32)
    assert _create_status(B, cfg, beta, u, None) == B.PA_EINVAL  # positions come in pairs
    assert _create_status(B, cfg, None) == B.PA_EINVAL
    fm = B.pa_config_default(7, 4, mode=B.PA_SINR_FINITE_M, M=0.0)
    assert _create_status(B, fm, beta) == B.PA_EINVAL


def test_status_strings_and_create_reason(B):
    for s in range(7):
        assert B.lib().pa_status_str(s)
    cfg = B.pa_config_default(7, 4, E=300)
    assert _create_status(B, cfg, np.ones((7, 7, 4))) == B.PA_EINVAL
    assert b"E must be" in B.lib().pa_last_error(None)
    with pytest.raises(B.PaError, match="E must be"):
        B.pa_create(cfg, np.ones((7, 7, 4)))


def test_null_and_invalid_handles_rejected(B):
    """Every entry point taking a handle rejects NULL (and invalid sizes)
    with PA_EINVAL before touching a GPU; destroy functions ignore NULL."""
    lib = B.lib()
    i32 = C.c_int32(0)
    u64 = C.c_uint64(0)
    assert lib.pa_eval_population(None, None, 1, None) == B.PA_EINVAL
    assert lib.pa_eval_population_host(None, None, 1, None) == B.PA_EINVAL
    assert lib.pa_ga_step(None, None, None, 0, None) == B.PA_EINVAL
    assert lib.pa_kmeans_seed(None, None, None) == B.PA_EINVAL
    assert lib.pa_step(None, 1) == B.PA_EINVAL
    assert lib.pa_solve(None, 1, None, None) == B.PA_EINVAL
    assert lib.pa_get_population(None, None, None, None) == B.PA_EINVAL
    assert lib.pa_set_population(None, None, 0) == B.PA_EINVAL
    assert lib.pa_set_seed(None, 1) == B.PA_EINVAL
    assert lib.pa_set_stream(None, None) == B.PA_EINVAL
    assert lib.pa_solve_cluster_ctas(None, C.byref(i32)) == B.PA_EINVAL
    assert lib.pa_load_instance(None, None, None, None) == B.PA_EINVAL
    lib.pa_destroy(None)
    # batches and servers
    out = C.c_void_p()
    assert lib.pa_batch_create(0, None, None, None, None, None, C.byref(out)) == B.PA_EINVAL
    assert lib.pa_batch_solve(None, 1, None, None) == B.PA_EINVAL
    assert lib.pa_batch_tune(None, 1, None) == B.PA_EINVAL
    assert lib.pa_batch_groups(None, None, None, None, None, None, None) == B.PA_EINVAL
    lib.pa_batch_destroy(None)
    cfg = B.pa_config_default(7, 4)
    assert lib.pa_server_create(C.byref(cfg), 0, 1, 1 << 30, None, C.byref(out)) == B.PA_EINVAL
    assert lib.pa_server_create(C.byref(cfg), 10, 0, 1 << 30, None, C.byref(out)) == B.PA_EINVAL
    assert lib.pa_server_create(C.byref(cfg), 10, 1, 0, None, C.byref(out)) == B.PA_EINVAL
    assert lib.pa_server_submit(None, 0, 7, 4, 0, None, None, None) == B.PA_EINVAL
    assert lib.pa_server_poll(None, 0, None, None, None, 0, None, C.byref(i32), None,
                              None) == B.PA_EINVAL
    assert lib.pa_server_stats(None, C.byref(u64), C.byref(i32), None) == B.PA_EINVAL
    assert lib.pa_server_cancel(None, 1) == B.PA_EINVAL
    assert lib.pa_server_inject_admission_failures(None, 1) == B.PA_EINVAL
    lib.pa_server_destroy(None)
    # islands
    assert lib.pa_island_cluster(None, None, 0, None, None) == B.PA_EINVAL
    assert lib.pa_island_step(None, None, None, None, 0, None) == B.PA_EINVAL
    assert lib.pa_get_islands(None, None) == B.PA_EINVAL
    # a server of islands is refused before any GPU work
    isl = B.pa_config_default(7, 4, islands=3)
    assert lib.pa_server_create(C.byref(isl), 10, 1, 1 << 30, None,
                                C.byref(out)) == B.PA_EUNSUPPORTED


def test_create_rejects_bad_island_configs(B):
    beta = np.ones((7, 7, 4))
    for kw in (dict(N=5000, islands=5), dict(N=32, islands=33), dict(islands=4, recluster=0),
               dict(islands=4, island_iter=0)):
        cfg = B.pa_config_default(7, 4, **kw)
        assert _create_status(B, cfg, beta) == B.PA_EINVAL, kw
