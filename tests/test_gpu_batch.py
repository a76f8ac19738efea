"""Batched solves of uneven instances (7, 19 and 37 cells, 4 to 16 users,
populations up to 128): every instance's result in the batch equals its
result solved alone (bit for bit), whatever cluster size the tuner picks;
FP64 instances equal the CPU oracle."""
import numpy as np
import pytest

from paper_2511_20511_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20511_gb300 import binding, build

    build.build()
    binding.lib()
    return binding


def _mixed(B, n, seed0=0):
    """Uneven instances: L in {7, 19, 37}, K in {4, 8, 10, 16}, N up to 128;
    every fourth one (from the second) is a 37-cell instance of 128 members,
    the group that holds most of the batched workload's gathers."""
    rng = np.random.default_rng(seed0)
    out = []
    for i in range(n):
        L = int(rng.choice([7, 19, 37]))
        K = int(rng.choice([4, 8, 10, 16]))
        N = int(rng.choice([32, 48, 64, 128]))
        if i % 4 == 1:
            L, N = 37, 128
        prec = B.PA_FP64 if i % 5 == 0 else B.PA_FP32
        mode = int(rng.integers(0, 2))
        inst = inputs.instance(L, K, seed=seed0 * 1000 + i, dtype=np.float32)
        cfg = B.pa_config_default(L, K, prec=prec, mode=mode, M=256.0, N=N, rho=inst["rho"],
                                  seed=100 + i)
        out.append(dict(cfg=cfg, beta=inst["beta"], user_xy_mm=inst["user_xy_mm"],
                        bs_xy_mm=inst["bs_xy_mm"]))
    return out


def _alone(B, d, G):
    with B.Context(d["cfg"], d["beta"], d["user_xy_mm"], d["bs_xy_mm"]) as ctx:
        best, bf = ctx.solve(G)
        pop, fit, _ = ctx.get_population()
    return best, bf, pop, fit


def test_batch_equals_alone_and_tuning_keeps_results(B, oracle):
    G = 15
    insts = _mixed(B, 24)
    batch = B.Batch(insts)
    try:
        rows, fits = batch.solve(G)
        sizes, group_of = batch.groups()
        assert len(sizes) >= 2
        for i, d in enumerate(insts):
            best, bf, pop, fit = _alone(B, d, G)
            assert (rows[i] == best).all(), i
            assert fits[i] == bf, i
            ctx = batch.context(i)
            cfg = d["cfg"]
            bpop = np.zeros((cfg.N, cfg.L, cfg.K), dtype=np.uint8)
            bfit = np.zeros(cfg.N, dtype=np.float64 if cfg.prec else np.float32)
            B.pa_get_population(ctx, bpop, bfit)
            assert (bpop == pop).all() and (bfit == fit).all()
            if cfg.prec == B.PA_FP64:
                sp = oracle.sinr_params(cfg.mode, cfg.tau_p, cfg.M, cfg.rho, cfg.sigma2)
                gp = oracle.ga_params(cfg.N, cfg.E, cfg.tour, cfg.pc_thresh, cfg.pm_thresh,
                                      cfg.seed)
                ref = oracle.solve(d["beta"], sp, gp, G, d["user_xy_mm"], d["bs_xy_mm"])
                assert (rows[i] == ref["best"]).all() and fits[i] == ref["best_fit"]
        chosen = batch.tune(3)
        assert len(chosen) == len(sizes)
        _, threads, _ = batch.group_shapes()
        assert set(threads.tolist()) <= {256, 1024}
        rows2, fits2 = batch.solve(G)
        rows3, fits3 = batch.solve(G)  # graph replay
        for i in range(len(insts)):
            assert (rows2[i] == rows[i]).all() and (rows3[i] == rows[i]).all()
        assert (fits2 == fits).all() and (fits3 == fits).all()
    finally:
        batch.close()


def test_batch_load_replaces_an_instance(B):
    G = 10
    insts = _mixed(B, 6, seed0=3)
    batch = B.Batch(insts)
    try:
        batch.solve(G)
        cfg = insts[2]["cfg"]
        new = inputs.instance(cfg.L, cfg.K, seed=999, dtype=np.float32)
        batch.load(2, new["beta"], new["user_xy_mm"], new["bs_xy_mm"])
        rows, fits = batch.solve(G)
        d = dict(insts[2], beta=new["beta"], user_xy_mm=new["user_xy_mm"],
                 bs_xy_mm=new["bs_xy_mm"])
        best, bf, _, _ = _alone(B, d, G)
        assert (rows[2] == best).all() and fits[2] == bf
    finally:
        batch.close()


def test_batch_small_ctas_equal_alone(B):
    """Every kernel-variant group forced to 256-thread CTAs (four per SM):
    results still equal the solves alone, bit for bit."""
    G = 8
    insts = _mixed(B, 10, seed0=7)
    batch = B.Batch(insts)
    try:
        rows0, fits0 = batch.solve(G)
        batch.tune(2)
        rows, fits = batch.solve(G)
        for i in range(len(insts)):
            assert (rows[i] == rows0[i]).all() and fits[i] == fits0[i]
        for i, d in enumerate(insts):
            best, bf, _, _ = _alone(B, d, G)
            assert (rows[i] == best).all() and fits[i] == bf
    finally:
        batch.close()
