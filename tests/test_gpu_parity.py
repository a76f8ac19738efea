"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars: FP64 mode bit-exact (fitness, GA step, K-means, seeding, whole solve
trajectory); FP32 fitness within 1e-5 relative of the FP64 oracle; GA step
and seeding bit-exact given the same fitness vector (integer work)."""
import numpy as np
import pytest

from paper_2511_20511_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_RTOL = 1e-5


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20511_gb300 import binding, build

    build.build()
    binding.lib()
    return binding


def _cfg(B, L, K, prec, mode=0, M=256.0, **kw):
    inst_rho = 10.0 / 500.0 ** -3.8
    return B.pa_config_default(L, K, prec=prec, mode=mode, M=M, rho=inst_rho, tau_p=K, **kw)


def _sp(oracle, cfg):
    return oracle.sinr_params(cfg.mode, cfg.tau_p, cfg.M, cfg.rho, cfg.sigma2)


def _gp(oracle, cfg):
    return oracle.ga_params(cfg.N, cfg.E, cfg.tour, cfg.pc_thresh, cfg.pm_thresh, cfg.seed)


def _eval(B, ctx, pop_np, prec):
    pop = torch.from_numpy(pop_np).cuda()
    fit = torch.empty(pop_np.shape[0], dtype=torch.float64 if prec == B.PA_FP64 else torch.float32,
                      device="cuda")
    B.pa_eval_population(ctx, pop, fit)
    torch.cuda.synchronize()
    return fit.cpu().numpy().astype(np.float64)


# ------------------------------------------------------------------ fitness
@pytest.mark.parametrize("L,K", [(2, 2), (7, 4), (19, 10), (7, 1), (37, 16)])
@pytest.mark.parametrize("mode", [0, 1])
def test_fp64_fitness_bit_exact(B, oracle, L, K, mode):
    inst = inputs.instance(L if L != 2 else 7, K, seed=L * 100 + K)
    beta = np.ascontiguousarray(inst["beta"][:L, :L, :])
    cfg = _cfg(B, L, K, B.PA_FP64, mode)
    ctx = B.pa_create(cfg, beta)
    try:
        for n in (1, 37, 300):
            pop = inputs.random_population(n, L, K, seed=n)
            got = _eval(B, ctx, pop, B.PA_FP64)
            ref = oracle.fitness_batch(beta, pop, _sp(oracle, cfg))
            assert (got == ref).all(), np.max(np.abs(got - ref))
    finally:
        B.pa_destroy(ctx)


@pytest.mark.parametrize("L,K", [(2, 2), (7, 4), (19, 10), (7, 1), (19, 13), (37, 16), (19, 17),
                                 (7, 32), (37, 4), (19, 64), (47, 5), (61, 32), (61, 12), (53, 20)])
@pytest.mark.parametrize("mode", [0, 1])
def test_fp32_fitness_within_tolerance(B, oracle, L, K, mode):
    rings_L = {2: 7, 47: 61, 53: 61}.get(L, L)
    inst = inputs.instance(rings_L, K, seed=L * 7 + K, dtype=np.float32)
    beta = np.ascontiguousarray(inst["beta"][:L, :L, :])
    cfg = _cfg(B, L, K, B.PA_FP32, mode)
    ctx = B.pa_create(cfg, beta)
    try:
        for n in (1, 5, 257, 1031):
            pop = inputs.random_population(n, L, K, seed=3 * n + 1)
            got = _eval(B, ctx, pop, B.PA_FP32)
            ref = oracle.fitness_batch(beta, pop, _sp(oracle, cfg))
            rel = np.abs(got - ref) / np.abs(ref)
            assert rel.max() <= F32_RTOL, rel.max()
    finally:
        B.pa_destroy(ctx)


def test_fp32_large_batch_sampled(B, oracle):
    """2^20 chromosomes on the 19-cell, 10-user instance, as timed by the
    benchmark; 2000 sampled outputs checked against the oracle one by one."""
    L, K, n = 19, 10, 1 << 20
    inst = inputs.instance(L, K, seed=0, dtype=np.float32)
    for mode in (0, 1):
        cfg = _cfg(B, L, K, B.PA_FP32, mode)
        ctx = B.pa_create(cfg, inst["beta"])
        try:
            pop = inputs.random_population_torch(n, L, K, seed=1, device="cuda")
            fit = torch.empty(n, dtype=torch.float32, device="cuda")
            B.pa_eval_population(ctx, pop, fit)
            torch.cuda.synchronize()
            idx = np.sort(np.random.default_rng(0).choice(n, 2000, replace=False))
            idx = np.concatenate([idx, [0, n - 1]])
            sub = pop[torch.from_numpy(idx).cuda()].cpu().numpy()
            ref = oracle.fitness_batch(inst["beta"], sub, _sp(oracle, cfg))
            got = fit.cpu().numpy()[idx].astype(np.float64)
            assert (np.abs(got - ref) / ref).max() <= F32_RTOL
            assert np.isfinite(fit.cpu().numpy()).all()
        finally:
            B.pa_destroy(ctx)


@pytest.mark.parametrize("L,K", [(19, 10), (7, 4), (24, 16), (13, 3), (5, 16), (3, 1)])
def test_fp32_staged_and_direct_decode_agree(B, oracle, L, K):
    """The per-pilot FP32 kernel takes full member tiles into shared memory
    by bulk copies and decodes partial tiles (or a population that is not
    16-byte aligned) straight from global memory: both routes give the same
    bits, for tile counts that leave ragged tails, and match the oracle."""
    rings_L = 7 if L <= 7 else (19 if L <= 19 else 37)
    inst = inputs.instance(rings_L, K, seed=L + 5 * K, dtype=np.float32)
    beta = np.ascontiguousarray(inst["beta"][:L, :L, :])
    for mode in (0, 1):
        cfg = _cfg(B, L, K, B.PA_FP32, mode)
        ctx = B.pa_create(cfg, beta)
        try:
            for n in (1, 23, 24, 25, 97, 4099):
                pop_np = inputs.random_population(n, L, K, seed=n + L)
                aligned = _eval(B, ctx, pop_np, B.PA_FP32)
                raw = torch.zeros(n * L * K + 16, dtype=torch.uint8, device="cuda")
                view = raw[1:1 + n * L * K].view(n, L, K)
                view.copy_(torch.from_numpy(pop_np).cuda())
                fit = torch.empty(n, dtype=torch.float32, device="cuda")
                B.pa_eval_population(ctx, view, fit)
                torch.cuda.synchronize()
                assert (fit.cpu().numpy().astype(np.float64) == aligned).all()
                ref = oracle.fitness_batch(beta, pop_np, _sp(oracle, cfg))
                assert (np.abs(aligned - ref) / np.abs(ref)).max() <= F32_RTOL
        finally:
            B.pa_destroy(ctx)


def test_eval_edge_cases(B, oracle):
    L, K = 7, 4
    inst = inputs.instance(L, K, seed=5)
    for prec in (B.PA_FP32, B.PA_FP64):
        ctx = B.pa_create(_cfg(B, L, K, prec), inst["beta"])
        try:
            empty = torch.empty((0, L, K), dtype=torch.uint8, device="cuda")
            fit = torch.empty(0, dtype=torch.float32, device="cuda")
            B.pa_eval_population(ctx, empty, fit)  # n == 0: no-op
            # host-buffer entry point equals the device one
            pop = inputs.random_population(100, L, K, seed=2)
            dev = _eval(B, ctx, pop, prec)
            host = np.zeros(100, dtype=np.float64 if prec else np.float32)
            B.pa_eval_population_host(ctx, pop, host)
            assert (host.astype(np.float64) == dev).all()
            # rows that are not permutations are caught by validation and
            # evaluate without touching memory out of bounds
            bad = pop.copy()
            bad[3, 2, 1] = 200
            bad[7, 0, :] = 0
            t = torch.from_numpy(bad).cuda()
            assert B.pa_validate_population(ctx, t) == 3
            assert B.pa_validate_population(ctx, torch.from_numpy(pop).cuda()) == -1
            out = _eval(B, ctx, bad, prec)
            keep = np.ones(100, bool)
            keep[[3, 7]] = False
            assert (out[keep] == dev[keep]).all()
        finally:
            B.pa_destroy(ctx)


# ------------------------------------------------------------------ GA step
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("L,K,N,E,tour", [(7, 4, 32, 2, 3), (19, 10, 256, 2, 3), (3, 1, 9, 0, 1),
                                          (37, 16, 130, 5, 4), (2, 64, 1000, 64, 2)])
def test_ga_step_bit_exact(B, oracle, prec, L, K, N, E, tour):
    inst = inputs.instance(7 if L < 7 else L, K, seed=1)
    beta = np.ascontiguousarray(inst["beta"][:L, :L, :])
    cfg = _cfg(B, L, K, prec, N=N, E=E, tour=tour, seed=1234567, pm_thresh=B.pa_prob_to_thresh(0.3))
    ctx = B.pa_create(cfg, beta)
    try:
        pop = inputs.random_population(N, L, K, seed=N)
        fit_np = np.random.default_rng(N).random(N)
        fit_np[N // 3] = fit_np[N // 2] = fit_np.max()  # a tie
        if prec == B.PA_FP32:
            fit_np = fit_np.astype(np.float32)
        fit = torch.from_numpy(fit_np).cuda()
        d_pop = torch.from_numpy(pop).cuda()
        nxt = torch.empty_like(d_pop)
        for gen in (0, 1, 77):
            B.pa_ga_step(ctx, d_pop, fit, gen, nxt)
            torch.cuda.synchronize()
            ref = oracle.ga_step(pop, fit_np.astype(np.float64), _gp(oracle, cfg), gen)
            assert (nxt.cpu().numpy() == ref).all()
    finally:
        B.pa_destroy(ctx)


# ------------------------------------------------------------------ K-means + seeding
@pytest.mark.parametrize("L,K,N,kk", [(7, 4, 32, 4), (19, 10, 256, 10), (37, 16, 128, 16),
                                      (61, 32, 64, 32), (19, 10, 17, 3)])
def test_kmeans_seed_bit_exact(B, oracle, L, K, N, kk):
    inst = inputs.instance(L, K, seed=11)
    # seeding does not depend on the arithmetic mode; the 61-cell instance uses
    # FP64 (its FP32 table exceeds shared memory)
    prec = B.PA_FP64 if L in (7, 61) else B.PA_FP32
    cfg = _cfg(B, L, K, prec, N=N, kmeans_k=kk, seed=99, n_seeded=(N + 1) // 2)
    ctx = B.pa_create(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    try:
        labels = np.zeros((L, K), dtype=np.int32)
        cent = np.zeros((kk, 2))
        B.pa_kmeans_seed(ctx, labels, cent)
        pop = np.zeros((N, L, K), dtype=np.uint8)
        B.pa_get_population(ctx, pop, None)
        fx, fy = oracle.features(inst["user_xy_mm"], inst["bs_xy_mm"])
        lab, cx, cy, _ = oracle.kmeans(fx, fy, kk, 100, 99)
        assert (labels.reshape(-1) == lab).all()
        assert (cent[:, 0] == cx).all() and (cent[:, 1] == cy).all()
        ref = oracle.seed_population(L, K, N, (N + 1) // 2, 99, lab, fx, fy, cx, cy)
        assert (pop == ref).all()
    finally:
        B.pa_destroy(ctx)


def test_random_seed_without_positions(B, oracle):
    L, K, N = 19, 10, 64
    inst = inputs.instance(L, K, seed=3)
    cfg = _cfg(B, L, K, B.PA_FP32, N=N, seed=5)
    ctx = B.pa_create(cfg, inst["beta"])
    try:
        B.pa_kmeans_seed(ctx)
        pop = np.zeros((N, L, K), dtype=np.uint8)
        B.pa_get_population(ctx, pop, None)
        assert (pop == oracle.seed_population(L, K, N, 0, 5)).all()
    finally:
        B.pa_destroy(ctx)


# ------------------------------------------------------------------ whole solve
@pytest.mark.parametrize("L,K,N,G,mode", [(7, 4, 32, 50, 0), (7, 4, 32, 50, 1),
                                          (19, 10, 256, 200, 1)])
def test_fp64_trajectory_bit_exact(B, oracle, L, K, N, G, mode):
    _fp64_trajectory(B, oracle, L, K, N, G, mode)


@pytest.mark.parametrize("E", [0, 1, 5, 8, 12, 31])
def test_fp64_trajectory_elite_counts(B, oracle, E):
    """Every elite path of the fused solve (none; rounds of a warp argmax for
    E <= 8; striped search and merge for larger E) against the oracle."""
    _fp64_trajectory(B, oracle, 7, 4, 48, 30, 1, E=E)


def _fp64_trajectory(B, oracle, L, K, N, G, mode, **kw):
    """FP64 mode reproduces the oracle's whole solve: K-means seeding, every
    generation's fitness, selection, crossover and mutation, bit for bit."""
    inst = inputs.instance(L, K, seed=0, dtype=np.float64 if L == 7 else np.float32)
    cfg = _cfg(B, L, K, B.PA_FP64, mode, M=128.0 if L == 7 else 256.0, N=N, seed=0, **kw)
    ctx = B.pa_create(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    try:
        best = np.zeros((L, K), dtype=np.uint8)
        bf = B.pa_solve(ctx, G, best)
        pop = np.zeros((N, L, K), dtype=np.uint8)
        fit = np.zeros(N)
        g = B.pa_get_population(ctx, pop, fit)
        ref = oracle.solve(inst["beta"], _sp(oracle, cfg), _gp(oracle, cfg), G, inst["user_xy_mm"],
                           inst["bs_xy_mm"])
        assert g == G
        assert (pop == ref["pop"]).all()
        assert (fit == ref["fit"]).all()
        assert (best == ref["best"]).all() and bf == ref["best_fit"]
    finally:
        B.pa_destroy(ctx)


def test_fp32_solve_consistent(B, oracle):
    L, K, N, G = 19, 10, 256, 200
    inst = inputs.instance(L, K, seed=0, dtype=np.float32)
    cfg = _cfg(B, L, K, B.PA_FP32, 1, N=N)
    ctx = B.pa_create(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    try:
        best = np.zeros((L, K), dtype=np.uint8)
        bf = B.pa_solve(ctx, G, best)
        assert (np.sort(best, axis=-1) == np.arange(K)).all()
        ref = oracle.fitness(inst["beta"], best, _sp(oracle, cfg))
        assert abs(bf - ref) / ref <= F32_RTOL
        pop = np.zeros((N, L, K), dtype=np.uint8)
        fit = np.zeros(N, dtype=np.float32)
        B.pa_get_population(ctx, pop, fit)
        assert fit.max() == np.float32(bf)
        # the GA improves on the K-means seed
        seed_ref = oracle.solve(inst["beta"], _sp(oracle, cfg), _gp(oracle, cfg), 0,
                                inst["user_xy_mm"], inst["bs_xy_mm"])
        assert bf > seed_ref["best_fit"]
    finally:
        B.pa_destroy(ctx)


def test_checkpoint_resume_bit_exact(B):
    """The GA state is (population, generation, seed): stopping after G1
    generations and resuming in a fresh context gives the same result as
    running G1 + G2 generations in one go."""
    L, K, N = 7, 4, 32
    inst = inputs.instance(L, K, seed=4)
    cfg = _cfg(B, L, K, B.PA_FP64, N=N, seed=3)
    a = B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    a.kmeans_seed()
    a.step(30)
    full, ffit, g = a.get_population()
    assert g == 30
    b = B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    b.kmeans_seed()
    b.step(12)
    mid, _, _ = b.get_population(with_fitness=False)
    c = B.Context(cfg, inst["beta"])
    c.set_population(mid, 12)
    c.step(18)
    res, rfit, g2 = c.get_population()
    assert g2 == 30 and (res == full).all() and (rfit == ffit).all()
    bad = mid.copy()
    bad[0, 0, 0] = bad[0, 0, 1]
    with pytest.raises(B.PaError):
        c.set_population(bad, 0)
    for x in (a, b, c):
        x.close()


@pytest.mark.parametrize("L,K,N,E,mode", [(19, 10, 256, 2, 1), (7, 4, 32, 2, 0), (37, 16, 130, 5, 1),
                                          (19, 17, 100, 3, 0), (7, 1, 9, 0, 1), (19, 10, 200, 12, 1),
                                          (7, 4, 64, 8, 0)])
def test_fused_generations_equal_per_generation_kernels(B, L, K, N, E, mode):
    """pa_step runs all generations in one cluster launch; the same
    generations driven one kernel pair at a time through pa_eval_population
    and pa_ga_step must give the identical population and fitness (FP32: the
    arithmetic per member is the same in both kernels)."""
    inst = inputs.instance(L, K, seed=21, dtype=np.float32)
    cfg = _cfg(B, L, K, B.PA_FP32, mode, N=N, E=E, seed=77, pm_thresh=B.pa_prob_to_thresh(0.2))
    ctx = B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    try:
        ctx.kmeans_seed()
        start, _, _ = ctx.get_population(with_fitness=False)
        G = 25
        ctx.step(G)
        fused, ffit, g = ctx.get_population()
        assert g == G
        pop = torch.from_numpy(start).cuda()
        fit = torch.empty(N, dtype=torch.float32, device="cuda")
        nxt = torch.empty_like(pop)
        for gen in range(G):
            B.pa_eval_population(ctx.handle, pop, fit)
            B.pa_ga_step(ctx.handle, pop, fit, gen, nxt)
            pop, nxt = nxt, pop
        B.pa_eval_population(ctx.handle, pop, fit)
        torch.cuda.synchronize()
        assert (pop.cpu().numpy() == fused).all()
        assert (fit.cpu().numpy() == ffit).all()
    finally:
        ctx.close()


def test_streamed_table_solve_steps(B, oracle):
    """61 cells x 32 users: the FP32 gain table (476 KB) exceeds shared
    memory, so evaluation streams BS-column tiles and generations run as
    per-generation kernels; the elite never decreases and the final fitness
    agrees with the oracle."""
    L, K, N = 61, 32, 64
    inst = inputs.instance(L, K, seed=5, dtype=np.float32)
    cfg = _cfg(B, L, K, B.PA_FP32, 1, M=512.0, N=N, seed=2)
    ctx = B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    try:
        ctx.kmeans_seed()
        hist = []
        for _ in range(4):
            ctx.step(3)
            pop, fit, _ = ctx.get_population()
            hist.append(fit.max())
        assert all(b >= a for a, b in zip(hist, hist[1:]))
        ref = oracle.fitness_batch(inst["beta"], pop[:16], _sp(oracle, cfg))
        assert (np.abs(fit[:16].astype(np.float64) - ref) / ref).max() <= F32_RTOL
    finally:
        ctx.close()
