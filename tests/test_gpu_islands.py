"""GPU parity of the PK-means GA (Sec. 4.3, Alg. 2) through the C ABI
against the FP64 CPU oracle: the population K-means (labels and pass count
bit-exact, counts in shared and in global memory), one island generation
(bit-exact given the same fitness and labels, FP64 and FP32 fitness), and
whole island solves (FP64 trajectories bit-exact, FP32 consistent)."""
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


def _cfg(B, L, K, prec=1, mode=1, **kw):
    return B.pa_config_default(L, K, prec=prec, mode=mode, M=256.0, rho=10.0 / 500.0 ** -3.8,
                               tau_p=K, **kw)


def _sp(oracle, cfg):
    return oracle.sinr_params(cfg.mode, cfg.tau_p, cfg.M, cfg.rho, cfg.sigma2,
                              objective=cfg.objective)


def _gp(oracle, cfg):
    return oracle.ga_params(cfg.N, cfg.E, cfg.tour, cfg.pc_thresh, cfg.pm_thresh, cfg.seed)


def _grouped(N, L, K, groups, seed):
    """A population of `groups` clusters around random bases (so that K-means
    runs several passes and moves members), shuffled."""
    rng = np.random.default_rng(seed)
    bases = inputs.random_population(groups, L, K, seed=seed + 1)
    pop = bases[rng.integers(0, groups, size=N)].copy()
    for n in range(N):
        for _ in range(int(rng.integers(0, 2 * L))):
            l = rng.integers(L)
            i, j = rng.choice(K, 2, replace=False)
            pop[n, l, i], pop[n, l, j] = pop[n, l, j], pop[n, l, i]
    return pop


@pytest.mark.parametrize("N,L,K,C,structured", [(64, 7, 4, 5, True), (256, 19, 10, 5, True),
                                                (256, 19, 10, 5, False), (120, 7, 8, 8, True),
                                                (33, 7, 4, 2, False), (2048, 19, 10, 5, True),
                                                (512, 61, 32, 5, True), (4096, 7, 4, 64, False)])
def test_island_kmeans_bit_exact(B, oracle, N, L, K, C, structured):
    """Labels and pass counts equal the oracle's; (61, 32) keeps its counts in
    global memory (5 x 1952 x 32 words), the others in shared memory."""
    inst = inputs.instance(L, K, seed=1, dtype=np.float32)
    cfg = _cfg(B, L, K, prec=0, N=N, islands=C, island_iter=60, seed=9)
    pop = _grouped(N, L, K, 2 * C, seed=N) if structured else inputs.random_population(N, L, K, 3)
    ctx = B.pa_create(cfg, inst["beta"])
    try:
        dpop = torch.from_numpy(pop).cuda()
        labels = torch.full((N,), -7, dtype=torch.int32, device="cuda")
        for gen in (0, 3):
            passes = B.pa_island_cluster(ctx, dpop, gen, labels)
            want, wpasses = oracle.pop_kmeans(pop, C, 60, cfg.seed, gen)
            assert passes == wpasses
            assert (labels.cpu().numpy() == want).all()
    finally:
        B.pa_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("E,C", [(2, 5), (0, 3), (5, 4), (1, 16)])
def test_island_step_bit_exact(B, oracle, prec, E, C):
    """One island generation from the same population, fitness and labels
    (fitness with many ties; an empty island; labels from K-means and
    arbitrary ones): children bit-exact."""
    L, K, N = 19, 10, 160
    inst = inputs.instance(L, K, seed=2, dtype=np.float32)
    cfg = _cfg(B, L, K, prec=prec, N=N, E=E, islands=C, seed=11,
               pm_thresh=B.pa_prob_to_thresh(0.3))
    pop = inputs.random_population(N, L, K, seed=4)
    rng = np.random.default_rng(C)
    fit = rng.integers(0, 12, size=N).astype(np.float64) + 0.5  # ties
    fdt = torch.float64 if prec else torch.float32
    ctx = B.pa_create(cfg, inst["beta"])
    try:
        dpop = torch.from_numpy(pop).cuda()
        dfit = torch.from_numpy(fit).to(fdt).cuda()
        km, _ = oracle.pop_kmeans(pop, C, cfg.island_iter, cfg.seed, 0)
        arb = rng.integers(0, C, size=N).astype(np.int32)
        arb[arb == C - 1] = 0  # island C-1 empty
        for labels in (km, arb):
            dlab = torch.from_numpy(labels.astype(np.int32)).cuda()
            nxt = torch.empty_like(dpop)
            for gen in (0, 7):
                B.pa_island_step(ctx, dpop, dfit, dlab, gen, nxt)
                torch.cuda.synchronize()
                want = oracle.island_step(pop, fit, _gp(oracle, cfg), gen, labels, C)
                assert (nxt.cpu().numpy() == want).all()
    finally:
        B.pa_destroy(ctx)


def test_one_island_step_is_the_ga_step(B):
    L, K, N = 7, 6, 64
    inst = inputs.instance(L, K, seed=5, dtype=np.float32)
    cfg = _cfg(B, L, K, prec=0, N=N, islands=2, seed=3)
    pop = torch.from_numpy(inputs.random_population(N, L, K, seed=6)).cuda()
    ctx = B.pa_create(cfg, inst["beta"])
    try:
        fit = torch.empty(N, dtype=torch.float32, device="cuda")
        B.pa_eval_population(ctx, pop, fit)
        zeros = torch.zeros(N, dtype=torch.int32, device="cuda")
        a = torch.empty_like(pop)
        b = torch.empty_like(pop)
        B.pa_island_step(ctx, pop, fit, zeros, 4, a)
        B.pa_ga_step(ctx, pop, fit, 4, b)
        torch.cuda.synchronize()
        assert (a == b).all()
    finally:
        B.pa_destroy(ctx)


@pytest.mark.parametrize("L,K,N,C,R,E,mode", [(7, 4, 32, 3, 3, 2, 1), (19, 10, 128, 5, 3, 2, 1),
                                              (19, 10, 96, 4, 1, 1, 0), (7, 8, 64, 8, 2, 0, 1),
                                              (37, 16, 64, 5, 3, 3, 0)])
def test_island_solve_fp64_trajectory(B, oracle, L, K, N, C, R, E, mode):
    inst = inputs.instance(L, K, seed=L * K)
    cfg = _cfg(B, L, K, prec=1, mode=mode, N=N, E=E, islands=C, recluster=R, seed=13)
    G = 20
    with B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"]) as ctx:
        best, bf = ctx.solve(G)
        pop, fit, g = ctx.get_population()
        labels = B.pa_get_islands(ctx.handle, N)
    ref = oracle.solve_islands(inst["beta"], _sp(oracle, cfg), _gp(oracle, cfg), G, C, R,
                               cfg.island_iter, inst["user_xy_mm"], inst["bs_xy_mm"])
    assert g == G
    assert (pop == ref["pop"]).all() and (fit == ref["fit"]).all()
    assert (best == ref["best"]).all() and bf == ref["best_fit"]
    assert (labels == ref["label"]).all()


@pytest.mark.parametrize("L,K,N,C,R,E", [(19, 10, 1024, 5, 3, 2), (7, 4, 48, 3, 2, 9)])
def test_island_solve_fallback_paths_fp64(B, oracle, L, K, N, C, R, E):
    """The island solve where one launch cannot hold it: N = 1024 (the staged
    population of the re-clustering does not fit beside the solve: K-means
    and list kernels between fused launches per block, the K-means from
    global memory), and E = 9 (island mode takes E <= 8: one generation at a
    time by the evaluation and island-generation kernels) -- FP64
    trajectories bit-exact against the oracle."""
    inst = inputs.instance(L, K, seed=L * K + N)
    cfg = _cfg(B, L, K, prec=1, mode=1, N=N, E=E, islands=C, recluster=R, seed=21)
    G = 7
    with B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"]) as ctx:
        best, bf = ctx.solve(G)
        pop, fit, g = ctx.get_population()
        labels = B.pa_get_islands(ctx.handle, N)
    ref = oracle.solve_islands(inst["beta"], _sp(oracle, cfg), _gp(oracle, cfg), G, C, R,
                               cfg.island_iter, inst["user_xy_mm"], inst["bs_xy_mm"])
    assert g == G
    assert (pop == ref["pop"]).all() and (fit == ref["fit"]).all()
    assert (best == ref["best"]).all() and bf == ref["best_fit"]
    assert (labels == ref["label"]).all()


def test_island_solve_in_pieces_equals_whole(B, oracle):
    """pa_step in pieces (re-clustering keyed by the generation counter)
    gives the same population as one solve."""
    L, K, N, C = 19, 10, 64, 5
    inst = inputs.instance(L, K, seed=3)
    cfg = _cfg(B, L, K, prec=1, N=N, islands=C, seed=2)
    with B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"]) as ctx:
        ctx.kmeans_seed()
        for g in (4, 1, 5, 2):
            ctx.step(g)
        pop, fit, gen = ctx.get_population()
    ref = oracle.solve_islands(inst["beta"], _sp(oracle, cfg), _gp(oracle, cfg), 12, C, 3,
                               cfg.island_iter, inst["user_xy_mm"], inst["bs_xy_mm"])
    assert gen == 12 and (pop == ref["pop"]).all()


@pytest.mark.parametrize("prec,E,R", [(0, 2, 3), (0, 0, 2), (1, 3, 3), (0, 8, 4)])
def test_island_fused_blocks_equal_per_generation_kernels(B, prec, E, R):
    """pa_step runs the generations between re-clusterings as one cluster
    launch (island mode of the fused solve); composing the per-generation
    kernels through the ABI -- pa_island_cluster every R generations,
    pa_eval_population, pa_island_step -- gives the same population and
    labels bit for bit."""
    L, K, N, C, G = 19, 10, 128, 5, 10
    inst = inputs.instance(L, K, seed=12, dtype=np.float32)
    cfg = _cfg(B, L, K, prec=prec, N=N, E=E, islands=C, recluster=R, seed=4)
    with B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"]) as ctx:
        ctx.kmeans_seed()
        pop0, _, _ = ctx.get_population(with_fitness=False)
        ctx.step(G)
        fused, _, gen = ctx.get_population(with_fitness=False)
        labels_fused = B.pa_get_islands(ctx.handle, N)
        cur = torch.from_numpy(pop0).cuda()
        lab = torch.empty(N, dtype=torch.int32, device="cuda")
        for g in range(G):
            if g % R == 0:
                B.pa_island_cluster(ctx.handle, cur, g, lab)
            fit = ctx.eval_population(cur)
            nxt = torch.empty_like(cur)
            B.pa_island_step(ctx.handle, cur, fit, lab, g, nxt)
            cur = nxt
        torch.cuda.synchronize()
    assert gen == G
    assert (cur.cpu().numpy() == fused).all()
    assert (lab.cpu().numpy() == labels_fused).all()


def test_island_solve_fp32(B, oracle):
    L, K, N, C = 19, 10, 256, 5
    inst = inputs.instance(L, K, seed=7, dtype=np.float32)
    cfg = _cfg(B, L, K, prec=0, N=N, islands=C, seed=1)
    with B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"]) as ctx:
        best, bf = ctx.solve(60)
        pop, fit, _ = ctx.get_population()
        labels = B.pa_get_islands(ctx.handle, N)
    sp = _sp(oracle, cfg)
    assert (np.sort(pop, axis=-1) == np.arange(K)).all()
    want = oracle.fitness_batch(inst["beta"], pop, sp)
    assert (np.abs(fit.astype(np.float64) - want) / want).max() <= F32_RTOL
    assert abs(bf - oracle.fitness(inst["beta"], best, sp)) <= F32_RTOL * bf
    assert set(np.unique(labels)) <= set(range(C))


def test_islands_rejected_where_unsupported(B):
    cfg = _cfg(B, 7, 4, prec=0, N=5000, islands=5)
    with pytest.raises(B.PaError) as e:
        B.pa_create(cfg, np.ones((7, 7, 4)))
    assert e.value.status == B.PA_EINVAL
    plain = _cfg(B, 7, 4, prec=0, N=32)
    ctx = B.pa_create(plain, np.ones((7, 7, 4)))
    try:
        pop = torch.zeros((32, 7, 4), dtype=torch.uint8, device="cuda")
        lab = torch.zeros(32, dtype=torch.int32, device="cuda")
        with pytest.raises(B.PaError):
            B.pa_island_cluster(ctx, pop, 0, lab)
    finally:
        B.pa_destroy(ctx)
