"""Continuous-batching server: every request's result equals the same solve
alone (bit for bit) and, in FP64, the CPU oracle's, however requests are
interleaved, ticked and admitted; the device-memory budget bounds the
resident slots, also with two shape classes competing for it; host-side
fault injection: malformed and oversized requests are rejected at submit,
failed admissions complete with an error status while the others finish,
cancelled requests never come back, and no completion is lost when a poll
returns fewer than finished."""
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


def _requests(n, seed0=0):
    rng = np.random.default_rng(seed0)
    out = []
    for i in range(n):
        L = int(rng.choice([7, 19]))
        K = int(rng.choice([8, 16]))
        inst = inputs.instance(L, K, seed=seed0 * 100 + i, dtype=np.float32)
        out.append(dict(id=1000 + i, L=L, K=K, seed=77 + i, inst=inst))
    return out


def _alone(B, base, r, G):
    cfg = B.pa_config_default(r["L"], r["K"])
    for f, _ in B.pa_config._fields_:
        if f not in ("L", "K", "tau_p", "kmeans_k", "seed", "reserved"):
            setattr(cfg, f, getattr(base, f))
    cfg.tau_p = r["K"]
    cfg.kmeans_k = r["K"]
    cfg.seed = r["seed"]
    inst = r["inst"]
    with B.Context(cfg, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"]) as ctx:
        return ctx.solve(G)


def _serve(B, base, reqs, G, tick, budget, per_poll=3):
    srv = B.Server(base, G, tick, budget)
    results = {}
    it = iter(reqs)
    pending = True
    max_slots = 0
    try:
        while pending or len(results) < len(reqs):
            for _ in range(per_poll):
                r = next(it, None)
                if r is None:
                    pending = False
                    break
                inst = r["inst"]
                srv.submit(r["id"], r["L"], r["K"], r["seed"], inst["beta"], inst["user_xy_mm"],
                           inst["bs_xy_mm"])
            done, _, _ = srv.poll()
            for rid, best, fit in done:
                results[rid] = (best.copy(), fit)
            max_slots = max(max_slots, srv.stats()["slots"])
            if not done:
                srv.wait(2000)
        return results, max_slots
    finally:
        srv.close()


def _oracle_solve(oracle, base, r, G):
    sp = oracle.sinr_params(base.mode, r["K"], base.M, base.rho, base.sigma2,
                            objective=base.objective)
    gp = oracle.ga_params(base.N, base.E, base.tour, base.pc_thresh, base.pm_thresh, r["seed"])
    inst = r["inst"]
    return oracle.solve(inst["beta"], sp, gp, G, inst["user_xy_mm"], inst["bs_xy_mm"])


@pytest.mark.parametrize("prec,mode,obj", [(0, 1, 0), (1, 0, 0), (1, 1, 1)])
def test_server_results_equal_alone_and_oracle(B, oracle, prec, mode, obj):
    G, tick = 12, 5
    base = B.pa_config_default(7, 8, prec=prec, mode=mode, M=256.0, N=32,
                               rho=10.0 / 500.0 ** -3.8, objective=obj)
    reqs = _requests(14, seed0=prec + 2 * obj)
    results, _ = _serve(B, base, reqs, G, tick, budget=1 << 32)
    assert len(results) == len(reqs)
    for r in reqs:
        best, fit = results[r["id"]]
        ab, af = _alone(B, base, r, G)
        LK = r["L"] * r["K"]
        assert (best[:LK].reshape(r["L"], r["K"]) == ab).all()
        assert fit == af
        if prec == 1:
            ref = _oracle_solve(oracle, base, r, G)
            assert (best[:LK].reshape(r["L"], r["K"]) == ref["best"]).all()
            assert fit == ref["best_fit"]


def test_server_budget_bounds_slots(B):
    G, tick = 6, 6
    base = B.pa_config_default(7, 8, mode=1, M=256.0, N=32, rho=10.0 / 500.0 ** -3.8)
    reqs = [dict(r, L=7, K=8, inst=inputs.instance(7, 8, seed=i, dtype=np.float32))
            for i, r in enumerate(_requests(10, seed0=5))]
    # bytes one slot of this shape holds, then room for two slots only
    probe = B.Server(base, G, tick, 1 << 40)
    inst = reqs[0]["inst"]
    probe.submit(0, 7, 8, 1, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
    probe.poll()
    one = probe.stats()["used_bytes"]
    probe.close()
    budget = 2 * one + one // 2
    results, max_slots = _serve(B, base, reqs, G, tick, budget, per_poll=5)
    assert len(results) == len(reqs)
    assert 1 <= max_slots <= 2


def _slot_bytes(B, base, L, K, G=4):
    probe = B.Server(base, G, G, 1 << 40)
    try:
        inst = inputs.instance(L, K, seed=0, dtype=np.float32)
        probe.submit(0, L, K, 1, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
        probe.poll()
        return probe.stats()["used_bytes"]
    finally:
        probe.close()


def test_server_two_classes_share_a_tight_budget(B):
    """Two (L, K) classes and room for about 2.5 slots of the larger one: idle
    slots of one class are destroyed when the other needs the memory, every
    request completes, and results still equal the solves alone."""
    G, tick = 8, 4
    base = B.pa_config_default(7, 8, mode=1, M=256.0, N=32, rho=10.0 / 500.0 ** -3.8)
    big = _slot_bytes(B, base, 19, 16)
    small = _slot_bytes(B, base, 7, 8)
    assert big > small
    budget = 2 * big + big // 2
    rng = np.random.default_rng(4)
    reqs = []
    for i in range(16):
        L, K = ((19, 16), (7, 8))[int(rng.integers(0, 2))]
        reqs.append(dict(id=2000 + i, L=L, K=K, seed=300 + i,
                         inst=inputs.instance(L, K, seed=700 + i, dtype=np.float32)))
    srv = B.Server(base, G, tick, budget)
    results = {}
    try:
        for r in reqs:
            srv.submit(r["id"], r["L"], r["K"], r["seed"], r["inst"]["beta"],
                       r["inst"]["user_xy_mm"], r["inst"]["bs_xy_mm"])
        polls = 0
        while len(results) < len(reqs):
            done, _, _ = srv.poll()
            polls += 1
            assert polls < 2000, "server made no progress"
            assert srv.stats()["used_bytes"] <= budget
            for rid, best, fit in done:
                results[rid] = (best, fit)
            if not done:
                srv.wait(2000)
    finally:
        srv.close()
    for r in reqs:
        best, fit = results[r["id"]]
        ab, af = _alone(B, base, r, G)
        LK = r["L"] * r["K"]
        assert (best[:LK].reshape(r["L"], r["K"]) == ab).all() and fit == af


def test_server_rejects_malformed_and_oversized_requests(B):
    G = 6
    base = B.pa_config_default(7, 8, mode=1, M=256.0, N=32, rho=10.0 / 500.0 ** -3.8)
    one = _slot_bytes(B, base, 7, 8)
    srv = B.Server(base, G, G, one + one // 2)  # room for one (7, 8) slot only
    good = _requests(3, seed0=9)
    for r in good:
        r["L"], r["K"] = 7, 8
        r["inst"] = inputs.instance(7, 8, seed=r["id"], dtype=np.float32)
    try:
        inst = good[0]["inst"]
        srv.submit(1, 7, 8, 1, inst["beta"], inst["user_xy_mm"], inst["bs_xy_mm"])
        bad_beta = inst["beta"].copy()
        bad_beta[2, 3, 1] = np.nan
        cases = [(7, 8, bad_beta, B.PA_EINVAL), (7, 8, -inst["beta"], B.PA_EINVAL)]
        for L, K, beta, want in cases:
            with pytest.raises(B.PaError) as e:
                srv.submit(99, L, K, 1, beta, inst["user_xy_mm"], inst["bs_xy_mm"])
            assert e.value.status == want
        for L, K in [(-3, 8), (1, 8), (7, 0), (7, 65), (300, 4)]:
            shape_beta = np.ones((max(L, 1), max(L, 1), max(K, 1)))
            with pytest.raises(B.PaError) as e:
                srv.submit(98, L, K, 1, shape_beta, np.zeros((max(L, 1), max(K, 1), 2)),
                           np.zeros((max(L, 1), 2)))
            assert e.value.status == B.PA_EINVAL
        big = inputs.instance(19, 16, seed=1, dtype=np.float32)
        with pytest.raises(B.PaError) as e:
            srv.submit(97, 19, 16, 1, big["beta"], big["user_xy_mm"], big["bs_xy_mm"])
        assert e.value.status == B.PA_EBUSY
        for r in good[1:]:
            srv.submit(r["id"], 7, 8, r["seed"], r["inst"]["beta"], r["inst"]["user_xy_mm"],
                       r["inst"]["bs_xy_mm"])
        got = {rid: fit for rid, _, fit in srv.run_until_idle()}
        assert set(got) == {1, good[1]["id"], good[2]["id"]}
        assert all(np.isfinite(list(got.values())))
    finally:
        srv.close()


def test_server_failed_admission_completes_with_error(B):
    """Host-side fault injection: two admissions fail as if their slot could
    not be created; those requests come back with PA_ECUDA and NaN fitness,
    the queue keeps moving and the other requests equal their solves alone."""
    G, tick = 6, 3
    base = B.pa_config_default(7, 8, mode=1, M=256.0, N=32, rho=10.0 / 500.0 ** -3.8)
    reqs = _requests(6, seed0=11)
    srv = B.Server(base, G, tick, 1 << 32)
    out = {}
    try:
        srv.inject_admission_failures(2)
        for r in reqs:
            inst = r["inst"]
            srv.submit(r["id"], r["L"], r["K"], r["seed"], inst["beta"], inst["user_xy_mm"],
                       inst["bs_xy_mm"])
        for rid, best, fit, st in srv.run_until_idle(with_status=True):
            out[rid] = (best, fit, st)
    finally:
        srv.close()
    assert len(out) == len(reqs)
    failed = [rid for rid, v in out.items() if v[2] != B.PA_OK]
    assert sorted(failed) == [reqs[0]["id"], reqs[1]["id"]]  # admission order
    for rid in failed:
        assert out[rid][2] == B.PA_ECUDA and np.isnan(out[rid][1])
    for r in reqs[2:]:
        best, fit, _ = out[r["id"]]
        ab, af = _alone(B, base, r, G)
        LK = r["L"] * r["K"]
        assert (best[:LK].reshape(r["L"], r["K"]) == ab).all() and fit == af


def test_server_cancel(B):
    G, tick = 9, 3
    base = B.pa_config_default(7, 8, mode=1, M=256.0, N=32, rho=10.0 / 500.0 ** -3.8)
    reqs = _requests(6, seed0=12)
    srv = B.Server(base, G, tick, 1 << 32)
    out = {}
    try:
        for r in reqs:
            inst = r["inst"]
            srv.submit(r["id"], r["L"], r["K"], r["seed"], inst["beta"], inst["user_xy_mm"],
                       inst["bs_xy_mm"])
        srv.cancel(reqs[0]["id"])          # still queued
        srv.poll()                         # the others are admitted, a tick is in flight
        srv.cancel(reqs[1]["id"])          # running: released once its tick has finished
        with pytest.raises(B.PaError) as e:
            srv.cancel(123456789)
        assert e.value.status == B.PA_EINVAL
        for rid, best, fit in srv.run_until_idle():
            out[rid] = (best, fit)
    finally:
        srv.close()
    assert set(out) == {r["id"] for r in reqs[2:]}
    for r in reqs[2:]:
        best, fit = out[r["id"]]
        ab, af = _alone(B, base, r, G)
        LK = r["L"] * r["K"]
        assert (best[:LK].reshape(r["L"], r["K"]) == ab).all() and fit == af


def test_server_completions_are_not_lost_when_polls_return_fewer(B):
    G = 4
    base = B.pa_config_default(7, 8, mode=1, M=256.0, N=32, rho=10.0 / 500.0 ** -3.8)
    reqs = _requests(7, seed0=13)
    srv = B.Server(base, G, G, 1 << 32)
    ids = []
    try:
        for r in reqs:
            inst = r["inst"]
            srv.submit(r["id"], r["L"], r["K"], r["seed"], inst["beta"], inst["user_xy_mm"],
                       inst["bs_xy_mm"])
        held = False
        for _ in range(5000):
            done, active, pending = srv.poll(max_done=2)
            ids += [d[0] for d in done]
            # completions beyond the two a poll returns stay queued
            held |= srv.stats()["completed"] > len(ids)
            if len(ids) == len(reqs):
                break
            if not done:
                srv.wait(2000)
        assert held
    finally:
        srv.close()
    assert sorted(ids) == sorted(r["id"] for r in reqs)
