"""Continuous-batching server: every request's result equals the same solve
alone (bit for bit) however requests are interleaved, ticked and admitted;
the device-memory budget bounds the number of resident slots."""
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
        return results, max_slots
    finally:
        srv.close()


@pytest.mark.parametrize("prec,mode", [(0, 1), (1, 0)])
def test_server_results_equal_alone(B, prec, mode):
    G, tick = 12, 5
    base = B.pa_config_default(7, 8, prec=prec, mode=mode, M=256.0, N=32,
                               rho=10.0 / 500.0 ** -3.8)
    reqs = _requests(14, seed0=prec)
    results, _ = _serve(B, base, reqs, G, tick, budget=1 << 32)
    assert len(results) == len(reqs)
    for r in reqs:
        best, fit = results[r["id"]]
        ab, af = _alone(B, base, r, G)
        LK = r["L"] * r["K"]
        assert (best[:LK].reshape(r["L"], r["K"]) == ab).all()
        assert fit == af


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
