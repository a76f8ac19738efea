"""Bounded waits: an evaluation whose chromosome copies are announced but
never issued (PA_FLAG_TEST_STALL_COPIES, one-shot) gives up after about a
second per block, returns normally and is reported as PA_ETIMEOUT by the
next synchronous call; the same context then evaluates correctly."""
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


def test_stalled_copies_time_out_and_context_recovers(B, oracle):
    L, K, n = 19, 10, 4096
    inst = inputs.instance(L, K, seed=3, dtype=np.float32)
    cfg = B.pa_config_default(L, K, mode=B.PA_SINR_FINITE_M, M=256.0, rho=inst["rho"])
    cfg.flags = B.PA_FLAG_TEST_STALL_COPIES
    ctx = B.pa_create(cfg, inst["beta"])
    try:
        pop = inputs.random_population(n, L, K, seed=11)
        fit = np.zeros(n, dtype=np.float32)
        with pytest.raises(B.PaError) as e:
            B.pa_eval_population_host(ctx, pop, fit)
        assert e.value.status == B.PA_ETIMEOUT
        # one-shot: the context is usable and the next evaluation is right
        B.pa_eval_population_host(ctx, pop, fit)
        sp = oracle.sinr_params(cfg.mode, cfg.tau_p, cfg.M, cfg.rho, cfg.sigma2)
        ref = oracle.fitness_batch(inst["beta"], pop, sp)
        assert (np.abs(fit.astype(np.float64) - ref) / ref).max() <= 1e-5
    finally:
        B.pa_destroy(ctx)
