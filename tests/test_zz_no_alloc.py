"""The allocation-free evaluation entry point against the regular one.

pa_eval_population_noalloc serves callers that cannot allocate device memory
(a real-time scheduling loop that must not take cudaMalloc's implicit device
synchronisation, a framework that owns all device memory).  It keeps its
instance data in one static device array shared by every call, so this test
calls it twice in a row on different instances and populations and checks
each result against pa_create + pa_eval_population on the same inputs, at
the tolerance of the other parity tests (FP32: 1e-5 relative; FP64:
identical).  The cases cover both FP32 evaluation kernels (K <= 16 and
K > 16) and a caller stream other than the default one.  The file runs last
so that a failure here leaves every other test already run.
"""
import ctypes as C

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


def _regular(B, cfg, beta, pop):
    ctx = B.pa_create(cfg, beta)
    try:
        fit = torch.empty(pop.shape[0], dtype=torch.float64 if cfg.prec else torch.float32,
                          device="cuda")
        B.pa_eval_population(ctx, pop, fit)
        torch.cuda.synchronize()
        return fit.cpu().numpy()
    finally:
        B.pa_destroy(ctx)


def _noalloc(B, cfg, beta, pop, stream=None):
    fit = torch.full((pop.shape[0],), -1.0, dtype=torch.float64 if cfg.prec else torch.float32,
                     device="cuda")
    handle = None
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())  # pop and fit are ready
        handle = C.c_void_p(stream.cuda_stream)
    st = B.lib().pa_eval_population_noalloc(C.byref(cfg),
                                            np.ascontiguousarray(beta).ctypes.data_as(C.c_void_p),
                                            C.c_void_p(pop.data_ptr()), pop.shape[0],
                                            C.c_void_p(fit.data_ptr()), handle)
    assert st == B.PA_OK, B.lib().pa_last_error(None)
    assert B.lib().pa_last_error(None) == b""
    torch.cuda.synchronize()
    return fit.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_regular_two_calls_in_a_row(B, prec):
    # (L, K, mode, n): each call overwrites the array the previous one used;
    # K = 20 takes the second FP32 kernel; the last call runs on a side stream
    cases = [(19, 10, 1, 5000), (7, 4, 0, 777), (7, 20, 1, 1500)]
    side = torch.cuda.Stream()
    results = []
    for L, K, mode, n in cases:
        inst = inputs.instance(L, K, seed=L + prec, dtype=np.float32)
        cfg = B.pa_config_default(L, K, prec=prec, mode=mode, M=256.0, rho=inst["rho"])
        pop = inputs.random_population_torch(n, L, K, seed=n, device="cuda")
        got = _noalloc(B, cfg, inst["beta"], pop, stream=side if K == 20 else None)
        want = _regular(B, cfg, inst["beta"], pop)
        results.append((got, want))
    for got, want in results:
        if prec == 1:
            assert (got == want).all()
        else:
            assert (np.abs(got.astype(np.float64) - want) / np.abs(want)).max() <= 1e-5
    # and the first instance again, after the second one has used the array
    L, K, mode, n = cases[0]
    inst = inputs.instance(L, K, seed=L + prec, dtype=np.float32)
    cfg = B.pa_config_default(L, K, prec=prec, mode=mode, M=256.0, rho=inst["rho"])
    pop = inputs.random_population_torch(n, L, K, seed=n, device="cuda")
    again = _noalloc(B, cfg, inst["beta"], pop)
    assert (again == results[0][0]).all()


def test_noalloc_rejects_instances_beyond_the_array(B):
    L, K = 61, 32  # gains alone need 61*61*32*8 = 952,576 bytes
    cfg = B.pa_config_default(L, K, prec=B.PA_FP64)
    beta = np.ones((L, L, K))
    pop = torch.zeros((1, L, K), dtype=torch.uint8, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = B.lib().pa_eval_population_noalloc(C.byref(cfg), beta.ctypes.data_as(C.c_void_p),
                                            C.c_void_p(pop.data_ptr()), 1,
                                            C.c_void_p(fit.data_ptr()), None)
    assert st == B.PA_EUNSUPPORTED
    assert b"bytes of scratch" in B.lib().pa_last_error(None)
