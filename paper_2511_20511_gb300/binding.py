"""Thin Python binding of libpa.so (include/pa.h): argument marshalling only.

Every function has the C name and forwards to it; device buffers are torch
CUDA tensors (passed by data_ptr()), host buffers numpy arrays.  Streams are
torch.cuda streams (the raw cudaStream_t is passed).  All computation runs
in the library's CUDA kernels: if libpa.so is missing this module raises --
there is no fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpa.so")

PA_OK, PA_EINVAL, PA_ENOMEM, PA_ECUDA, PA_ETIMEOUT, PA_EUNSUPPORTED, PA_EBUSY = range(7)
PA_FLAG_TEST_STALL_COPIES = 1
PA_FP32, PA_FP64 = 0, 1
PA_SINR_ASYMPTOTIC, PA_SINR_FINITE_M = 0, 1
PA_OBJ_SUM_SE, PA_OBJ_MIN_SINR = 0, 1


class pa_config(C.Structure):
    _fields_ = [("L", C.c_int32), ("K", C.c_int32), ("tau_p", C.c_int32), ("mode", C.c_int32),
                ("M", C.c_double), ("rho", C.c_double), ("sigma2", C.c_double),
                ("prec", C.c_int32), ("N", C.c_int32), ("E", C.c_int32), ("tour", C.c_int32),
                ("pc_thresh", C.c_uint64), ("pm_thresh", C.c_uint64), ("seed", C.c_uint64),
                ("kmeans_k", C.c_int32), ("kmeans_max_iter", C.c_int32),
                ("n_seeded", C.c_int32), ("flags", C.c_int32), ("objective", C.c_int32),
                ("islands", C.c_int32), ("recluster", C.c_int32), ("island_iter", C.c_int32),
                ("reserved", C.c_int64 * 2)]


assert C.sizeof(pa_config) == 128


class PaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


_lib = None

_SIGS = {
    "pa_config_default": (C.c_int, [C.POINTER(pa_config), C.c_int32, C.c_int32]),
    "pa_prob_to_thresh": (C.c_uint64, [C.c_double]),
    "pa_create": (C.c_int, [C.POINTER(pa_config), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(C.c_void_p)]),
    "pa_load_instance": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pa_destroy": (None, [C.c_void_p]),
    "pa_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pa_set_seed": (C.c_int, [C.c_void_p, C.c_uint64]),
    "pa_eval_population": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "pa_eval_population_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "pa_ga_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "pa_kmeans_seed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pa_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "pa_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_double)]),
    "pa_get_population": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "pa_set_population": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "pa_population_device": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "pa_validate_population": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64,
                                         C.POINTER(C.c_int64)]),
    "pa_island_cluster": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                    C.POINTER(C.c_int32)]),
    "pa_island_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                 C.c_void_p]),
    "pa_get_islands": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pa_status_str": (C.c_char_p, [C.c_int]),
    "pa_last_error": (C.c_char_p, [C.c_void_p]),
    "pa_kernel_launches": (C.c_uint64, []),
    "pa_solve_cluster_ctas": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "pa_batch_create": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.POINTER(C.c_void_p)]),
    "pa_batch_destroy": (None, [C.c_void_p]),
    "pa_batch_load": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pa_batch_tune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "pa_batch_groups": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "pa_batch_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "pa_batch_context": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "pa_batch_completion_times": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pa_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "pa_server_create": (C.c_int, [C.POINTER(pa_config), C.c_int32, C.c_int32, C.c_uint64,
                                   C.c_void_p, C.POINTER(C.c_void_p)]),
    "pa_server_destroy": (None, [C.c_void_p]),
    "pa_server_submit": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_uint64,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "pa_server_poll": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_int64, C.c_void_p, C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pa_server_cancel": (C.c_int, [C.c_void_p, C.c_int64]),
    "pa_server_wait": (C.c_int, [C.c_void_p, C.c_int32]),
    "pa_server_inject_admission_failures": (C.c_int, [C.c_void_p, C.c_int32]),
    "pa_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int64)]),
    "pa_server_last_error": (C.c_char_p, [C.c_void_p]),
    "pa_eval_population_noalloc": (C.c_int, [C.POINTER(pa_config), C.c_void_p, C.c_void_p,
                                             C.c_int64, C.c_void_p, C.c_void_p]),
}


def lib():
    """Load libpa.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2511_20511_gb300.build` (no fallback path)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _check(st, ctx=None):
    if st != PA_OK:
        msg = lib().pa_status_str(st).decode()
        detail = lib().pa_last_error(ctx).decode()  # ctx None: this thread's last create error
        if detail:
            msg = f"{msg}: {detail}"
        raise PaError(st, msg)


def _host_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ free functions
def pa_config_default(L, K, **overrides):
    cfg = pa_config()
    _check(lib().pa_config_default(C.byref(cfg), int(L), int(K)))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        setattr(cfg, k, v)
    if "N" in overrides and "n_seeded" not in overrides:
        cfg.n_seeded = (cfg.N + 1) // 2
    return cfg


def pa_prob_to_thresh(p):
    return int(lib().pa_prob_to_thresh(float(p)))


def pa_create(cfg, beta, user_xy_mm=None, bs_xy_mm=None, stream=None):
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    if beta.shape != (cfg.L, cfg.L, cfg.K):
        raise ValueError(f"beta must be (L, L, K) = {(cfg.L, cfg.L, cfg.K)}, got {beta.shape}")
    u = None if user_xy_mm is None else np.ascontiguousarray(user_xy_mm, dtype=np.int32)
    b = None if bs_xy_mm is None else np.ascontiguousarray(bs_xy_mm, dtype=np.int32)
    if u is not None and u.shape != (cfg.L, cfg.K, 2):
        raise ValueError("user_xy_mm must be (L, K, 2)")
    if b is not None and b.shape != (cfg.L, 2):
        raise ValueError("bs_xy_mm must be (L, 2)")
    out = C.c_void_p()
    st = lib().pa_create(C.byref(cfg), _host_ptr(beta), _host_ptr(u), _host_ptr(b),
                         _stream_handle(stream), C.byref(out))
    _check(st, None)
    return out


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def pa_load_instance(ctx, beta, user_xy_mm=None, bs_xy_mm=None):
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    u = None if user_xy_mm is None else np.ascontiguousarray(user_xy_mm, dtype=np.int32)
    b = None if bs_xy_mm is None else np.ascontiguousarray(bs_xy_mm, dtype=np.int32)
    _check(lib().pa_load_instance(ctx, _host_ptr(beta), _host_ptr(u), _host_ptr(b)), ctx)
    return beta, u, b  # keep the arrays alive until the stream has consumed them


def pa_eval_population_noalloc(cfg, beta, pop, fit, stream=None):
    """Evaluation without any device allocation (see include/pa.h)."""
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    if beta.shape != (cfg.L, cfg.L, cfg.K):
        raise ValueError(f"beta must be (L, L, K) = {(cfg.L, cfg.L, cfg.K)}, got {beta.shape}")
    _check(lib().pa_eval_population_noalloc(C.byref(cfg), _host_ptr(beta), _dev_ptr(pop),
                                            int(pop.shape[0]), _dev_ptr(fit),
                                            _stream_handle(stream)), None)


def pa_kernel_launches():
    return int(lib().pa_kernel_launches())


def pa_solve_cluster_ctas(ctx):
    v = C.c_int32(-1)
    _check(lib().pa_solve_cluster_ctas(ctx, C.byref(v)), ctx)
    return int(v.value)


def pa_destroy(ctx):
    lib().pa_destroy(ctx)


def pa_set_seed(ctx, seed):
    _check(lib().pa_set_seed(ctx, int(seed)), ctx)


def pa_set_stream(ctx, stream):
    _check(lib().pa_set_stream(ctx, _stream_handle(stream)), ctx)


def pa_eval_population(ctx, pop, fit, n=None):
    n = pop.shape[0] if n is None else n
    _check(lib().pa_eval_population(ctx, _dev_ptr(pop), int(n), _dev_ptr(fit)), ctx)


def pa_eval_population_host(ctx, pop, fit):
    pop = np.ascontiguousarray(pop, dtype=np.uint8)
    _check(lib().pa_eval_population_host(ctx, _host_ptr(pop), int(pop.shape[0]),
                                         _host_ptr(fit)), ctx)
    return fit


def pa_ga_step(ctx, pop, fit, generation, next_pop):
    _check(lib().pa_ga_step(ctx, _dev_ptr(pop), _dev_ptr(fit), int(generation),
                            _dev_ptr(next_pop)), ctx)


def pa_kmeans_seed(ctx, labels=None, centroids=None):
    _check(lib().pa_kmeans_seed(ctx, _host_ptr(labels), _host_ptr(centroids)), ctx)


def pa_step(ctx, generations):
    _check(lib().pa_step(ctx, int(generations)), ctx)


def pa_solve(ctx, generations, best):
    bf = C.c_double(0.0)
    _check(lib().pa_solve(ctx, int(generations), _host_ptr(best), C.byref(bf)), ctx)
    return bf.value


def pa_get_population(ctx, pop=None, fit=None):
    g = C.c_int32(0)
    _check(lib().pa_get_population(ctx, _host_ptr(pop), _host_ptr(fit), C.byref(g)), ctx)
    return g.value


def pa_set_population(ctx, pop, generation):
    pop = np.ascontiguousarray(pop, dtype=np.uint8)
    _check(lib().pa_set_population(ctx, _host_ptr(pop), int(generation)), ctx)


def pa_population_device(ctx):
    p = C.c_void_p()
    f = C.c_void_p()
    _check(lib().pa_population_device(ctx, C.byref(p), C.byref(f)), ctx)
    return p.value, f.value


def pa_validate_population(ctx, pop, n=None):
    n = pop.shape[0] if n is None else n
    bad = C.c_int64(0)
    _check(lib().pa_validate_population(ctx, _dev_ptr(pop), int(n), C.byref(bad)), ctx)
    return bad.value


def pa_island_cluster(ctx, pop, generation, labels):
    """K-means of a device population into islands (labels: device int32 N);
    returns the number of assignment passes."""
    passes = C.c_int32(0)
    _check(lib().pa_island_cluster(ctx, _dev_ptr(pop), int(generation), _dev_ptr(labels),
                                   C.byref(passes)), ctx)
    return passes.value


def pa_island_step(ctx, pop, fit, labels, generation, next_pop):
    _check(lib().pa_island_step(ctx, _dev_ptr(pop), _dev_ptr(fit), _dev_ptr(labels),
                                int(generation), _dev_ptr(next_pop)), ctx)


def pa_get_islands(ctx, n):
    out = np.zeros(n, dtype=np.int32)
    _check(lib().pa_get_islands(ctx, _host_ptr(out)), ctx)
    return out


# ------------------------------------------------------------------ convenience
class Context:
    """Owns one pa_ctx.  Methods mirror the C entry points."""

    def __init__(self, cfg, beta, user_xy_mm=None, bs_xy_mm=None, stream=None):
        self.cfg = cfg
        self.L, self.K, self.N = cfg.L, cfg.K, cfg.N
        self.fit_dtype = np.float64 if cfg.prec == PA_FP64 else np.float32
        self.handle = pa_create(cfg, beta, user_xy_mm, bs_xy_mm, stream)

    def close(self):
        if self.handle:
            pa_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def torch_fit_dtype(self):
        import torch

        return torch.float64 if self.cfg.prec == PA_FP64 else torch.float32

    def eval_population(self, pop, fit=None):
        import torch

        if fit is None:
            fit = torch.empty(pop.shape[0], dtype=self.torch_fit_dtype(), device=pop.device)
        pa_eval_population(self.handle, pop, fit)
        return fit

    def eval_population_host(self, pop):
        fit = np.zeros(pop.shape[0], dtype=self.fit_dtype)
        return pa_eval_population_host(self.handle, pop, fit)

    def ga_step(self, pop, fit, generation, next_pop=None):
        import torch

        if next_pop is None:
            next_pop = torch.empty_like(pop)
        pa_ga_step(self.handle, pop, fit, generation, next_pop)
        return next_pop

    def kmeans_seed(self, want_outputs=False):
        if want_outputs:
            labels = np.zeros((self.L, self.K), dtype=np.int32)
            cent = np.zeros((self.cfg.kmeans_k, 2), dtype=np.float64)
            pa_kmeans_seed(self.handle, labels, cent)
            return labels, cent
        pa_kmeans_seed(self.handle)
        return None

    def step(self, generations):
        pa_step(self.handle, generations)

    def solve(self, generations):
        best = np.zeros((self.L, self.K), dtype=np.uint8)
        f = pa_solve(self.handle, generations, best)
        return best, f

    def get_population(self, with_fitness=True):
        pop = np.zeros((self.N, self.L, self.K), dtype=np.uint8)
        fit = np.zeros(self.N, dtype=self.fit_dtype) if with_fitness else None
        g = pa_get_population(self.handle, pop, fit)
        return pop, fit, g

    def set_population(self, pop, generation):
        pa_set_population(self.handle, pop, generation)

    def validate_population(self, pop):
        return pa_validate_population(self.handle, pop)


class Batch:
    """Many instances solved together (pa_batch_*).  instances: list of dicts
    with keys cfg, beta, and optionally user_xy_mm, bs_xy_mm."""

    def __init__(self, instances, stream=None):
        n = len(instances)
        self.n = n
        self.cfgs = (pa_config * n)(*[d["cfg"] for d in instances])
        self._keep = []
        betas = (C.c_void_p * n)()
        have_pos = all(d.get("user_xy_mm") is not None for d in instances)
        ux = (C.c_void_p * n)()
        bx = (C.c_void_p * n)()
        self.shapes = []
        for i, d in enumerate(instances):
            cfg = d["cfg"]
            b = np.ascontiguousarray(d["beta"], dtype=np.float64)
            assert b.shape == (cfg.L, cfg.L, cfg.K)
            self._keep.append(b)
            betas[i] = b.ctypes.data
            self.shapes.append((cfg.L, cfg.K))
            if have_pos:
                u = np.ascontiguousarray(d["user_xy_mm"], dtype=np.int32)
                s = np.ascontiguousarray(d["bs_xy_mm"], dtype=np.int32)
                self._keep += [u, s]
                ux[i] = u.ctypes.data
                bx[i] = s.ctypes.data
        out = C.c_void_p()
        st = lib().pa_batch_create(n, C.cast(self.cfgs, C.c_void_p), C.cast(betas, C.c_void_p),
                                   C.cast(ux, C.c_void_p) if have_pos else None,
                                   C.cast(bx, C.c_void_p) if have_pos else None,
                                   _stream_handle(stream), C.byref(out))
        _check(st, None)
        self.handle = out
        self.offsets = np.cumsum([0] + [L * K for L, K in self.shapes])

    def _bcheck(self, st):
        if st != PA_OK:
            raise PaError(st, lib().pa_status_str(st).decode() + ": " +
                          lib().pa_batch_last_error(self.handle).decode())

    def tune(self, generations):
        ng = C.c_int32(0)
        self._bcheck(lib().pa_batch_groups(self.handle, C.byref(ng), None, None, None, None,
                                           None))
        chosen = np.zeros(max(1, ng.value), dtype=np.int32)
        self._bcheck(lib().pa_batch_tune(self.handle, int(generations), _host_ptr(chosen)))
        return chosen[:ng.value]

    def groups(self):
        """(cluster size per group, group of each instance)."""
        cs, _, gi = self.group_shapes()
        return cs, gi

    def group_shapes(self):
        """(cluster size per group, CTA threads per group, group of each instance)."""
        cs, th, _, _, gi = self.group_tiling()
        return cs, th, gi

    def group_tiling(self):
        """(cluster size, CTA threads, latency column split, persistent clusters
        launched per group, group of each instance)."""
        ng = C.c_int32(0)
        self._bcheck(lib().pa_batch_groups(self.handle, C.byref(ng), None, None, None, None,
                                           None))
        cs = np.zeros(max(1, ng.value), dtype=np.int32)
        th = np.zeros(max(1, ng.value), dtype=np.int32)
        lat = np.zeros(max(1, ng.value), dtype=np.int32)
        rc = np.zeros(max(1, ng.value), dtype=np.int32)
        gi = np.zeros(self.n, dtype=np.int32)
        self._bcheck(lib().pa_batch_groups(self.handle, None, _host_ptr(cs), _host_ptr(th),
                                           _host_ptr(lat), _host_ptr(rc), _host_ptr(gi)))
        return cs[:ng.value], th[:ng.value], lat[:ng.value], rc[:ng.value], gi

    def solve(self, generations):
        best = np.zeros(int(self.offsets[-1]), dtype=np.uint8)
        fit = np.zeros(self.n, dtype=np.float64)
        self._bcheck(lib().pa_batch_solve(self.handle, int(generations), _host_ptr(best),
                                          _host_ptr(fit)))
        rows = [best[self.offsets[i]:self.offsets[i + 1]].reshape(self.shapes[i])
                for i in range(self.n)]
        return rows, fit

    def completion_times_ms(self):
        """Per-instance completion latency (ms) of the last solve."""
        out = np.zeros(self.n, dtype=np.float64)
        self._bcheck(lib().pa_batch_completion_times(self.handle, _host_ptr(out)))
        return out

    def load(self, i, beta, user_xy_mm=None, bs_xy_mm=None):
        b = np.ascontiguousarray(beta, dtype=np.float64)
        u = None if user_xy_mm is None else np.ascontiguousarray(user_xy_mm, dtype=np.int32)
        s = None if bs_xy_mm is None else np.ascontiguousarray(bs_xy_mm, dtype=np.int32)
        self._bcheck(lib().pa_batch_load(self.handle, int(i), _host_ptr(b), _host_ptr(u),
                                         _host_ptr(s)))
        self._keep.append((b, u, s))

    def context(self, i):
        out = C.c_void_p()
        self._bcheck(lib().pa_batch_context(self.handle, int(i), C.byref(out)))
        return out

    def close(self):
        if self.handle:
            lib().pa_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (pa_server_*)."""

    MAX_LK = 64 * 64

    def __init__(self, base_cfg, generations, tick, budget_bytes, stream=None, max_done=4096):
        out = C.c_void_p()
        _check(lib().pa_server_create(C.byref(base_cfg), int(generations), int(tick),
                                      int(budget_bytes), _stream_handle(stream), C.byref(out)),
               None)
        self.handle = out
        self.max_done = max_done
        self._ids = np.zeros(max_done, dtype=np.int64)
        self._st = np.zeros(max_done, dtype=np.int32)
        self._best = np.zeros((max_done, self.MAX_LK), dtype=np.uint8)
        self._fit = np.zeros(max_done, dtype=np.float64)

    def _scheck(self, st):
        if st != PA_OK:
            raise PaError(st, lib().pa_status_str(st).decode() + ": " +
                          lib().pa_server_last_error(self.handle).decode())

    def submit(self, rid, L, K, seed, beta, user_xy_mm, bs_xy_mm):
        b = np.ascontiguousarray(beta, dtype=np.float64)
        u = np.ascontiguousarray(user_xy_mm, dtype=np.int32)
        s = np.ascontiguousarray(bs_xy_mm, dtype=np.int32)
        self._scheck(lib().pa_server_submit(self.handle, int(rid), int(L), int(K), int(seed),
                                            _host_ptr(b), _host_ptr(u), _host_ptr(s)))

    def poll(self, max_done=None, with_status=False):
        """One tick; returns ([(id, best row bytes, fitness[, status]) ...],
        active slots, queued requests)."""
        md = self.max_done if max_done is None else min(int(max_done), self.max_done)
        nd, na, npd = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        self._scheck(lib().pa_server_poll(self.handle, md, _host_ptr(self._ids),
                                          _host_ptr(self._st), _host_ptr(self._best), self.MAX_LK,
                                          _host_ptr(self._fit), C.byref(nd), C.byref(na),
                                          C.byref(npd)))
        k = nd.value
        if with_status:
            out = [(int(self._ids[i]), self._best[i].copy(), float(self._fit[i]),
                    int(self._st[i])) for i in range(k)]
        else:
            out = [(int(self._ids[i]), self._best[i].copy(), float(self._fit[i]))
                   for i in range(k)]
        return out, na.value, npd.value

    def wait(self, timeout_us=-1):
        """Block until a tick in flight finishes (at most timeout_us when >= 0)."""
        self._scheck(lib().pa_server_wait(self.handle, int(timeout_us)))

    def run_until_idle(self, max_done=None, with_status=False):
        """Poll (waiting for ticks in between) until nothing is queued or running;
        returns every completion."""
        out = []
        while True:
            done, active, pending = self.poll(max_done, with_status)
            out += done
            if not done and active == 0 and pending == 0:
                return out
            if not done:
                self.wait()

    def cancel(self, rid):
        self._scheck(lib().pa_server_cancel(self.handle, int(rid)))

    def inject_admission_failures(self, count):
        self._scheck(lib().pa_server_inject_admission_failures(self.handle, int(count)))

    def stats(self):
        u, ns, c = C.c_uint64(0), C.c_int32(0), C.c_int64(0)
        self._scheck(lib().pa_server_stats(self.handle, C.byref(u), C.byref(ns), C.byref(c)))
        return dict(used_bytes=u.value, slots=ns.value, completed=c.value)

    def close(self):
        if self.handle:
            lib().pa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

