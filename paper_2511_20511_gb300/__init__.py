"""GB300-native pilot assignment: K-means-seeded 2D genetic algorithm for
massive-MIMO uplink pilot assignment (arXiv 2511.20511).

The compute path is libpa.so (hand-written CUDA for sm_103a, C ABI in
include/pa.h); ``binding`` is its thin ctypes binding and ``inputs`` the
seeded synthetic workload generator.
"""
from . import binding  # noqa: F401
from .binding import (PA_FP32, PA_FP64, PA_SINR_ASYMPTOTIC, PA_SINR_FINITE_M,  # noqa: F401
                      Context, PaError, pa_config, pa_config_default)
