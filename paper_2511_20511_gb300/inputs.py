"""Seeded synthetic inputs: hexagonal multi-cell layouts, user drops and
large-scale fading coefficients beta, plus random pilot populations.

This module generates the *workload* only -- it holds none of the method's
arithmetic (fitness, GA operators, K-means).  The same arrays feed both the
CUDA library and the CPU oracle.

Model (paper Sec. 3.1, Eq. 1-2; Sec. 6.1 hexagonal cells, i.i.d. Rayleigh):
  * L = 1 + 3 r (r + 1) flat-top hexagonal cells in r rings, circumradius R,
    BS at each centre, no wrap-around.  Cells are ordered ring by ring, each
    ring counter-clockwise starting from the +q axial direction.
  * K users per cell, uniform in the hexagon by rejection from its bounding
    box, at least d_min from the own BS; positions quantised to integer mm.
  * beta[j][l][k] = d^-alpha * 10^(z/10), z ~ N(0, sigma_dB^2) i.i.d. per
    (BS j, user (l,k)), d the distance in metres from the quantised positions
    (Eq. 2: log-normal shadowing over path loss).
"""
import math

import numpy as np

SQRT3 = math.sqrt(3.0)

# axial directions, counter-clockwise
_AXIAL_DIRS = [(1, 0), (1, -1), (0, -1), (-1, 0), (-1, 1), (0, 1)]


def rings_for(L):
    """Number of hex rings r with 1 + 3r(r+1) == L (ValueError otherwise)."""
    r = 0
    while 1 + 3 * r * (r + 1) < L:
        r += 1
    if 1 + 3 * r * (r + 1) != L:
        raise ValueError(f"L={L} is not a full hexagonal layout (1, 7, 19, 37, 61, ...)")
    return r


def hex_centres(L, R=500.0):
    """(L, 2) BS positions in metres for a full hexagonal layout of L cells."""
    rings = rings_for(L)
    cells = [(0, 0)]
    for ring in range(1, rings + 1):
        # start at ring * dir[4] and walk ring steps along each direction
        q, r = _AXIAL_DIRS[4][0] * ring, _AXIAL_DIRS[4][1] * ring
        for d in range(6):
            for _ in range(ring):
                cells.append((q, r))
                q += _AXIAL_DIRS[d][0]
                r += _AXIAL_DIRS[d][1]
    out = np.array([[R * 1.5 * q, R * SQRT3 * (r + q / 2.0)] for q, r in cells])
    return out


def _in_hex(x, y, R):
    ax, ay = np.abs(x), np.abs(y)
    return (ay <= SQRT3 / 2.0 * R) & (SQRT3 * ax + ay <= SQRT3 * R)


def instance(L, K, seed=0, R=500.0, alpha=3.8, sigma_db=8.0, d_min=35.0, dtype=np.float64):
    """One pilot-assignment instance.

    Returns a dict with
      beta       (L, L, K) float64 -- rounded to float32 first if dtype is float32
      user_xy_mm (L, K, 2) int32   -- user positions, mm
      bs_xy_mm   (L, 2)    int32   -- BS positions, mm
      rho        float             -- SNR scale giving 10 dB at distance R
                                      without shadowing (sigma2 = 1)
    """
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    centres = hex_centres(L, R)
    bs_mm = np.round(centres * 1000.0).astype(np.int64)
    users = np.zeros((L, K, 2), dtype=np.int64)
    for l in range(L):
        got = 0
        while got < K:
            cand = rng.uniform(low=[-R, -SQRT3 / 2 * R], high=[R, SQRT3 / 2 * R], size=(4 * K, 2))
            ok = _in_hex(cand[:, 0], cand[:, 1], R) & (np.hypot(cand[:, 0], cand[:, 1]) >= d_min)
            # candidates in draw order; the quantised position must still be
            # at least d_min from the BS; the first K - got of them are taken
            rel = np.round(cand[ok] * 1000.0).astype(np.int64)
            far = ~(np.hypot(rel[:, 0].astype(np.float64), rel[:, 1].astype(np.float64)) / 1000.0
                    < d_min)
            take = rel[far][:K - got]
            users[l, got:got + len(take)] = take + bs_mm[l]
            got += len(take)
    # distances from every BS j to every user (l, k), metres
    dx = users[None, :, :, 0] - bs_mm[:, None, None, 0]
    dy = users[None, :, :, 1] - bs_mm[:, None, None, 1]
    d = np.hypot(dx.astype(np.float64), dy.astype(np.float64)) / 1000.0
    z = rng.normal(0.0, sigma_db, size=(L, L, K))
    beta = d ** (-alpha) * 10.0 ** (z / 10.0)
    if np.dtype(dtype) == np.float32:
        beta = beta.astype(np.float32).astype(np.float64)
    rho = 10.0 / (R ** (-alpha))
    return dict(beta=np.ascontiguousarray(beta), user_xy_mm=users.astype(np.int32),
                bs_xy_mm=bs_mm.astype(np.int32), rho=float(rho), sigma2=1.0)


def random_population(n, L, K, seed=0):
    """(n, L, K) uint8: every row an independent uniformly random permutation."""
    rng = np.random.Generator(np.random.Philox(key=int(seed) ^ 0x5EED))
    keys = rng.random((n, L, K))
    return np.argsort(keys, axis=-1).astype(np.uint8)


def random_population_torch(n, L, K, seed, device):
    """Same distribution as random_population, generated on a torch device
    (for populations too large to build on the host quickly)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    keys = torch.rand((n, L, K), generator=g, device=device)
    return torch.argsort(keys, dim=-1).to(torch.uint8).contiguous()
