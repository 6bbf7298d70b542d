"""Seeded synthetic input generators shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the method itself: only random fields, random
vectors and workload descriptions.  Every generator is deterministic in its seed.

Workloads (sizes and structure of the paper's poroelastic test class, §Numerical
Simulations; the paper prints no data, so every field here is synthetic):

* layered permeability: log-permeability g constant inside horizontal layers of a
  fixed number of cells, i.i.d. N(0, std^2) across layers; K = exp(g) * K0;
* correlated 2-D field: white noise per cell convolved with a separable Gaussian
  kernel (periodic wrap), renormalised to a sample standard deviation;
* unit-RMS random directions for finite-difference checks;
* the ragged batch instance list (mesh size n and time order r per instance).
"""
from __future__ import annotations

import numpy as np

K0 = 1.0e-2  # base permeability of the synthetic media


def layered_logk(n, layer_cells: int = 4, std: float = 1.5, seed: int = 1801) -> np.ndarray:
    """Cellwise log-permeability, constant within `layer_cells`-thick layers of the
    last axis (z in 3-D, y in 2-D).  Returned in cell-lexicographic order (x fastest)."""
    n = tuple(int(v) for v in n)
    nz = n[-1]
    nlayers = (nz + layer_cells - 1) // layer_cells
    rng = np.random.default_rng(seed)
    vals = rng.normal(0.0, std, size=nlayers)
    layer_of = np.arange(nz) // layer_cells
    g_z = vals[layer_of]
    shape = n[::-1]  # (nz, ny, nx) for C-order with x fastest
    g = np.broadcast_to(g_z.reshape((nz,) + (1,) * (len(n) - 1)), shape)
    return np.ascontiguousarray(g).reshape(-1).astype(np.float64)


def correlated_logk_2d(n: int, std: float = 1.0, corr_cells: float = 8.0, seed: int = 1801) -> np.ndarray:
    """2-D Gaussian random field on an n x n cell grid: white noise convolved with a
    separable Gaussian kernel of width `corr_cells` (periodic), renormalised to
    sample std `std`.  Returned x-fastest."""
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 1.0, size=(n, n))
    k = np.arange(n)
    d = np.minimum(k, n - k).astype(np.float64)
    ker = np.exp(-0.5 * (d / corr_cells) ** 2)
    kf = np.fft.fft(ker)
    f = np.fft.ifft2(np.fft.fft2(w) * kf[None, :] * kf[:, None]).real
    f -= f.mean()
    s = f.std()
    if s > 0:
        f *= std / s
    return np.ascontiguousarray(f).reshape(-1)


def fd_directions(ncells: int, count: int = 20, seed: int = 4984) -> np.ndarray:
    """`count` random directions in R^ncells, each normalised to unit RMS."""
    rng = np.random.default_rng(seed)
    d = rng.normal(0.0, 1.0, size=(count, ncells))
    d /= np.sqrt(np.mean(d * d, axis=1, keepdims=True))
    return d


def batch_instances(count: int = 256, seed: int = 1801, sizes=(16, 32, 64, 128), orders=(0, 1, 2)):
    """Ragged batch description: list of dicts (n, r, seed) drawn uniformly."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        out.append({"n": int(rng.choice(sizes)), "r": int(rng.choice(orders)), "seed": seed + i})
    return out


def random_vector(size: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform(-1, 1) * scale, float64."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1.0, 1.0, size=size) * scale).astype(np.float64)
