"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no step of the Monte Carlo method: it only draws couplings
and starting spins.  It imports neither the CUDA binding nor the oracle.

Arrays are site-major, the paper's indexing (Sec. 2): site ``i = x + y*L +
z*L*L``; ``J[3*i + d]`` is the coupling of the bond from ``i`` to ``i + e_d``
(d = 0, 1, 2 for x, y, z) and ``s[3*i + a]`` the spin component ``a``.

The paper's workload is a synthetic L^3 cube with Gaussian couplings of mean 0
and variance 1 (Sec. 2 and Sec. 4, L = 128), so these generators stand in for
it; no dataset is involved.
"""
from __future__ import annotations

import numpy as np

# Stream tags keep the coupling and spin draws of one seed independent.
_TAG_COUPLINGS = 0x4A
_TAG_SPINS = 0x53


def _rng(seed: int, sample: int, tag: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(sample), int(tag)])


def gaussian_couplings(L: int, seed: int, sample: int = 0, dtype=np.float64) -> np.ndarray:
    """J ~ N(0, 1) on the 3 L^3 bonds, site-major ``J[3*i + d]``."""
    n = 3 * L ** 3
    return _rng(seed, sample, _TAG_COUPLINGS).standard_normal(n, dtype=np.dtype(dtype).type)


def uniform_couplings(L: int, value: float = 1.0, axes=(0, 1, 2), dtype=np.float64) -> np.ndarray:
    """J = value on the bonds along ``axes`` and 0 on the others."""
    J = np.zeros((L ** 3, 3), dtype=dtype)
    for d in axes:
        J[:, d] = value
    return J.reshape(-1)


def random_spins(L: int, seed: int, sample: int = 0, dtype=np.float64) -> np.ndarray:
    """Unit spins, isotropic (normalised Gaussian triples), site-major."""
    g = _rng(seed, sample, _TAG_SPINS).standard_normal((L ** 3, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g.astype(dtype).reshape(-1)


def aligned_spins(L: int, direction=(0.0, 0.0, 1.0), dtype=np.float64) -> np.ndarray:
    """All spins along one unit direction."""
    v = np.asarray(direction, dtype=np.float64)
    v = v / np.linalg.norm(v)
    return np.tile(v, L ** 3).astype(dtype)


def round_to_f32(a: np.ndarray) -> np.ndarray:
    """Values rounded to fp32 and held in fp64 (what the GPU path stores)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)
