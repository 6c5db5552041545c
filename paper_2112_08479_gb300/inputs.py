"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds none of the method's arithmetic: it only draws seeded random
numbers (perturbations, directions, adjoint seeds).  Each side adds its own
lattice weights, equilibria or scalings to what is drawn here.
"""
from __future__ import annotations

import numpy as np


def uniform(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform(-scale, scale) float64 array."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=shape)


def normal(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Normal(0, scale^2) float64 array."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=shape)


def unit_direction(shape, seed: int) -> np.ndarray:
    """Gaussian direction of unit 2-norm (finite-difference directions)."""
    d = normal(shape, seed)
    return d / np.linalg.norm(d.ravel())


def distinct_values(shape, seed: int) -> np.ndarray:
    """Pairwise distinct float32-representable values in (-1, 1), as float64.

    Used to follow individual populations through a streaming permutation.
    """
    n = int(np.prod(shape))
    rng = np.random.default_rng(seed)
    k = rng.permutation(n).astype(np.float64)
    return ((k + 1.0) / (n + 2.0) * 2.0 - 1.0).astype(np.float32).astype(np.float64).reshape(shape)


def torch_uniform(shape, seed: int, scale: float = 1.0, device="cuda"):
    """Uniform(-scale, scale) float32 tensor drawn on `device` by a seeded
    torch generator (for inputs too large to draw on the host)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    t = torch.rand(shape, generator=g, device=device, dtype=torch.float32)
    return t.mul_(2.0 * scale).sub_(scale)
