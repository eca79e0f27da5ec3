"""Per-element coefficients and input vectors."""

import numpy as np

from .rng import normal, uniform


def lognormal(seed: int, count: int) -> np.ndarray:
    """kappa_e = exp(z_e), z_e ~ N(0,1) (natural log)."""
    return np.exp(normal(seed, count))


def x_uniform(seed: int, count: int) -> np.ndarray:
    """Input vector entries ~ U[-1, 1]."""
    return uniform(seed, count, -1.0, 1.0)


def rho_uniform(seed: int, count: int, lo: float = 0.2, hi: float = 1.0) -> np.ndarray:
    """Design densities rho_e ~ U[lo, hi]."""
    return uniform(seed, count, lo, hi)
