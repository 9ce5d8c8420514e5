"""Derived outputs of a steady solve (oracle; test infrastructure only)."""
from __future__ import annotations

import math

import numpy as np


def mean_concentration(c: np.ndarray) -> float:
    """cbar: the average over all cells, blob interiors included (Sec. IV.A)."""
    return float(np.mean(c))


def overall_rate(lam: np.ndarray, c: np.ndarray) -> float:
    """K from K cbar = N^-1 sum_i lambda_i (Sec. I.A)."""
    return float(np.sum(lam)) / (len(lam) * mean_concentration(c))


def reaction_radius(lam: np.ndarray, c: np.ndarray, chi: float) -> float:
    """a_L = K / (4 pi chi); for one blob with s = 1/V_Omega this is
    [4 pi chi cbar]^-1 (Sec. IV.A, Eq. beta0_low_phi)."""
    return overall_rate(lam, c) / (4.0 * math.pi * chi)


RADIUS_SERIES_COEFFICIENT = 2.84  # Eq. a_phi


def extrapolated_radius(a_L: float, L: int, h: float, k: float = RADIUS_SERIES_COEFFICIENT) -> float:
    """a ~ a_L - k a_L^2 / (L h): the first-order inversion of Eq. a_phi that
    Sec. IV.A uses for the translational-invariance study at L = 128. Its
    error against the exact inverse of the series is second order in a / L."""
    return a_L - k * a_L * a_L / (L * h)


def radius_from_series(a_L: float, L: int, h: float, k: float = RADIUS_SERIES_COEFFICIENT) -> float:
    """The a that solves Eq. a_phi truncated after its quadratic term,
    a_L = a [1 + k a/(L h) + (k a/(L h))^2], by fixed-point iteration from
    a = a_L (a contraction while k a_L / (L h) < 1/2)."""
    a = a_L
    for _ in range(200):
        x = k * a / (L * h)
        a = a_L / (1.0 + x + x * x)
    return a


def beta0(cbar: float, s: float, a: float, chi: float, n_blobs: int, volume: float) -> float:
    """Normalized rate, Eq. beta_P_disc with phi = N (4 pi a^3 / 3) / V_Omega."""
    phi = n_blobs * (4.0 * math.pi * a ** 3 / 3.0) / volume
    return (s * a * a / chi) * (1.0 - phi) / (3.0 * phi) / cbar


def beta0_cubic_fit(phi: float, b: float = -0.92, c: float = 17.4) -> float:
    """Eq. beta_cubic: the cubic-lattice fit with the paper's b, c."""
    t = phi ** (1.0 / 3.0)
    return 1.0 + 1.76 * t + 1.76 ** 2 * t * t + b * phi + c * phi * t
