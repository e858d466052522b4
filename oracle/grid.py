"""Imaginary-time grid, quadrature weights and fermionic reflection (oracle).

Test infrastructure; see the package docstring.

* Sec. II A defines G(tau) on [0, beta] (Eq. G_def).  The paper evaluates it on
  sparse-ir grids (Sec. III A); the stand-in grid here is Chebyshev-Lobatto,
  which contains both end points and is symmetric under tau -> beta - tau.
* The algorithms of Sec. II C use G(-tau) (static chain: the A intermediate;
  dynamic chain: Eq. GG).  For fermions G(-tau) = -G(beta - tau), so on a
  symmetric grid G(-tau_j) = -G(tau_{n-1-j}).
"""
from __future__ import annotations

import numpy as np


def chebyshev_lobatto(n_tau: int, beta: float) -> np.ndarray:
    """tau_j = (beta/2) (1 - cos(pi j / (n_tau - 1))), j = 0..n_tau-1."""
    j = np.arange(n_tau, dtype=np.float64)
    return 0.5 * beta * (1.0 - np.cos(np.pi * j / (n_tau - 1)))


def clenshaw_curtis(n_tau: int, beta: float) -> np.ndarray:
    """Weights w_j with sum_j w_j f(tau_j) ~ int_0^beta f(tau) d tau on the nodes above.

    Clenshaw-Curtis on [-1, 1] with nodes x_j = cos(pi j / M), M = n_tau - 1:
        w_j = (c_j / M) * (1 - sum_{k=1}^{floor(M/2)} b_k cos(2 pi j k / M) / (4 k^2 - 1)),
    c_j = 1 at the two ends and 2 inside, b_k = 1 for k = M/2 (M even) and 2
    otherwise; the map tau = (beta/2)(1 - x) scales them by beta/2.
    """
    M = n_tau - 1
    if M < 1:
        raise ValueError("need at least two nodes")
    j = np.arange(n_tau, dtype=np.float64)
    w = np.ones(n_tau)
    for k in range(1, M // 2 + 1):
        b = 1.0 if (2 * k == M) else 2.0
        w -= b * np.cos(2.0 * np.pi * j * k / M) / (4.0 * k * k - 1.0)
    c = np.full(n_tau, 2.0)
    c[0] = c[-1] = 1.0
    return 0.5 * beta * c * w / M


def reflect(n_tau: int) -> np.ndarray:
    """Index map j -> n_tau - 1 - j that takes tau_j to beta - tau_j."""
    return np.arange(n_tau)[::-1].copy()


def g_minus_tau(G_tau: np.ndarray) -> np.ndarray:
    """G(-tau_j) = -G(beta - tau_j) = -G(tau_{n-1-j}) along the tau axis (axis -3)."""
    return -np.flip(G_tau, axis=-3)
