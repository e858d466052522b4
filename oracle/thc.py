"""Tensor-hypercontraction pieces (oracle).  Test infrastructure.

Sec. II C writes the two-electron integrals in THC form

    (ij|sr) = sum_PQ (X^{k_i}_{iP})^* X^{k_j}_{jP} U^q_{PQ} (X^{k_s}_{sQ})^* X^{k_r}_{rQ},
    q = k_i - k_j,

with momenta set to zero for molecules.  Arrays here store the collocation
matrix as ``X[P, p]`` (= X_{pP}), so that N x n is one row per THC point.
"""
from __future__ import annotations

import numpy as np


def eri(X_i: np.ndarray, X_j: np.ndarray, U: np.ndarray, X_s: np.ndarray, X_r: np.ndarray,
        scale: float = 1.0) -> np.ndarray:
    """Reconstructed 4-index tensor v[i, j, s, r] = (ij|sr) of Sec. II C.

    ``X_a`` are [N, n] slices; the first of each pair is complex-conjugated.
    """
    left = np.einsum("Pi,Pj->ijP", X_i.conj(), X_j)       # pair function of electron 1
    right = np.einsum("Qs,Qr->srQ", X_s.conj(), X_r)      # pair function of electron 2
    return scale * np.einsum("ijP,PQ,srQ->ijsr", left, U, right, optimize=True)


def project_full(X: np.ndarray, G: np.ndarray) -> np.ndarray:
    """G^{PQ} = sum_pq X_{pP} G_pq X_{qQ}^* (molecules: X real)."""
    return X @ G @ X.conj().T


def project_left(X: np.ndarray, G: np.ndarray) -> np.ndarray:
    """G_{Rq} = sum_u X_{uR} G_{uq}  (second projection of the static chain)."""
    return X @ G


def project_right(X: np.ndarray, G: np.ndarray) -> np.ndarray:
    """G_{wP} = sum_p G_{wp} X_{pP}^*  (third projection of the static chain).

    The printed sum index reads "uq"; it is a sum over p.
    """
    return G @ X.conj().T
