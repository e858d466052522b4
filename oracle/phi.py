"""Luttinger-Ward functional of the SOX diagram and its gradients (oracle).

Test infrastructure; see the package docstring.

The paper invokes the conserving (Phi-derivable) property (Sec. II A) but never
writes Phi for SOX.  The reading used here ties it to the tau form of the
dynamical Galitskii-Migdal energy (Eq. E2b): with the Matsubara sum
(1/beta) sum_n A(i w_n) B(i w_n) = int_0^beta A(tau) B(-tau) d tau,

    Phi = 1/4 sum_j w_j Tr[Sigma(tau_j) G(-tau_j)],

so that 4 Phi is E_dyn's SOX part.  Phi is quartic in G and for bare SOX
d Phi / d G_rt(tau_j) = -w_j Sigma_tr(beta - tau_j) on a mirror-symmetric grid
with symmetric weights.

Gradients with respect to G, X and V come from PyTorch CPU autograd over the
plain formula (a library step); they are pinned by central finite differences
and by the identity above in the tests.
"""
from __future__ import annotations

import numpy as np

from . import grid, sox, thc


def phi_trace(Sigma_tau: np.ndarray, G_tau: np.ndarray, w: np.ndarray) -> complex:
    """Phi = 1/4 sum_j w_j sum_tr Sigma_tr(tau_j) G_rt(-tau_j) for one spin block."""
    Gm = grid.g_minus_tau(G_tau)
    return 0.25 * np.einsum("j,jtr,jrt->", w, Sigma_tau, Gm)


def phi_thc_direct(X: np.ndarray, U1: np.ndarray, U2: np.ndarray, G_tau: np.ndarray,
                   w: np.ndarray) -> complex:
    """Independent route: Phi = -1/4 sum_j w_j sum_PQRS U1_PQ U2_RS G^SP G^RQ G^QS(-) G^PR(-)."""
    Gm_tau = grid.g_minus_tau(G_tau)
    tot = 0.0
    for j in range(G_tau.shape[0]):
        gp = thc.project_full(X, G_tau[j])
        gm = thc.project_full(X, Gm_tau[j])
        tot = tot - 0.25 * w[j] * np.einsum("PQ,RS,SP,RQ,QS,PR->", U1, U2, gp, gp, gm, gm,
                                             optimize=True)
    return tot


def phi_sox(X: np.ndarray, V: np.ndarray, G: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Phi per spin for bare SOX, library layout (G [n_spin][1][n_tau][n][n]); returns [n_spin]."""
    out = []
    for s in range(G.shape[0]):
        sig = sox.sigma_tau(X[0], V[0], V[0], G[s, 0])
        out.append(phi_trace(sig, np.asarray(G[s, 0], complex), w))
    return np.array(out)


def phi_torch(X, U1, U2, G_tau, w):
    """Phi for one spin block written with torch CPU ops (float64), for autograd.

    Same formula as ``phi_thc_direct``; G(-tau) is built by the reflection so the
    gradient with respect to G(tau) collects both the +tau and -tau lines.
    """
    import torch

    Gm = -torch.flip(G_tau, dims=(0,))
    gp = X @ G_tau @ X.T                    # [n_tau, N, N]  G^PQ(tau)
    gm = X @ Gm @ X.T                       # G^PQ(-tau)
    # sum_PQRS U1_PQ U2_RS G^SP G^RQ G^QS(-) G^PR(-)
    t1 = torch.einsum("RS,jQS,jSP->jRQP", U2, gm, gp)
    t2 = torch.einsum("PQ,jRQ,jRQP,jPR->j", U1, gp, t1, gm)
    return -0.25 * torch.sum(w * t2)


def phi_and_grads(X: np.ndarray, V: np.ndarray, G_tau: np.ndarray, w: np.ndarray,
                  U2: np.ndarray | None = None):
    """Phi and d Phi/d(G, X, V) for one spin block (real data), by torch CPU autograd.

    With ``U2`` given the functional is built from SOX(V, U2); V is then the
    first-slot interaction and only its gradient is returned for V.
    Gradients are with respect to the unsymmetrised entries (single-entry
    finite differences reproduce them).
    """
    import torch

    tX = torch.tensor(np.asarray(X, np.float64), requires_grad=True)
    tV = torch.tensor(np.asarray(V, np.float64), requires_grad=True)
    tG = torch.tensor(np.asarray(G_tau, np.float64), requires_grad=True)
    tw = torch.tensor(np.asarray(w, np.float64))
    tU2 = tV if U2 is None else torch.tensor(np.asarray(U2, np.float64))
    val = phi_torch(tX, tV, tU2, tG, tw)
    val.backward()
    return float(val.detach()), tG.grad.numpy(), tX.grad.numpy(), tV.grad.numpy()
