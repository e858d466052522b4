"""Second-order exchange self-energy with static interactions (oracle, molecules).

Test infrastructure; see the package docstring.

Eq. (sox), Sec. II B-C: for two interactions U(1), U(2)

    Sigma_tr(tau) = - sum_{pqsuvw} U1_(pr|qs) U2_(tu|vw) G_wp(tau_wp) G_uq(tau_uq) G_sv(tau_sv)

(the printed time label of G_uq reads tau_up; it is tau_uq).  With both
interactions static the times collapse to tau_wp = tau_uq = tau, tau_sv = -tau
(Sec. II C), so every route below takes G(tau) and G(-tau) of one grid point.

Three independent routes compute the same number:

1. ``sigma_bruteforce``  the definition over reconstructed 4-index tensors, O(n^5);
2. ``sigma_thc_direct``  the definition with the THC form substituted and the
   orbital sums done first, Sigma_RP = -sum_QS U1_PQ U2_RS G^SP G^RQ G^QS(-tau),
   O(N^4) — it shares no intermediate with the chain;
3. ``sigma_chain``       the paper's algorithm (Eq. U_contraction and the steps
   after it, k = 0): mixed tensor U_Pqs, projections G_Rq and G_wP, A, B, C, D,
   Sigma_RP = -D_PR, back-projection to orbitals.

Arrays: X[P, p] (N x n), U1/U2 [N, N], G and Gm (= G(-tau)) [n, n].
"""
from __future__ import annotations

import numpy as np

from . import grid, thc


def sigma_bruteforce(v1: np.ndarray, v2: np.ndarray, G: np.ndarray, Gm: np.ndarray) -> np.ndarray:
    """Eq. (sox) over 4-index tensors v1[p,r,q,s] = U1_(pr|qs), v2[t,u,v,w] = U2_(tu|vw)."""
    f1 = np.einsum("prqs,wp->rqsw", v1, G)        # sum over p
    f2 = np.einsum("rqsw,uq->rswu", f1, G)        # sum over q
    f3 = np.einsum("rswu,sv->rwuv", f2, Gm)       # sum over s
    return -np.einsum("tuvw,rwuv->tr", v2, f3)    # sum over u, v, w


def sigma_thc_direct(X: np.ndarray, U1: np.ndarray, U2: np.ndarray,
                     G: np.ndarray, Gm: np.ndarray) -> np.ndarray:
    """Definition with THC substituted: Sigma_RP = -sum_QS U1_PQ U2_RS G^SP G^RQ G^QS(-tau)."""
    gp = thc.project_full(X, G)       # G^{AB}(tau)
    gm = thc.project_full(X, Gm)      # G^{AB}(-tau)
    # M[R, Q, P] = sum_S U2_RS G^{QS}(-) G^{SP}
    M = np.einsum("RS,QS,SP->RQP", U2, gm, gp, optimize=True)
    sig_RP = -np.einsum("PQ,RQ,RQP->RP", U1, gp, M, optimize=True)
    # back to orbitals: Sigma_tr = sum_PR X_tR Sigma_RP X_rP
    return X.T @ sig_RP @ X


def mixed_tensor(U: np.ndarray, X: np.ndarray) -> np.ndarray:
    """U_Pqs = sum_Q U_PQ X_qQ X_sQ  (Eq. U_contraction at k = 0), shape [N, n, n]."""
    return np.einsum("PQ,Qq,Qs->Pqs", U, X, X, optimize=True)


def sigma_chain(X: np.ndarray, U1: np.ndarray, U2: np.ndarray, G: np.ndarray, Gm: np.ndarray,
                U1_mixed: np.ndarray | None = None, U2_mixed: np.ndarray | None = None,
                return_RP: bool = False):
    """The paper's static THC-SOX algorithm, Sec. II C, molecular case (k = 0)."""
    Um1 = mixed_tensor(U1, X) if U1_mixed is None else U1_mixed      # U_Pqs
    Um2 = mixed_tensor(U2, X) if U2_mixed is None else U2_mixed      # U(2)_Rvw
    G_Rq = thc.project_left(X, G)                                     # G_Rq(tau)
    G_wP = thc.project_right(X, G)                                    # G_wP(tau)
    A = np.einsum("Pqs,sv->Pqv", Um1, Gm, optimize=True)                             # A_Pqv
    B = np.einsum("Pqv,Rq->PRv", A, G_Rq, optimize=True)                             # B_PRv
    C = np.einsum("Rvw,wP->RvP", Um2, G_wP, optimize=True)                           # C_RvP
    D = np.einsum("RvP,PRv->PR", C, B, optimize=True)                                # D_PR
    sig_RP = -D.T                                                     # Sigma_RP = -D_PR
    sig = X.T @ sig_RP @ X                                            # Sigma_tr
    if return_RP:
        return sig, sig_RP
    return sig


def sigma_tau(X: np.ndarray, U1: np.ndarray, U2: np.ndarray, G_tau: np.ndarray,
              route: str = "chain", taus=None, dtype=np.complex128) -> np.ndarray:
    """Sigma(tau_j) for every grid point (or the listed ``taus``) of one spin block.

    G_tau: [n_tau, n, n] on a symmetric grid; G(-tau_j) = -G(tau_{n-1-j}).
    """
    G_tau = np.asarray(G_tau, dtype=dtype)
    X = np.asarray(X, dtype=dtype)
    U1 = np.asarray(U1, dtype=dtype)
    U2 = np.asarray(U2, dtype=dtype)
    Gm_tau = grid.g_minus_tau(G_tau)
    n_tau = G_tau.shape[0]
    idx = range(n_tau) if taus is None else taus
    if route == "brute":
        v1 = thc.eri(X, X, U1, X, X)
        v2 = thc.eri(X, X, U2, X, X)
        out = [sigma_bruteforce(v1, v2, G_tau[j], Gm_tau[j]) for j in idx]
    elif route == "direct":
        out = [sigma_thc_direct(X, U1, U2, G_tau[j], Gm_tau[j]) for j in idx]
    elif route == "chain":
        m1 = mixed_tensor(U1, X)
        m2 = m1 if U2 is U1 else mixed_tensor(U2, X)
        out = [sigma_chain(X, U1, U2, G_tau[j], Gm_tau[j], m1, m2) for j in idx]
    else:
        raise ValueError(route)
    return np.stack(out)


def sox_sigma(X: np.ndarray, V: np.ndarray, G: np.ndarray, route: str = "chain", taus=None,
              dtype=np.complex128) -> np.ndarray:
    """Bare SOX, SOX(v, v), for G in the library layout [n_spin][1][n_tau][n][n].

    Same-spin only (Sec. II C), so spin blocks are independent.  Returns the
    same layout (or [n_spin][1][len(taus)][n][n]).
    """
    X0, V0 = X[0], V[0]
    return np.stack([sigma_tau(X0, V0, V0, G[s, 0], route, taus, dtype)
                     for s in range(G.shape[0])])[:, None]


def sosex_static_sigma(X: np.ndarray, V: np.ndarray, W: np.ndarray, G: np.ndarray,
                       slot: int = 1, route: str = "chain", taus=None,
                       dtype=np.complex128) -> np.ndarray:
    """Statically screened SOSEX: SOX(U1 = W(0), U2 = v) for slot 1, SOX(v, W(0)) for slot 2.

    Sec. II B screens the first interaction; the G3W2 decomposition of Sec. III C
    writes SOSEX with W in the second slot, so both are offered.
    """
    X0, V0, W0 = X[0], V[0], W[0] if W.ndim == 3 else W
    U1, U2 = (W0, V0) if slot == 1 else (V0, W0)
    return np.stack([sigma_tau(X0, U1, U2, G[s, 0], route, taus, dtype)
                     for s in range(G.shape[0])])[:, None]


def g3w2_static_sigma(X: np.ndarray, W: np.ndarray, G: np.ndarray, route: str = "chain", taus=None,
                      dtype=np.complex128) -> np.ndarray:
    """G3W2 with static screening: both interactions screened, SOX(W(0), W(0)) (Sec. III C)."""
    return sox_sigma(X, W if W.ndim == 3 else W[None], G, route, taus, dtype)


def sosex2_static_sigma(X: np.ndarray, V: np.ndarray, W: np.ndarray, G: np.ndarray, route: str = "chain",
                        taus=None, dtype=np.complex128) -> np.ndarray:
    """2SOSEX with static screening, the paper's decomposition of Sec. III C with
    W_d = W(0) - v:  SOX(v, v) + SOX(v, W_d) + SOX(W_d, v)."""
    X0, V0 = X[0], V[0]
    W0 = W[0] if W.ndim == 3 else W
    Wd = W0 - V0
    out = []
    for s in range(G.shape[0]):
        terms = [sigma_tau(X0, U1, U2, G[s, 0], route, taus, dtype) for U1, U2 in ((V0, V0), (V0, Wd), (Wd, V0))]
        out.append(terms[0] + terms[1] + terms[2])
    return np.stack(out)[:, None]
