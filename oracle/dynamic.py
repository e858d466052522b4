"""Dynamically screened SOSEX (oracle, molecules).  Test infrastructure.

Sec. II C, Eq. GG and the steps after it: with a frequency-dependent first
interaction W(tau) the times no longer collapse.  With the screened part
W_d = W - v (the static v part is SOX(v, v), Sec. III C) in slot U(1),

    Sigma_d,tr(tau) = - sum v_(tu|vw) G_wp(tau) int_0^beta ds W_d,(pr|qs)(tau - s) G_uq(s) G_sv(-s)

and the convolution is taken through bosonic frequencies with the caller's
transform pair: conv(tau_i) = sum_m T_inv[i][m] W_d(i Omega_m) sum_j T_fwd[m][j] (.)(tau_j).

Two routes: ``sigma_d_bruteforce`` (4-index tensors, tiny sizes) and
``sigma_d_chain`` (the paper's algorithm with v in the outer loop: GG, FT,
W_d GEMM, IFT, B, C, D, back-projection).
"""
from __future__ import annotations

import numpy as np

from . import grid, sox, thc


def sigma_d_bruteforce(X, V, Wd, T_fwd, T_inv, G_tau):
    """Definition over 4-index tensors for one spin block; returns Sigma_d [n_tau][n][n]."""
    Gm_tau = grid.g_minus_tau(G_tau)
    v2 = thc.eri(X, X, V, X, X)                                   # v_(tu|vw)
    wd = np.stack([thc.eri(X, X, Wd[m], X, X) for m in range(Wd.shape[0])])   # W_d,m (pr|qs)
    # F[m][u,q,s,v] = sum_j T_fwd[m][j] G_uq(tau_j) G_sv(-tau_j)
    F = np.einsum("mj,juq,jsv->muqsv", T_fwd, G_tau, Gm_tau, optimize=True)
    # conv[i][p,r,u,v] = sum_m T_inv[i][m] sum_{q,s} W_d,m(pr|qs) F[m][u,q,s,v]
    conv = np.einsum("im,mprqs,muqsv->ipruv", T_inv, wd, F, optimize=True)
    return -np.einsum("tuvw,iwp,ipruv->itr", v2, G_tau, conv, optimize=True)


def sigma_d_chain(X, V, Wd, T_fwd, T_inv, G_tau):
    """The paper's dynamic THC algorithm (Sec. II C), v outermost, one spin block."""
    Gm_tau = grid.g_minus_tau(G_tau)
    n_tau, n = G_tau.shape[0], G_tau.shape[1]
    U2 = sox.mixed_tensor(V, X)                                    # U(2)_Rvw
    G_uQ = np.einsum("juq,Qq->juQ", G_tau, X)                      # sum_q G_uq X_qQ
    G_Qv = np.einsum("Qs,jsv->jQv", X, Gm_tau)                     # sum_s X_sQ G_sv(-tau)
    G_wP = np.einsum("jwp,Pp->jwP", G_tau, X)                      # sum_p G_wp X_pP
    D = 0.0
    for v in range(n):
        GG = np.einsum("juQ,jQ->jQu", G_uQ, G_Qv[:, :, v])         # GG_Quv(tau_j)
        GGw = np.einsum("mj,jQu->mQu", T_fwd, GG)                  # FT
        Aw = np.einsum("mPQ,mQu->mPu", Wd, GGw)                    # A_Puv(i Omega_m)
        At = np.einsum("im,mPu->iPu", T_inv, Aw)                   # IFT
        B = np.einsum("iPu,uR->iPR", At, X.T)                      # B_PRv(tau_i) = sum_u X_uR A_Puv
        C = np.einsum("Rw,iwP->iPR", U2[:, v, :], G_wP)            # C_RvP(tau_i), stored [i][P][R]
        D = D + B * C
    sig_RP = -np.transpose(D, (0, 2, 1))
    return np.einsum("Rt,iRP,Pr->itr", X, sig_RP, X)


def sosex_dynamic_sigma(X, V, Wd, T_fwd, T_inv, G, route="chain"):
    """SOX(v, v) + Sigma_d in the library layout G [n_spin][1][n_tau][n][n] (complex128)."""
    f = sigma_d_chain if route == "chain" else sigma_d_bruteforce
    stat = sox.sox_sigma(X, V, G)
    dyn = np.stack([f(X[0].astype(complex), V[0].astype(complex), Wd.astype(complex), T_fwd, T_inv,
                      G[s, 0].astype(complex)) for s in range(G.shape[0])])[:, None]
    return stat + dyn
