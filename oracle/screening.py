"""Static screening for SOSEX-stat (oracle, molecules).  Test infrastructure.

Sec. II B: statically screened SOSEX replaces the first bare interaction by the
screened interaction at zero bosonic frequency, W(i Omega = 0).  The RPA form
used by the statically screened workload is

    Pi_PQ(0) = sum_j w_j G^PQ(tau_j) G^QP(-tau_j)          (quadrature of int_0^beta)
    W        = V^1/2 (1 - V^1/2 Pi(0) V^1/2)^-1 V^1/2

with G^PQ = X G X^T.  The printed Pi(0) carries an extra minus sign; with the
sign above Pi(0) is negative semidefinite and W <= V (screening).
"""
from __future__ import annotations

import numpy as np

from . import grid, thc


def pi0_quadrature(X: np.ndarray, G_tau: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Pi_PQ(0) = sum_j w_j G^PQ(tau_j) G^QP(-tau_j) for one spin block G_tau [n_tau, n, n]."""
    Gm_tau = grid.g_minus_tau(G_tau)
    Pi = np.zeros((X.shape[0], X.shape[0]), dtype=np.result_type(X, G_tau))
    for j in range(G_tau.shape[0]):
        gp = thc.project_full(X, G_tau[j])
        gm = thc.project_full(X, Gm_tau[j])
        Pi += w[j] * gp * gm.T
    return Pi


def pi0_pole_sum(X: np.ndarray, eps: np.ndarray, U: np.ndarray, mu: float, beta: float) -> np.ndarray:
    """Exact int_0^beta G^PQ(tau) G^QP(-tau) d tau for G = -U diag(e^{-xi tau}/(1+e^{-beta xi})) U^T.

    With y = X U and occupations f_a = 1/(1 + e^{beta xi_a}) the integral is
        Pi_PQ = -sum_ab y_Pa y_Qa y_Pb y_Qb (f_b - f_a)/(xi_a - xi_b),
    whose diagonal limit (xi_a = xi_b) is beta f_a (1 - f_a).
    """
    xi = eps - mu
    f = 0.5 * (1.0 - np.tanh(0.5 * beta * xi))
    d = xi[:, None] - xi[None, :]
    same = np.abs(d) < 1e-12
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.where(same, beta * f[:, None] * (1.0 - f[:, None]), (f[None, :] - f[:, None]) / np.where(same, 1.0, d))
    y = X @ U
    return -np.einsum("Pa,Qa,ab,Pb,Qb->PQ", y, y, c, y, y, optimize=True)


def pi_omega_pole_sum(X: np.ndarray, eps: np.ndarray, U: np.ndarray, mu: float, beta: float,
                      omegas: np.ndarray) -> np.ndarray:
    """Exact int_0^beta e^{i Omega tau} G^PQ(tau) G^QP(-tau) d tau at bosonic Omega_m for
    G = -U diag(e^{-xi tau}/(1+e^{-beta xi})) U^T.

    With y = X U and f_a = 1/(1 + e^{beta xi_a}), G^PQ(tau) = -sum_a y_Pa y_Qa (1-f_a) e^{-xi_a tau}
    and G^QP(-tau) = sum_b y_Qb y_Pb f_b e^{xi_b tau}; since e^{i Omega beta} = 1 and
    (1-f_a) f_b (e^{beta (xi_b - xi_a)} - 1) = f_a - f_b the integral is
        Pi_PQ(i Omega) = -sum_ab y_Pa y_Qa y_Pb y_Qb (f_a - f_b) / (i Omega - xi_a + xi_b),
    the a = b terms vanishing for Omega != 0 and giving pi0_pole_sum's limit at Omega = 0.
    """
    xi = eps - mu
    f = 0.5 * (1.0 - np.tanh(0.5 * beta * xi))
    y = X @ U
    out = []
    for om in np.atleast_1d(omegas):
        if om == 0.0:
            out.append(pi0_pole_sum(X, eps, U, mu, beta).astype(complex))
            continue
        c = (f[:, None] - f[None, :]) / (1j * om - xi[:, None] + xi[None, :])
        out.append(-np.einsum("Pa,Qa,ab,Pb,Qb->PQ", y, y, c, y, y, optimize=True))
    return np.stack(out)


def w_static(V: np.ndarray, Pi: np.ndarray) -> np.ndarray:
    """W = V^1/2 (1 - V^1/2 Pi V^1/2)^-1 V^1/2 with V^1/2 from the eigendecomposition of V."""
    lam, Q = np.linalg.eigh(V)
    s = np.sqrt(np.clip(lam, 0.0, None))
    Vh = (Q * s) @ Q.conj().T
    K = np.eye(V.shape[0]) - Vh @ Pi @ Vh
    return Vh @ np.linalg.solve(K, Vh)


def pi_omega(X: np.ndarray, G_tau: np.ndarray, T_fwd: np.ndarray) -> np.ndarray:
    """Pi_PQ(i Omega_m) = sum_j T_fwd[m][j] G^PQ(tau_j) G^QP(-tau_j): the transform of the
    bosonic polarisability Pi(tau) = G^PQ(tau) G^QP(-tau) (THC form of the RPA bubble)."""
    Gm_tau = grid.g_minus_tau(G_tau)
    pit = np.stack([thc.project_full(X, G_tau[j]) * thc.project_full(X, Gm_tau[j]).T
                    for j in range(G_tau.shape[0])])
    return np.einsum("mj,jPQ->mPQ", T_fwd, pit)


def w_dynamic(V: np.ndarray, Pi_om: np.ndarray) -> np.ndarray:
    """W_d(i Omega_m) = W(i Omega_m) - V with W = V^1/2 (1 - V^1/2 Pi V^1/2)^-1 V^1/2 per m;
    real for a real molecule (Pi(i Omega) is real and even in Omega)."""
    out = []
    for m in range(Pi_om.shape[0]):
        P = Pi_om[m].real
        out.append(w_static(V, 0.5 * (P + P.T)) - V)
    return np.stack(out)
