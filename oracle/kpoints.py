"""SOX self-energy of a periodic solid: the momentum-resolved forms (oracle).

Test infrastructure; see the package docstring.

Orbitals carry a momentum k (Sec. II A: G is block diagonal in k).  The THC
integrals of Sec. II C are

    (ij|sr) = sum_PQ (X^{k_i}_{iP})^* X^{k_j}_{jP} U^q_{PQ} (X^{k_s}_{sQ})^* X^{k_r}_{rQ},  q = k_i - k_j,

non-zero only when k_i - k_j = k_r - k_s.  Inserting them into Eq. (sox) with
the static time collapse leaves two free transfers q1 (of U1) and q2 (of U2):
for the external momentum k (k_t = k_r = k)

    Sigma^k_tr(tau) = -1/N_k^2 sum_{q1,q2} sum_{pqsuvw} U1^{q1}_(pr|qs) U2^{q2}_(tu|vw)
                       G^{k+q1}_wp(tau) G^{k-q2}_uq(tau) G^{k+q1-q2}_sv(-tau)

(the printed chain carries 1/N_k twice and garbled momentum labels; reading
both normalisations as one 1/N_k^2 and all labels as k - q with q = k_i - k_j
makes n_k = 1 the molecular formula and matches the brute force below).

Arrays: X[k][P][p] = X^k_{pP}, V[q][P][Q] = U^q_{PQ}, G[k][n][n] at one tau;
k labels are row-major integer triples of the mesh (``synth.kmesh``).
Three routes: brute force over block-diagonal "big" matrices, the pure-THC
form, and the paper's chain with mixed tensors U^{q,k}.
"""
from __future__ import annotations

import numpy as np

from . import grid


def _kadd(ks: np.ndarray, nk: tuple, a: int, b: int, sign: int = 1) -> int:
    m = np.mod(ks[a] + sign * ks[b], nk)
    return int((m[0] * nk[1] + m[1]) * nk[2] + m[2])


def k_tables(nk: tuple):
    """add[a][b] = index of k_a + k_b, sub[a][b] = index of k_a - k_b."""
    g = np.stack(np.meshgrid(*[np.arange(d) for d in nk], indexing="ij"), axis=-1).reshape(-1, 3)
    n = g.shape[0]
    add = np.array([[_kadd(g, nk, a, b, 1) for b in range(n)] for a in range(n)])
    sub = np.array([[_kadd(g, nk, a, b, -1) for b in range(n)] for a in range(n)])
    return add, sub


def eri_big(X: np.ndarray, U: np.ndarray, nk: tuple) -> np.ndarray:
    """4-index tensor over (k, orbital) with momentum conservation and the 1/N_k of a
    per-cell integral: v[(a,i),(b,j),(c,s),(d,r)] = (ij|sr) / N_k, q = k_a - k_b."""
    add, sub = k_tables(nk)
    n_k, N, n = X.shape
    v = np.zeros((n_k, n, n_k, n, n_k, n, n_k, n), dtype=complex)
    for a in range(n_k):
        for b in range(n_k):
            q = sub[a, b]
            left = np.einsum("Pi,Pj->ijP", X[a].conj(), X[b])
            for c in range(n_k):
                d = add[c, q]          # k_d - k_c = q  (k_r - k_s = k_i - k_j)
                right = np.einsum("Qs,Qr->srQ", X[c].conj(), X[d])
                v[a, :, b, :, c, :, d, :] = np.einsum("ijP,PQ,srQ->ijsr", left, U[q], right) / n_k
    nt = n_k * n
    return v.reshape(nt, nt, nt, nt)


def sigma_bruteforce(X, U1, U2, Gk, Gmk, nk):
    """Eq. (sox) over the big matrices; returns (Sigma^k blocks, the full big Sigma)."""
    from .sox import sigma_bruteforce as mol

    n_k, _, n = X.shape
    nt = n_k * n
    Gb = np.zeros((nt, nt), complex)
    Gmb = np.zeros((nt, nt), complex)
    for k in range(n_k):
        Gb[k * n:(k + 1) * n, k * n:(k + 1) * n] = Gk[k]
        Gmb[k * n:(k + 1) * n, k * n:(k + 1) * n] = Gmk[k]
    big = mol(eri_big(X, U1, nk), eri_big(X, U2, nk), Gb, Gmb)
    blocks = np.stack([big[k * n:(k + 1) * n, k * n:(k + 1) * n] for k in range(n_k)])
    return blocks, big


def _proj(Xa, G, Xb):
    """G^{AB} = sum_ab X_a[A][a] G[a][b] conj(X_b[B][b])."""
    return Xa @ G @ Xb.conj().T


def sigma_thc_direct(X, U1, U2, Gk, Gmk, nk):
    """Sigma^k_RP = -1/N_k^2 sum_{q1,q2} sum_QS U1^{q1}_PQ U2^{q2}_RS
                     G^{SP}(k+q1) G^{RQ}(k-q2) G^{QS}(k+q1-q2, -tau);  Sigma^k = X_k^H Sigma_RP X_k."""
    add, sub = k_tables(nk)
    n_k = X.shape[0]
    gp = [_proj(X[k], Gk[k], X[k]) for k in range(n_k)]
    gm = [_proj(X[k], Gmk[k], X[k]) for k in range(n_k)]
    out = []
    for k in range(n_k):
        S_RP = 0.0
        for q1 in range(n_k):
            kp = add[k, q1]
            for q2 in range(n_k):
                ku = sub[k, q2]
                ks = sub[kp, q2]
                M = np.einsum("RS,QS,SP->RQP", U2[q2], gm[ks], gp[kp], optimize=True)
                S_RP = S_RP - np.einsum("PQ,RQ,RQP->RP", U1[q1], gp[ku], M, optimize=True)
        S_RP = S_RP / n_k ** 2
        out.append(X[k].conj().T @ S_RP @ X[k])
    return np.stack(out)


def mixed_tensors(U, X, nk):
    """U^{q,k'}[P][a][b] = sum_Q U^q_PQ conj(X^{k'-q}_{aQ}) X^{k'}_{bQ}  for every (q, k')."""
    add, sub = k_tables(nk)
    n_k = X.shape[0]
    out = np.empty((n_k, n_k) + (X.shape[1], X.shape[2], X.shape[2]), complex)
    for q in range(n_k):
        for kk in range(n_k):
            out[q, kk] = np.einsum("PQ,Qa,Qb->Pab", U[q], X[sub[kk, q]].conj(), X[kk], optimize=True)
    return out


def sigma_chain(X, U1, U2, Gk, Gmk, nk, M1=None, M2=None, k_list=None):
    """The paper's THC-SOX algorithm for solids (Sec. II C): mixed tensors, projections,
    A, B per (q1, k_s), C per (q2, k_w), then the n_k^3 D step and back-projection.
    k_list restricts the output to those external momenta (all by default)."""
    add, sub = k_tables(nk)
    n_k, N, n = X.shape
    M1 = mixed_tensors(U1, X, nk) if M1 is None else M1
    M2 = mixed_tensors(U2, X, nk) if M2 is None else M2
    GR = np.stack([X[k] @ Gk[k] for k in range(n_k)])                    # G_Rq (k_u)
    GW = np.stack([Gk[k] @ X[k].conj().T for k in range(n_k)])           # G_wP (k_p)
    # B^{q1,k_s}_{PRv} and C^{q2,k_w}_{RvP}
    B = np.empty((n_k, n_k, N, N, n), complex)
    C = np.empty((n_k, n_k, N, n, N), complex)
    for q in range(n_k):
        for kk in range(n_k):
            A = np.einsum("Pqs,sv->Pqv", M1[q, kk], Gmk[kk], optimize=True)  # k_s = kk
            B[q, kk] = np.einsum("Pqv,Rq->PRv", A, GR[sub[kk, q]], optimize=True)  # k_q = k_s - q1
            C[q, kk] = np.einsum("Rvw,wP->RvP", M2[q, kk], GW[kk], optimize=True)  # k_w = kk
    out = []
    for k in (range(n_k) if k_list is None else k_list):
        D = 0.0
        for q1 in range(n_k):
            kw = add[k, q1]                        # k_w = k_p = k + q1
            for q2 in range(n_k):
                ks = sub[kw, q2]                   # k_s = k + q1 - q2
                D = D + np.einsum("RvP,PRv->PR", C[q2, kw], B[q1, ks], optimize=True)
        S_RP = -D.T / n_k ** 2
        out.append(X[k].conj().T @ S_RP @ X[k])
    return np.stack(out)


def sox_sigma(X, V, G, nk, route="chain", taus=None, U2=None, k_list=None):
    """Bare SOX (or SOX(V, U2)) for a solid, library layout G [n_spin][n_k][n_tau][n][n];
    k_list (chain route) restricts the output to those k."""
    U2 = V if U2 is None else U2
    n_spin, n_k, n_tau = G.shape[:3]
    idx = range(n_tau) if taus is None else taus
    n_out = n_k if k_list is None else len(k_list)
    res = np.empty((n_spin, n_out, len(list(idx)), G.shape[-1], G.shape[-1]), complex)
    M1 = mixed_tensors(V, X, nk) if route == "chain" else None
    M2 = (M1 if U2 is V else mixed_tensors(U2, X, nk)) if route == "chain" else None
    for s in range(n_spin):
        Gm = grid.g_minus_tau(np.asarray(G[s], complex))
        for o, j in enumerate(idx):
            Gk, Gmk = G[s][:, j], Gm[:, j]
            if route == "chain":
                res[s, :, o] = sigma_chain(X, V, U2, Gk, Gmk, nk, M1, M2, k_list)
            elif route == "direct":
                res[s, :, o] = sigma_thc_direct(X, V, U2, Gk, Gmk, nk)
            else:
                res[s, :, o] = sigma_bruteforce(X, V, U2, Gk, Gmk, nk)[0]
    return res


# ---------------------------------------------------------------------------
# Dynamically screened SOSEX for solids: W_d^{q1}(i Omega) in slot U(1), bare v
# in U(2), the convolution over the time of the W vertex taken through the
# caller's transform pair (Sec. II C, Eq. GG onward, with momenta).
# ---------------------------------------------------------------------------

def sigma_d_bruteforce(X, V, Wd, T_fwd, T_inv, G_tau, nk):
    """Definition over big matrices: momentum-conserving 4-index tensors for v and for every
    W_d(i Omega_m), block-diagonal G; returns Sigma_d^k [n_tau][n_k][n][n]."""
    n_k, N, n = X.shape
    nt = n_k * n
    T = G_tau.shape[1]
    Gm_tau = grid.g_minus_tau(np.asarray(G_tau, complex))   # [n_k][n_tau][n][n]: reflect tau
    def big(Gk):
        b = np.zeros((nt, nt), complex)
        for k in range(n_k):
            b[k * n:(k + 1) * n, k * n:(k + 1) * n] = Gk[k]
        return b
    Gb = np.stack([big(G_tau[:, j]) for j in range(T)])
    Gmb = np.stack([big(Gm_tau[:, j]) for j in range(T)])
    v2 = eri_big(X, V, nk)
    wd = np.stack([eri_big(X, Wd[:, m], nk) for m in range(Wd.shape[1])])
    F = np.einsum("mj,juq,jsv->muqsv", T_fwd, Gb, Gmb, optimize=True)
    conv = np.einsum("im,mprqs,muqsv->ipruv", T_inv, wd, F, optimize=True)
    sig = -np.einsum("tuvw,iwp,ipruv->itr", v2, Gb, conv, optimize=True)
    return np.stack([[sig[i, k * n:(k + 1) * n, k * n:(k + 1) * n] for k in range(n_k)] for i in range(T)])


def sigma_d_chain(X, V, Wd, T_fwd, T_inv, G_tau, nk):
    """The paper's dynamic algorithm with momenta, v outermost.  For every (q1, k_s):
    GG_Quv(tau_j) = G^{k_u}_uQ(tau_j) G^{k_s}_Qv(-tau_j) with k_u = k_s - q1, transform,
    A_Puv(i Omega) = sum_Q W_d^{q1}_PQ(i Omega) GG_Quv(i Omega), inverse transform,
    B_PRv(tau) = sum_u X^{k_u}_uR A_Puv(tau); C and the n_k^3 D step as in the static chain.
    Wd: [n_q][n_omega][N][N]; G_tau: [n_k][n_tau][n][n]; returns [n_tau][n_k][n][n]."""
    add, sub = k_tables(nk)
    n_k, N, n = X.shape
    T = G_tau.shape[1]
    Gm_tau = grid.g_minus_tau(np.asarray(G_tau, complex))   # [n_k][n_tau][n][n]: reflect tau
    M2 = mixed_tensors(V, X, nk)
    GuQ = np.einsum("kjuq,kQq->kjuQ", G_tau, X.conj())                  # G^{k}_uQ(tau_j)
    GQv = np.einsum("kQs,kjsv->kjQv", X, Gm_tau)                         # G^{k}_Qv(-tau_j)
    GwP = np.einsum("kjwp,kPp->kjwP", G_tau, X.conj())                   # G^{k}_wP(tau_i)
    D = np.zeros((T, n_k, N, N), complex)
    for v in range(n):
        B = np.empty((n_k, n_k, T, N, N), complex)
        C = np.empty((n_k, n_k, T, N, N), complex)
        for q in range(n_k):
            for ks in range(n_k):
                ku = sub[ks, q]
                GG = np.einsum("juQ,jQ->jQu", GuQ[ku], GQv[ks][:, :, v])
                GGw = np.einsum("mj,jQu->mQu", T_fwd, GG)
                Aw = np.einsum("mPQ,mQu->mPu", Wd[q], GGw)
                At = np.einsum("im,mPu->iPu", T_inv, Aw)
                B[q, ks] = np.einsum("iPu,Ru->iPR", At, X[ku])                  # B^{q1,ks}_PRv(tau_i)
                C[q, ks] = np.einsum("Rw,iwP->iPR", M2[q, ks][:, v, :], GwP[ks])  # C^{q2,kw}_RvP(tau_i)
        for k in range(n_k):
            for q1 in range(n_k):
                kw = add[k, q1]
                for q2 in range(n_k):
                    D[:, k] += C[q2, kw] * B[q1, sub[kw, q2]]
    out = np.empty((T, n_k, n, n), complex)
    for k in range(n_k):
        for i in range(T):
            out[i, k] = X[k].conj().T @ (-D[i, k].T / n_k ** 2) @ X[k]
    return out


def sosex_dynamic_sigma(X, V, Wd, T_fwd, T_inv, G, nk, route="chain"):
    """SOX(v, v) + Sigma_d for a solid, library layout G [n_spin][n_k][n_tau][n][n];
    Wd [n_q][n_omega][N][N]."""
    f = sigma_d_chain if route == "chain" else sigma_d_bruteforce
    stat = sox_sigma(X, V, G, nk)
    dyn = np.stack([f(X, V, Wd, T_fwd, T_inv, G[s], nk).transpose(1, 0, 2, 3) for s in range(G.shape[0])])
    return stat + dyn


def pi_omega(X, G_tau, T_fwd, nk):
    """Pi^q_PQ(i Omega_m) = 1/N_k sum_k sum_j T_fwd[m][j] G^{PQ}_{k+q, k}(tau_j) G^{QP}_{k, k+q}(-tau_j):
    the THC RPA bubble of transfer q, G^{PQ}_{a,b} = sum X^{a}[P][p] G^{a}[p][p'] conj(X^{a}[Q][p'])
    mixed with the momenta of the two propagators.  Used to build test inputs for the
    dynamic solid path."""
    add, sub = k_tables(nk)
    n_k = X.shape[0]
    Gm = grid.g_minus_tau(np.asarray(G_tau, complex))   # [n_k][n_tau][n][n]: reflect tau
    out = np.zeros((n_k, T_fwd.shape[0], X.shape[1], X.shape[1]), complex)
    for q in range(n_k):
        acc = 0.0
        for k in range(n_k):
            kq = add[k, q]
            a = np.einsum("Pp,jpr,Qr->jPQ", X[kq], G_tau[kq], X[kq].conj(), optimize=True)
            b = np.einsum("Qs,jst,Pt->jQP", X[k], Gm[k], X[k].conj(), optimize=True)
            acc = acc + a * np.transpose(b, (0, 2, 1))
        out[q] = np.einsum("mj,jPQ->mPQ", T_fwd, acc) / n_k
    return out


def pi_omega_pole_sum(X, eps, U, mu, beta, omegas, nk):
    """Exact bubble of transfer q at bosonic Omega for G^k(tau) = -U_k diag(e^{-xi tau}/(1+e^{-beta xi})) U_k^H:
    with y^k = X^k U_k and f^k_a = 1/(1 + e^{beta xi^k_a}),
        Pi^q_PQ(i Omega) = -1/N_k sum_k sum_ab y^{k+q}_Pa conj(y^{k+q}_Qa) y^k_Qb conj(y^k_Pb) c_ab,
        c_ab = (f^{k+q}_a - f^k_b) / (i Omega - xi^{k+q}_a + xi^k_b),
    (the k-resolved form of the molecular pole sum), with c_ab = beta f (1 - f) where Omega = 0
    and the two energies coincide."""
    add, _ = k_tables(nk)
    n_k = X.shape[0]
    xi = np.asarray(eps) - mu
    f = 0.5 * (1.0 - np.tanh(0.5 * beta * xi))
    y = np.einsum("kPp,kpa->kPa", X, U)
    out = np.zeros((n_k, len(omegas), X.shape[1], X.shape[1]), complex)
    for q in range(n_k):
        for k in range(n_k):
            kq = add[k, q]
            d = xi[kq][:, None] - xi[k][None, :]
            df = f[kq][:, None] - f[k][None, :]
            for m, om in enumerate(omegas):
                den = 1j * om - d
                same = np.abs(den) < 1e-12
                c = np.where(same, beta * f[kq][:, None] * (1.0 - f[kq][:, None]), df / np.where(same, 1.0, den))
                out[q, m] -= np.einsum("Pa,Qa,ab,Qb,Pb->PQ", y[kq], y[kq].conj(), c, y[k], y[k].conj(),
                                       optimize=True) / n_k
    return out


def w_dynamic(V, Pi_om):
    """W_d^q(i Omega_m) = W^q(i Omega_m) - V^q, W^q = V^q^1/2 (1 - V^q^1/2 Pi^q V^q^1/2)^-1 V^q^1/2
    per transfer q and frequency m (V^q Hermitian PSD).  Builds test inputs only."""
    from .screening import w_static

    return np.stack([np.stack([w_static(V[q], Pi_om[q, m]) - V[q] for m in range(Pi_om.shape[1])])
                     for q in range(V.shape[0])])
