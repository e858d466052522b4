"""The self-consistent loop around Sigma for molecules (Sec. II A): the Dyson equation,
the chemical-potential update and the Galitskii-Migdal energies (oracle).

Test infrastructure; see the package docstring.

* Eqs. Dyson and G0: G(i w_n)^-1 = (i w_n + mu) S - H0 - Sigma[G](i w_n) on the fermionic
  Matsubara frequencies w_n = (2n+1) pi / beta, with S = 1 (orthonormal orbitals).
* Sigma[G] = Sigma_HF[gamma] + Sigma_dyn[G]: the static Hartree-Fock part from the
  correlated density matrix (Sec. II A prints gamma_pq = -G_qp(0^-), which gives negative
  occupations for G(tau) = -<T c(tau) c^+>; read gamma_pq = G_qp(0^-) = -G_qp(beta^-)) in THC form,
  and a dynamic part given in imaginary time (SOX, Eq. sox), carried to i w_n by the
  Fourier integral F(i w) = int_0^beta e^{i w tau} F(tau) d tau of its interpolant on the
  Chebyshev-Lobatto nodes.
* G(tau) = (1/beta) sum_n e^{-i w_n tau} G(i w_n): the first three terms of the
  high-frequency expansion G = 1/(iw) + c2/(iw)^2 + c3/(iw)^3 + ... are subtracted from
  the finite sum and added back through their closed-form tau images.
* mu is set at every iteration to the target electron count (Sec. II A); the iteration
  mixes old and new G linearly (the paper's CDIIS is out of scope).
* E_inf and E_dyn (Eqs. E1b and E2b), summed over spin blocks.
"""
from __future__ import annotations

import numpy as np

from . import grid


def fermionic_frequencies(beta: float, n_max: int) -> np.ndarray:
    """w_n = (2n+1) pi / beta for n = -n_max .. n_max-1 (a set closed under w -> -w)."""
    n = np.arange(-n_max, n_max)
    return (2 * n + 1) * np.pi / beta


def _cardinal(tau: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Values at the points s of the Lagrange cardinal polynomials L_j of the Chebyshev-Lobatto
    nodes tau (barycentric form, weights (-1)^j halved at the two ends); [len(s)][len(tau)]."""
    bw = np.array([(-1.0) ** j for j in range(tau.size)])
    bw[0] *= 0.5
    bw[-1] *= 0.5
    d = s[:, None] - tau[None, :]
    hit = np.abs(d) < 1e-300
    d = np.where(hit, 1.0, d)
    ratio = bw[None, :] / d
    L = ratio / ratio.sum(axis=1, keepdims=True)
    rows = hit.any(axis=1)
    L[rows] = hit[rows].astype(float)
    return L


def tau_to_iw(F_tau: np.ndarray, tau: np.ndarray, beta: float, omegas: np.ndarray, n_gl: int = 16,
              chunk: int = 64) -> np.ndarray:
    """F(i w) = int_0^beta e^{i w tau} F(tau) d tau of the interpolant of F_tau [n_tau, ...].

    Composite Gauss-Legendre with n_gl points per panel and at least two panels per period of
    the highest frequency, so the oscillatory integral is exact to rounding for the
    interpolant.  Returns [len(omegas), ...] complex."""
    wmax = float(np.abs(omegas).max()) if omegas.size else 0.0
    n_pan = max(8, int(np.ceil(wmax * beta / np.pi)) + 1)
    x, wg = np.polynomial.legendre.leggauss(n_gl)
    edges = np.linspace(0.0, beta, n_pan + 1)
    h = 0.5 * np.diff(edges)
    s = (edges[:-1, None] + h[:, None] * (x[None, :] + 1.0)).ravel()
    ws = (h[:, None] * wg[None, :]).ravel()
    L = _cardinal(tau, s)                                   # [n_s][n_tau]
    flat = F_tau.reshape(tau.size, -1)
    vals = L @ flat                                         # interpolant at the quadrature points
    out = np.empty((omegas.size, flat.shape[1]), complex)
    for a in range(0, omegas.size, chunk):
        E = np.exp(1j * omegas[a:a + chunk, None] * s[None, :]) * ws[None, :]
        out[a:a + chunk] = E @ vals
    return out.reshape((omegas.size,) + F_tau.shape[1:])


def tail_images(tau: np.ndarray, beta: float):
    """tau images on (0, beta) of 1/(iw), 1/(iw)^2, 1/(iw)^3 summed over all fermionic w_n:
    -1/2, (2 tau - beta)/4 and tau (beta - tau)/4 (their transforms give back the powers)."""
    t = np.asarray(tau, float)
    return -0.5 * np.ones_like(t), (2.0 * t - beta) / 4.0, t * (beta - t) / 4.0


def iw_to_tau(F_iw: np.ndarray, omegas: np.ndarray, tau: np.ndarray, beta: float, c1, c2, c3) -> np.ndarray:
    """F(tau) = (1/beta) sum_n e^{-i w_n tau} F(i w_n) for [len(omegas), n, n] with the tails
    c1/(iw) + c2/(iw)^2 + c3/(iw)^3 ([n, n] each) summed exactly; tau on [0, beta] with the end
    points read as 0^+ and beta^-.  Returns [len(tau), n, n] complex."""
    iw = (1j * omegas)[:, None, None]
    R = F_iw - c1[None] / iw - c2[None] / iw ** 2 - c3[None] / iw ** 3
    ph = np.exp(-1j * np.asarray(tau)[:, None] * omegas[None, :]) / beta
    t1, t2, t3 = tail_images(tau, beta)
    out = np.einsum("tw,wpq->tpq", ph, R)
    return out + t1[:, None, None] * c1[None] + t2[:, None, None] * c2[None] + t3[:, None, None] * c3[None]


def sigma_hf(X: np.ndarray, V: np.ndarray, gammas: np.ndarray) -> np.ndarray:
    """Hartree-Fock self-energy per spin block from the THC interaction
    (pq|rs) = sum_PQ X_Pp X_Pq V_PQ X_Qr X_Qs:  J_pq = sum_rs (pq|rs) rho_rs with rho the
    spin-summed density, K^s_pq = sum_rs (pr|sq) gamma^s_rs, Sigma_HF^s = J - K^s.
    X [N][n], V [N][N], gammas [n_spin][n][n] -> [n_spin][n][n]."""
    rho = gammas.sum(axis=0)
    d = np.einsum("Qr,Qs,rs->Q", X, X, rho)
    J = np.einsum("Pp,Pq,PQ,Q->pq", X, X, V, d)
    out = []
    for g in gammas:
        Gam = X @ g @ X.T                                   # Gam_PQ = sum_rs X_Pr g_rs X_Qs
        K = np.einsum("Pp,Qq,PQ,PQ->pq", X, X, V, Gam)
        out.append(J - K)
    return np.stack(out)


def dyson(omegas: np.ndarray, mu: float, F: np.ndarray, Sigma_iw: np.ndarray) -> np.ndarray:
    """G(i w_n) = [(i w_n + mu) 1 - F - Sigma(i w_n)]^-1 (Eqs. Dyson, G0 with S = 1 and the
    static part F = H0 + Sigma_HF); [n_w, n, n]."""
    n = F.shape[0]
    A = (1j * omegas + mu)[:, None, None] * np.eye(n)[None] - F[None] - Sigma_iw
    return np.linalg.inv(A)


def green_tails(F: np.ndarray, mu: float, Sigma_tau: np.ndarray):
    """High-frequency coefficients of G = [iw - (F - mu) - Sigma(iw)]^-1:
    c1 = 1, c2 = F - mu, c3 = (F - mu)^2 + Sigma_1 with Sigma(iw) ~ Sigma_1 / (iw) and
    Sigma_1 = -(Sigma(beta^-) + Sigma(0^+)) (the jump of the antiperiodic Sigma(tau))."""
    n = F.shape[0]
    A = F - mu * np.eye(n)
    S1 = -(Sigma_tau[-1] + Sigma_tau[0])
    return np.eye(n, dtype=complex), A.astype(complex), (A @ A + S1).astype(complex)


class LoopState:
    """Converged (or last) iterate: G(tau) [n_spin][n_tau][n][n], mu, gamma, Sigma_HF,
    Sigma_dyn(tau), Sigma_dyn(i w), G(i w), the iteration count and the last change."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def _gamma_at(omegas, tau_end, beta, mu, F, S_iw, S_tau):
    G_iw = dyson(omegas, mu, F, S_iw)
    c1, c2, c3 = green_tails(F, mu, S_tau)
    Gb = iw_to_tau(G_iw, omegas, np.array([tau_end]), beta, c1, c2, c3)[0]
    return -Gb.real.T                                        # gamma_pq = -G_qp(beta^-)


def find_mu(omegas, beta, target, Fs, S_iws, S_taus, lo=-50.0, hi=50.0, iters=200, tol=1e-13):
    """mu with sum_s Tr gamma^s(mu) = target by bisection (the count rises with mu)."""
    def count(mu):
        return sum(np.trace(_gamma_at(omegas, beta, beta, mu, F, Si, St)) for F, Si, St in zip(Fs, S_iws, S_taus))

    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if count(mid) < target:
            lo = mid
        else:
            hi = mid
        if hi - lo < tol:
            break
    return 0.5 * (lo + hi)


def sc_loop(H0: np.ndarray, X: np.ndarray, V: np.ndarray, beta: float, n_tau: int, n_elec: float,
            sigma_dyn, n_spin: int = 2, n_max: int = 1000, mix: float = 0.5, max_iter: int = 200,
            tol: float = 1e-10, G_start: np.ndarray | None = None) -> LoopState:
    """Fixed point G = G[Sigma_HF[gamma(G)] + sigma_dyn(G)] at the target electron count.

    sigma_dyn(G_tau [n_spin][n_tau][n][n]) -> Sigma_dyn(tau) of the same layout (pass a
    function returning zeros for Hartree-Fock alone).  The start is G0 of H0 at its own mu
    unless G_start is given."""
    tau = grid.chebyshev_lobatto(n_tau, beta)
    om = fermionic_frequencies(beta, n_max)
    n = H0.shape[0]
    zeros_t = np.zeros((n_tau, n, n))
    zeros_w = np.zeros((om.size, n, n), complex)
    if G_start is None:
        mu0 = find_mu(om, beta, n_elec, [H0] * n_spin, [zeros_w] * n_spin, [zeros_t] * n_spin)
        G_tau = np.stack([_g_tau(om, tau, beta, mu0, H0, zeros_w, zeros_t) for _ in range(n_spin)])
    else:
        G_tau = np.array(G_start, dtype=float)
    change = np.inf
    for it in range(1, max_iter + 1):
        gammas = np.stack([-g[-1].T for g in G_tau])           # gamma_pq = -G_qp(beta^-)
        S_hf = sigma_hf(X, V, gammas)
        S_tau = np.asarray(sigma_dyn(G_tau), dtype=float)
        S_iw = [tau_to_iw(S_tau[s], tau, beta, om) for s in range(n_spin)]
        Fs = [H0 + S_hf[s] for s in range(n_spin)]
        mu = find_mu(om, beta, n_elec, Fs, S_iw, list(S_tau))
        new = np.stack([_g_tau(om, tau, beta, mu, Fs[s], S_iw[s], S_tau[s]) for s in range(n_spin)])
        change = float(np.abs(new - G_tau).max())
        G_tau = (1.0 - mix) * G_tau + mix * new
        if change < tol:
            G_tau = new
            break
    gammas = np.stack([-g[-1].T for g in G_tau])
    S_hf = sigma_hf(X, V, gammas)
    S_tau = np.asarray(sigma_dyn(G_tau), dtype=float)
    S_iw = np.stack([tau_to_iw(S_tau[s], tau, beta, om) for s in range(n_spin)])
    Fs = [H0 + S_hf[s] for s in range(n_spin)]
    G_iw = np.stack([dyson(om, mu, Fs[s], S_iw[s]) for s in range(n_spin)])
    return LoopState(G_tau=G_tau, mu=mu, gamma=gammas, sigma_hf=S_hf, sigma_tau=S_tau, sigma_iw=S_iw,
                     G_iw=G_iw, omegas=om, tau=tau, beta=beta, iterations=it, change=change)


def _g_tau(om, tau, beta, mu, F, S_iw, S_tau):
    G_iw = dyson(om, mu, F, S_iw)
    c1, c2, c3 = green_tails(F, mu, S_tau)
    return iw_to_tau(G_iw, om, tau, beta, c1, c2, c3).real


def energy_inf(H0: np.ndarray, st: LoopState) -> float:
    """E_inf = sum_s sum_pq (h_pq + Sigma_HF^s_pq / 2) gamma^s_pq (Eq. E1b, h = H0)."""
    return float(sum(np.sum((H0 + 0.5 * st.sigma_hf[s]) * st.gamma[s]) for s in range(st.gamma.shape[0])))


def energy_dyn_matsubara(st: LoopState) -> float:
    """E_dyn = (1/beta) sum_n sum_s sum_pq G^s_qp(i w_n) Sigma^s_pq(i w_n) (Eq. E2b): the
    finite sum plus the exact sum of its leading tail Tr[Sigma_1] / (iw)^2 (value -beta/4)."""
    beta, om = st.beta, st.omegas
    total = 0.0
    for s in range(st.G_iw.shape[0]):
        tr = np.einsum("wpq,wqp->w", st.sigma_iw[s], st.G_iw[s])
        S1 = -(st.sigma_tau[s][-1] + st.sigma_tau[s][0])
        lead = np.trace(S1) / (1j * om) ** 2
        total += float(((tr - lead).sum() / beta).real + np.trace(S1).real * (-beta / 4.0))
    return total


def energy_dyn_tau(st: LoopState) -> float:
    """The same energy in imaginary time: E_dyn = sum_s int_0^beta Tr[Sigma^s(-tau) G^s(tau)] d tau
    = -sum_s sum_j w_j Tr[Sigma^s(tau_{n-1-j}) G^s(tau_j)] (Clenshaw-Curtis, symmetric grid)."""
    w = grid.clenshaw_curtis(st.tau.size, st.beta)
    total = 0.0
    for s in range(st.G_tau.shape[0]):
        total -= float(np.einsum("j,jpq,jqp->", w, st.sigma_tau[s][::-1], st.G_tau[s]))
    return total
