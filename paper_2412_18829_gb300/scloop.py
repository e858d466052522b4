"""The self-consistent loop around Sigma for molecules (Sec. II A), driven on the GPU.

Every arithmetic step is a library call: the density matrix gamma = G(0^-) from G(tau), the
Hartree-Fock self-energy and the Fock matrix F = H0 + Sigma_HF[gamma] (THC form), the
dynamic self-energy Sigma[G](tau) (bare SOX, Eq. sox), its transform to the fermionic
Matsubara frequencies, the chemical potential for the target electron count, the Dyson
equation on every frequency, the tail-corrected return to imaginary time and the linear
mixing of the iteration; this module only sequences them.  The paper's CDIIS accelerator
is not part of the library (linear mixing stands in for it).
"""
from __future__ import annotations

from dataclasses import dataclass

from . import _binding as b


@dataclass
class LoopResult:
    G_tau: object         # [n_spin][n_tau][n][n]
    mu: float
    gamma: object         # [n_spin][n][n]
    sigma_hf: object      # [n_spin][n][n]
    sigma_tau: object     # [n_spin][n_tau][n][n] (dynamic part)
    iterations: int
    change: float
    energies: object      # [2]: E_inf, E_dyn


def run(h: b.Handle, p: b.sox_problem, H0, X, V, n_elec: float, omegas, T_w, tau, w, dynamic: bool = True,
        mix: float = 0.5, tol: float = 1e-10, max_iter: int = 200, mu_bounds=(-50.0, 50.0), stream=None):
    """Fixed point G = G[Sigma_HF[gamma(G)] + Sigma_SOX[G]] at the target electron count.

    Device tensors (torch, FP64): H0 [n][n], X [1][N][n], V [1][N][N], omegas [n_w] (fermionic),
    T_w [n_w][n_tau] complex (the tau -> i w transform of the grid), tau and w [n_tau] (the
    mirror-symmetric grid and its weights).  dynamic=False runs Hartree-Fock alone.  The
    start is G0 of H0 at its own mu."""
    import torch

    n, S, T = p.n, p.n_spin, p.n_tau
    dev = H0.device
    f64 = dict(dtype=torch.float64, device=dev)
    F = torch.empty(S, n, n, **f64)
    for s in range(S):
        F[s].copy_(H0)
    Siw = torch.zeros(S, omegas.shape[0], n, n, dtype=torch.complex128, device=dev)
    Giw = torch.empty_like(Siw)
    Stau = torch.zeros(S, T, n, n, **f64)
    tails = torch.empty(S, 3, n, n, **f64)
    gamma = torch.empty(S, n, n, **f64)
    Shf = torch.empty(S, n, n, **f64)
    G = torch.empty(S, T, n, n, **f64)
    Gnew = torch.empty_like(G)
    lo, hi = mu_bounds

    def green(mu_, Fm, Si, St, out):
        b.sox_dyson(h, p, omegas, mu_, Fm, Si, Giw, stream)
        b.sox_green_tails(h, p, mu_, Fm, St, tails, stream)
        b.sox_iw_to_tau(h, p, omegas, Giw, tails, tau, out, stream)

    mu = b.sox_find_mu(h, p, omegas, n_elec, F, None, None, lo, hi)
    green(mu, F, None, None, G)
    change = float("inf")
    it = 0
    for it in range(1, max_iter + 1):
        b.sox_density_matrix(h, p, G, gamma, stream)
        b.sox_sigma_hf(h, p, X, V, gamma, Shf, H0=H0, F=F, stream=stream)
        if dynamic:
            b.sox_sigma(h, p, G, X, V, Stau, stream)   # layout [n_spin][1][n_tau][n][n]
            b.sox_tau_to_iw(h, p, T_w, Stau, Siw, stream)
        mu = b.sox_find_mu(h, p, omegas, n_elec, F, Siw if dynamic else None, Stau if dynamic else None, lo, hi)
        green(mu, F, Siw if dynamic else None, Stau if dynamic else None, Gnew)
        change = b.sox_mix_green(h, G, Gnew, mix, stream)
        if change < tol:
            G.copy_(Gnew)
            break
    # the final iterate's parts and energies (Eqs. E1b, E2b)
    b.sox_density_matrix(h, p, G, gamma, stream)
    b.sox_sigma_hf(h, p, X, V, gamma, Shf, H0=H0, F=F, stream=stream)
    if dynamic:
        b.sox_sigma(h, p, G, X, V, Stau, stream)
    E = torch.empty(2, **f64)
    b.sox_gm_energies(h, p, H0, Shf, gamma, Stau, G, w, E, stream)
    return LoopResult(G_tau=G, mu=mu, gamma=gamma, sigma_hf=Shf, sigma_tau=Stau, iterations=it, change=change,
                      energies=E)

