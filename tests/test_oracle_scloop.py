"""Pins for the oracle's self-consistent loop (Dyson equation, chemical potential,
Galitskii-Migdal energies), CPU only."""
import numpy as np
import pytest

import synth
from oracle import grid, phi, scloop, sox


@pytest.mark.parametrize("xi", [-1.3, 0.7])
def test_fermionic_transform_pair_on_a_pole(xi):
    """g(tau) = -e^{-xi tau}/(1+e^{-beta xi}) has g(i w) = 1/(i w - xi) exactly; its tails are
    1, xi, xi^2.  Forward through the interpolant, back through the tail-corrected sum."""
    beta = 4.0
    tau = grid.chebyshev_lobatto(65, beta)
    om = scloop.fermionic_frequencies(beta, 2000)
    g_tau = -np.exp(-xi * tau) / (1.0 + np.exp(-beta * xi))
    g_iw = 1.0 / (1j * om - xi)
    low = np.abs(om) < 100.0
    fwd = scloop.tau_to_iw(g_tau, tau, beta, om[low])
    assert np.abs(fwd - g_iw[low]).max() < 1e-12
    one = np.eye(1)
    back = scloop.iw_to_tau(g_iw[:, None, None], om, tau, beta, one, xi * one, xi ** 2 * one)[:, 0, 0]
    err = np.abs(back - g_tau).max()
    assert err < 1e-9
    # the third tail term matters: without it the error is orders of magnitude larger
    worse = scloop.iw_to_tau(g_iw[:, None, None], om, tau, beta, one, xi * one, 0 * one)[:, 0, 0]
    assert np.abs(worse - g_tau).max() > 100 * err


def test_tail_images_transform_back_to_their_powers():
    beta = 3.0
    tau = grid.chebyshev_lobatto(41, beta)
    om = scloop.fermionic_frequencies(beta, 5)
    for k, img in enumerate(scloop.tail_images(tau, beta), start=1):
        got = scloop.tau_to_iw(img, tau, beta, om)
        assert np.abs(got - 1.0 / (1j * om) ** k).max() < 1e-12


def test_hartree_fock_matches_the_four_index_contraction():
    rng = np.random.default_rng(3)
    n, N = 4, 9
    X = rng.standard_normal((N, n)) / np.sqrt(n)
    Z = rng.standard_normal((N, N)) / N
    V = Z @ Z.T
    gam = rng.standard_normal((2, n, n))
    gam = 0.5 * (gam + np.swapaxes(gam, 1, 2))
    v = np.einsum("Pp,Pq,PQ,Qr,Qs->pqrs", X, X, V, X, X)    # (pq|rs)
    J = np.einsum("pqrs,rs->pq", v, gam.sum(axis=0))
    for s in range(2):
        K = np.einsum("prsq,rs->pq", v, gam[s])
        assert np.abs(scloop.sigma_hf(X, V, gam)[s] - (J - K)).max() < 1e-13 * np.abs(J).max()


def _molecule(n=4, N=10, beta=4.0, scale=0.6, seed=11):
    rng = np.random.default_rng(seed)
    h, _, _ = synth.random_hamiltonian(rng, n)
    X = rng.standard_normal((N, n)) / np.sqrt(n)
    Z = rng.standard_normal((N, N)) / N
    V = scale * (Z @ Z.T)
    return h, X, V, beta


def test_hartree_fock_loop_reaches_the_pole_form_of_its_fock_matrix():
    """With no dynamic part the fixed point is self-consistent Hartree-Fock: G(tau) is the
    pole form of F = H0 + Sigma_HF[gamma] at the converged mu, and the count is the target."""
    h, X, V, beta = _molecule()
    n, n_tau, n_elec = h.shape[0], 33, 4.0
    st = scloop.sc_loop(h, X, V, beta, n_tau, n_elec, lambda G: np.zeros_like(G), n_max=400, tol=1e-11)
    assert st.change < 1e-10
    assert abs(sum(np.trace(g) for g in st.gamma) - n_elec) < 1e-9
    for s in range(2):
        eps, U = np.linalg.eigh(h + st.sigma_hf[s])
        exact = synth.green_tau(eps, U, st.mu, st.tau, beta)
        assert np.abs(st.G_tau[s] - exact).max() < 1e-7
        # fermionic jump: G(0+) + G(beta-) = -1
        assert np.abs(st.G_tau[s][0] + st.G_tau[s][-1] + np.eye(n)).max() < 1e-7


def test_sox_loop_is_conserving_and_its_energies_agree():
    """SOX as the dynamic part: at the fixed point the count is the target, E_dyn through the
    Matsubara sum equals E_dyn through the tau trace, and that equals 4 sum_s Phi_s computed
    by the independent pure-THC form of Phi."""
    h, X, V, beta = _molecule()
    n, n_tau, n_elec = h.shape[0], 33, 4.0

    def sigma_sox(G):
        return sox.sox_sigma(X[None], V[None], G[:, None], dtype=np.float64)[:, 0].real

    st = scloop.sc_loop(h, X, V, beta, n_tau, n_elec, sigma_sox, n_max=400, tol=1e-10)
    assert st.change < 1e-9
    assert abs(sum(np.trace(g) for g in st.gamma) - n_elec) < 1e-9
    e_w = scloop.energy_dyn_matsubara(st)
    e_t = scloop.energy_dyn_tau(st)
    assert abs(e_t) > 1e-6                                   # the dynamic part is not empty
    assert abs(e_w - e_t) < 1e-6 * abs(e_t)
    w = grid.clenshaw_curtis(n_tau, beta)
    phis = sum(phi.phi_thc_direct(X, V, V, st.G_tau[s], w).real for s in range(2))
    assert abs(e_t - 4.0 * phis) < 1e-10 * abs(e_t)
    # the fixed point: the Dyson residual vanishes on every frequency
    for s in range(2):
        F = h + st.sigma_hf[s]
        A = (1j * st.omegas + st.mu)[:, None, None] * np.eye(n) - F - st.sigma_iw[s]
        assert np.abs(np.einsum("wpq,wqr->wpr", A, st.G_iw[s]) - np.eye(n)).max() < 1e-10
    # E_inf is the one-body energy plus half the Hartree-Fock interaction
    e_inf = scloop.energy_inf(h, st)
    direct = sum(np.sum(h * st.gamma[s]) + 0.5 * np.sum(st.sigma_hf[s] * st.gamma[s]) for s in range(2))
    assert abs(e_inf - direct) < 1e-12 * abs(direct)
