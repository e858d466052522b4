"""Pins for the oracle's Pi(0) and W(i Omega = 0) (CPU only)."""
import numpy as np

import synth
from oracle import grid, screening


def _small_system(beta=2.0, n_tau=65, n=5, N=9, seed=4):
    rng = np.random.default_rng(seed)
    h, e, u = synth.random_hamiltonian(rng, n)
    mu = synth.half_filling_mu(e)
    tau = grid.chebyshev_lobatto(n_tau, beta)
    G = synth.green_tau(e, u, mu, tau, beta)
    X = rng.standard_normal((N, n)) / np.sqrt(n)
    return X, G, e, u, mu, tau


def test_pi0_quadrature_converges_to_pole_sum():
    beta = 2.0
    X, G, e, u, mu, tau = _small_system(beta=beta)
    wt = grid.clenshaw_curtis(tau.size, beta)
    quad = screening.pi0_quadrature(X, G, wt)
    exact = screening.pi0_pole_sum(X, e, u, mu, beta)
    assert np.abs(quad - exact).max() < 1e-12 * np.abs(exact).max()


def test_pi0_is_negative_semidefinite_and_symmetric():
    w = synth.config(0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    Pi = screening.pi0_quadrature(w.X[0], w.G[0, 0], wt)
    assert np.abs(Pi - Pi.T).max() < 1e-14 * np.abs(Pi).max()
    exact = screening.pi0_pole_sum(w.X[0], w.extras["eps"], w.extras["U"], w.extras["mu"], w.beta)
    assert np.linalg.eigvalsh(exact).max() <= 1e-12 * np.abs(exact).max()
    assert np.linalg.eigvalsh(Pi).max() <= 1e-3 * np.abs(Pi).max()


def test_w_static_push_through_identity_and_screening():
    w = synth.config(0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    V = w.V[0]
    Pi = screening.pi0_quadrature(w.X[0], w.G[0, 0], wt)
    Pi = 0.5 * (Pi + Pi.T)
    W = screening.w_static(V, Pi)
    # (1 - V Pi)^-1 V equals V^1/2 (1 - V^1/2 Pi V^1/2)^-1 V^1/2
    alt = np.linalg.solve(np.eye(w.N) - V @ Pi, V)
    assert np.abs(W - alt).max() < 1e-10 * np.abs(W).max()
    # screening: W <= V in the PSD order when Pi <= 0
    lam = np.linalg.eigvalsh(0.5 * ((V - W) + (V - W).T))
    assert lam.min() > -1e-10 * np.abs(V).max()
    # no polarisation -> no screening
    np.testing.assert_allclose(screening.w_static(V, np.zeros_like(V)), V, atol=1e-12 * np.abs(V).max())


def test_pi_omega_converges_to_pole_sum_at_every_frequency():
    """The bubble through the caller's transform equals the exact transform of the pole
    form at Omega_m = 2 pi m / beta, m = -3..3 (real, even in Omega)."""
    beta, M = 2.0, 3
    X, G, e, u, mu, tau = _small_system(beta=beta)
    om, Tf, _ = synth.bosonic_transforms(tau, beta, M)
    quad = screening.pi_omega(X, G, Tf)
    exact = screening.pi_omega_pole_sum(X, e, u, mu, beta, om)
    assert np.abs(quad - exact).max() < 1e-11 * np.abs(exact).max()
    assert np.abs(exact.imag).max() < 1e-13 * np.abs(exact).max()
    assert np.abs(exact - exact[::-1]).max() < 1e-13 * np.abs(exact).max()
    # a dropped transform sign or a misplaced reflection would break the nonzero rows
    assert np.abs(exact[0] - exact[M]).max() > 1e-3 * np.abs(exact).max()
