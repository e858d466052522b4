"""Pins for the oracle's tau grid, quadrature and fermionic reflection (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import grid


@pytest.mark.parametrize("n_tau", [2, 3, 5, 8, 31])
def test_nodes_symmetric_and_match_generator(n_tau):
    beta = 7.5
    t = grid.chebyshev_lobatto(n_tau, beta)
    assert t[0] == 0.0 and abs(t[-1] - beta) < 1e-14
    np.testing.assert_allclose(t[::-1], beta - t, atol=1e-13)
    np.testing.assert_allclose(synth.tau_nodes(n_tau, beta), t, atol=1e-13)


def test_clenshaw_curtis_textbook_values():
    # On [-1, 1]: 3 nodes -> Simpson (1/3, 4/3, 1/3); 5 nodes -> (1, 8, 12, 8, 1)/15.
    # tau = (beta/2)(1 - x), so beta = 2 reproduces the [-1, 1] weights.
    np.testing.assert_allclose(grid.clenshaw_curtis(3, 2.0), [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    np.testing.assert_allclose(grid.clenshaw_curtis(5, 2.0), np.array([1, 8, 12, 8, 1]) / 15, atol=1e-15)


@pytest.mark.parametrize("n_tau", [4, 9, 30])
def test_clenshaw_curtis_exact_on_polynomials(n_tau):
    beta = 3.0
    t = grid.chebyshev_lobatto(n_tau, beta)
    w = grid.clenshaw_curtis(n_tau, beta)
    for k in range(n_tau):
        exact = beta ** (k + 1) / (k + 1)
        assert abs(np.dot(w, t ** k) - exact) <= 1e-12 * exact
    np.testing.assert_allclose(w, w[::-1], atol=1e-15)


def test_clenshaw_curtis_converges_on_exponential():
    beta, a = 10.0, 1.3
    exact = (1 - np.exp(-a * beta)) / a
    err = [abs(np.dot(grid.clenshaw_curtis(n, beta), np.exp(-a * grid.chebyshev_lobatto(n, beta))) - exact)
           for n in (9, 17, 33, 65)]
    assert err[-1] < 1e-13 and err[0] > err[-1]


def test_reflection_matches_pole_form_of_g_minus_tau():
    # G(-tau) for G = -U diag(e^{-xi tau}(1 - f)) U^T is +U diag(e^{xi tau} f) U^T
    # (f the Fermi occupation); the oracle's reflection -G(beta - tau) must agree.
    rng = np.random.default_rng(3)
    n, beta, n_tau = 6, 9.0, 13
    h, e, u = synth.random_hamiltonian(rng, n)
    mu = 0.1
    tau = grid.chebyshev_lobatto(n_tau, beta)
    G = synth.green_tau(e, u, mu, tau, beta)
    xi = e - mu
    f = 1.0 / (1.0 + np.exp(beta * xi))
    direct = np.einsum("pa,ja,qa->jpq", u, f[None, :] * np.exp(xi[None, :] * tau[:, None]), u)
    np.testing.assert_allclose(grid.g_minus_tau(G), direct, atol=1e-13)
    # and G(0+) - G(0-) = -1 (fermionic jump)
    np.testing.assert_allclose(G[0] - direct[0], -np.eye(n), atol=1e-13)
