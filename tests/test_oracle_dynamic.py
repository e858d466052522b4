"""Pins for the oracle's dynamically screened SOSEX and its transforms (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import dynamic, grid, screening, sox, thc


def test_zero_frequency_row_is_clenshaw_curtis():
    tau = synth.tau_nodes(17, 7.0)
    _, Tf, _ = synth.bosonic_transforms(tau, 7.0, 4)
    # the integral of the Chebyshev-Lobatto interpolant is the Clenshaw-Curtis rule
    np.testing.assert_allclose(Tf[4], grid.clenshaw_curtis(17, 7.0), atol=1e-13)


def test_transform_round_trip_of_a_band_limited_bosonic_function():
    beta, M = 10.0, 5
    tau = synth.tau_nodes(40, beta)
    _, Tf, Ti = synth.bosonic_transforms(tau, beta, M)
    f = np.cos(2 * np.pi * 2 * tau / beta) + 0.3 * np.sin(2 * np.pi * tau / beta)
    back = (Ti @ (Tf @ f)).real
    assert np.abs(back - f).max() < 1e-10


def _case(n=4, N=7, n_tau=5, beta=3.0, M=3, seed=7):
    w = synth.tiny(n, N, n_tau=n_tau, beta=beta, seed=seed)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
    Wd = screening.w_dynamic(w.V[0], screening.pi_omega(w.X[0], w.G[0, 0], Tf))
    return w, Tf, Ti, Wd


@pytest.mark.parametrize("n,N,n_tau,M", [(4, 7, 5, 3), (3, 9, 6, 2)])
def test_chain_equals_definition(n, N, n_tau, M):
    w, Tf, Ti, Wd = _case(n, N, n_tau, M=M)
    args = (w.X[0].astype(complex), w.V[0].astype(complex), Wd.astype(complex), Tf, Ti, w.G[0, 0].astype(complex))
    a = dynamic.sigma_d_bruteforce(*args)
    b = dynamic.sigma_d_chain(*args)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    assert np.abs(a.imag).max() < 1e-12 * np.abs(a).max()      # real molecule, even W_d(i Omega)


def test_static_limit_of_the_convolution():
    # W_d(i Omega_m) = beta C delta_{m0}: the convolution no longer depends on tau_i and
    # equals C (x) sum_j w_j G_uq(tau_j) G_sv(-tau_j) (w_j: Clenshaw-Curtis weights)
    w, Tf, Ti, _ = _case()
    M = (Tf.shape[0] - 1) // 2
    rng = np.random.default_rng(3)
    z = rng.standard_normal((w.N, w.N)) / w.N
    C = z @ z.T
    Wd = np.zeros((Tf.shape[0], w.N, w.N))
    Wd[M] = w.beta * C
    X, V, G = w.X[0], w.V[0], w.G[0, 0]
    got = dynamic.sigma_d_chain(X.astype(complex), V.astype(complex), Wd.astype(complex), Tf, Ti, G.astype(complex))
    wts = grid.clenshaw_curtis(w.n_tau, w.beta)
    Gm = grid.g_minus_tau(G)
    cint = np.einsum("j,juq,jsv->uqsv", wts, G, Gm)
    c4 = thc.eri(X, X, C, X, X)
    v2 = thc.eri(X, X, V, X, X)
    ref = -np.einsum("tuvw,iwp,prqs,uqsv->itr", v2, G, c4, cint, optimize=True)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_full_sosex_dynamic_includes_the_bare_sox():
    w, Tf, Ti, Wd = _case()
    full = dynamic.sosex_dynamic_sigma(w.X, w.V, Wd, Tf, Ti, w.G)
    only_d = full - sox.sox_sigma(w.X, w.V, w.G)
    direct = dynamic.sigma_d_chain(w.X[0].astype(complex), w.V[0].astype(complex), Wd.astype(complex), Tf, Ti,
                                   w.G[0, 0].astype(complex))
    assert np.abs(only_d[0, 0] - direct).max() < 1e-15 * 100 * np.abs(direct).max()
