"""Pins for the oracle's momentum-resolved SOX (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import dynamic, grid, kpoints, screening, sox


@pytest.mark.parametrize("nk,n,N", [((1, 1, 2), 3, 5), ((1, 2, 2), 3, 4), ((1, 1, 3), 2, 4), ((2, 1, 1), 3, 6)])
def test_three_routes_agree_and_momentum_is_conserved(nk, n, N):
    w = synth.solid(9, nk, n, N, 3, 4.0)
    Gm = grid.g_minus_tau(w.G[0])
    for j in range(w.n_tau):
        brute, big = kpoints.sigma_bruteforce(w.X, w.V, w.V, w.G[0][:, j], Gm[:, j], nk)
        scale = np.abs(brute).max()
        assert np.abs(kpoints.sigma_thc_direct(w.X, w.V, w.V, w.G[0][:, j], Gm[:, j], nk) - brute).max() < 1e-12 * scale
        assert np.abs(kpoints.sigma_chain(w.X, w.V, w.V, w.G[0][:, j], Gm[:, j], nk) - brute).max() < 1e-12 * scale
        nkt = w.X.shape[0]
        for a in range(nkt):
            for b in range(nkt):
                if a != b:     # the big self-energy is block diagonal in k
                    assert np.abs(big[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < 1e-15 * scale


def test_two_interactions_and_slot_swap():
    w = synth.solid(11, (1, 1, 2), 3, 5, 3, 4.0)
    # a physical second interaction obeys W^{-q} = conj(W^q); on a 1x1x2 mesh every
    # q equals -q, so each W^q is real symmetric
    rng = np.random.default_rng(0)
    W = np.stack([(lambda z: z @ z.T)(rng.standard_normal((5, 5)) / 5) for _ in range(2)]).astype(complex)
    Gm = grid.g_minus_tau(w.G[0])
    a = kpoints.sigma_bruteforce(w.X, W, w.V, w.G[0][:, 1], Gm[:, 1], (1, 1, 2))[0]
    b = kpoints.sigma_chain(w.X, W, w.V, w.G[0][:, 1], Gm[:, 1], (1, 1, 2))
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    # SOX(V, W) = SOX(W, V)^dagger for Hermitian data
    c = kpoints.sigma_chain(w.X, w.V, W, w.G[0][:, 1], Gm[:, 1], (1, 1, 2))
    assert np.abs(c - np.conj(np.swapaxes(b, -1, -2))).max() < 1e-12 * np.abs(b).max()


def test_single_k_point_is_the_molecule():
    wm = synth.molecule(5, 4, 9, 3, 4.0)
    Gm = grid.g_minus_tau(wm.G[0, 0])
    c = kpoints.sigma_chain(wm.X.astype(complex), wm.V.astype(complex), wm.V.astype(complex),
                            wm.G[0, 0][None, 1].astype(complex), Gm[None, 1].astype(complex), (1, 1, 1))
    m = sox.sigma_chain(wm.X[0], wm.V[0], wm.V[0], wm.G[0, 0, 1], Gm[1])
    assert np.abs(c[0] - m).max() < 1e-15 * np.abs(m).max() * 10


def test_solid_sigma_hermitian():
    w = synth.solid(12, (1, 2, 2), 4, 7, 3, 6.0)
    s = kpoints.sox_sigma(w.X, w.V, w.G, w.nk)
    assert np.abs(s - np.conj(np.swapaxes(s, -1, -2))).max() < 1e-14 * np.abs(s).max()


def _dyn_case(nk, n=3, N=4, n_tau=4, M=2, seed=21):
    w = synth.solid(seed, nk, n, N, n_tau, 4.0)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
    rng = np.random.default_rng(seed)
    # a generic complex W_d (no symmetry), so a transposed or conjugated operand shows up
    Wd = (rng.standard_normal((w.X.shape[0], 2 * M + 1, N, N))
          + 1j * rng.standard_normal((w.X.shape[0], 2 * M + 1, N, N))) / N
    return w, Tf, Ti, Wd


@pytest.mark.parametrize("nk", [(1, 1, 2), (1, 1, 3), (2, 1, 2)])
def test_dynamic_chain_equals_definition(nk):
    w, Tf, Ti, Wd = _dyn_case(nk, N=4 if nk != (2, 1, 2) else 3, n=3 if nk != (2, 1, 2) else 2)
    a = kpoints.sigma_d_bruteforce(w.X, w.V, Wd, Tf, Ti, w.G[0], nk)
    b = kpoints.sigma_d_chain(w.X, w.V, Wd, Tf, Ti, w.G[0], nk)
    assert np.abs(a).max() > 1e-6
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_dynamic_single_k_point_is_the_molecule():
    w, Tf, Ti, _ = _dyn_case((1, 1, 1))
    wm = synth.molecule(5, 3, 7, w.n_tau, w.beta)
    rng = np.random.default_rng(2)
    Wd = rng.standard_normal((1, Tf.shape[0], 7, 7)) + 1j * rng.standard_normal((1, Tf.shape[0], 7, 7))
    X, V, G = wm.X.astype(complex), wm.V.astype(complex), wm.G[0].astype(complex)
    c = kpoints.sigma_d_chain(X, V, Wd, Tf, Ti, G, (1, 1, 1))[:, 0]
    b = kpoints.sigma_d_bruteforce(X, V, Wd, Tf, Ti, G, (1, 1, 1))[:, 0]
    m = dynamic.sigma_d_bruteforce(X[0], V[0], Wd[0], Tf, Ti, G[0])
    assert np.abs(c - m).max() < 1e-13 * np.abs(m).max()
    assert np.abs(b - m).max() < 1e-13 * np.abs(m).max()
    # the solid bubble at one k point is the molecular bubble
    p = kpoints.pi_omega(X, G, Tf, (1, 1, 1))[0]
    assert np.abs(p - screening.pi_omega(X[0], G[0], Tf)).max() < 1e-13 * np.abs(p).max()


def test_physical_screened_interaction_frequency_symmetry():
    # G_k(tau) is Hermitian, so conj(G^{PQ}_k) = G^{QP}_k and Pi^q(i Omega_{-m}) = Pi^q(i Omega_m)^H;
    # with V^q Hermitian the same holds for W_d^q
    nk = (1, 1, 3)
    w, Tf, Ti, _ = _dyn_case(nk, N=4)
    Pi = kpoints.pi_omega(w.X, w.G[0], Tf, nk)
    Wd = kpoints.w_dynamic(w.V, Pi)
    H = lambda a: np.conj(np.swapaxes(a, -1, -2))
    assert np.abs(Pi[:, ::-1] - H(Pi)).max() < 1e-12 * np.abs(Pi).max()
    assert np.abs(Wd[:, ::-1] - H(Wd)).max() < 1e-12 * np.abs(Wd).max()
    # SOX(v, v) + Sigma_d through both routes with the physical W_d
    a = kpoints.sosex_dynamic_sigma(w.X, w.V, Wd, Tf, Ti, w.G, nk)
    b = kpoints.sosex_dynamic_sigma(w.X, w.V, Wd, Tf, Ti, w.G, nk, route="brute")
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_chain_restricted_to_listed_k_points():
    w = synth.solid(13, (1, 1, 3), 3, 5, 3, 4.0)
    full = kpoints.sox_sigma(w.X, w.V, w.G, w.nk, taus=[1])
    part = kpoints.sox_sigma(w.X, w.V, w.G, w.nk, taus=[1], k_list=[2, 0])
    assert np.array_equal(part[:, 0], full[:, 2]) and np.array_equal(part[:, 1], full[:, 0])


def test_solid_bubble_converges_to_pole_sum_for_every_transfer():
    """The k-resolved bubble through the caller's transform equals the exact transform of
    the pole form for every transfer q and frequency (a dropped momentum shift, a swapped
    pair of propagators or a misplaced conjugate changes the q != 0 blocks)."""
    nk = (1, 2, 2)
    beta, M = 2.0, 2
    w = synth.solid(21, nk, 4, 6, 65, beta)
    om, Tf, _ = synth.bosonic_transforms(w.tau, beta, M)
    quad = kpoints.pi_omega(w.X, w.G[0], Tf, nk)
    exact = kpoints.pi_omega_pole_sum(w.X, w.extras["eps"], w.extras["U"], w.extras["mu"], beta, om, nk)
    scale = np.abs(exact).max()
    assert np.abs(quad - exact).max() < 1e-11 * scale
    assert np.abs(exact[1:] - exact[:1]).max() > 1e-3 * scale    # the transfers differ
    assert np.abs(exact[:, M] - exact[:, M + 1]).max() > 1e-3 * scale   # so do the frequencies
