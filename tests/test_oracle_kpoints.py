"""Pins for the oracle's momentum-resolved SOX (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import grid, kpoints, sox


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
