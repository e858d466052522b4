"""Pins for the oracle's SOX / SOSEX-stat self-energy (CPU only).

Each check ties the oracle to something other than itself: the literal
definition (Eq. sox) over 4-index tensors, closed forms, exact THC
reconstruction of a generic 4-index tensor, and the invariants of the
self-energy.
"""
import numpy as np
import pytest

import synth
from oracle import grid, sox, thc


def _general_case(n=4, N=7, seed=1):
    """Non-symmetric G, U1 != U2 (non-symmetric) so transposes and swaps show up."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, n))
    U1 = rng.standard_normal((N, N))
    U2 = rng.standard_normal((N, N))
    G = rng.standard_normal((n, n))
    Gm = rng.standard_normal((n, n))
    return X, U1, U2, G, Gm


def _definition_loops(v1, v2, G, Gm):
    """Eq. (sox) as six explicit sums (pure Python; tiny sizes only)."""
    n = G.shape[0]
    out = np.zeros((n, n))
    r6 = range(n)
    for t in r6:
        for r in r6:
            acc = 0.0
            for p in r6:
                for q in r6:
                    for s in r6:
                        for u in r6:
                            for v in r6:
                                for w in r6:
                                    acc += v1[p, r, q, s] * v2[t, u, v, w] * G[w, p] * G[u, q] * Gm[s, v]
            out[t, r] = -acc
    return out


def test_bruteforce_equals_explicit_loops():
    X, U1, U2, G, Gm = _general_case(n=3, N=4)
    v1 = thc.eri(X, X, U1, X, X)
    v2 = thc.eri(X, X, U2, X, X)
    np.testing.assert_allclose(sox.sigma_bruteforce(v1, v2, G, Gm), _definition_loops(v1, v2, G, Gm),
                               rtol=1e-12, atol=1e-12)


def test_eri_is_the_thc_product():
    X, U1, _, _, _ = _general_case(n=3, N=5)
    v = thc.eri(X, X, U1, X, X)
    i, j, s, r = 2, 0, 1, 2
    ref = sum(X[P, i] * X[P, j] * U1[P, Q] * X[Q, s] * X[Q, r] for P in range(5) for Q in range(5))
    assert abs(v[i, j, s, r] - ref) < 1e-12


@pytest.mark.parametrize("n,N,seed", [(4, 7, 1), (5, 3, 2), (3, 11, 3)])
def test_three_routes_agree_general(n, N, seed):
    X, U1, U2, G, Gm = _general_case(n, N, seed)
    v1 = thc.eri(X, X, U1, X, X)
    v2 = thc.eri(X, X, U2, X, X)
    ref = sox.sigma_bruteforce(v1, v2, G, Gm)
    scale = np.abs(ref).max()
    assert np.abs(sox.sigma_thc_direct(X, U1, U2, G, Gm) - ref).max() < 1e-12 * scale
    assert np.abs(sox.sigma_chain(X, U1, U2, G, Gm) - ref).max() < 1e-12 * scale


def test_three_routes_agree_c0():
    w = synth.config(0)
    taus = [0, 7, 29]
    a = sox.sox_sigma(w.X, w.V, w.G, route="brute", taus=taus)
    b = sox.sox_sigma(w.X, w.V, w.G, route="direct", taus=taus)
    c = sox.sox_sigma(w.X, w.V, w.G, route="chain", taus=taus)
    assert np.abs(a - b).max() < 1e-15 and np.abs(a - c).max() < 1e-15
    assert np.abs(a).max() > 1e-3


def test_single_level_closed_form():
    # n = N = 1, X = 1: Sigma(tau) = -V^2 G(tau)^2 G(-tau)
    beta, n_tau = 5.0, 9
    tau = grid.chebyshev_lobatto(n_tau, beta)
    xi, V = 0.3, 0.7
    g = -np.exp(-xi * tau) / (1 + np.exp(-beta * xi))
    G = g[:, None, None]
    sig = sox.sigma_tau(np.ones((1, 1)), np.full((1, 1), V), np.full((1, 1), V), G, route="chain")
    gm = -g[::-1]
    np.testing.assert_allclose(sig[:, 0, 0].real, -V * V * g * g * gm, rtol=1e-14)


def test_diagonal_closed_form():
    # X = I (N = n), V diagonal, G diagonal: Sigma_tt = -d_t^2 g_t(tau)^2 g_t(-tau), off-diagonal 0
    rng = np.random.default_rng(5)
    n = 4
    d = rng.random(n) + 0.5
    g, gm = rng.standard_normal(n), rng.standard_normal(n)
    sig = sox.sigma_chain(np.eye(n), np.diag(d), np.diag(d), np.diag(g), np.diag(gm))
    np.testing.assert_allclose(sig, np.diag(-d * d * g * g * gm), atol=1e-15)


def test_thc_exact_on_generic_four_index_tensor():
    # Pair functions Phi[(p r), P] = X_pP X_rP span the symmetric pair space when
    # N >= n(n+1)/2 generic points; V = Phi^+ M Phi^+T then reproduces any
    # pair-symmetric PSD M exactly, so THC-SOX must equal the 4-index SOX of M.
    rng = np.random.default_rng(11)
    n, N = 3, 9
    X = rng.standard_normal((N, n))
    Phi = np.einsum("Pp,Pr->prP", X, X).reshape(n * n, N)
    B = rng.standard_normal((n, n, 4))
    B = 0.5 * (B + B.transpose(1, 0, 2))
    M = np.einsum("prk,qsk->prqs", B, B)
    Pinv = np.linalg.pinv(Phi)
    V = Pinv @ M.reshape(n * n, n * n) @ Pinv.T
    np.testing.assert_allclose(thc.eri(X, X, V, X, X), M, atol=1e-10)
    G, Gm = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    ref = sox.sigma_bruteforce(M, M, G, Gm)
    np.testing.assert_allclose(sox.sigma_chain(X, V, V, G, Gm), ref, atol=1e-9 * np.abs(ref).max())


def test_symmetry_and_slot_swap_c0():
    w = synth.config(0)
    sig = sox.sox_sigma(w.X, w.V, w.G, taus=[0, 3, 15, 29])[0, 0]
    assert np.abs(sig - sig.transpose(0, 2, 1)).max() < 1e-17
    # SOX(V, W) = SOX(W, V)^T for any second symmetric interaction
    rng = np.random.default_rng(2)
    z = rng.standard_normal((w.N, w.N)) / w.N
    W = z @ z.T
    a = sox.sigma_tau(w.X[0], W, w.V[0], w.G[0, 0], taus=[4, 20])
    b = sox.sigma_tau(w.X[0], w.V[0], W, w.G[0, 0], taus=[4, 20])
    np.testing.assert_allclose(a, b.transpose(0, 2, 1), atol=1e-18)
    assert np.abs(a - a.transpose(0, 2, 1)).max() > 1e-8


def test_antiperiodicity_of_the_formula():
    # Evaluating the static formula with G(tau) and G(-tau) exchanged gives
    # Sigma(-tau_j) = -Sigma(beta - tau_j) = -Sigma(tau_{n-1-j}).
    w = synth.tiny(5, 9, n_tau=7)
    X, V, Gt = w.X[0], w.V[0], w.G[0, 0]
    Gm = grid.g_minus_tau(Gt)
    sig = sox.sigma_tau(X, V, V, Gt)
    for j in range(Gt.shape[0]):
        s_minus = sox.sigma_chain(X, V, V, Gm[j], Gt[j])
        np.testing.assert_allclose(s_minus, -sig[Gt.shape[0] - 1 - j], atol=1e-16)


def test_spin_blocks_are_independent():
    w = synth.molecule(9, 6, 14, 5, 3.0, n_spin=2)
    a = sox.sox_sigma(w.X, w.V, w.G)
    G2 = w.G.copy()
    G2[1] *= 1.7
    b = sox.sox_sigma(w.X, w.V, G2)
    np.testing.assert_allclose(a[0], b[0], atol=0)
    np.testing.assert_allclose(b[1], a[1] * 1.7 ** 3, rtol=1e-12, atol=1e-18)


def test_sosex_static_slots():
    w = synth.tiny(4, 8, n_tau=5)
    rng = np.random.default_rng(0)
    z = rng.standard_normal((w.N, w.N)) / w.N
    W = (z @ z.T)[None]
    s1 = sox.sosex_static_sigma(w.X, w.V, W, w.G, slot=1)
    s2 = sox.sosex_static_sigma(w.X, w.V, W, w.G, slot=2)
    v1 = thc.eri(w.X[0], w.X[0], W[0], w.X[0], w.X[0])
    v2 = thc.eri(w.X[0], w.X[0], w.V[0], w.X[0], w.X[0])
    Gm = grid.g_minus_tau(w.G[0, 0])
    for j in range(w.n_tau):
        np.testing.assert_allclose(s1[0, 0, j], sox.sigma_bruteforce(v1, v2, w.G[0, 0, j], Gm[j]), atol=1e-16)
        np.testing.assert_allclose(s2[0, 0, j], sox.sigma_bruteforce(v2, v1, w.G[0, 0, j], Gm[j]), atol=1e-16)


def test_screened_compositions_follow_the_dielectric_scalings():
    """With W = v / eps exactly, the paper's effective-dielectric argument (Sec. III C) is
    exact: SOSEX = SOX(v,v)/eps, G3W2 = SOX(v,v)/eps^2, 2SOSEX = (2 - eps)/eps SOX(v,v)."""
    w = synth.tiny(4, 9, n_tau=4)
    eps = 1.7
    W = w.V / eps
    base = sox.sox_sigma(w.X, w.V, w.G)
    scale = np.abs(base).max()
    assert np.abs(sox.sosex_static_sigma(w.X, w.V, W, w.G, slot=2) - base / eps).max() < 1e-14 * scale
    assert np.abs(sox.g3w2_static_sigma(w.X, W, w.G) - base / eps ** 2).max() < 1e-14 * scale
    assert np.abs(sox.sosex2_static_sigma(w.X, w.V, W, w.G) - (2 - eps) / eps * base).max() < 1e-14 * scale


def test_g3w2_decomposition_identity():
    """G3W2 = 2SOSEX + SOX(W_d, W_d) and 2SOSEX = SOSEX + SOX(W_d, v) with a generic symmetric
    W (Sec. III C), each term from the brute-force 4-index route."""
    w = synth.tiny(3, 7, n_tau=3)
    rng = np.random.default_rng(4)
    z = rng.standard_normal((7, 7)) / 7
    W = w.V[0] + z @ z.T - 0.3 * w.V[0]
    Wd = W - w.V[0]
    X, V, G = w.X[0], w.V[0], w.G[0, 0]
    br = lambda U1, U2: sox.sigma_tau(X, U1, U2, G, route="brute")   # noqa: E731
    g3w2 = sox.g3w2_static_sigma(w.X, W[None], w.G)[0, 0]
    two = sox.sosex2_static_sigma(w.X, w.V, W[None], w.G)[0, 0]
    sosex = sox.sosex_static_sigma(w.X, w.V, W[None], w.G, slot=2)[0, 0]
    scale = np.abs(g3w2).max()
    assert np.abs(g3w2 - (two + br(Wd, Wd))).max() < 1e-13 * scale
    assert np.abs(two - (sosex + br(Wd, V))).max() < 1e-13 * scale
    assert np.abs(g3w2 - br(W, W)).max() < 1e-13 * scale
