"""Pins for the oracle's Phi_SOX and its gradients (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import grid, phi, sox


def test_trace_form_equals_pure_thc_form_c0():
    w = synth.config(0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    sig = sox.sox_sigma(w.X, w.V, w.G)[0, 0]
    a = phi.phi_trace(sig, w.G[0, 0].astype(complex), wt)
    b = phi.phi_thc_direct(w.X[0], w.V[0], w.V[0], w.G[0, 0], wt)
    assert abs(a - b) < 1e-15 * 1e3 * abs(a)
    assert abs(a) > 1e-4


def test_torch_form_equals_numpy_form():
    w = synth.tiny(5, 11, n_tau=7)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    val, *_ = phi.phi_and_grads(w.X[0], w.V[0], w.G[0, 0], wt)
    ref = phi.phi_thc_direct(w.X[0], w.V[0], w.V[0], w.G[0, 0], wt)
    assert abs(val - ref.real) < 1e-14 * max(1.0, abs(ref))


@pytest.mark.parametrize("case", ["tiny", "c0"])
def test_gradient_wrt_G_is_sigma_reflected(case):
    # d Phi / d G_rt(tau_j) = -w_j Sigma_tr(beta - tau_j) for bare SOX
    w = synth.tiny(5, 11, n_tau=7) if case == "tiny" else synth.config(0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    _, gG, _, _ = phi.phi_and_grads(w.X[0], w.V[0], w.G[0, 0], wt)
    sig = sox.sox_sigma(w.X, w.V, w.G)[0, 0].real
    ident = -wt[:, None, None] * np.flip(sig, 0).transpose(0, 2, 1)
    assert np.abs(gG - ident).max() < 1e-12 * np.abs(ident).max()


def _fd(f, arr, idx, h):
    a = arr.copy(); a[idx] += h
    b = arr.copy(); b[idx] -= h
    return (f(a) - f(b)) / (2 * h)


def test_gradients_match_central_differences():
    w = synth.tiny(4, 9, n_tau=6, beta=3.0)
    X, V, G = w.X[0], w.V[0], w.G[0, 0]
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    _, gG, gX, gV = phi.phi_and_grads(X, V, G, wt)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(6):
        i = tuple(rng.integers(0, s) for s in X.shape)
        fd = _fd(lambda a: phi.phi_thc_direct(a, V, V, G, wt).real, X, i, h)
        assert abs(fd - gX[i]) < 1e-8 * max(1.0, np.abs(gX).max())
        i = tuple(rng.integers(0, s) for s in V.shape)
        fd = _fd(lambda a: phi.phi_thc_direct(X, a, a, G, wt).real, V, i, h)
        assert abs(fd - gV[i]) < 1e-8 * max(1.0, np.abs(gV).max())
        i = tuple(rng.integers(0, s) for s in G.shape)
        fd = _fd(lambda a: phi.phi_thc_direct(X, V, V, a, wt).real, G, i, h)
        assert abs(fd - gG[i]) < 1e-8 * max(1.0, np.abs(gG).max())


def test_sosex_functional_gradient_is_symmetrised():
    # With a fixed screened W in slot 1, d Phi/dG gives 1/2 [SOX(W, v) + SOX(v, W)]
    w = synth.tiny(4, 8, n_tau=6, beta=3.0)
    X, V, G = w.X[0], w.V[0], w.G[0, 0]
    rng = np.random.default_rng(1)
    z = rng.standard_normal((w.N, w.N)) / w.N
    W = z @ z.T
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    _, gG, _, _ = phi.phi_and_grads(X, W, G, wt, U2=V)
    a = sox.sigma_tau(X, W, V, G).real
    b = sox.sigma_tau(X, V, W, G).real
    sym = 0.5 * (a + b)
    ident = -wt[:, None, None] * np.flip(sym, 0).transpose(0, 2, 1)
    assert np.abs(gG - ident).max() < 1e-12 * np.abs(ident).max()
