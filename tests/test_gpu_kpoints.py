"""GPU parity of SOX for periodic solids (momentum-resolved chain, FP64 complex)."""
import numpy as np
import pytest

import synth
from oracle import kpoints, sox
from gpu_common import pkg_built, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    hs = {p: pkg.Handle(p) for p in ("fp64", "f16x2")}
    yield torch, pkg, hs
    for h in hs.values():
        h.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(env, w, prec="fp64", W=None, slot=None):
    torch, pkg, hs = env
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
    G, X, V = _dev(torch, w.G.astype(complex)), _dev(torch, w.X.astype(complex)), _dev(torch, w.V.astype(complex))
    S = torch.full_like(G, complex("nan"))
    if W is not None:
        pkg.sosex_static_sigma(hs[prec], p, G, X, V, _dev(torch, W), S, slot=slot)
    else:
        pkg.sox_sigma(hs[prec], p, G, X, V, S)
    torch.cuda.synchronize()
    return S.cpu().numpy()


@pytest.mark.parametrize("nk,n,N,n_tau", [((1, 1, 2), 3, 5, 3), ((1, 2, 2), 4, 7, 3), ((1, 1, 3), 5, 12, 4),
                                          ((2, 2, 2), 6, 20, 3), ((2, 1, 1), 9, 70, 2)])
def test_solid_matches_oracle_chain(env, nk, n, N, n_tau):
    w = synth.solid(9, nk, n, N, n_tau, 10.0)
    ref = kpoints.sox_sigma(w.X, w.V, w.G, nk)
    got = _run(env, w)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_single_k_complex_equals_real_molecule(env):
    w = synth.molecule(41, 13, 70, 5, 100.0, n_spin=2)
    got = _run(env, w)
    ref = sox.sox_sigma(w.X, w.V, w.G, dtype=np.float64)
    assert np.abs(got.imag).max() == 0.0
    assert np.abs(got.real - ref).max() <= 1e-12 * np.abs(ref).max()


def test_solid_sigma_is_hermitian_and_handle_precision_independent(env):
    w = synth.solid(3, (2, 2, 1), 8, 40, 4, 20.0)
    a = _run(env, w, "fp64")
    b = _run(env, w, "f16x2")
    assert np.abs(a - b).max() == 0.0          # solids always take the FP64 complex chain
    herm = np.abs(a - np.conj(np.swapaxes(a, -1, -2))).max()
    assert herm <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("slot", [1, 2])
def test_solid_sosex_static(env, slot):
    w = synth.solid(10, (1, 1, 2), 4, 9, 3, 10.0)
    rng = np.random.default_rng(1)
    W = np.empty_like(w.V)
    for q in range(W.shape[0]):
        z = (rng.standard_normal((w.N, w.N)) + 1j * rng.standard_normal((w.N, w.N))) / w.N
        W[q] = z @ z.conj().T
    U1, U2 = (W, w.V) if slot == 1 else (w.V, W)
    ref = kpoints.sox_sigma(w.X, U1, w.G, w.nk, U2=U2)
    got = _run(env, w, W=W, slot=slot)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
