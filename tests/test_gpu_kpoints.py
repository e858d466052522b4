"""GPU parity of SOX for periodic solids (momentum-resolved chain, FP64 complex)."""
import numpy as np
import pytest

import synth
from oracle import kpoints, sox
from gpu_common import check, pkg_built, torch_cuda

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


def test_solid_sigma_is_hermitian_in_both_precisions(env):
    w = synth.solid(3, (2, 2, 1), 8, 40, 4, 20.0)
    a = _run(env, w, "fp64")
    b = _run(env, w, "f16x2")
    for x in (a, b):
        herm = np.abs(x - np.conj(np.swapaxes(x, -1, -2))).max()
        assert herm <= (1e-13 if x is a else 1e-6) * np.abs(a).max()
    check(b, a, "f16x2", "split vs FP64 chain")


@pytest.mark.parametrize("nk,n,N,n_tau", [((1, 1, 2), 3, 5, 3), ((1, 2, 2), 4, 7, 3), ((1, 1, 3), 5, 12, 4),
                                          ((2, 2, 2), 6, 20, 3), ((2, 1, 1), 9, 70, 2), ((3, 1, 1), 26, 300, 3),
                                          ((1, 1, 4), 3, 8, 2), ((1, 1, 7), 2, 5, 2), ((1, 1, 2), 40, 161, 2),
                                          ((2, 1, 1), 70, 210, 2), ((3, 3, 3), 3, 7, 2), ((4, 4, 4), 2, 3, 2),
                                          ((2, 2, 4), 2, 5, 2), ((1, 1, 5), 3, 8, 2)])
def test_solid_split_precision_matches_oracle(env, nk, n, N, n_tau):
    """Meshes with sides up to 4 take the Fourier D step (sides of 1, 2, 3 and 4, mixed); n_k = 5
    the register form and n_k = 7 the generic one."""
    w = synth.solid(9, nk, n, N, n_tau, 10.0)
    ref = kpoints.sox_sigma(w.X, w.V, w.G, nk)
    got = _run(env, w, "f16x2")
    assert np.isfinite(got).all()
    check(got, ref, "f16x2", f"solid split {nk} n={n} N={N}", n=n, N=N)


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
@pytest.mark.parametrize("slot", [1, 2])
def test_solid_sosex_static(env, slot, prec):
    w = synth.solid(10, (1, 1, 2), 4, 9, 3, 10.0)
    rng = np.random.default_rng(1)
    W = np.empty_like(w.V)
    for q in range(W.shape[0]):
        z = (rng.standard_normal((w.N, w.N)) + 1j * rng.standard_normal((w.N, w.N))) / w.N
        W[q] = z @ z.conj().T
    U1, U2 = (W, w.V) if slot == 1 else (w.V, W)
    ref = kpoints.sox_sigma(w.X, U1, w.G, w.nk, U2=U2)
    got = _run(env, w, prec, W=W, slot=slot)
    check(got, ref, prec, f"solid SOSEX slot {slot}")


def _dynamic_inputs(nk, n, N, n_tau, M, seed, physical=True, n_spin=1):
    w = synth.solid(seed, nk, n, N, n_tau, 10.0)
    G = w.G
    if n_spin == 2:   # a second, different spin block: the propagator of another solid of the same mesh
        G = np.concatenate([G, synth.solid(seed + 1, nk, n, N, n_tau, 10.0).G], axis=0)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
    if physical:
        Wd = kpoints.w_dynamic(w.V, kpoints.pi_omega(w.X, w.G[0], Tf, nk))
    else:
        rng = np.random.default_rng(seed)
        shape = (w.X.shape[0], 2 * M + 1, N, N)
        Wd = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / N
    return w, np.ascontiguousarray(G), Tf, Ti, np.ascontiguousarray(Wd)


def _run_dynamic(env, w, G, Tf, Ti, Wd, handle=None, prec="fp64"):
    torch, pkg, hs = env
    h = hs[prec] if handle is None else handle
    p = pkg.problem(w.n, w.N, w.n_tau, G.shape[0], w.beta, nk=w.nk, dtype=1)
    Gd, X, V, W = (_dev(torch, a.astype(complex)) for a in (G, w.X, w.V, Wd))
    S = torch.full_like(Gd, complex("nan"))
    pkg.sosex_dynamic_sigma(h, p, Gd, X, V, W, _dev(torch, Tf), _dev(torch, Ti), Tf.shape[0], S)
    pkg.sox_check_device(h)
    torch.cuda.synchronize()
    return S.cpu().numpy()


_DYN_REF = {}


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
@pytest.mark.parametrize("nk,n,N,n_tau,M,physical,n_spin", [
    ((1, 1, 2), 3, 5, 4, 2, False, 1),
    ((1, 2, 2), 4, 9, 5, 3, True, 1),
    ((1, 1, 3), 5, 12, 4, 2, False, 2),
    ((2, 1, 1), 9, 70, 6, 3, True, 1),
    ((3, 3, 3), 2, 5, 3, 1, False, 1),
    ((2, 2, 4), 2, 5, 3, 1, False, 1),
    ((4, 4, 4), 2, 3, 3, 1, False, 1),
])
def test_solid_sosex_dynamic_matches_oracle(env, nk, n, N, n_tau, M, physical, n_spin, prec):
    w, G, Tf, Ti, Wd = _dynamic_inputs(nk, n, N, n_tau, M, 30 + n, physical, n_spin)
    key = (nk, n, N, n_tau, M, physical, n_spin)
    if key not in _DYN_REF:   # both precisions compare against one oracle run
        _DYN_REF[key] = kpoints.sosex_dynamic_sigma(w.X, w.V, Wd, Tf, Ti, G, nk)
    ref = _DYN_REF[key]
    got = _run_dynamic(env, w, G, Tf, Ti, Wd, prec=prec)
    assert np.isfinite(got).all()
    check(got, ref, prec, f"solid dynamic {nk} n={n} N={N}", n=n, N=N)


def test_solid_sosex_dynamic_zero_screening_is_bare_sox(env):
    w, G, Tf, Ti, Wd = _dynamic_inputs((1, 2, 1), 4, 10, 4, 2, 44)
    got = _run_dynamic(env, w, G, Tf, Ti, np.zeros_like(Wd))
    ref = kpoints.sox_sigma(w.X, w.V, G, w.nk)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_single_k_complex_dynamic_equals_real_molecule(env):
    from oracle import dynamic, screening
    wm = synth.molecule(42, 8, 36, 6, 20.0)
    _, Tf, Ti = synth.bosonic_transforms(wm.tau, wm.beta, 3)
    Wd = screening.w_dynamic(wm.V[0], screening.pi_omega(wm.X[0], wm.G[0, 0], Tf))
    got = _run_dynamic(env, wm, wm.G, Tf, Ti, Wd[None])
    ref = dynamic.sosex_dynamic_sigma(wm.X, wm.V, Wd, Tf, Ti, wm.G)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_solid_2sosex_static(env, prec):
    """2SOSEXstat for a solid: SOX(v, W0) + SOX(W0 - v, v) against the oracle's terms, at the
    solid workload's beta = 300 (max|Sigma| ~ 1e-2 Ha, so the split path meets 1e-8 Ha)."""
    torch, pkg, hs = env
    w = synth.solid(15, (1, 1, 2), 8, 40, 3, 300.0)   # the solid workload's temperature
    rng = np.random.default_rng(6)
    W = np.empty_like(w.V)
    for q in range(W.shape[0]):     # on a 1x1x2 mesh every q equals -q: real symmetric W^q
        z = rng.standard_normal((w.N, w.N)) / w.N
        W[q] = 0.6 * w.V[q].real + 0.05 * z @ z.T
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
    G, X, V, Wt = (_dev(torch, a.astype(complex)) for a in (w.G, w.X, w.V, W))
    S = torch.full_like(G, complex("nan"))
    pkg.sosex2_static_sigma(hs[prec], p, G, X, V, Wt, S)
    pkg.sox_check_device(hs[prec])
    ref = kpoints.sox_sigma(w.X, w.V, w.G, w.nk, U2=W) + kpoints.sox_sigma(w.X, W - w.V, w.G, w.nk, U2=w.V)
    check(S.cpu().numpy(), ref, prec, "solid 2SOSEXstat")
