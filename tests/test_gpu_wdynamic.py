"""GPU parity of the RPA screened interaction on the transform's frequencies
(sox_w_dynamic) against the oracle's bubble and W, for molecules and solids, and of the
dynamically screened SOSEX fed with it."""
import numpy as np
import pytest

import synth
from oracle import dynamic, kpoints, screening
from gpu_common import check, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

W_REL = 1e-10   # FP64 Gauss-Jordan against the oracle's eigen-decomposition route


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    h = pkg.Handle("fp64")
    yield torch, pkg, h
    h.close()


def _w_gpu(env, w, Tf, complex_data):
    torch, pkg, h = env
    nO = Tf.shape[0]
    if complex_data:
        p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
        cx = lambda a: np.ascontiguousarray(a, dtype=complex)   # noqa: E731
        G, X, V = to_dev(torch, cx(w.G), cx(w.X), cx(w.V))
        nq = w.X.shape[0]
        Wd = torch.full((nq, nO, w.N, w.N), complex("nan"), dtype=torch.complex128, device="cuda")
    else:
        p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
        G, X, V = to_dev(torch, w.G, w.X, w.V)
        Wd = torch.full((nO, w.N, w.N), float("nan"), dtype=torch.float64, device="cuda")
    F = torch.from_numpy(np.ascontiguousarray(Tf)).cuda()
    pkg.sox_w_dynamic(h, p, G, X, V, F, nO, Wd)
    return Wd.cpu().numpy()


@pytest.mark.parametrize("n,N,n_tau,M,n_spin", [(7, 30, 8, 4, 1), (13, 70, 10, 5, 2), (20, 150, 12, 6, 1)])
def test_molecule_w_dynamic_matches_oracle(env, n, N, n_tau, M, n_spin):
    w = synth.molecule(70 + n, n, N, n_tau, 20.0, n_spin=n_spin)
    _, Tf, _ = synth.bosonic_transforms(w.tau, w.beta, M)
    Pi = sum(screening.pi_omega(w.X[0], w.G[s, 0], Tf) for s in range(n_spin))
    ref = screening.w_dynamic(w.V[0], Pi)
    got = _w_gpu(env, w, Tf, False)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= W_REL * np.abs(ref).max()
    assert np.abs(ref).max() > 1e-6 * np.abs(w.V).max()   # the screening is not negligible


@pytest.mark.parametrize("nk,n,N,n_tau,M", [((1, 1, 2), 3, 7, 4, 2), ((1, 2, 2), 4, 9, 5, 2),
                                            ((3, 1, 1), 3, 11, 4, 1), ((2, 2, 2), 3, 8, 3, 1),
                                            ((1, 1, 4), 2, 6, 3, 1), ((3, 3, 3), 2, 5, 3, 1)])
def test_solid_w_dynamic_matches_oracle(env, nk, n, N, n_tau, M):
    w = synth.solid(80 + n, nk, n, N, n_tau, 10.0)
    _, Tf, _ = synth.bosonic_transforms(w.tau, w.beta, M)
    ref = kpoints.w_dynamic(w.V, kpoints.pi_omega(w.X, w.G[0], Tf, nk))
    got = _w_gpu(env, w, Tf, True)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= W_REL * np.abs(ref).max()
    # Pi^q(-Omega) = Pi^q(Omega)^H carries over to W_d
    H = np.conj(np.swapaxes(got, -1, -2))
    assert np.abs(got[:, ::-1] - H).max() <= W_REL * np.abs(ref).max()


def test_molecule_sosex_dynamic_with_gpu_w(env):
    """W_d built on the GPU feeds sosex_dynamic_sigma; Sigma equals the oracle's chain with
    the oracle's W_d."""
    torch, pkg, h = env
    w = synth.molecule(91, 9, 40, 8, 20.0)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, 4)
    Wd = _w_gpu(env, w, Tf, False)
    ref_w = screening.w_dynamic(w.V[0], screening.pi_omega(w.X[0], w.G[0, 0], Tf))
    ref = dynamic.sosex_dynamic_sigma(w.X, w.V, ref_w, Tf, Ti, w.G).real
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, W = to_dev(torch, w.G, w.X, w.V, Wd)
    F, I = to_dev(torch, Tf, Ti)
    S = torch.full_like(G, float("nan"))
    pkg.sosex_dynamic_sigma(h, p, G, X, V, W, F, I, Tf.shape[0], S)
    check(S.cpu().numpy(), ref, "fp64", "dynamic SOSEX with the GPU W_d")


def test_solid_sosex_dynamic_with_gpu_w(env):
    torch, pkg, h = env
    nk = (1, 2, 2)
    w = synth.solid(92, nk, 3, 8, 4, 10.0)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, 2)
    Wd = _w_gpu(env, w, Tf, True)
    ref_w = kpoints.w_dynamic(w.V, kpoints.pi_omega(w.X, w.G[0], Tf, nk))
    ref = kpoints.sosex_dynamic_sigma(w.X, w.V, ref_w, Tf, Ti, w.G, nk)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=nk, dtype=1)
    cx = lambda a: np.ascontiguousarray(a, dtype=complex)   # noqa: E731
    G, X, V, W, F, I = to_dev(torch, cx(w.G), cx(w.X), cx(w.V), cx(Wd), Tf, Ti)
    S = torch.full_like(G, complex("nan"))
    pkg.sosex_dynamic_sigma(h, p, G, X, V, W, F, I, Tf.shape[0], S)
    check(S.cpu().numpy(), ref, "fp64", "solid dynamic SOSEX with the GPU W_d")


def test_w_dynamic_rejects_wide_meshes(env):
    torch, pkg, h = env
    p = pkg.problem(2, 3, 3, 1, 10.0, nk=(9, 1, 1), dtype=1)
    G = torch.zeros(1, 9, 3, 2, 2, dtype=torch.complex128, device="cuda")
    X = torch.zeros(9, 3, 2, dtype=torch.complex128, device="cuda")
    V = torch.zeros(9, 3, 3, dtype=torch.complex128, device="cuda")
    F = torch.zeros(3, 3, dtype=torch.complex128, device="cuda")
    Wd = torch.zeros(9, 3, 3, 3, dtype=torch.complex128, device="cuda")
    with pytest.raises(pkg.SoxError) as e:
        pkg.sox_w_dynamic(h, p, G, X, V, F, 3, Wd)
    assert e.value.code == 2


def test_w_dynamic_without_the_frequency_symmetry(env):
    """Unpaired frequencies (a molecule's last transform row dropped) and a non-Hermitian G
    (a solid) take the full solve of every (q, Omega); both against the oracle."""
    w = synth.molecule(93, 8, 30, 8, 20.0)
    _, Tf, _ = synth.bosonic_transforms(w.tau, w.beta, 3)
    Tf = np.ascontiguousarray(Tf[:-1])
    ref = screening.w_dynamic(w.V[0], screening.pi_omega(w.X[0], w.G[0, 0], Tf))
    got = _w_gpu(env, w, Tf, False)
    assert np.abs(got - ref).max() <= W_REL * np.abs(ref).max()

    nk = (1, 1, 3)
    ws = synth.solid(94, nk, 3, 8, 4, 10.0)
    rng = np.random.default_rng(5)
    ws.G = ws.G + 1e-3 * np.abs(ws.G).max() * (rng.standard_normal(ws.G.shape)
                                               + 1j * rng.standard_normal(ws.G.shape))
    _, Tf, _ = synth.bosonic_transforms(ws.tau, ws.beta, 2)
    ref = kpoints.w_dynamic(ws.V, kpoints.pi_omega(ws.X, ws.G[0], Tf, nk))
    got = _w_gpu(env, ws, Tf, True)
    assert np.abs(got - ref).max() <= W_REL * np.abs(ref).max()
    # without Hermitian G the -Omega block is no conjugate transpose
    H = np.conj(np.swapaxes(ref, -1, -2))
    assert np.abs(ref[:, ::-1] - H).max() > 1e-6 * np.abs(ref).max()
