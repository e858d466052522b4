"""GPU parity with the smallest chunks: a handle whose workspace limit is one byte
runs every tau / v loop one point at a time.  The results must match the oracle to
the same bars as the default chunking."""
import numpy as np
import pytest

import synth
from oracle import grid, kpoints, phi, sox
from gpu_common import check, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    hs = {(p, lim): pkg.Handle(p, workspace_limit=lim) for p in ("fp64", "f16x2") for lim in (0, 1)}
    yield torch, pkg, hs
    for h in hs.values():
        h.close()


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_molecule_sigma_one_tau_per_chunk(env, prec):
    torch, pkg, hs = env
    w = synth.molecule(71, 11, 60, 5, 20.0, n_spin=2)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    out = {}
    for lim in (0, 1):
        S = torch.full_like(G, float("nan"))
        pkg.sox_sigma(hs[(prec, lim)], p, G, X, V, S)
        pkg.sox_check_device(hs[(prec, lim)])
        out[lim] = S.cpu().numpy()
    ref = sox.sox_sigma(w.X, w.V, w.G, dtype=np.float64)
    check(out[1], ref, prec, f"{prec} chunk 1")
    assert np.abs(out[1] - out[0]).max() <= 1e-13 * np.abs(ref).max()


def test_adjoint_one_tau_per_chunk(env):
    torch, pkg, hs = env
    w = synth.molecule(72, 7, 31, 5, 3.0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    d = torch.ones(1, dtype=torch.float64, device="cuda")
    dX, dV = torch.empty_like(X), torch.empty_like(V)
    pkg.phi_sox_backward(hs[("fp64", 1)], p, G, X, V, tw, d, None, dX, dV)
    _, _, rX, rV = phi.phi_and_grads(w.X[0], w.V[0], w.G[0, 0], wt)
    assert np.abs(dX.cpu().numpy()[0] - rX).max() <= 1e-11 * np.abs(rX).max()
    assert np.abs(dV.cpu().numpy()[0] - rV).max() <= 1e-11 * np.abs(rV).max()


def test_solid_static_one_v_per_chunk(env):
    torch, pkg, hs = env
    w = synth.solid(73, (1, 1, 3), 5, 12, 3, 10.0)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    S = torch.full_like(G, complex("nan"))
    pkg.sox_sigma(hs[("fp64", 1)], p, G, X, V, S)
    ref = kpoints.sox_sigma(w.X, w.V, w.G, w.nk)
    assert np.abs(S.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_solid_dynamic_one_tau_per_chunk(env, prec):
    torch, pkg, hs = env
    w = synth.solid(74, (1, 2, 1), 4, 9, 5, 10.0)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, 2)
    Wd = kpoints.w_dynamic(w.V, kpoints.pi_omega(w.X, w.G[0], Tf, w.nk))
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
    G, X, V, W, F, I = to_dev(torch, w.G, w.X, w.V, Wd, Tf, Ti)
    S = torch.full_like(G, complex("nan"))
    pkg.sosex_dynamic_sigma(hs[(prec, 1)], p, G, X, V, W, F, I, Tf.shape[0], S)
    pkg.sox_check_device(hs[(prec, 1)])
    ref = kpoints.sosex_dynamic_sigma(w.X, w.V, Wd, Tf, Ti, w.G, w.nk)
    check(S.cpu().numpy(), ref, prec, "solid dynamic, one tau per chunk")


def test_negative_workspace_limit_is_rejected(env):
    _, pkg, _ = env
    with pytest.raises(pkg.SoxError):
        pkg.Handle("fp64", workspace_limit=-1)
