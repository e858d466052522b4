"""GPU parity of Phi_SOX and its adjoint through the C ABI and the autograd Function."""
import numpy as np
import pytest

import synth
from oracle import grid, phi, sox
from gpu_common import pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    h = pkg.Handle("fp64")
    yield torch, pkg, h
    h.close()


@pytest.mark.parametrize("case", ["small2spin", "c0"])
def test_phi_and_dG_identity(env, case):
    torch, pkg, h = env
    w = synth.molecule(21, 18, 77, 9, 30.0, n_spin=2) if case == "small2spin" else synth.config(0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    sig_ref = sox.sox_sigma(w.X, w.V, w.G).real
    phi_ref = np.array([phi.phi_trace(sig_ref[s, 0], w.G[s, 0], wt) for s in range(w.n_spin)])
    Gg = G.clone().requires_grad_(True)
    val = pkg.PhiSOX.apply(Gg, X, V, tw, h, p)
    (val * torch.tensor([1.0, -0.5][: w.n_spin], dtype=torch.float64, device="cuda")).sum().backward()
    torch.cuda.synchronize()
    np.testing.assert_allclose(val.detach().cpu().numpy(), phi_ref, rtol=1e-12)
    # dPhi/dG_rt(tau_j) = -w_j Sigma_tr(beta - tau_j), times the cotangent
    cot = np.array([1.0, -0.5][: w.n_spin])[:, None, None, None, None]
    ident = -cot * wt[None, None, :, None, None] * np.flip(sig_ref, 2).transpose(0, 1, 2, 4, 3)
    got = Gg.grad.cpu().numpy()
    assert np.abs(got - ident).max() <= 1e-12 * np.abs(ident).max()


def test_phi_host_sigma_output(env):
    torch, pkg, h = env
    w = synth.molecule(22, 10, 40, 6, 10.0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    out_phi = np.zeros(1)
    out_sig = np.zeros_like(w.G)
    pkg.phi_sox(h, p, w.G, w.X, w.V, wt, out_phi, out_sig)
    sig_ref = sox.sox_sigma(w.X, w.V, w.G).real
    np.testing.assert_allclose(out_sig, sig_ref, atol=1e-12 * np.abs(sig_ref).max())
    np.testing.assert_allclose(out_phi[0], phi.phi_trace(sig_ref[0, 0], w.G[0, 0], wt).real, rtol=1e-12)
