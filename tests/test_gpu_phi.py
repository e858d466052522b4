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


def _grads(env, w, wt, dphi):
    torch, pkg, h = env
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    d = torch.tensor(dphi, dtype=torch.float64, device="cuda")
    dX = torch.empty_like(X)
    dV = torch.empty_like(V)
    pkg.phi_sox_backward(h, p, G, X, V, tw, d, None, dX, dV)
    torch.cuda.synchronize()
    return dX.cpu().numpy()[0], dV.cpu().numpy()[0]


@pytest.mark.parametrize("n,N,n_tau,n_spin", [(9, 30, 6, 1), (7, 41, 5, 2), (16, 70, 4, 1)])
def test_adjoint_X_V_matches_oracle_autograd(env, n, N, n_tau, n_spin):
    w = synth.molecule(23, n, N, n_tau, 3.0, n_spin=n_spin)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    dphi = [1.0, -0.5][:n_spin]
    gX, gV = _grads(env, w, wt, dphi)
    rX = np.zeros_like(gX)
    rV = np.zeros_like(gV)
    for s in range(n_spin):
        _, _, x, v = phi.phi_and_grads(w.X[0], w.V[0], w.G[s, 0], wt)
        rX += dphi[s] * x
        rV += dphi[s] * v
    assert np.abs(gX - rX).max() <= 1e-11 * np.abs(rX).max()
    assert np.abs(gV - rV).max() <= 1e-11 * np.abs(rV).max()


def test_phisox_autograd_returns_X_and_V_gradients(env):
    torch, pkg, h = env
    w = synth.molecule(24, 8, 25, 5, 3.0, n_spin=1)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    X.requires_grad_(True)
    V.requires_grad_(True)
    pkg.PhiSOX.apply(G, X, V, tw, h, p).sum().backward()
    _, _, rX, rV = phi.phi_and_grads(w.X[0], w.V[0], w.G[0, 0], wt)
    assert np.abs(X.grad.cpu().numpy()[0] - rX).max() <= 1e-11 * np.abs(rX).max()
    assert np.abs(V.grad.cpu().numpy()[0] - rV).max() <= 1e-11 * np.abs(rV).max()


@pytest.mark.parametrize("inst", synth.c4_smallest(3))
def test_adjoint_central_differences_on_smallest_batch_instances(env, inst):
    """Batch workload's three smallest instances (N = 6n, 120 tau): dPhi/dX and
    dPhi/dV against central differences (h = 1e-6) of the FP64 Phi at sampled entries."""
    torch, pkg, h = env
    w = synth.c4_instance(inst)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    out = torch.empty(1, dtype=torch.float64, device="cuda")

    def phi_of(Xa, Va):
        pkg.phi_sox(h, p, G, Xa, Va, tw, out)
        return float(out.item())

    gX, gV = _grads(env, w, wt, [1.0])
    rng = np.random.default_rng(inst)
    hstep = 1e-6
    for tensor, grad, name in ((X, gX, "X"), (V, gV, "V")):
        scale = np.abs(grad).max()
        for _ in range(8):
            i = tuple(int(rng.integers(0, s)) for s in grad.shape)
            if name == "V" and rng.random() < 0.5:   # favour the large leading block of V
                i = (int(rng.integers(0, 8)), int(rng.integers(0, 8)))
            base = tensor[(0,) + i].item()
            tensor[(0,) + i] = base + hstep
            fp = phi_of(X, V)
            tensor[(0,) + i] = base - hstep
            fm = phi_of(X, V)
            tensor[(0,) + i] = base
            fd = (fp - fm) / (2 * hstep)
            assert abs(fd - grad[i]) <= 1e-6 * scale + 1e-7 * abs(grad[i]), (name, i, fd, grad[i], scale)


def test_grad_G_from_kept_sigma_equals_backward(env):
    torch, pkg, h = env
    w = synth.molecule(25, 12, 50, 7, 20.0, n_spin=2)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    d = torch.tensor([0.7, -1.3], dtype=torch.float64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    S = torch.empty_like(G)
    pkg.phi_sox(h, p, G, X, V, tw, out, S)
    a, b = torch.empty_like(G), torch.empty_like(G)
    pkg.phi_sox_grad_G(h, p, S, tw, d, a)
    pkg.phi_sox_backward(h, p, G, X, V, tw, d, b, None, None)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    with pytest.raises(pkg.SoxError):
        pkg.phi_sox_grad_G(h, p, S, tw, d, S)


def _grads_with(torch, pkg, h, w, wt, dphi):
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    d = torch.tensor(dphi, dtype=torch.float64, device="cuda")
    dX = torch.full_like(X, float("nan"))
    dV = torch.full_like(V, float("nan"))
    pkg.phi_sox_backward(h, p, G, X, V, tw, d, None, dX, dV)
    pkg.sox_check_device(h)
    torch.cuda.synchronize()
    return dX.cpu().numpy()[0], dV.cpu().numpy()[0]


@pytest.mark.parametrize("n,N,n_tau,n_spin", [(9, 30, 6, 1), (7, 41, 5, 2), (16, 70, 4, 1), (33, 130, 3, 1)])
def test_split_adjoint_matches_oracle_autograd(env, n, N, n_tau, n_spin):
    """The tensor-core adjoint (FP16 pairs, FP32 accumulation) against the oracle's
    autograd gradients, to the split path's FP32-class bound (relative 2e-5)."""
    torch, pkg, _ = env
    w = synth.molecule(26, n, N, n_tau, 3.0, n_spin=n_spin)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    dphi = [1.0, -0.5][:n_spin]
    with pkg.Handle("f16x2") as h:
        gX, gV = _grads_with(torch, pkg, h, w, wt, dphi)
    rX = np.zeros_like(gX)
    rV = np.zeros_like(gV)
    for s in range(n_spin):
        _, _, x, v = phi.phi_and_grads(w.X[0], w.V[0], w.G[s, 0], wt)
        rX += dphi[s] * x
        rV += dphi[s] * v
    assert np.isfinite(gX).all() and np.isfinite(gV).all()
    assert np.abs(gX - rX).max() <= 2e-5 * np.abs(rX).max()
    assert np.abs(gV - rV).max() <= 2e-5 * np.abs(rV).max()


@pytest.mark.parametrize("n,N,n_tau", [(150, 300, 2), (131, 263, 3)])
def test_split_adjoint_beyond_one_k_tile(env, n, N, n_tau):
    """n > 128 and odd sizes: split rows of several 64-wide chunks, padded row lengths."""
    torch, pkg, h64 = env
    w = synth.molecule(27, n, N, n_tau, 3.0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    rX, rV = _grads_with(torch, pkg, h64, w, wt, [1.0])
    with pkg.Handle("f16x2") as h:
        gX, gV = _grads_with(torch, pkg, h, w, wt, [1.0])
    assert np.abs(gX - rX).max() <= 2e-5 * np.abs(rX).max()
    assert np.abs(gV - rV).max() <= 2e-5 * np.abs(rV).max()


def test_split_adjoint_matches_fp64_adjoint_on_smallest_batch_instance(env):
    torch, pkg, h64 = env
    w = synth.c4_instance(synth.c4_smallest(1)[0])
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    rX, rV = _grads_with(torch, pkg, h64, w, wt, [1.0])
    with pkg.Handle("f16x2") as h:
        gX, gV = _grads_with(torch, pkg, h, w, wt, [1.0])
    assert np.abs(gX - rX).max() <= 2e-5 * np.abs(rX).max()
    assert np.abs(gV - rV).max() <= 2e-5 * np.abs(rV).max()


@pytest.mark.parametrize("n,N,n_tau,n_spin", [(33, 130, 3, 1), (20, 90, 6, 2)])
def test_split_adjoint_one_tau_per_chunk(env, n, N, n_tau, n_spin):
    """The split adjoint with its tau chunk forced to one point (workspace_limit = 1 byte)
    equals the oracle's autograd gradients like the default (all points in one chunk)."""
    torch, pkg, _ = env
    w = synth.molecule(28, n, N, n_tau, 3.0, n_spin=n_spin)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    dphi = [1.0, -0.5][:n_spin]
    rX = np.zeros((w.N, w.n))
    rV = np.zeros((w.N, w.N))
    for s in range(n_spin):
        _, _, x, v = phi.phi_and_grads(w.X[0], w.V[0], w.G[s, 0], wt)
        rX += dphi[s] * x
        rV += dphi[s] * v
    for limit in (0, 1):
        with pkg.Handle("f16x2", workspace_limit=limit) as h:
            gX, gV = _grads_with(torch, pkg, h, w, wt, dphi)
        assert np.isfinite(gX).all() and np.isfinite(gV).all()
        assert np.abs(gX - rX).max() <= 2e-5 * np.abs(rX).max(), limit
        assert np.abs(gV - rV).max() <= 2e-5 * np.abs(rV).max(), limit


def test_split_adjoint_largest_batch_instance_against_fp64(env):
    """The batch's largest instance (n = 298, N = 1788: 14 P/R tiles, 5 K chunks) on a
    two-point mirror grid: the split adjoint against the FP64 adjoint (itself pinned to the
    oracle's autograd on small cases), relative 2e-5."""
    torch, pkg, h64 = env
    i = int(np.argmax(synth.batch_c4_sizes()))
    full = synth.c4_instance(i)
    j = full.n_tau // 4
    order = [j, full.n_tau - 1 - j]
    G = np.ascontiguousarray(full.G[:, :, order])
    wt = grid.clenshaw_curtis(full.n_tau, full.beta)[order]
    p = pkg.problem(full.n, full.N, 2, 1, full.beta)
    Gd, X, V, tw = to_dev(torch, G, full.X, full.V, np.ascontiguousarray(wt))
    d = torch.ones(1, dtype=torch.float64, device="cuda")
    out = {}
    for prec, h in (("fp64", h64), ("f16x2", None)):
        hh = h if h is not None else pkg.Handle("f16x2")
        dX = torch.full_like(X, float("nan"))
        dV = torch.full_like(V, float("nan"))
        pkg.phi_sox_backward(hh, p, Gd, X, V, tw, d, None, dX, dV)
        pkg.sox_check_device(hh)
        out[prec] = (dX.cpu().numpy(), dV.cpu().numpy())
        if h is None:
            hh.close()
    (rX, rV), (gX, gV) = out["fp64"], out["f16x2"]
    assert np.isfinite(gX).all() and np.isfinite(gV).all()
    eX = np.abs(gX - rX).max() / np.abs(rX).max()
    eV = np.abs(gV - rV).max() / np.abs(rV).max()
    print(f"largest instance: split vs FP64 adjoint, relative dX {eX:.2e}, dV {eV:.2e}")
    assert eX <= 2e-5 and eV <= 2e-5
