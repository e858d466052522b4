"""GPU parity at the full sizes of the benchmarked workloads, in the launch configuration
bench.py times (split precision), on outputs the oracle can compute one by one; the
dynamically screened solid additionally through properties that hold at any size."""
import numpy as np
import pytest

import synth
from oracle import grid, kpoints, screening, sox
from gpu_common import MIXED_ABS, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    h = pkg.Handle("f16x2")
    yield torch, pkg, h
    h.close()


def test_screened_molecule_full_size(env):
    """n=250, N=2000, 100 tau: Pi(0), W(0) and SOSEX on the GPU; the oracle builds its own
    Pi(0) and W(0) and evaluates Sigma at tau = 0, the largest point."""
    torch, pkg, h = env
    w = synth.config(2)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    _, wts = pkg.sox_tau_grid(w.n_tau, w.beta)
    G, X, V, wt = to_dev(torch, w.G, w.X, w.V, wts)
    Pi = torch.empty(1, w.N, w.N, dtype=torch.float64, device="cuda")
    W0 = torch.empty_like(Pi)
    S = torch.full_like(G, float("nan"))
    pkg.sox_pi0(h, p, G, X, wt, Pi)
    pkg.sox_w_static(h, p, V, Pi, W0)
    pkg.sosex_static_sigma(h, p, G, X, V, W0, S, slot=1)
    pkg.sox_check_device(h)
    got = S.cpu().numpy()
    assert np.isfinite(got).all()
    Pi_o = screening.pi0_quadrature(w.X[0], w.G[0, 0], grid.clenshaw_curtis(w.n_tau, w.beta)).real
    W_o = screening.w_static(w.V[0], 0.5 * (Pi_o + Pi_o.T))
    assert np.abs(W0[0].cpu().numpy() - W_o).max() <= 1e-10 * np.abs(W_o).max()
    ref = sox.sigma_tau(w.X[0], W_o, w.V[0], w.G[0, 0], taus=[0], dtype=np.float64)
    assert np.abs(got[0, 0, [0]] - ref).max() <= MIXED_ABS


def test_solid_dynamic_full_size(env):
    """3x3x3 mesh, n=26, N=300, 60 tau, 59 frequencies.  W_d = 0 leaves SOX(v, v), checked
    against the oracle at tau = 0 for two k points; Sigma is affine in W_d, checked with
    W_d and 2 W_d (every chunk and pair of the dynamic part contributes)."""
    torch, pkg, h = env
    w = synth.config(3)
    M = (w.n_tau - 1) // 2
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
    Wd = synth.pole_screening(w.V, w.beta, M)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
    cx = lambda a: np.ascontiguousarray(a, dtype=complex)   # noqa: E731
    G, X, V, F, I = to_dev(torch, cx(w.G), cx(w.X), cx(w.V), cx(Tf), cx(Ti))
    out = []
    for scale in (0.0, 1.0, 2.0):
        (Wdev,) = to_dev(torch, cx(scale * Wd))
        S = torch.full_like(G, complex("nan"))
        pkg.sosex_dynamic_sigma(h, p, G, X, V, Wdev, F, I, 2 * M + 1, S)
        pkg.sox_check_device(h)
        out.append(S.cpu().numpy())
        del Wdev
    s0, s1, s2 = out
    assert all(np.isfinite(x).all() for x in out)
    ref = kpoints.sox_sigma(w.X, w.V, w.G, w.nk, taus=[0], k_list=[0, 13])
    assert np.abs(s0[:, [0, 13]][:, :, [0]] - ref).max() <= MIXED_ABS
    d1, d2 = s1 - s0, s2 - s1
    assert np.abs(d1).max() > 1e-7                      # the dynamic part is not empty
    assert np.abs(d2 - d1).max() <= MIXED_ABS


def test_batch_largest_instance_full_size(env):
    """Largest instance of the uneven batch (N = 6n, 120 tau): Phi and Sigma on the GPU,
    Sigma against the oracle at tau = 0, and dPhi/dG from the kept Sigma equal to the
    identity -w_j Sigma(beta - tau_j)^T."""
    torch, pkg, h = env
    i = int(np.argmax(synth.batch_c4_sizes()))
    w = synth.c4_instance(i)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    _, wts = pkg.sox_tau_grid(w.n_tau, w.beta)
    G, X, V, wt = to_dev(torch, w.G, w.X, w.V, wts)
    phi = torch.empty(1, dtype=torch.float64, device="cuda")
    S = torch.full_like(G, float("nan"))
    pkg.phi_sox(h, p, G, X, V, wt, phi, S)
    dG = torch.empty_like(G)
    d = torch.tensor([0.75], dtype=torch.float64, device="cuda")
    pkg.phi_sox_grad_G(h, p, S, wt, d, dG)
    pkg.sox_check_device(h)
    got = S.cpu().numpy()
    ref = sox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[0, 0], taus=[0], dtype=np.float64)
    assert np.abs(got[0, 0, [0]] - ref).max() <= MIXED_ABS
    ident = -0.75 * wts[:, None, None] * np.swapaxes(got[0, 0, ::-1], -1, -2)
    assert np.abs(dG.cpu().numpy()[0, 0] - ident).max() <= 1e-15 * np.abs(ident).max()
    assert np.isfinite(phi.item())


def _golden():
    import importlib.util
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_solid_dynamic_fullsize.py")
    spec = importlib.util.spec_from_file_location("make_solid_dynamic_fullsize", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", ["solid_dynamic_k311_n26_N300_t4", "solid_dynamic_k222_n26_N300_t3",
                                  "solid_dynamic_k333_n12_N130_t3"])
def test_solid_dynamic_full_tiles_against_stored_oracle(env, name):
    """Dynamically screened SOSEX of a solid at the full solid's tile counts (N = 300: three
    128-row P/R tiles; 3x3x3 with N = 130: two), every element against the oracle's stored
    result (tests/golden/make_solid_dynamic_fullsize.py, which calls only synth/ and
    oracle/): FP64 to 1e-12 relative, split precision to 1e-8 Ha with the default chunking
    and with one tau point per chunk (workspace_limit = 1 byte)."""
    torch, pkg, _ = env
    gold = _golden()
    nk, n, N, T = gold.CASES[name]
    w, Tf, Ti, Wd = gold.inputs(name)
    stored = np.load(gold.path(name))
    assert np.allclose(stored["fingerprint"], gold.fingerprint(w, Tf, Ti, Wd), rtol=1e-10, atol=0.0), \
        "stored oracle result belongs to other inputs: rerun tests/golden/make_solid_dynamic_fullsize.py"
    ref = stored["sigma"]
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
    cx = lambda a: np.ascontiguousarray(a, dtype=complex)   # noqa: E731
    G, X, V, W, F, I = to_dev(torch, cx(w.G), cx(w.X), cx(w.V), cx(Wd), cx(Tf), cx(Ti))
    for prec, limit in (("fp64", 0), ("f16x2", 0), ("f16x2", 1)):
        with pkg.Handle(prec, workspace_limit=limit) as hh:
            S = torch.full_like(G, complex("nan"))
            pkg.sosex_dynamic_sigma(hh, p, G, X, V, W, F, I, Tf.shape[0], S)
            pkg.sox_check_device(hh)
            got = S.cpu().numpy()
        assert np.isfinite(got).all()
        err = float(np.abs(got - ref).max())
        scale = float(np.abs(ref).max())
        bar = 1e-12 * scale if prec == "fp64" else MIXED_ABS
        print(f"{name} {prec} limit={limit}: max|dSigma| {err:.3e} Ha (max|Sigma| {scale:.3e})")
        assert err <= bar, f"{name} {prec} limit={limit}: max|dSigma| {err:.3e} > {bar:.1e}"
