"""GPU parity of the self-consistent loop's device steps (Sec. II A) against the oracle's
loop (oracle/scloop.py, pinned in tests/test_oracle_scloop.py): Dyson on the Matsubara
frequencies, the tail-corrected return to imaginary time, the forward transform, the
chemical potential, THC Hartree-Fock, the Galitskii-Migdal energies, and whole loops."""
import numpy as np
import pytest

import synth
from oracle import grid, scloop, sox
from gpu_common import pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _molecule(n=4, N=10, beta=4.0, scale=0.6, seed=11):
    rng = np.random.default_rng(seed)
    h, _, _ = synth.random_hamiltonian(rng, n)
    X = rng.standard_normal((N, n)) / np.sqrt(n)
    Z = rng.standard_normal((N, N)) / N
    V = scale * (Z @ Z.T)
    return h, X, V, beta


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    h = pkg.Handle("fp64")
    yield torch, pkg, h
    h.close()


def test_dyson_and_tail_corrected_return(env):
    torch, pkg, h = env
    rng = np.random.default_rng(5)
    n, n_tau, beta, n_max, mu = 5, 21, 4.0, 300, 0.3
    F = rng.standard_normal((2, n, n))
    F = 0.5 * (F + np.swapaxes(F, 1, 2))
    tau = grid.chebyshev_lobatto(n_tau, beta)
    om = scloop.fermionic_frequencies(beta, n_max)
    S_tau = 0.05 * rng.standard_normal((2, n_tau, n, n))
    S_tau = 0.5 * (S_tau + np.swapaxes(S_tau, 2, 3))
    S_iw = np.stack([scloop.tau_to_iw(S_tau[s], tau, beta, om) for s in range(2)])
    p = pkg.problem(n, 8, n_tau, 2, beta)
    Fd, Sd, St, omd, taud = to_dev(torch, F, S_iw, S_tau, om, tau)
    Giw = torch.empty(2, om.size, n, n, dtype=torch.complex128, device="cuda")
    pkg.sox_dyson(h, p, omd, mu, Fd, Sd, Giw)
    tails = torch.empty(2, 3, n, n, dtype=torch.float64, device="cuda")
    pkg.sox_green_tails(h, p, mu, Fd, St, tails)
    Gt = torch.empty(2, n_tau, n, n, dtype=torch.float64, device="cuda")
    pkg.sox_iw_to_tau(h, p, omd, Giw, tails, taud, Gt)
    torch.cuda.synchronize()
    for s in range(2):
        ref_iw = scloop.dyson(om, mu, F[s], S_iw[s])
        assert np.abs(Giw[s].cpu().numpy() - ref_iw).max() <= 1e-12 * np.abs(ref_iw).max()
        c1, c2, c3 = scloop.green_tails(F[s], mu, S_tau[s])
        got_tails = tails[s].cpu().numpy()
        for k, c in enumerate((c1, c2, c3)):
            assert np.abs(got_tails[k] - c.real).max() <= 1e-13 * max(1.0, np.abs(c).max())
        ref_t = scloop.iw_to_tau(ref_iw, om, tau, beta, c1, c2, c3).real
        assert np.abs(Gt[s].cpu().numpy() - ref_t).max() <= 1e-11


def test_forward_transform_with_the_grid_transform(env):
    """sox_tau_to_iw with synth's fermionic transform equals the oracle's Fourier integral of
    the interpolant, both on a pole function (exact: 1/(i w - xi))."""
    torch, pkg, h = env
    beta, n_tau, xi = 4.0, 65, 0.7
    tau = grid.chebyshev_lobatto(n_tau, beta)
    om, Tw = synth.fermionic_transform(tau, beta, 200)
    g = (-np.exp(-xi * tau) / (1.0 + np.exp(-beta * xi)))[None, :, None, None]   # [1][T][1][1]
    p = pkg.problem(1, 4, n_tau, 1, beta)
    Twd, gd = to_dev(torch, Tw, np.ascontiguousarray(g))
    out = torch.empty(1, om.size, 1, 1, dtype=torch.complex128, device="cuda")
    pkg.sox_tau_to_iw(h, p, Twd, gd, out)
    got = out.cpu().numpy()[0, :, 0, 0]
    ref = scloop.tau_to_iw(g[0, :, 0, 0], tau, beta, om)
    assert np.abs(got - ref).max() < 1e-12
    assert np.abs(got - 1.0 / (1j * om - xi)).max() < 1e-10


def test_hartree_fock_energies_and_mu(env):
    torch, pkg, h = env
    hm, X, V, beta = _molecule()
    n, N, n_tau = hm.shape[0], X.shape[0], 17
    rng = np.random.default_rng(9)
    gam = rng.standard_normal((2, n, n)) * 0.2
    gam = 0.5 * (gam + np.swapaxes(gam, 1, 2))
    p = pkg.problem(n, N, n_tau, 2, beta)
    Xd, Vd, gd, Hd = to_dev(torch, X[None], V[None], gam, hm)
    S = torch.empty(2, n, n, dtype=torch.float64, device="cuda")
    F = torch.empty_like(S)
    pkg.sox_sigma_hf(h, p, Xd, Vd, gd, S, H0=Hd, F=F)
    ref = scloop.sigma_hf(X, V, gam)
    assert np.abs(S.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(F.cpu().numpy() - (hm[None] + ref)).max() <= 1e-13 * np.abs(ref).max()
    # energies of an arbitrary (G, Sigma) pair against the oracle's formulas
    tau = grid.chebyshev_lobatto(n_tau, beta)
    w = grid.clenshaw_curtis(n_tau, beta)
    G = rng.standard_normal((2, n_tau, n, n))
    Sg = rng.standard_normal((2, n_tau, n, n)) * 0.1
    st = scloop.LoopState(G_tau=G, sigma_tau=Sg, tau=tau, beta=beta, gamma=gam, sigma_hf=ref)
    E = np.zeros(2)
    Gd, Sgd, wd = to_dev(torch, G, Sg, w)
    pkg.sox_gm_energies(h, p, Hd, S, gd, Sgd, Gd, wd, E)
    assert abs(E[0] - scloop.energy_inf(hm, st)) <= 1e-12 * abs(E[0])
    assert abs(E[1] - scloop.energy_dyn_tau(st)) <= 1e-12 * abs(E[1])
    # chemical potential of the bare Fock problem at the half-filling count
    om = scloop.fermionic_frequencies(beta, 400)
    omd, = to_dev(torch, om)
    mu = pkg.sox_find_mu(h, p, omd, 4.0, F)
    zt = np.zeros((n_tau, n, n))
    zw = np.zeros((om.size, n, n), complex)
    ref_mu = scloop.find_mu(om, beta, 4.0, [hm + ref[0], hm + ref[1]], [zw, zw], [zt, zt])
    assert abs(mu - ref_mu) < 1e-10


@pytest.mark.parametrize("dynamic", [False, True])
def test_whole_loop_matches_the_oracle_loop(env, dynamic):
    """Hartree-Fock alone, and HF + SOX as the dynamic part: the GPU loop (library calls
    sequenced by paper_2412_18829_gb300.scloop) against the oracle's loop -- mu, G(tau), the
    electron count and both Galitskii-Migdal energies."""
    torch, pkg, h = env
    from paper_2412_18829_gb300 import scloop as gloop

    hm, X, V, beta = _molecule()
    n, N, n_tau, n_elec, n_max = hm.shape[0], X.shape[0], 33, 4.0, 400

    def sigma_sox(G):
        return sox.sox_sigma(X[None], V[None], G[:, None], dtype=np.float64)[:, 0].real

    zero = lambda G: np.zeros_like(G)   # noqa: E731
    ref = scloop.sc_loop(hm, X, V, beta, n_tau, n_elec, sigma_sox if dynamic else zero, n_max=n_max,
                         tol=1e-11 if not dynamic else 1e-10)
    tau = grid.chebyshev_lobatto(n_tau, beta)
    w = grid.clenshaw_curtis(n_tau, beta)
    om, Tw = synth.fermionic_transform(tau, beta, n_max)
    p = pkg.problem(n, N, n_tau, 2, beta)
    Hd, Xd, Vd, omd, Twd, taud, wd = to_dev(torch, hm, X[None], V[None], om, Tw, tau, w)
    res = gloop.run(h, p, Hd, Xd, Vd, n_elec, omd, Twd, taud, wd, dynamic=dynamic,
                    tol=1e-11 if not dynamic else 1e-10)
    torch.cuda.synchronize()
    assert res.change < (1e-10 if not dynamic else 1e-9)
    assert abs(res.mu - ref.mu) < 1e-8
    assert np.abs(res.G_tau.cpu().numpy() - ref.G_tau).max() < 1e-8
    assert abs(float(res.gamma.cpu().numpy().trace(axis1=1, axis2=2).sum()) - n_elec) < 1e-8
    E = res.energies.cpu().numpy()
    e_inf = scloop.energy_inf(hm, ref)
    assert abs(E[0] - e_inf) < 1e-8 * abs(e_inf)
    if dynamic:
        e_dyn = scloop.energy_dyn_tau(ref)
        assert abs(E[1] - e_dyn) < 1e-7 * abs(e_dyn)
    else:
        assert E[1] == 0.0
