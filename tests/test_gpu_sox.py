"""GPU parity of SOX / SOSEX-stat / projections through the C ABI against the CPU oracle."""
import numpy as np
import pytest

import synth
from oracle import grid, screening, sox, thc
from gpu_common import check, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu
PRECS = ["fp64", "f16x2"]


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    handles = {p: pkg.Handle(p) for p in PRECS}
    yield torch, pkg, handles
    for h in handles.values():
        h.close()


def _sigma(env, prec, w, U1=None, U2=None, slot=None):
    torch, pkg, hs = env
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    S = torch.full_like(G, float("nan"))
    if slot is not None:
        (W,) = to_dev(torch, U1)
        pkg.sosex_static_sigma(hs[prec], p, G, X, V, W, S, slot=slot)
    elif U1 is not None:
        A1, A2 = to_dev(torch, U1, U2)
        pkg.sox_sigma_general(hs[prec], p, G, X, A1, A2, S)
    else:
        pkg.sox_sigma(hs[prec], p, G, X, V, S)
    pkg.sox_check_device(hs[prec])
    return S.cpu().numpy()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,N,n_tau,n_spin", [(13, 70, 6, 2), (1, 1, 4, 1), (5, 3, 2, 1), (33, 130, 5, 1),
                                              (64, 128, 3, 1)])
def test_sox_small_and_ragged(env, prec, n, N, n_tau, n_spin):
    w = synth.molecule(11, n, N, n_tau, 100.0, n_spin=n_spin, name="ragged")
    ref = sox.sox_sigma(w.X, w.V, w.G).real
    check(_sigma(env, prec, w), ref, prec, f"n={n} N={N}", n=n, N=N)


@pytest.mark.parametrize("prec", PRECS)
def test_sox_c0_all_tau(env, prec):
    w = synth.config(0)
    ref = sox.sox_sigma(w.X, w.V, w.G).real
    err, scale = check(_sigma(env, prec, w), ref, prec, "c0")
    print(f"c0 {prec}: max|dSigma| {err:.3e} Ha, relative {err / scale:.3e}")


@pytest.mark.parametrize("prec", PRECS)
def test_sox_c1_full_size_sampled_tau(env, prec):
    """c1 (n=120, N=600, 80 tau, 2 spins) in the benchmark's launch; oracle on sampled tau."""
    w = synth.config(1)
    out = _sigma(env, prec, w)
    assert np.isfinite(out).all()
    taus = [0, 17, 40, 79]
    for s in range(w.n_spin):
        ref = sox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[s, 0], taus=taus, dtype=np.float64)
        err, scale = check(out[s, 0, taus], ref, prec, f"c1 spin {s}")
        print(f"c1 {prec} spin {s}: max|dSigma| {err:.3e} Ha, relative {err / scale:.3e}")


@pytest.mark.parametrize("prec", PRECS)
def test_general_two_interactions_nonsymmetric(env, prec):
    w = synth.molecule(12, 19, 75, 5, 100.0, n_spin=1)
    rng = np.random.default_rng(3)
    z = rng.standard_normal((w.N, w.N)) / w.N
    U1 = np.ascontiguousarray((z @ z.T + 0.3 * z)[None])     # non-symmetric on purpose
    U2 = np.ascontiguousarray(w.V)
    ref = np.stack([sox.sigma_tau(w.X[0], U1[0], U2[0], w.G[0, 0]).real])[:, None]
    assert np.abs(ref).max() > 1e-4
    check(_sigma(env, prec, w, U1, U2), ref, prec, "general")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("slot", [1, 2])
def test_sosex_static_c0(env, prec, slot):
    w = synth.config(0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    Pi = screening.pi0_quadrature(w.X[0], w.G[0, 0], wt)
    W = np.ascontiguousarray(screening.w_static(w.V[0], 0.5 * (Pi + Pi.T))[None])
    ref = sox.sosex_static_sigma(w.X, w.V, W, w.G, slot=slot).real
    check(_sigma(env, prec, w, W, slot=slot), ref, prec, f"sosex slot {slot}")


def test_thc_project_G(env):
    torch, pkg, hs = env
    w = synth.molecule(13, 21, 90, 4, 10.0, n_spin=2)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X = to_dev(torch, w.G, w.X)
    shp = (w.n_spin, 1, w.n_tau)
    GR = torch.empty(*shp, w.N, w.n, dtype=torch.float64, device="cuda")
    GW = torch.empty(*shp, w.n, w.N, dtype=torch.float64, device="cuda")
    GPQ = torch.empty(*shp, w.N, w.N, dtype=torch.float64, device="cuda")
    pkg.thc_project_G(hs["fp64"], p, G, X, GR, GW, GPQ)
    torch.cuda.synchronize()
    for s in range(w.n_spin):
        for j in range(w.n_tau):
            g = w.G[s, 0, j]
            np.testing.assert_allclose(GR[s, 0, j].cpu().numpy(), thc.project_left(w.X[0], g), atol=1e-14)
            np.testing.assert_allclose(GW[s, 0, j].cpu().numpy(), thc.project_right(w.X[0], g), atol=1e-14)
            np.testing.assert_allclose(GPQ[s, 0, j].cpu().numpy(), thc.project_full(w.X[0], g), atol=1e-13)


def test_pi0_and_w_static(env):
    torch, pkg, hs = env
    w = synth.config(0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    Pi = torch.empty(1, w.N, w.N, dtype=torch.float64, device="cuda")
    pkg.sox_pi0(hs["fp64"], p, G, X, tw, Pi)
    torch.cuda.synchronize()
    ref = screening.pi0_quadrature(w.X[0], w.G[0, 0], wt)
    np.testing.assert_allclose(Pi[0].cpu().numpy(), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    W = torch.empty(w.N, w.N, dtype=torch.float64, device="cuda")
    pkg.sox_w_static(hs["fp64"], p, V[0].contiguous(), Pi[0].contiguous(), W)
    torch.cuda.synchronize()
    refW = screening.w_static(w.V[0], Pi[0].cpu().numpy())
    np.testing.assert_allclose(W.cpu().numpy(), refW, rtol=0, atol=1e-11 * np.abs(refW).max())


def test_w_static_reports_singular_system(env):
    torch, pkg, hs = env
    N = 4
    p = pkg.problem(2, N, 4, 1, 1.0)
    V = torch.eye(N, dtype=torch.float64, device="cuda")
    Pi = torch.eye(N, dtype=torch.float64, device="cuda")   # 1 - V Pi = 0
    W = torch.empty_like(V)
    with pytest.raises(pkg.SoxError) as e:
        pkg.sox_w_static(hs["fp64"], p, V, Pi, W)
    assert e.value.code == 1


@pytest.mark.parametrize("prec", PRECS)
def test_host_buffers_through_the_c_abi(env, prec):
    torch, pkg, hs = env
    w = synth.molecule(14, 17, 66, 5, 100.0, n_spin=1)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    S = np.full_like(w.G, np.nan)
    pkg.sox_sigma(hs[prec], p, w.G, w.X, w.V, S)
    check(S, sox.sox_sigma(w.X, w.V, w.G).real, prec, "host buffers")


def test_error_paths(env):
    torch, pkg, hs = env
    h = hs["fp64"]
    G = torch.zeros(1, 1, 4, 3, 3, dtype=torch.float64, device="cuda")
    X = torch.zeros(1, 5, 3, dtype=torch.float64, device="cuda")
    V = torch.zeros(1, 5, 5, dtype=torch.float64, device="cuda")
    S = torch.zeros_like(G)
    bad = [pkg.problem(0, 5, 4), pkg.problem(3, 5, 1), pkg.problem(3, 5, 4, n_spin=3),
           pkg.problem(3, 5, 4, beta=-1.0), pkg.problem(3, 5, 4, nk=(2, 1, 1)),
           pkg.problem(3, 5, 4, dtype=7), pkg.problem(2000, 5, 4)]
    codes = []
    for p in bad:   # every descriptor is rejected before any buffer is touched
        with pytest.raises(pkg.SoxError) as e:
            pkg.sox_sigma(h, p, G, X, V, S)
        codes.append(e.value.code)
    assert codes == [2, 2, 2, 1, 3, 1, 2]
    with pytest.raises(pkg.SoxError):
        pkg.sox_sigma(h, pkg.problem(3, 5, 4), G, X, V, None)
    with pytest.raises(pkg.SoxError):
        pkg.sosex_static_sigma(h, pkg.problem(3, 5, 4), G, X, V, V, S, slot=3)


@pytest.mark.parametrize("n,N,n_tau", [(130, 300, 3), (200, 260, 2)])
def test_split_path_beyond_one_k_tile(env, n, N, n_tau):
    """n > 128: the A intermediate takes its a-priori scale and K spans several chunks."""
    w = synth.molecule(15, n, N, n_tau, 100.0, n_spin=1)
    ref = sox.sox_sigma(w.X, w.V, w.G, dtype=np.float64)
    check(_sigma(env, "f16x2", w), ref, "f16x2", f"n={n}")


def test_bounded_waits_report_timeout_and_context_survives(env):
    """With an iteration cap of 1 the tensor-core kernels give up their first
    waits, set the status word and return; the call reports SOX_ERR_TIMEOUT and
    the context stays usable for a normal call afterwards."""
    torch, pkg, hs = env
    w = synth.molecule(16, 64, 256, 4, 100.0, n_spin=1)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    S = torch.empty_like(G)
    with pkg.Handle("f16x2", spin_limit=1) as h1:
        pkg.sox_sigma(h1, p, G, X, V, S)
        with pytest.raises(pkg.SoxError) as e:
            pkg.sox_check_device(h1)
        assert e.value.code == 6
        pkg.sox_check_device(h1)          # status was cleared
    pkg.sox_sigma(hs["f16x2"], p, G, X, V, S)
    pkg.sox_check_device(hs["f16x2"])
    check(S.cpu().numpy(), sox.sox_sigma(w.X, w.V, w.G, dtype=np.float64), "f16x2", "after timeout")


@pytest.mark.parametrize("prec", PRECS)
def test_nonsymmetric_G_takes_the_general_projection(env, prec):
    """G(tau) is symmetric for real molecular orbitals, and the split path then
    reuses G_Rq for G_wP^T; a non-symmetric G must still give the definition."""
    w = synth.molecule(17, 26, 130, 5, 100.0, n_spin=2)
    rng = np.random.default_rng(5)
    G = w.G.copy()
    G[1] += 0.05 * np.abs(G[1]).max() * rng.standard_normal(G[1].shape)   # spin 1 only
    w.G = np.ascontiguousarray(G)
    ref = sox.sox_sigma(w.X, w.V, w.G, dtype=np.float64)
    check(_sigma(env, prec, w), ref, prec, "non-symmetric G")


@pytest.mark.parametrize("prec", PRECS)
def test_capture_in_cuda_graph_and_replay(env, prec):
    """After one un-captured call sizes the workspace, a whole build is one
    graph: no allocation, no host synchronisation inside the call."""
    torch, pkg, hs = env
    w = synth.molecule(18, 40, 200, 6, 100.0, n_spin=2)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    eager = torch.empty_like(G)
    pkg.sox_sigma(hs[prec], p, G, X, V, eager)          # sizes the workspace
    torch.cuda.synchronize()
    out = torch.full_like(G, float("nan"))
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            pkg.sox_sigma(hs[prec], p, G, X, V, out)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()                        # capture ran nothing
    for k in range(2):
        G.mul_(1.0 + 0.01 * k)                           # new inputs in the captured buffers
        graph.replay()
        ref = torch.empty_like(G)
        pkg.sox_sigma(hs[prec], p, G, X, V, ref)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    pkg.sox_check_device(hs[prec])


@pytest.mark.parametrize("n,N", [(40, 200), (150, 300)])
def test_autotuned_and_fixed_fused_kernel_agree(env, n, N):
    """The autotuner times the fused kernel's variants on the first call for a shape;
    whichever it keeps, the result meets the parity bar and matches the fixed choice."""
    torch, pkg, _ = env
    w = synth.molecule(19, n, N, 4, 100.0)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    out = {}
    for tune in (True, False):
        with pkg.Handle("f16x2", autotune=tune) as h:
            for _ in range(2):                       # first call tunes, second uses the kept choice
                S = torch.full_like(G, float("nan"))
                pkg.sox_sigma(h, p, G, X, V, S)
            pkg.sox_check_device(h)
            out[tune] = S.cpu().numpy()
    ref = sox.sox_sigma(w.X, w.V, w.G, dtype=np.float64)
    for r in out.values():
        check(r, ref, "f16x2", "autotune")
    assert np.abs(out[True] - out[False]).max() <= 1e-9


@pytest.mark.parametrize("prec", PRECS)
def test_g3w2_and_2sosex_static(env, prec):
    """The screened compositions of Sec. III C on the GPU against the oracle's decomposition."""
    torch, pkg, hs = env
    w = synth.molecule(28, 18, 90, 6, 100.0, n_spin=2)
    rng = np.random.default_rng(5)
    z = rng.standard_normal((w.N, w.N)) / w.N
    W = (0.6 * w.V[0] + 0.05 * z @ z.T)[None]
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, Wd = to_dev(torch, w.G, w.X, w.V, W)
    S = torch.full_like(G, float("nan"))
    pkg.g3w2_static_sigma(hs[prec], p, G, X, Wd, S)
    check(S.cpu().numpy(), sox.g3w2_static_sigma(w.X, W, w.G, dtype=np.float64), prec, "G3W2stat")
    S.fill_(float("nan"))
    pkg.sosex2_static_sigma(hs[prec], p, G, X, V, Wd, S)
    pkg.sox_check_device(hs[prec])
    check(S.cpu().numpy(), sox.sosex2_static_sigma(w.X, w.V, W, w.G, dtype=np.float64), prec, "2SOSEXstat")
    Sh = np.full_like(w.G, np.nan)
    pkg.sosex2_static_sigma(hs[prec], p, w.G, X, V, W, Sh)      # host G and Sigma are staged
    assert np.array_equal(Sh, S.cpu().numpy())


@pytest.mark.parametrize("prec", PRECS)
def test_tau_shards_through_the_library_reassemble_the_build(env, prec):
    """One build split by mirror-pair tau shards (three ranks, run one after the other on
    this GPU): each shard's sox_sigma on its compact G, reassembled, equals the whole build."""
    from paper_2412_18829_gb300 import sharding

    torch, pkg, hs = env
    w = synth.molecule(29, 21, 100, 9, 100.0, n_spin=2)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    full = torch.empty_like(G)
    pkg.sox_sigma(hs[prec], pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta), G, X, V, full)
    orders = sharding.tau_shards(w.n_tau, 3)
    parts = []
    for order in orders:
        Gc = G[:, :, order].contiguous()
        Sc = torch.full_like(Gc, float("nan"))
        pkg.sox_sigma(hs[prec], pkg.problem(w.n, w.N, len(order), w.n_spin, w.beta), Gc, X, V, Sc)
        parts.append(Sc)
    got = sharding.assemble(parts, orders, w.n_tau)
    pkg.sox_check_device(hs[prec])
    err = float((got - full).abs().max())
    assert err <= (1e-14 if prec == "fp64" else 1e-9) * float(full.abs().max())
    check(got.cpu().numpy(), sox.sox_sigma(w.X, w.V, w.G, dtype=np.float64), prec, "tau shards")
