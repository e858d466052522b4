"""GPU tests of batch plans: the sox_sigma sequence of an uneven batch recorded once into a
CUDA graph and replayed, against the eager batch call and the oracle."""
import numpy as np
import pytest

import synth
from oracle import sox
from gpu_common import check, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [(13, 70, 6, 2), (40, 200, 5, 1), (150, 300, 4, 1)]   # n, N, n_tau, n_spin


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    yield torch, pkg


def _batch(torch, pkg):
    ws = [synth.molecule(60 + i, n, N, T, 100.0, n_spin=s) for i, (n, N, T, s) in enumerate(SHAPES)]
    probs = [pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta) for w in ws]
    dev = [to_dev(torch, w.G, w.X, w.V) for w in ws]
    G, X, V = [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev]
    return ws, probs, G, X, V


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_plan_replays_the_batch_with_new_inputs(env, prec):
    torch, pkg = env
    ws, probs, G, X, V = _batch(torch, pkg)
    S = [torch.full_like(g, float("nan")) for g in G]
    R = [torch.empty_like(g) for g in G]
    with pkg.Handle(prec) as h, pkg.SigmaBatchPlan(h, probs, G, X, V, S) as plan:
        for k in range(2):
            for g in G:                     # new values in the recorded buffers
                g.mul_(1.0 + 0.02 * (k + 1))
            for s in S:
                s.fill_(float("nan"))
            plan.launch()
            plan.check_device()
            pkg.sox_sigma_batch(h, probs, G, X, V, R)
            torch.cuda.synchronize()
            for s, r in zip(S, R):
                assert torch.isfinite(s).all()
                scale = float(r.abs().max())
                tol = 1e-14 if prec == "fp64" else 1e-9
                assert float((s - r).abs().max()) <= tol * max(scale, 1e-300)
        # the last replay against the oracle, on the largest instance
        w = ws[-1]
        Gh = G[-1].cpu().numpy()
        ref = sox.sox_sigma(w.X, w.V, Gh, dtype=np.float64)
        check(S[-1].cpu().numpy(), ref, prec, "plan replay")


def test_plan_rejects_host_tensors_and_solids(env):
    torch, pkg = env
    ws, probs, G, X, V = _batch(torch, pkg)
    S = [torch.empty_like(g) for g in G]
    with pkg.Handle("fp64") as h:
        host_G = [g.cpu() for g in G]
        with pytest.raises(pkg.SoxError) as e:
            pkg.SigmaBatchPlan(h, probs, host_G, X, V, S)
        assert e.value.code == 1
        solid = [pkg.problem(3, 5, 3, 1, 10.0, nk=(1, 1, 2), dtype=1)]
        with pytest.raises(pkg.SoxError) as e:
            pkg.SigmaBatchPlan(h, solid, G[:1], X[:1], V[:1], S[:1])
        assert e.value.code == 3


UNEVEN = [(57, 342, 4, 1), (150, 900, 2, 1), (79, 474, 3, 2), (33, 300, 3, 1), (13, 70, 5, 2)]


def _uneven(torch, pkg, shapes=UNEVEN):
    ws = [synth.molecule(80 + i, n, N, T, 100.0, n_spin=s) for i, (n, N, T, s) in enumerate(shapes)]
    probs = [pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta) for w in ws]
    dev = [to_dev(torch, w.G, w.X, w.V) for w in ws]
    return ws, probs, [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev]


@pytest.mark.parametrize("limit", [0, 1])
def test_batched_fused_launch_equals_the_instances_built_alone(env, limit):
    """The split path's uneven batch runs the fused step of every tau chunk of every instance
    as one persistent launch (n from 13 to 150, Kp 64 to 192, one and two spins, odd and even
    tile counts); with the streamed kernel forced on the single builds, every instance's Sigma
    is bit-identical to its own build, with the default chunking and with one batch per chunk
    (limit = 1), and the smallest and largest instances meet the oracle."""
    torch, pkg = env
    ws, probs, G, X, V = _uneven(torch, pkg)
    S = [torch.full_like(g, float("nan")) for g in G]
    with pkg.Handle("f16x2", workspace_limit=limit) as hb, pkg.Handle("f16x2") as hs:
        pkg.sox_set_kernel_variant(hs, "streamed")
        pkg.sox_sigma_batch(hb, probs, G, X, V, S)
        pkg.sox_check_device(hb)
        for i, w in enumerate(ws):
            R = torch.full_like(G[i], float("nan"))
            pkg.sox_sigma(hs, probs[i], G[i], X[i], V[i], R)
            pkg.sox_check_device(hs)
            assert torch.equal(S[i], R), f"instance {i}"
    for i in (0, 1):   # largest n first in UNEVEN[1], smallest N x n in UNEVEN[4]
        w = ws[[1, 4][i]]
        ref = sox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[0, 0], taus=[0, w.n_tau - 1], dtype=np.float64)
        got = S[[1, 4][i]].cpu().numpy()[0, 0, [0, w.n_tau - 1]]
        check(got, ref, "f16x2", f"batched instance n={w.n}", n=w.n, N=w.N)


def test_batched_fused_launch_keeps_the_v_range(env):
    torch, pkg = env
    ws, probs, G, X, V = _uneven(torch, pkg, UNEVEN[:3])
    with pkg.Handle("f16x2") as hb, pkg.Handle("f16x2") as hs:
        pkg.sox_set_kernel_variant(hs, "streamed")
        for h in (hb, hs):
            pkg.sox_set_v_range(h, 5, 40)
        S = [torch.full_like(g, float("nan")) for g in G]
        pkg.sox_sigma_batch(hb, probs, G, X, V, S)
        for i in range(len(ws)):
            R = torch.full_like(G[i], float("nan"))
            pkg.sox_sigma(hs, probs[i], G[i], X[i], V[i], R)
            assert torch.equal(S[i], R), f"instance {i}"


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_phi_sox_batch_matches_phi_sox(env, prec):
    torch, pkg = env
    ws, probs, G, X, V = _uneven(torch, pkg, UNEVEN[:3])
    wts = [torch.from_numpy(np.ascontiguousarray(pkg.sox_tau_grid(w.n_tau, w.beta)[1])).cuda() for w in ws]
    S = [torch.full_like(g, float("nan")) for g in G]
    phi = [torch.full((w.n_spin,), float("nan"), dtype=torch.float64, device="cuda") for w in ws]
    with pkg.Handle(prec) as hb, pkg.Handle(prec) as hs:
        if prec == "f16x2":
            pkg.sox_set_kernel_variant(hs, "streamed")
        pkg.phi_sox_batch(hb, probs, G, X, V, wts, phi, S)
        for i in range(len(ws)):
            R = torch.full_like(G[i], float("nan"))
            p1 = torch.full((ws[i].n_spin,), float("nan"), dtype=torch.float64, device="cuda")
            pkg.phi_sox(hs, probs[i], G[i], X[i], V[i], wts[i], p1, R)
            assert torch.equal(S[i], R) and torch.equal(phi[i], p1), f"instance {i}"
