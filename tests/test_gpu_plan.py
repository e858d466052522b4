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
