"""A build split over the orbital index v (sox_set_v_range): the partial results of a
partition of [0, n), summed, equal the whole build -- every path, both precisions (GPU,
the ranks emulated as successive calls on one handle)."""
import numpy as np
import pytest

import synth
from oracle import grid
from paper_2412_18829_gb300 import sharding
from gpu_common import MIXED_ABS, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _bar(prec, ref):
    scale = float(np.abs(ref).max())
    return 1e-12 * scale if prec == "fp64" else MIXED_ABS


def _split_sum(pkg, h, n, world, run):
    """sum over the shards of run() with the handle restricted to each shard's v range."""
    total = None
    for v0, v1 in sharding.v_shards(n, world):
        pkg.sox_set_v_range(h, v0, v1)
        part = run()
        total = part if total is None else total + part
    pkg.sox_set_v_range(h, 0, 0)
    return total


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_v_split_static_molecule(prec):
    torch = torch_cuda()
    pkg = pkg_built()
    w = synth.molecule(81, 21, 140, 6, 100.0, n_spin=2)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    with pkg.Handle(prec) as h:
        def run():
            S = torch.full_like(G, float("nan"))
            pkg.sox_sigma(h, p, G, X, V, S)
            return S.cpu().numpy()
        full = run()
        got = _split_sum(pkg, h, w.n, 3, run)
    assert np.abs(got - full).max() <= _bar(prec, full)


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_v_split_dynamic_molecule(prec):
    torch = torch_cuda()
    pkg = pkg_built()
    w = synth.molecule(82, 12, 60, 6, 100.0)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, 2)
    Wd = synth.pole_screening(w.V, w.beta, 2)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, W, F, I = to_dev(torch, w.G, w.X, w.V, Wd, Tf, Ti)
    with pkg.Handle(prec) as h:
        def run():
            S = torch.full_like(G, float("nan"))
            pkg.sosex_dynamic_sigma(h, p, G, X, V, W, F, I, Tf.shape[0], S)
            return S.cpu().numpy()
        full = run()
        got = _split_sum(pkg, h, w.n, 2, run)
    assert np.abs(got - full).max() <= _bar(prec, full)


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_v_split_dynamic_solid(prec):
    torch = torch_cuda()
    pkg = pkg_built()
    w = synth.solid(83, (2, 1, 1), 6, 30, 4, 300.0)
    M = 1
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
    Wd = synth.pole_screening(w.V, w.beta, M)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta, nk=w.nk, dtype=1)
    cx = lambda a: np.ascontiguousarray(a, dtype=complex)   # noqa: E731
    G, X, V, W, F, I = to_dev(torch, cx(w.G), cx(w.X), cx(w.V), cx(Wd), cx(Tf), cx(Ti))
    with pkg.Handle(prec) as h:
        def run():
            S = torch.full_like(G, complex("nan"))
            pkg.sosex_dynamic_sigma(h, p, G, X, V, W, F, I, Tf.shape[0], S)
            return S.cpu().numpy()
        full = run()
        got = _split_sum(pkg, h, w.n, 3, run)
    assert np.abs(got - full).max() <= _bar(prec, full)


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
def test_v_split_phi_and_its_x_v_adjoint(prec):
    torch = torch_cuda()
    pkg = pkg_built()
    w = synth.molecule(84, 14, 70, 5, 3.0)
    wt = grid.clenshaw_curtis(w.n_tau, w.beta)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, tw = to_dev(torch, w.G, w.X, w.V, wt)
    d = torch.ones(1, dtype=torch.float64, device="cuda")
    with pkg.Handle(prec) as h:
        def run():
            phi = torch.empty(1, dtype=torch.float64, device="cuda")
            dX, dV = torch.empty_like(X), torch.empty_like(V)
            pkg.phi_sox(h, p, G, X, V, tw, phi)
            pkg.phi_sox_backward(h, p, G, X, V, tw, d, None, dX, dV)
            return np.concatenate([phi.cpu().numpy().ravel(), dX.cpu().numpy().ravel(), dV.cpu().numpy().ravel()])
        full = run()
        got = _split_sum(pkg, h, w.n, 2, run)
        pkg.sox_set_v_range(h, 0, 5)
        with pytest.raises(pkg.SoxError):   # dG needs the whole Sigma
            pkg.phi_sox_backward(h, p, G, X, V, tw, d, torch.empty_like(G), None, None)
        pkg.sox_set_v_range(h, 0, 0)
    rel = 1e-12 if prec == "fp64" else 2e-5
    assert abs(got[0] - full[0]) <= rel * abs(full[0])
    assert np.abs(got[1:] - full[1:]).max() <= rel * np.abs(full[1:]).max()
