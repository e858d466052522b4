"""The allocation-free entry point against the handle-based FP64 entry point (GPU).

sox_sigma_fp64_noalloc serves callers that may not allocate device memory (a
handle allocates its workspace with cudaMalloc).  It must give the handle
path's result, also on a second call that reuses the library's fixed scratch
array and after a call of a different size left other contents in it.  This
file is collected last so a stop-at-first-failure run has already run every
other test.
"""
import numpy as np
import pytest

import synth
from gpu_common import FP64_REL, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _handle_result(torch, pkg, p, G, X, V):
    S = torch.empty_like(G)
    with pkg.Handle("fp64") as h:
        pkg.sox_sigma(h, p, G, X, V, S)
    torch.cuda.synchronize()
    return S.cpu().numpy()


@pytest.mark.parametrize("dims", [(18, 96, 7, 2), (33, 140, 5, 1)])
def test_noalloc_matches_handle_path_on_two_calls(dims):
    torch = torch_cuda()
    pkg = pkg_built()
    n, N, T, S_ = dims
    w = synth.molecule(31, n, N, T, 100.0, n_spin=S_)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    ref = _handle_result(torch, pkg, p, G, X, V)
    scale = np.abs(ref).max()
    assert scale > 0
    # a call of another size first, so the shared scratch holds other contents
    w2 = synth.molecule(32, 11, 50, 4, 100.0)
    p2 = pkg.problem(w2.n, w2.N, w2.n_tau, w2.n_spin, w2.beta)
    G2, X2, V2 = to_dev(torch, w2.G, w2.X, w2.V)
    pkg.sox_sigma_fp64_noalloc(p2, G2, X2, V2, torch.empty_like(G2))
    for _ in range(2):
        out = torch.full_like(G, float("nan"))
        pkg.sox_sigma_fp64_noalloc(p, G, X, V, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= FP64_REL * scale


def test_noalloc_chunks_tau_near_its_scratch_bound_on_a_side_stream():
    """n = 80, N = 480 leaves room for one tau point per chunk in the 64 MiB array, so
    the chunk loop runs n_tau times (the G(-tau) stride then starts at T-1-t0 with t0 > 0);
    the calls are queued on a non-default stream and checked against the handle path."""
    torch = torch_cuda()
    pkg = pkg_built()
    w = synth.molecule(33, 80, 480, 6, 100.0, n_spin=2)
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    ref = _handle_result(torch, pkg, p, G, X, V)
    scale = np.abs(ref).max()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        outs = [torch.full_like(G, float("nan")) for _ in range(2)]
        for out in outs:   # two calls in a row on the side stream
            pkg.sox_sigma_fp64_noalloc(p, G, X, V, out, stream=side)
    side.synchronize()
    for out in outs:
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= FP64_REL * scale


def test_noalloc_rejects_problems_beyond_its_scratch():
    torch = torch_cuda()
    pkg = pkg_built()
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.SoxError) as e:
        pkg.sox_sigma_fp64_noalloc(pkg.problem(120, 600, 4), t, t, t, t)
    assert e.value.code == 2
    with pytest.raises(pkg.SoxError) as e:
        pkg.sox_sigma_fp64_noalloc(pkg.problem(4, 8, 4), np.zeros(64), t, t, t)
    assert e.value.code == 1
