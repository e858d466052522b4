"""Every variant of the split path's fused B/C/D kernel (Sec. II C, the B, C and D steps) -
G_Rq / G_wP^T resident, all operands streamed, and streamed on CTA pairs - against the
oracle at the 1e-8 Ha bar: one and several P/R tiles, odd and even tile counts (the pair's
second CTA then idles on the last P pair or not), ragged N, n beyond one K chunk with a
partial last chunk, two interactions, a partial v range and the mid-size molecule."""
import numpy as np
import pytest

import synth
from oracle import sox
from gpu_common import check, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu
VARIANTS = ["resident", "streamed", "pair"]


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    hs = {}
    for v in VARIANTS:
        h = pkg.Handle("f16x2")
        pkg.sox_set_kernel_variant(h, v)
        hs[v] = h
    yield torch, pkg, hs
    for h in hs.values():
        h.close()


def _sigma(env, variant, w, U1=None, U2=None):
    torch, pkg, hs = env
    h = hs[variant]
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V = to_dev(torch, w.G, w.X, w.V)
    S = torch.full_like(G, float("nan"))
    if U1 is not None:
        A1, A2 = to_dev(torch, U1, U2)
        pkg.sox_sigma_general(h, p, G, X, A1, A2, S)
    else:
        pkg.sox_sigma(h, p, G, X, V, S)
    pkg.sox_check_device(h)
    return S.cpu().numpy()


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,N,n_tau,n_spin", [(13, 70, 6, 2), (64, 128, 3, 1), (40, 250, 3, 1), (33, 300, 4, 1),
                                              (70, 520, 2, 2), (150, 300, 2, 1), (5, 3, 2, 1)])
def test_variant_matches_oracle(env, variant, n, N, n_tau, n_spin):
    w = synth.molecule(21, n, N, n_tau, 100.0, n_spin=n_spin, name="variants")
    ref = sox.sox_sigma(w.X, w.V, w.G).real
    err, scale = check(_sigma(env, variant, w), ref, "f16x2", f"{variant} n={n} N={N}", n=n, N=N)
    print(f"{variant} n={n} N={N}: max|dSigma| {err:.3e} Ha (max|Sigma| {scale:.3e})")


@pytest.mark.parametrize("variant", ["streamed", "pair"])
def test_variant_two_interactions(env, variant):
    w = synth.molecule(22, 27, 260, 3, 100.0, n_spin=1)
    rng = np.random.default_rng(5)
    z = rng.standard_normal((w.N, w.N)) / w.N
    U1 = np.ascontiguousarray((z @ z.T + 0.3 * z)[None])
    U2 = np.ascontiguousarray(w.V)
    ref = np.stack([sox.sigma_tau(w.X[0], U1[0], U2[0], w.G[0, 0]).real])[:, None]
    check(_sigma(env, variant, w, U1, U2), ref, "f16x2", f"{variant} general", n=w.n, N=w.N)


def test_pair_partial_v_ranges_sum_to_the_build(env):
    torch, pkg, hs = env
    w = synth.molecule(23, 36, 290, 3, 100.0, n_spin=1)
    ref = sox.sox_sigma(w.X, w.V, w.G).real
    parts = []
    for v0, v1 in ((0, 11), (11, 36)):
        pkg.sox_set_v_range(hs["pair"], v0, v1)
        try:
            parts.append(_sigma(env, "pair", w))
        finally:
            pkg.sox_set_v_range(hs["pair"], 0, 0)
    check(parts[0] + parts[1], ref, "f16x2", "pair, two v ranges", n=w.n, N=w.N)


@pytest.mark.parametrize("variant", ["pair"])
def test_variant_mid_size_molecule_sampled_tau(env, variant):
    """n=120, N=600, 80 tau, 2 spins (five P tiles: the last pair half-empty)."""
    w = synth.config(1)
    out = _sigma(env, variant, w)
    assert np.isfinite(out).all()
    taus = [0, 40, 79]
    for s in range(w.n_spin):
        ref = sox.sigma_tau(w.X[0], w.V[0], w.V[0], w.G[s, 0], taus=taus, dtype=np.float64)
        err, scale = check(out[s, 0, taus], ref, "f16x2", f"{variant} mid-size spin {s}")
        print(f"{variant} mid-size spin {s}: max|dSigma| {err:.3e} Ha (max|Sigma| {scale:.3e})")


def test_sigma_is_bitwise_independent_of_tau_chunking(env):
    """Every (spin, tau) batch is computed with its own scales, so Sigma is bit-identical for
    one batch per chunk, the default chunking and a non-default caller stream, and meets the
    oracle."""
    torch, pkg, _ = env
    w = synth.molecule(24, 30, 260, 10, 100.0, n_spin=2)
    ref = sox.sox_sigma(w.X, w.V, w.G).real
    outs = []
    for limit, use_stream in ((0, False), (1, False), (0, True)):
        with pkg.Handle("f16x2", workspace_limit=limit) as h:
            pkg.sox_set_kernel_variant(h, "streamed")
            p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
            G, X, V = to_dev(torch, w.G, w.X, w.V)
            S = torch.full_like(G, float("nan"))
            if use_stream:
                st = torch.cuda.Stream()
                with torch.cuda.stream(st):
                    pkg.sox_sigma(h, p, G, X, V, S, stream=st.cuda_stream)
                st.synchronize()
            else:
                pkg.sox_sigma(h, p, G, X, V, S)
            pkg.sox_check_device(h)
            outs.append(S.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    check(outs[0], ref, "f16x2", "tau chunking", n=w.n, N=w.N)
