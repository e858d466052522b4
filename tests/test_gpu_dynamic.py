"""GPU parity of dynamically screened SOSEX for molecules against the CPU oracle."""
import numpy as np
import pytest

import synth
from oracle import dynamic, screening
from gpu_common import check, pkg_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    pkg = pkg_built()
    hs = {p: pkg.Handle(p) for p in ("fp64", "f16x2")}
    yield torch, pkg, hs
    for h in hs.values():
        h.close()


def _inputs(n, N, n_tau, beta, M, n_spin, seed):
    w = synth.molecule(seed, n, N, n_tau, beta, n_spin=n_spin)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
    Wd = screening.w_dynamic(w.V[0], screening.pi_omega(w.X[0], w.G[0, 0], Tf))
    return w, Tf, Ti, np.ascontiguousarray(Wd)


def _run(env, prec, w, Tf, Ti, Wd):
    """prec: "fp64" / "f16x2" (the module's handles) or a Handle of its own."""
    torch, pkg, hs = env
    h = hs[prec] if isinstance(prec, str) else prec
    p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
    G, X, V, W = to_dev(torch, w.G, w.X, w.V, Wd)
    F = torch.from_numpy(Tf).cuda()
    I = torch.from_numpy(Ti).cuda()
    S = torch.full_like(G, float("nan"))
    pkg.sosex_dynamic_sigma(h, p, G, X, V, W, F, I, Tf.shape[0], S)
    pkg.sox_check_device(h)
    return S.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "f16x2"])
@pytest.mark.parametrize("n,N,n_tau,M,n_spin", [(7, 30, 8, 4, 1), (13, 70, 10, 5, 2), (20, 80, 12, 6, 1)])
def test_sosex_dynamic_matches_oracle(env, prec, n, N, n_tau, M, n_spin):
    w, Tf, Ti, Wd = _inputs(n, N, n_tau, 20.0, M, n_spin, seed=50 + n)
    ref = dynamic.sosex_dynamic_sigma(w.X, w.V, Wd, Tf, Ti, w.G).real
    got = _run(env, prec, w, Tf, Ti, Wd)
    check(got, ref, prec, f"dynamic n={n}", n=n, N=N)


def test_dynamic_part_alone_with_zero_screening_is_bare_sox(env):
    w, Tf, Ti, Wd = _inputs(9, 40, 6, 10.0, 3, 1, seed=60)
    got = _run(env, "fp64", w, Tf, Ti, np.zeros_like(Wd))
    from oracle import sox
    ref = sox.sox_sigma(w.X, w.V, w.G).real
    check(got, ref, "fp64", "W_d = 0")


def test_sosex_dynamic_split_two_tiles_and_tau_chunks(env):
    """Split precision on the tensor cores (transforms, W_d product, fused B/C/D) at two
    128-row P/R tiles and beta = 100, with the default tau chunk and with one tau point per
    chunk (workspace_limit = 1 byte), every element against the oracle at 1e-8 Ha."""
    torch, pkg, _ = env
    w, Tf, Ti, Wd = _inputs(40, 200, 10, 100.0, 5, 1, seed=70)
    ref = dynamic.sosex_dynamic_sigma(w.X, w.V, Wd, Tf, Ti, w.G).real
    for limit in (0, 1):
        with pkg.Handle("f16x2", workspace_limit=limit) as h:
            got = _run(env, h, w, Tf, Ti, Wd)
        err, scale = check(got, ref, "f16x2", f"dynamic split, workspace_limit={limit}", n=w.n, N=w.N)
        print(f"dynamic split limit={limit}: max|dSigma| {err:.3e} Ha (max|Sigma| {scale:.3e})")
