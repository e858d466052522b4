"""Small-case drivers for ncu captures (one process, one GPU, a few GB at most).

    python -m paper_2412_18829_gb300.probes.profile_case molecule [f16x2|fp64] [n_tau]
        sox_sigma twice on the mid-size molecule's shapes (n=120, N=600, 2 spins), 8 tau by default
    python -m paper_2412_18829_gb300.probes.profile_case solid [f16x2|fp64] [n_tau] [mesh] [n,N]
        one sosex_dynamic_sigma on the 3x3x3 solid's shapes (n=26, N=300), 4 tau by default,
        with the synthetic single-pole W_d; another mesh ("4,4,4") and sizes ("10,100") optional
    python -m paper_2412_18829_gb300.probes.profile_case screened [f16x2|fp64] [n_tau]
        sox_sigma twice on the screened molecule's shapes (n=250, N=2000), 4 tau by default
    python -m paper_2412_18829_gb300.probes.profile_case wdyn [-] [n_tau]
        sox_w_dynamic (RPA W_d for every transfer and frequency, FP64) on the 3x3x3 solid's
        shapes (n=26, N=300), 60 tau and 59 frequencies by default
    python -m paper_2412_18829_gb300.probes.profile_case adjoint [f16x2|fp64] [n_tau]
        phi_sox_backward (dX, dV) twice on the largest batch instance's shapes (n=298,
        N=1788), 8 tau by default
"""
from __future__ import annotations

import sys

import numpy as np


def main(argv):
    import torch

    import paper_2412_18829_gb300 as pkg
    import synth

    kind = argv[1] if len(argv) > 1 else "molecule"
    prec = argv[2] if len(argv) > 2 else "f16x2"
    if kind == "molecule":
        T = int(argv[3]) if len(argv) > 3 else 8
        w = synth.molecule(1, 120, 600, T, 100.0, n_spin=2)
        p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
        G, X, V = [torch.from_numpy(a).cuda() for a in (w.G, w.X, w.V)]
        S = torch.empty_like(G)
        with pkg.Handle(prec) as h:
            for _ in range(2):
                pkg.sox_sigma(h, p, G, X, V, S)
            pkg.sox_check_device(h)
    elif kind == "screened":
        T = int(argv[3]) if len(argv) > 3 else 4
        w = synth.molecule(2, 250, 2000, T, 100.0, 1)
        p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
        G, X, V = [torch.from_numpy(a).cuda() for a in (w.G, w.X, w.V)]
        S = torch.empty_like(G)
        with pkg.Handle(prec) as h:
            for _ in range(2):
                pkg.sox_sigma(h, p, G, X, V, S)
            pkg.sox_check_device(h)
    elif kind == "solid":
        T = int(argv[3]) if len(argv) > 3 else 4
        mesh = tuple(int(x) for x in argv[4].split(",")) if len(argv) > 4 else (3, 3, 3)
        n, N = (int(x) for x in argv[5].split(",")) if len(argv) > 5 else (26, 300)
        w = synth.solid(3, mesh, n, N, T, 300.0)
        M = (T - 1) // 2
        _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
        Wd = synth.pole_screening(w.V, w.beta, M)
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=complex)).cuda()   # noqa: E731
        G, X, V, W, F, I = (to(a) for a in (w.G, w.X, w.V, Wd, Tf, Ti))
        S = torch.empty_like(G)
        p = pkg.problem(w.n, w.N, T, 1, w.beta, nk=w.nk, dtype=1)
        with pkg.Handle(prec) as h:
            pkg.sosex_dynamic_sigma(h, p, G, X, V, W, F, I, 2 * M + 1, S)
            pkg.sox_check_device(h)
    elif kind == "adjoint":
        T = int(argv[3]) if len(argv) > 3 else 8
        n = int(synth.batch_c4_sizes().max())
        w = synth.molecule(4, n, 6 * n, T, 100.0, 1)
        _, wts = pkg.sox_tau_grid(w.n_tau, w.beta)
        p = pkg.problem(w.n, w.N, w.n_tau, w.n_spin, w.beta)
        G, X, V, tw = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w.G, w.X, w.V, wts)]
        d = torch.ones(1, dtype=torch.float64, device="cuda")
        dX, S = torch.empty_like(X), torch.empty_like(V)
        with pkg.Handle(prec) as h:
            for _ in range(2):
                pkg.phi_sox_backward(h, p, G, X, V, tw, d, None, dX, S)
            pkg.sox_check_device(h)
    elif kind == "wdyn":
        T = int(argv[3]) if len(argv) > 3 else 60
        w = synth.solid(3, (3, 3, 3), 26, 300, T, 300.0)
        M = (T - 1) // 2
        _, Tf, _ = synth.bosonic_transforms(w.tau, w.beta, M)
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=complex)).cuda()   # noqa: E731
        G, X, V, F = (to(a) for a in (w.G, w.X, w.V, Tf))
        S = torch.empty(27, 2 * M + 1, w.N, w.N, dtype=torch.complex128, device="cuda")
        p = pkg.problem(w.n, w.N, T, 1, w.beta, nk=w.nk, dtype=1)
        with pkg.Handle("fp64") as h:
            pkg.sox_w_dynamic(h, p, G, X, V, F, 2 * M + 1, S)
    else:
        raise SystemExit(f"unknown case {kind}")
    torch.cuda.synchronize()
    print("ok", float(S.abs().max()))


if __name__ == "__main__":
    main(sys.argv)
