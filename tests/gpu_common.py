"""Shared helpers for the GPU parity tests (inputs from synth/, expectations from oracle/)."""
import numpy as np
import pytest

# Parity bars.  FP64 path: rounding-order differences only.  Split-precision
# tensor-core path: the absolute bound max|dSigma| <= 1e-8 Ha of the target, on
# every shape, with one exception that the check decides by itself (no caller can
# opt in): degenerate shapes, with fewer THC points than orbitals (N < n) or a
# self-energy of order 1 Ha (max|Sigma| >= 0.05 Ha: more than three times the
# largest |Sigma| of any molecular or solid workload, 1.5e-2 Ha, reached only by toy
# inputs at beta = 10 or with N < n), are held to the FP32-class relative bound
# 2e-6 max|Sigma| instead.
FP64_REL = 1e-12
MIXED_ABS = 1e-8
MIXED_REL = 2e-6
DEGENERATE_SIGMA = 0.05


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    return torch


def pkg_built():
    from paper_2412_18829_gb300 import build

    build.build()
    import paper_2412_18829_gb300 as pkg

    pkg.lib()
    return pkg


def to_dev(torch, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def check(out, ref, prec, what="", n=None, N=None):
    """Element-wise parity of `out` with the oracle's `ref`; returns (max|d|, max|ref|).
    n, N (orbitals, THC points) let the check recognise the N < n degenerate case."""
    err = float(np.abs(out - ref).max())
    scale = float(np.abs(ref).max())
    if prec == "fp64":
        assert err <= FP64_REL * max(scale, 1e-300), f"{what}: fp64 max|d| {err:.3e} vs max|ref| {scale:.3e}"
        return err, scale
    degenerate = (n is not None and N is not None and N < n) or scale >= DEGENERATE_SIGMA
    bar = max(MIXED_ABS, MIXED_REL * scale) if degenerate else MIXED_ABS
    assert err <= bar, (f"{what}: {prec} max|d| {err:.3e} Ha > {bar:.1e} (max|ref| {scale:.3e}"
                        f"{', degenerate shape' if degenerate else ''})")
    return err, scale
