"""Shared helpers for the GPU parity tests (inputs from synth/, expectations from oracle/)."""
import numpy as np
import pytest

# Parity bars.  FP64 path: rounding-order differences only.  Split-precision
# tensor-core path: the absolute bound max|dSigma| <= 1e-8 Ha on the workloads
# (strict=True); on degenerate shapes whose |Sigma| is far above a molecule's
# (N < n, tiny beta) the FP32-class relative bound 2e-6 max|Sigma| applies.
FP64_REL = 1e-12
MIXED_ABS = 1e-8
MIXED_REL = 2e-6


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


def check(out, ref, prec, what="", strict=False):
    err = float(np.abs(out - ref).max())
    scale = float(np.abs(ref).max())
    if prec == "fp64":
        assert err <= FP64_REL * max(scale, 1e-300), f"{what}: fp64 max|d| {err:.3e} vs max|ref| {scale:.3e}"
    elif strict:
        assert err <= MIXED_ABS, f"{what}: {prec} max|d| {err:.3e} Ha (max|ref| {scale:.3e})"
    else:
        assert err <= max(MIXED_ABS, MIXED_REL * scale), f"{what}: {prec} max|d| {err:.3e} (max|ref| {scale:.3e})"
    return err, scale
