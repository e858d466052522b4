"""The C-ABI library builds, loads and exports every declared entry point (CPU only)."""
import glob
import os
import re

import numpy as np
import pytest

from oracle import grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2412_18829_gb300 import build

    build.build()
    import paper_2412_18829_gb300 as p

    p.lib()
    return p


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names |= set(re.findall(r"^SOX_API\s+(?:int|const char \*)\s*(\w+)\(", open(h).read(), flags=re.M))
    return names


def test_every_declared_symbol_is_exported(pkg):
    declared = _declared()
    assert len(declared) >= 16
    lib = pkg.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(pkg.EXPORTED)


def test_only_the_c_abi_is_exported(pkg):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", pkg._binding.LIB_PATH], capture_output=True,
                         text=True).stdout
    text = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert text == _declared()


@pytest.mark.parametrize("n_tau,beta", [(2, 1.0), (3, 2.0), (30, 100.0), (101, 7.0)])
def test_tau_grid_matches_oracle(pkg, n_tau, beta):
    tau, w = pkg.sox_tau_grid(n_tau, beta)
    np.testing.assert_allclose(tau, grid.chebyshev_lobatto(n_tau, beta), atol=1e-13 * beta)
    np.testing.assert_allclose(w, grid.clenshaw_curtis(n_tau, beta), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(tau[::-1], beta - tau, rtol=0, atol=4e-16 * beta)


def test_tau_grid_rejects_bad_arguments(pkg):
    with pytest.raises(pkg.SoxError):
        pkg.sox_tau_grid(1, 1.0)
    with pytest.raises(pkg.SoxError):
        pkg.sox_tau_grid(5, -1.0)


def test_create_without_gpu_fails_cleanly(pkg):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.SoxError):
        pkg.Handle("fp64")


def test_binding_rejects_wrong_dtype(pkg):
    from paper_2412_18829_gb300 import _binding

    with pytest.raises(ValueError):
        _binding._ptr(np.zeros(3, np.float32))
    with pytest.raises(ValueError):
        _binding._ptr(np.zeros((3, 3))[:, ::2])
