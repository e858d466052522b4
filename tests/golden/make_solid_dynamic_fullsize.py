"""Writes the oracle's dynamically screened SOSEX of a solid at tile counts of the full-size
solid (N = 300: three 128-row P/R tiles; 3x3x3 with N = 130: two), for the GPU parity test
tests/test_gpu_fullsize.py::test_solid_dynamic_full_tiles_against_stored_oracle.

The oracle (oracle/kpoints.py, the dynamic chain of Sec. II C with momenta, plus the static
SOX(v, v)) needs minutes per case in numpy, so its results are stored here once:

    python tests/golden/make_solid_dynamic_fullsize.py

Inputs come from synth/ (the solid recipe at beta = 300, the Chebyshev-Lobatto transform pair
with M = 1, the single-pole W_d); each file also stores fingerprints of those inputs, which the
tests compare before trusting the stored Sigma.  Only synth/ and oracle/ are called.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# name -> (k-mesh, n, N, n_tau); M = 1 (three bosonic frequencies)
CASES = {
    "solid_dynamic_k311_n26_N300_t4": ((3, 1, 1), 26, 300, 4),
    "solid_dynamic_k222_n26_N300_t3": ((2, 2, 2), 26, 300, 3),
    "solid_dynamic_k333_n12_N130_t3": ((3, 3, 3), 12, 130, 3),
}
M = 1
BETA = 300.0


def inputs(name):
    import synth

    nk, n, N, T = CASES[name]
    w = synth.solid(3, nk, n, N, T, BETA)
    _, Tf, Ti = synth.bosonic_transforms(w.tau, w.beta, M)
    Wd = synth.pole_screening(w.V, w.beta, M)
    return w, Tf, Ti, Wd


def fingerprint(w, Tf, Ti, Wd) -> np.ndarray:
    """sum |x|, sum |Re x| and sum |Im x| over every input tensor: sums of non-negative terms,
    so machines that round the generator's arithmetic differently agree to ~1e-14 relative."""
    out = []
    for a in (w.G, w.X, w.V, Wd, Tf, Ti):
        a = np.asarray(a, dtype=complex)
        out += [float(np.abs(a).sum()), float(np.abs(a.real).sum()), float(np.abs(a.imag).sum())]
    return np.array(out)


def path(name):
    return os.path.join(HERE, name + ".npz")


def main():
    from oracle import kpoints

    for name, (nk, n, N, T) in CASES.items():
        w, Tf, Ti, Wd = inputs(name)
        ref = kpoints.sosex_dynamic_sigma(w.X, w.V, Wd, Tf, Ti, w.G, nk)
        np.savez_compressed(path(name), sigma=ref, fingerprint=fingerprint(w, Tf, Ti, Wd))
        print(name, "max|Sigma|", float(np.abs(ref).max()))


if __name__ == "__main__":
    main()
