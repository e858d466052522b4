"""The stored oracle results under tests/golden/ belong to the inputs synth/ generates now
(CPU: regenerates the inputs and compares their fingerprints, no oracle run)."""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    path = os.path.join(HERE, "golden", "make_solid_dynamic_fullsize.py")
    spec = importlib.util.spec_from_file_location("make_solid_dynamic_fullsize", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", ["solid_dynamic_k311_n26_N300_t4", "solid_dynamic_k222_n26_N300_t3",
                                  "solid_dynamic_k333_n12_N130_t3"])
def test_stored_solid_dynamic_results_match_the_generated_inputs(name):
    gold = _golden()
    assert name in gold.CASES
    stored = np.load(gold.path(name))
    w, Tf, Ti, Wd = gold.inputs(name)
    assert np.allclose(stored["fingerprint"], gold.fingerprint(w, Tf, Ti, Wd), rtol=1e-10, atol=0.0)
    nk, n, N, T = gold.CASES[name]
    assert stored["sigma"].shape == (1, nk[0] * nk[1] * nk[2], T, n, n)
    assert np.isfinite(stored["sigma"]).all()
