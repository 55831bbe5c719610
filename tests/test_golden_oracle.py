"""The oracle reproduces its stored fixtures (written by tests/golden/make_golden.py).

Tolerance 1e-13 relative rather than bit equality: the right-hand side is
formed by scipy's sparse product, whose build may fuse multiply-adds on some
hosts and so move b by an ulp.
"""

import json
import os

import numpy as np
import pytest

from synthetic import single_problem

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("key,name,size,k", [("c1_seed0", "c1", None, 1), ("c2_n32_seed0", "c2", 32, 10)])
def test_oracle_matches_fixture(orc, key, name, size, k):
    with open(os.path.join(HERE, "golden", "oracle_pcg_history.json")) as f:
        g = json.load(f)[key]
    p = single_problem(name, seed=0, size=size)
    r = orc.pcg(p.A, p.b, rtol=1e-8, check_every=k, hist_len=10)
    assert r["iters"] == g["iters"] and r["reason"] == g["reason"]
    for h in ("alpha", "beta"):
        ref = np.array([float.fromhex(v) for v in g[h]])
        assert np.allclose(r[h], ref, rtol=1e-13, atol=0)
    assert abs(r["rr"] - float.fromhex(g["rr_final"])) <= 1e-6 * float.fromhex(g["rr_final"])
