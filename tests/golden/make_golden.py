"""Write the stored oracle fixtures in this folder.

Calls only the CPU oracle (``oracle/``) on seeded synthetic inputs.  The
fixture pins the oracle's own output across hosts (x86 and Arm builds must
agree bit for bit, the oracle being compiled without fused multiply-add) and
across later edits of the oracle.  The paper prints no worked example, so no
stored value here comes from the paper.

Usage: python tests/golden/make_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from synthetic import single_problem  # noqa: E402


def main():
    out = {}
    p = single_problem("c1", seed=0)
    r = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=1, hist_len=10)
    out["c1_seed0"] = {
        "workload": "2-D 5-point Laplacian 64x64, x_true ~ U[-1,1] seed 0, b = A x_true, x0 = 0, rtol 1e-8, k = 1",
        "iters": r["iters"],
        "reason": r["reason"],
        "alpha": [float(v).hex() for v in r["alpha"]],
        "beta": [float(v).hex() for v in r["beta"]],
        "rr_final": float(r["rr"]).hex(),
    }
    p = single_problem("c2", seed=0, size=32)
    r = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=10, hist_len=10)
    out["c2_n32_seed0"] = {
        "workload": "3-D 7-point Laplacian 32^3, x_true ~ U[-1,1] seed 0, b = A x_true, x0 = 0, rtol 1e-8, k = 10",
        "iters": r["iters"],
        "reason": r["reason"],
        "alpha": [float(v).hex() for v in r["alpha"]],
        "beta": [float(v).hex() for v in r["beta"]],
        "rr_final": float(r["rr"]).hex(),
    }
    p = single_problem("c2", seed=0)
    r = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=10, hist_len=10)
    out["c2_full_seed0"] = {
        "workload": "3-D 7-point Laplacian 128^3, x_true ~ U[-1,1] seed 0, b = A x_true, x0 = 0, rtol 1e-8, k = 10",
        "iters": r["iters"],
        "reason": r["reason"],
        "alpha": [float(v).hex() for v in r["alpha"]],
        "beta": [float(v).hex() for v in r["beta"]],
        "rr_final": float(r["rr"]).hex(),
    }
    with open(os.path.join(HERE, "oracle_pcg_history.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
