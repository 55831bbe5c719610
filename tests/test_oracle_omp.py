"""The multi-threaded timing variant of the float64 oracle (the CPU baseline on all host cores) runs the
same steps as the sequential oracle: same iteration count and the same iterate up to summation order, for
every thread count, on a 2-D and a 3-D Laplacian, a variable-coefficient 27-point system and a ragged
random SPD matrix; a bad diagonal and a non-finite right-hand side give the oracle's reasons."""

import numpy as np
import pytest

from synthetic import laplace_2d_5pt, random_spd_csr, rhs_from_solution, single_problem


@pytest.fixture(scope="module")
def omp(orc):
    if orc.build_omp() is None:
        pytest.skip("gcc without OpenMP")
    return orc


@pytest.mark.parametrize("threads", [1, 3, 8])
@pytest.mark.parametrize("case", ["c1", "c2", "c3", "random"])
def test_omp_variant_matches_sequential_oracle(omp, case, threads):
    if case == "random":
        rng = np.random.default_rng(9)
        A = random_spd_csr(3001, 0.003, rng, dominance=0.3)
        b = rhs_from_solution(A, rng.uniform(-1, 1, A.n))
    else:
        p = single_problem(case, seed=1, size={"c1": 40, "c2": 14, "c3": 9}[case])
        A, b = p.A, p.b
    ref = omp.pcg(A, b, rtol=1e-10, check_every=3)
    got = omp.pcg_omp(A, b, rtol=1e-10, check_every=3, threads=threads)
    assert got["reason"] == ref["reason"] == "converged"
    assert got["iters"] == ref["iters"]
    assert np.linalg.norm(got["x"] - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-12
    fixed = omp.pcg_omp(A, b, rtol=0.0, max_it=7, threads=threads)
    assert fixed["iters"] == 7 and fixed["reason"] == "not_converged"
    assert np.linalg.norm(fixed["x"] - omp.pcg(A, b, rtol=0.0, max_it=7)["x"]) <= 1e-13 * np.linalg.norm(fixed["x"])


def test_omp_variant_failure_reasons(omp):
    A = laplace_2d_5pt(10)
    b = np.ones(A.n)
    b[3] = np.nan
    assert omp.pcg_omp(A, b, threads=2)["reason"] == "breakdown"
    A.val[A.rowptr[5]:A.rowptr[6]][A.col[A.rowptr[5]:A.rowptr[6]] == 5] = 0.0
    assert omp.pcg_omp(A, np.ones(A.n), threads=2)["reason"] == "bad_diagonal"
