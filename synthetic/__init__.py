"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds matrices and right-hand sides only.  It holds none of the
solver's arithmetic (no preconditioner, no Krylov step, no reduction); the
one product it forms, b = A x_true, is delegated to ``scipy.sparse``.

The workloads follow the experiments of Sec. 4.1 (finite-difference Laplace
operators with 5/7/27-point stencils, Jacobi preconditioning) and the
extensions built on them (variable-coefficient diffusion, shifted and
anisotropic batches).  Every generator is deterministic given its seed.
"""

from .stencils import (  # noqa: F401
    CSR,
    laplace_2d_5pt,
    laplace_2d_9pt,
    laplace_3d_7pt,
    laplace_3d_27pt,
    diffusion_3d_27pt,
    aniso_3d_7pt_fp32exact,
    diagonal_csr,
    random_spd_csr,
    graph_laplacian_csr,
    convection_diffusion_2d,
    stencil_terms,
    stencil_matrix,
    sine_mode_2d,
    sine_mode_3d,
    rhs_from_solution,
)
from .problems import (  # noqa: F401
    Problem,
    Batch,
    single_problem,
    batch_shifted_5pt,
    batch_aniso_7pt,
    PROBLEMS,
)
