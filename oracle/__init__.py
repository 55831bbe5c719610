"""CPU oracle for the Jacobi-preconditioned CG and TFQMR paths and the stencil operator (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path never does; it shares no code
with it.
"""

from .oracle import (  # noqa: F401
    REASON,
    build,
    load,
    dot,
    spmv,
    spmv_f32,
    diagonal,
    pcg,
    tfqmr,
    stencil_apply,
    pcg_f32,
    ir,
    pcg_omp,
    build_omp,
    host_cores,
    host_cpu_model,
)
from .expr_oracle import expr_eval  # noqa: F401
