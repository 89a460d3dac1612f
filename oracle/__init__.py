"""Oracle: a plain, slow, FP64 CPU implementation of the DACG-Newton eigensolver
with the BFGS-updated IC preconditioner (Bergamaschi & Martinez, arXiv:1312.1553).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, the smoke check in
``__graft_entry__.py`` and the CPU-baseline leg of ``bench.py`` may import it.
The CUDA library (``paper_1312_1553_gb300``) never imports, links or calls it,
and the two share no code: the only common module is ``workloads`` (seeded
input generators, no solver arithmetic).

Layout
  nle_oracle.c   IC(lfil, tau) factor, level sets, SpMV, triangular solves
                 (plain C, FP64, built with -O2 -ffp-contract=off).
  ic.py          ctypes bindings of the C file.
  solver.py      Algorithm 3.1 (preconditioner application), PCG on the
                 correction equation (Section 4.3), DACG (Section 4.1),
                 Algorithm 3.2 (DACG-Newton) and the adjoint of the
                 eigenpairs (not in the paper).

Parity status of each function is stated in its docstring.
"""
from .ic import ICFactor, build_library, ic_factor, levels, level_sets, spmv, lsolve, usolve  # noqa: F401
from .solver import (  # noqa: F401
    OracleOptions,
    adjoint_grad,
    bfgs_apply,
    dacg,
    dacg_newton,
    fix_sign,
    pcg_correction,
    projected_solve,
)
