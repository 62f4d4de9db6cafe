"""FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA solver
in ``paper_1803_07772_gb300``; the two meet only at the seeded inputs drawn by
``hcran_inputs``.
"""
from .oracle import (  # noqa: F401
    OracleResult,
    bruteforce,
    build,
    psi,
    scale_coeffs,
    solve,
)
