"""FP64 CPU oracle for the randomized LU decomposition (Shabat, Shmueli, Aizenbud,
Averbuch, "Randomized LU Decomposition", Algorithm 1, with power iterations and the
rank-deficient least squares of Algorithm 3), its fast variant (Algorithm 4, complex128)
and the orthogonal-basis range finder of Algorithm 2, the comparator of Section 5.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may call it. It shares no code with the CUDA path; the only module
both sides use is the seeded input generator ``paper_1310_7202_gb300.synth``, which holds
none of the method's arithmetic.

Every function cites the passage of the paper it follows. Pins (tests that tie the oracle
to something other than itself) live in ``tests/test_oracle_*.py``.
"""
from .rlu_oracle import (  # noqa: F401
    PHILOX_M0, PHILOX_M1, PHILOX_W0, PHILOX_W1,
    philox4x32_10, philox_stream,
    series_ln, series_sincos_2pi, box_muller, gaussian,
    box_muller_f32, gaussian_f32,
    lu_partial_pivot, lu_column_pivot, pinv_apply, project,
    rlu_factor, reconstruct_error, spectral_norm, rdls_apply, rdls_solve,
    lu_normalize, randomized_orth, orth_error, halko_bound,
    theorem1_constant, theorem1_success_probability, theorem1_failure_terms,
    check_dims,
)
from .frlu_oracle import (  # noqa: F401
    cabs1, srft_matrix, srft_apply, clu_partial_pivot, clu_column_pivot, id_from_lu,
    cpinv_apply, frlu_factor, creconstruct_error,
)
