"""FP64 CPU oracle for Semi-Global Weighted Least Squares (SG-WLS).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA library; the
only thing both sides use is the seeded input generator in ``synth``.

Contents (each function cites the passage of Liu et al., "Semi-Global
Weighted Least Squares in Image Filtering", ICCV 2017, that it follows):

* ``sgwls``       -- the method: Sec. 2.1 neighbourhood construction,
                     Eq. 5 subsystems formed like Eq. 4 with Eq. 2 weights,
                     solved exactly, inverse construction and averaging
                     (the four steps of Sec. 2.3), T alternating passes.
* ``rband_lu``    -- the paper's own r-band LU decomposition, Eqs. 6-20,
                     written out in the paper's notation (small cases only).
* ``wls2d``       -- the full 2D WLS model, Eqs. 1-4, solved densely
                     (tiny images only; used for the closeness check).
* ``adjoint``     -- the reverse-mode derivative of ``sgwls`` with respect to
                     the input, the guidance and lambda (derived from
                     Eqs. 2, 4, 5; the paper has no backward pass).

Parity pins: see ``tests/test_oracle*.py``.  The whole-method output is
"parity unpinned" against printed values: the paper prints no numeric
SG-WLS output (its numbers are timings and MAD values on a dataset that is
not available); the oracle is pinned by the paper's structural statements,
closed forms, invariants, brute force on tiny inputs and finite differences.
"""
from .sgwls import (  # noqa: F401
    Params,
    COLUMN,
    ROW,
    centre_indices,
    neighbourhood_construction,
    guidance_weight,
    subsystem_band,
    solve_subsystem,
    coverage_counts,
    sgwls_pass,
    sgwls,
    sgwls_interpolate,
)
