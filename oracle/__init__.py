"""CPU oracle of the SAT + 2D CA-CFAR radar chain (test infrastructure).

This package is test infrastructure, not part of the product: only the tests,
the smoke check of the package entry point and the benchmark's CPU-baseline
leg may import it. It is written from the paper (Rohman, Andra, Nishimoto,
"Optimized 2D CA-CFAR for Drone-Mounted Radar Signal Processing Using Integral
Image Algorithm") in plain numpy, FP64 throughout, with no blocking, fusion or
reordering beyond what each definition states, and shares no code with the
CUDA path.

Modules
  preprocess : Sec. II.A chain -- fast-time DC-shift removal and linear-trend
               subtraction, slow-time mean filter, normalisation, slow-time
               DFT restricted to the 0.3-0.8 Hz respiration band, magnitude.
  cfar       : Sec. II.B -- eq. 2 threshold factor (with the exponent's sign
               corrected), eq. 3 summed-area table, eq. 4 four-corner region
               sum, the direct sliding-window CA-CFAR and the SAT CA-CFAR
               (eq. 1 decisions), and the decision comparison with a margin.

Readings where the paper is silent or garbled are stated in each function's
docstring. Parity status: every function is pinned by the `not gpu` tests in
tests/test_oracle_*.py except the composition of the whole chain on real radar
data, which has no printed worked example ("parity unpinned" for that
composition; each of its steps is pinned on its own).
"""
from .preprocess import (  # noqa: F401
    band_plan,
    detrend_fast_time,
    mean_filter_slow_time,
    normalise,
    normalise_row_zscore,
    band_dft_magnitude,
    preprocess_frame,
)
from .cfar import (  # noqa: F401
    alpha,
    n_ref,
    sat,
    box_sum,
    cfar_direct,
    cfar_sat,
    cfar_chain,
    compare_decisions,
    run_chain,
)
