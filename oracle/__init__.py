"""FP64 CPU oracle for the stochastic Henry problem and its MLMC estimator.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may use it. It shares no code with the CUDA path.

Modules
  henry    -- discretisation (cell-centred finite volumes, implicit Euler),
              exact Jacobian by complex-step differentiation, Newton with a
              sparse direct solver, quantities of interest.
  mlmc     -- two-pass level statistics, the telescoping estimator and the
              optimal sample allocation (paper section 3).
  adjoint  -- discrete adjoint of a QoI through the implicit time stepping.
  qmc      -- sample quantiles, exceedance fractions and randomised-QMC
              replicate estimates (paper section 4, tests A1-A3).

Parity status: every function here is pinned by `tests/test_oracle_pins.py`
against closed forms, invariants or the paper's printed numbers, except the
physical QoI values of the random-field model, which the paper does not print
("parity unpinned" for absolute QoI values; their ingredients are pinned).
The paper's porosity model (Eq. poro_2levels) is pinned factor by factor:
the layer factor C0 through row means over a period, C1 and C2 through the
exact spectra of phi along x and along y (frequencies, amplitudes, sine or
cosine, signs), the Kozeny-Carman scale through Table 1.
"""
