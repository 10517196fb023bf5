"""CPU oracle for the collision-integral hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 restatement of what the paper's method computes, written
to check the CUDA library against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path never
does, and it shares no code with ``paper_2603_28848_gb300``.

Modules (each function cites the passage of the paper it restates):
  philox       Philox4x32-10 (Salmon et al., SC'11) and the uniform streams
  vegas        VEGAS map, per-bin training data, refinement, iteration combine
  spline       cubic spline in linear scale + equilibrium-form tails (Sec. 3B)
  tasks        identical-particle decomposition and particle roles (Sec. 2C, App. A)
  collision    the Monte Carlo integrand and C_a(p_i) (Sec. 2B-2D, App. A)
  step         log-space Euler / Heun with adaptive dt (Sec. 3C)
  reference    independent exact-energy reductions used as pins (Sec. 4, App. B)
  width        fractional Gaussian width and its error-threshold controller (App. C)
  stratified   adaptive stratified sampling on top of the map (the vegas library's default)
  moments      number and energy densities for conservation checks (Sec. 5C)
  budget       variance-driven per-task sample budgets (Sec. 3D integrator reuse, App. C)
  adjoint      the fixed-sample integral as a torch function; its reverse and forward derivatives
  implicit     backward-Euler log-space step by dense-Jacobian Newton

Parity pins live in ``tests/test_oracle_*.py``.  Items without an external
pin are marked "parity unpinned" in their docstrings.
"""
