"""CPU FP64 oracle for the dynamic-circuit MPS simulator -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and reference legs of
``bench.py`` may import this package.  The product (``paper_2609_26516_b300``) never imports it, and it
never imports the product: the two share no code besides the seeded circuit generators in
``circuits``.

Contents (each function cites the passage of the paper it follows):

* ``philox``      -- Philox4x32-10 counter-based uniforms (Salmon et al., SC'11), the
  random numbers the single-path strategy draws.
* ``statevector`` -- O1: dense FP64 state-vector simulation with mid-circuit measurement,
  classically controlled gates, single-path (Alg. 1) and multi-path (Alg. 2) drivers.
* ``layers``      -- chunk construction (Sec. "Handling unitary chunks in dynamic
  circuits", with the one-layer reading) and the per-chunk MPO.
* ``mps``         -- O2: FP64 MPS, the variational compression step (Sec. "Simulating
  unitary quantum circuits with DMRG"), measurement/collapse on the MPS (Sec. "Mid-circuit
  measurements"), an exact gate-by-gate mode.
* ``drivers``     -- Alg. 1 and Alg. 2 on the MPS, top-M selection.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against values the
paper prints, closed forms, brute force or library routines, except the truncated-regime
result of the compression, which the paper does not fix (parity unpinned there; it is
checked only through the invariants that hold at any size: f <= 1, sweeps never lower f,
exactness when chi is large enough).
"""
