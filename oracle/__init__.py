"""FP64 CPU oracle for the Ehrenfest-regularised lattice Boltzmann step.

Test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
It shares no code with the CUDA library (``paper_0705_4371_gb300``) and never
imports it; the two meet only in the seeded input generators, which hold
none of the method's arithmetic.

Modules:
  build  -- compiles ``lbm_oracle.c`` (plain C, FP64, OpenMP) with gcc.
  core   -- ctypes wrapper: equilibria, dS, selection, Newton, whole runs.
  mlp    -- numpy FP64 forward / backward / Adam of the 4-64-64-4 network on
            bf16-rounded tensors (reference for the GPU training kernels).

Parity status: every function is pinned by a ``-m "not gpu"`` test to a fact
that the paper or mathematics fixes (closed forms, invariants, brute force,
special cases); see the test names in ``tests/test_oracle_*.py``.
"""
