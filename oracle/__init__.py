"""CPU FP64 oracle for CTMRG and SI-CTMRG (arXiv 2607.15158).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
reference that the CUDA path is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the product path never does, and the two share no code (they meet only in
the seeded input module ``ctm_synth``).

Modules
  ctmrg   -- standard truncated-SVD CTMRG and SI-CTMRG on Lx x Ly unit cells
  exact   -- brute-force contractions of small finite networks (pins)
  ising   -- closed forms of the 2D Ising model (Onsager, Yang) (pins)

Parity pins: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, brute force, invariants); the pin of
each function is named in its docstring. No function is "parity unpinned".
"""
