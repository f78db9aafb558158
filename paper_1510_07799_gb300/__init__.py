"""hp-fRG on GB300: the one-loop fRG flow of the single-impurity Anderson model
(vertex + self-energy, Matsubara frequencies, Omega-scheme cutoff) with its
right-hand side and Dormand-Prince integrator in hand-written sm_103a CUDA.

The compute path lives in the shared library built from csrc/ and is reached
through the C ABI declared in include/frg.h.  Submodules:
  frg     -- the thin ctypes binding to that library (import it explicitly)
  inputs  -- seeded synthetic workloads and states
"""
