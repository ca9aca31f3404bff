"""Plain, slow, obviously correct FP64 CPU oracle for the k.p hole eigensolve.

TEST INFRASTRUCTURE.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / reference leg of `bench.py` may import or run anything in
this package.  It shares no code with the CUDA path (`paper_2607_08447_b300`)
and imports nothing from it; the two meet only in the seeded generators of
the `inputs` package.

Modules
  kp           CSR assembly of H_NI = H_DKK + H_SOI + H'_PB + V (+ B field)
  eig          dense LAPACK and thick-restarted block Lanczos lowest states
  observables  hole density and Hellmann-Feynman gradients
"""
from . import kp, eig, observables  # noqa: F401
