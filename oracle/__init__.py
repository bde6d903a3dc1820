"""FP64 CPU oracle for the MM NMF iteration (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference arm may import this package.  See ``nmf_oracle`` for the float64
iteration, ``exact`` for the exact-rational elementwise form,
``poisson_oracle`` and ``qn_oracle`` for the Poisson variant and the
quasi-Newton scheme, and ``pet_oracle`` for penalised PET reconstruction
(Section 3.2, Algorithm 2).
"""
from . import nmf_oracle, exact  # noqa: F401
