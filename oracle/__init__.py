"""FP64 CPU oracle for the MM NMF iteration (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference arm may import this package.  See ``nmf_oracle`` for the float64
iteration and ``exact`` for the exact-rational elementwise form.
"""
from . import nmf_oracle, exact  # noqa: F401
