"""GB300-native multiplicative-update NMF (Zhou, Lange & Suchard, Section 3.1).

The compute path is the C-ABI library ``libnmf.so`` (hand-written sm_103a
kernels, declared in ``include/nmf.h``); ``nmf`` is its thin ctypes binding and
``synth`` draws the seeded synthetic inputs.  Submodules are imported lazily so
that ``synth`` can be used on machines without the built library.
"""
__all__ = ["nmf", "synth", "build"]
