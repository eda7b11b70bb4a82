"""FP64 CPU oracle of the micro-continuum DBS-VOF time step (test infrastructure).

Only tests, ``__graft_entry__.smoke()`` and the cpu_baseline / reference leg of
``bench.py`` import this package.  The product path never calls it: there is
no CPU fallback.  It shares no code with the CUDA library.
"""
