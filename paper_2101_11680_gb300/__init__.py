"""GB300-native confocal time-of-flight DOT (arXiv 2101.11680).

``ctof``  -- the Python binding of the C ABI in ``include/ctof.h``.
``synth`` -- seeded phantoms and Poisson noise (inputs only).
``build`` -- compiles ``libctof.so`` for sm_103a.
"""
