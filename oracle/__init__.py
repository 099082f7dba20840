"""CPU oracle of the two-phase lattice Boltzmann update (arXiv 2112.01975).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only users. The product library never imports, links or
executes anything here, and nothing here imports the product library (the
seeded input generators in ``paper_2112_01975_gb300.inputs`` are the one
shared module, and hold none of the method's arithmetic).

``lbm_oracle.c`` is a plain single-threaded FP64 C restatement of the update;
``lbm.py`` wraps it with ctypes; ``physics.py`` holds host-side closed forms
(Maxwell construction, second-gradient interface profile, surface tension,
equimolar radius) used to pin it.
"""
