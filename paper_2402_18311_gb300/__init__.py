"""GB300 (sm_103a) electrostatic global placement: the inner loop that Hybro
(arXiv 2402.18311, Algorithm 1) re-runs after every perturbation.

``place`` is the ctypes binding of ``libhybro_place.so`` (the C ABI in
``include/hybro_place.h``); ``synth`` draws seeded synthetic workloads;
``build`` compiles the library.  Importing the package loads nothing; the
binding loads the library on first use and fails loudly if it is missing.
"""
