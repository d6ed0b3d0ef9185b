"""libfst: GB300-native (sm_103a) evaluation and randomized least-squares refit of
functional sparse Tucker models (arXiv 1907.05884).

``paper_1907_05884_gb300.fst`` is the ctypes binding of the C ABI declared in
``include/fst.h``; importing it loads ``libfst.so`` and fails loudly when the
library has not been built.  ``paper_1907_05884_gb300.synth`` draws seeded
synthetic inputs.  This package module itself imports neither, so the input
generator can be used without the CUDA library.
"""
