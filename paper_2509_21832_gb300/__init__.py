"""GB300-native micro-macro KFVS step for the Boltzmann-ES-BGK equation.

The compute path is the CUDA library libmmkfvs.so (C ABI, include/mmkfvs.h); the Python side is
argument marshalling only.  Import ``paper_2509_21832_gb300.api`` for the binding and
``paper_2509_21832_gb300.inputs`` for seeded problem set-up.
"""
