"""GB300 (sm_103a) Cherenkov photon generation and propagation.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/cherenkov.h``); ``binding`` marshals arguments to it through ctypes
and ``synth`` generates seeded synthetic inputs.
"""
