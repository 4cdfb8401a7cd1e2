"""GB300-native SDP-BSREM PET reconstruction (arXiv 2111.07886).

The compute path is the CUDA library ``libpet.so`` (sources in ``csrc/``, C-ABI declared
in ``include/pet.h``); ``pet`` is its thin ctypes binding and ``synth`` the seeded
synthetic-workload generator.  Importing the package loads nothing; the library is
loaded on first use of ``pet``.
"""
