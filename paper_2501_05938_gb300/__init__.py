"""GB300-native tridiagonal partition-method solver.

The compute path is the CUDA library ``libtps.so`` (sources in ``csrc/``,
C ABI in ``include/tps.h``); ``binding`` marshals arguments to it through
ctypes.  ``synth`` generates the seeded synthetic systems used by the tests
and the bench.  Importing this package loads nothing; the library is loaded
on first use and its absence is an error.
"""
__all__ = ["binding", "build", "synth"]
