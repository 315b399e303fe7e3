"""GB300-native block simulation of mixed-radix (qubit-qudit) state vectors.

The compute path is ``libqudit.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/qudit.h``); ``binding`` marshals arguments to it.
Importing this package does not load the library; ``binding`` does, and it
raises if the library is missing.
"""
__all__ = ["inputs", "binding"]
