"""GB300-native exact-exchange (EXX) pair path for localized orbitals.

The compute path lives in the CUDA library ``libexx`` (see ``exx.py`` for the
ctypes binding); ``synth`` builds seeded synthetic inputs.  Importing the
package does not load the CUDA library.
"""
__all__ = ["synth", "exx"]
