"""GB300-native light-field Richardson-Lucy deconvolution.

The compute path is the CUDA library ``liblfd.so`` (built from ``csrc/`` for
sm_103a); ``lfd`` is its thin ctypes binding and ``synth`` generates seeded
synthetic inputs. Importing the package loads nothing; ``lfd.load()`` loads the
library and raises if it is missing.
"""
__all__ = ["lfd", "synth"]
