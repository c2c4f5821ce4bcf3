"""GB300-native hot path of the RPNN cloud renderer (Kallweit et al., "Deep Scattering").

The compute lives in a C-ABI CUDA library (``csrc/``, declared in ``include/rpnn.h``);
``api`` is its thin ctypes binding.  ``workloads`` generates the seeded synthetic
inputs.  Importing the package does not load the CUDA library; calling any op does,
and fails loudly when the library has not been built.
"""
__all__ = ["api", "workloads"]
