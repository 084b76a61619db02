"""GB300-native (sm_103a) Fast-AGMS sketch build and sketch-merging join-size estimation
of COMPASS (arXiv 2102.02440), behind the C ABI declared in include/compass.h.

Submodules: `compass` (ctypes binding of libcompass), `pipeline` (device orchestration
over the binding), `datagen` (seeded synthetic inputs), `build_lib` (nvcc build).
Importing the package loads nothing; the library is loaded on first use.
"""
__all__ = ["compass", "pipeline", "datagen", "build_lib"]
