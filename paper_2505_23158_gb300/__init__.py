"""GB300 (sm_103a) LODGE frame renderer: LOD + chunked 3D Gaussian Splatting.

The CUDA library (``_build/liblodge.so``, built by ``build.build()``) does
all of the work; ``api.Lodge`` wraps its C ABI (``include/lodge.h``) with
PyTorch device memory and streams.  ``synth`` draws the seeded synthetic
scenes and cameras.  Importing this package loads nothing; ``api`` loads the
library on first use and raises if it is missing.
"""

__all__ = ["api", "build", "synth"]
