"""GB300-native (sm_103a) Embedded-Atom-Method molecular dynamics.

The compute path is the CUDA library built from `csrc/` (C ABI:
include/eammd.h); `binding.MD` is its Python face.  `inputs` holds the
seeded synthetic workloads.  Importing the package does not load the CUDA
library; `binding.load()` does, and fails loudly if it is missing.
"""

__all__ = ["inputs", "binding", "build"]
