"""GB300-native Polylla: terminal-edge-region polygon meshes from half-edge
triangulations (arXiv 2403.14723), as hand-written sm_103a CUDA kernels
behind a C ABI (``include/polylla.h``).

Submodules (imported lazily, so the input generator works without a GPU):

* ``polylla``  -- ctypes binding of libpolylla (names follow the C ABI);
* ``build``    -- builds libpolylla.so in-tree with nvcc for sm_103a;
* ``meshgen``  -- seeded synthetic triangulations in the half-edge layout.
"""

__all__ = ["polylla", "build", "meshgen"]
