"""GB300-native finite-element assembly of convection-diffusion-reaction transport
equations into CSR (arXiv 2107.11541, Sec. 4.2).

* ``fea``      -- ctypes binding of the C ABI (``include/fea.h``), same names.
* ``meshgen``  -- seeded synthetic meshes and fields (inputs only).
* ``build``    -- compiles the CUDA library for sm_103a.
"""
__all__ = ["fea", "meshgen", "build"]
