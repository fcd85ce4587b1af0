"""GB300 (sm_103a) implementation of the Octree-GS LOD renderer hot path (arXiv 2403.17898).

The compute path is the C-ABI library ``libogs.so`` built from ``csrc/`` (declared in
``include/ogs.h``) by ``build.build()``; ``abi`` is its thin Python binding and ``render``
composes a frame.
"""
