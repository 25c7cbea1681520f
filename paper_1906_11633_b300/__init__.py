"""B300-native batched renderer for visually randomized robotics scenes.

The data-parallel hot path of ORRB (arXiv 1906.11633): many small scenes
(an articulated capsule hand, a block and a table) rendered in one batch into
RGB, depth, view-space normal and segmentation channels (Sec. 4.4), with
geometry shared across samples (Single Scene Multiple States, Sec. 3) and all
randomization drawn on the host from a seeded counter-based generator
(Sec. 4.3).

Submodules:
  scenegen  -- seeded synthetic scenes and randomizer parameters (inputs only)
  lib       -- ctypes binding of the C-ABI library ``liborrb.so``
  render    -- torch-level helpers (device buffers, ShadeFn autograd wrapper)
  tune      -- tile-shape autotuner
  serve     -- continuous-batching request loop

Nothing is imported eagerly: ``import paper_1906_11633_b300.scenegen`` does
not load the CUDA library.
"""

__all__ = ["scenegen", "lib", "render", "tune", "serve"]
