"""GB300 (sm_103a) Hough-transform track finder.

Modules:
  ht     -- binding of libht.so (the C ABI in include/ht.h); no CPU fallback
  build  -- in-tree nvcc build of libht.so
  synth  -- seeded synthetic trigger events (inputs only)
  serve  -- continuous-batching trigger request loop over the C ABI

Importing the package loads nothing; ``ht.load()`` opens the library.
"""
