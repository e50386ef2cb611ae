"""GB300-native energy-based DG / Galerkin-difference wave solver.

The compute path is the C-ABI library ``libgdg.so`` (hand-written CUDA for
sm_103a); ``gdg`` is its thin ctypes binding.  Importing this package does
not load the library; ``gdg.lib()`` does, and fails loudly if it is absent.
"""
