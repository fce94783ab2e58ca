"""CPU oracle for the curved-surface MD hot path (TEST INFRASTRUCTURE ONLY).

Plain FP64 C (window propagation, forces, face walk, dynamics) behind ctypes,
plus a definitional brute-force geodesic solver in pure Python (``brute``).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares nothing with the CUDA library.
"""
