"""FP64 CPU oracle of the Monte-Carlo dust-temperature solve (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library does not, and must not, depend on it.
"""
