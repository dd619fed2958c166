"""Delayed-asynchronous pull-based PageRank and Bellman-Ford SSSP on GB300.

The compute path is the CUDA library ``libdag.so`` (built from ``csrc/``),
reached through the ctypes binding in ``dag.py``. Importing this package does
not load the library; the first call into ``dag`` does, and raises if it is
missing.
"""
