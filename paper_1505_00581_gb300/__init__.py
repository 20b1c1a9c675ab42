"""hgm: exact chain hypergraph matching of space-time interest points on GB300.

The compute path is the CUDA library ``libhgm.so`` (see ``include/hgm.h``);
``paper_1505_00581_gb300.hgm`` is its thin ctypes binding. ``synth`` draws
seeded synthetic models and scenes. Importing the package does not load the
CUDA library; the binding does, and fails loudly when it is missing.
"""
__all__ = ["synth"]
