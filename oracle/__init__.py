"""FP64 CPU oracle for the exact chain hypergraph matching -- TEST INFRASTRUCTURE ONLY.

Importable only from tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference leg. The CUDA library never imports it.
"""
from .oracle import ChainOracle, Oracle, build  # noqa: F401
