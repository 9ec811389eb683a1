"""GB300-native consistent neural message passing (arXiv 2410.01657).

The compute path is ``libgnnmp.so`` (hand-written sm_103a CUDA behind the C ABI
in ``include/gnnmp.h``); ``binding`` marshals arguments to it, ``graph`` wraps
graph generation / partitioning and the device-side graph, and ``nn`` holds the
autograd Functions and the encode-process-decode network.
"""
from ._build import build  # noqa: F401

__all__ = ["build", "binding", "graph", "nn"]
