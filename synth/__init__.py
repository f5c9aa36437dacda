"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and bench.py.

This module only builds inputs: graph Laplacians in CSR form and node sets.  It holds none
of the Krylov arithmetic.  Every generator is deterministic for a given seed on any machine.

The graphs follow the shapes the kernel-column problem is posed on (Section 2.1, Eq.
(generalizedLaplacian)): the standard Laplacian L = D - A of a simple undirected graph, or
its weighted form L = D_w - W.  The CSR arrays describe all of L, diagonal included, with
int32 indices sorted within each row and float32 values.
"""
from .graphs import (CSRGraph, path_graph, cycle_graph, grid_graph, random_geometric_graph,
                     barabasi_albert_graph, from_edges, sample_nodes, random_weighted_graph)

__all__ = ["CSRGraph", "path_graph", "cycle_graph", "grid_graph", "random_geometric_graph",
           "barabasi_albert_graph", "from_edges", "sample_nodes", "random_weighted_graph"]
