"""Seeded synthetic graph generators shared by the tests, the benchmark and the oracle checks.

This package draws random graphs and labels only; it holds none of the embedding
arithmetic (no degrees, no normalisation, no label weights), so that neither the CUDA
path nor the CPU oracle depends on the other through it.
"""
from .graphs import (  # noqa: F401
    Graph,
    sbm,
    chung_lu,
    zipf_labels,
    batch_specs,
    batch_graph,
    random_tiny,
    edge_density,
    expected_sbm_edges,
)
