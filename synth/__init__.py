"""Seeded synthetic instance generators shared by the oracle tests and the CUDA path.

This package holds no arithmetic of the method (no tensors, no semiring, no
contraction): it only draws graphs, couplings, fields and weights from a
counter-based generator, so that both sides are fed identical inputs.
"""
from .instances import (  # noqa: F401
    SplitMix64, Instance, square_lattice, cubic_lattice, kings_subgraph, kings_mask_graph,
    random_regular_graph, erdos_renyi, path_graph, cycle_graph, complete_graph,
    empty_graph, star_graph, random_tree, config_seed, write_instance, read_instance,
)
