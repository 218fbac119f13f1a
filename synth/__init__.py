"""Seeded synthetic graph generators (edge lists only).

This module produces raw edge lists -- possibly with duplicates and self-loops
-- for the workloads the closeness estimators are measured on.  It holds none
of the estimators' arithmetic: no CSR building, no traversal, no sampling of
the sources.  Both the GPU library's tests and the CPU oracle consume its
output.
"""
from .graphs import (  # noqa: F401
    splitmix64_at,
    uniform_at,
    rmat_edges,
    grid_edges,
    watts_strogatz_edges,
    rgg_edges,
    road_like_edges,
    path_edges,
    star_edges,
    cycle_edges,
    complete_edges,
    random_weights,
    pareto_node_weights,
    edge_lengths_to_weights,
)
