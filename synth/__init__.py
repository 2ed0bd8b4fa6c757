"""Seeded synthetic inputs: planted-partition attributed bipartite graphs.

This package only draws inputs (edges, weights, attributes, ground-truth
clusters). It holds none of the clustering arithmetic; both the FP64 oracle
and the CUDA path consume what it produces.
"""
from .planted import (  # noqa: F401
    ABG,
    make_config1,
    make_config2,
    make_config3,
    make_config4_graph,
    make_config5_request,
    config5_arrivals,
    make_small,
    bf16_bits_to_f32,
    f32_to_bf16_bits,
    CONFIG_PARAMS,
)
