"""Seeded synthetic netlist hypergraphs and random start blocks.

This package only draws random inputs; it holds none of the resistance
method's arithmetic, so both the FP64 oracle and the GPU path can read the
same instances without sharing any of the computation.
"""
from .synth import (  # noqa: F401
    Netlist,
    WORKLOADS,
    grid_netlist,
    start_block,
    workload,
    window_subhypergraph,
)
