"""GB300-native hyperedge effective-resistance estimation (HyperEF 2.0,
Algorithm 1): a CUDA library (libhef.so, C ABI in include/hef.h) and its thin
Python binding."""
from ._binding import (  # noqa: F401
    HEF_CLIQUE_HYPEREDGE,
    HEF_CLIQUE_PAPER,
    HEF_F32,
    HEF_F64,
    HEF_REDUCE_MAX,
    HEF_REDUCE_SUM,
    HefError,
    Incidence,
    Pipeline,
    build_incidence,
    edge_resistance,
    hyperedge_resistance,
    krylov_basis,
    launch_count,
    lib,
    trace_kernels,
    trace_read,
    orthonormalize,
    padded_ld,
)
