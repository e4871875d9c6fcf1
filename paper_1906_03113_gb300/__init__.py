"""GB300-native algebraic BFS by submatrix multiplication.

The library is libabfs.so (C-ABI in include/abfs.h, CUDA kernels for
sm_103a); this package is its Python binding.  Importing the package does not
load the library; the first call does, and fails loudly if it was not built.
"""
from .binding import (  # noqa: F401
    MODE_PLAIN,
    MODE_SUBMATRIX,
    AbfsError,
    BatchPlan,
    batch_tune,
    Graph,
    Server,
    ServeCfg,
    serve_default_cfg,
    Params,
    Stats,
    default_params,
    declared_symbols,
    graph_create,
    graph_destroy,
    load,
    run,
    run_counts,
    calibrate,
    run_batch,
    run_host,
    run_host_many,
    graph_relabel,
    relabel_order,
    run_trace,
    strerror,
    tune,
)


def build(force: bool = False) -> str:
    """Compiles libabfs.so for sm_103a in-tree and returns its path."""
    from ._build import build as _b
    return _b(force=force)
