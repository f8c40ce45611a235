"""GB300-native visual matrix ordering (VMO): CUDA library for sm_103a behind a
C-ABI (include/vmo.h) with a thin Python binding (``vmo``)."""
from . import server, vmo  # noqa: F401
from .vmo import (HostMatrix, Hypergraph, Params, VmoError, autotune, batch_layout, batch_order, default_params,  # noqa: F401
                  get_tuning, init_coords, kmeans, load, perfect_matching, read_matrix_market, set_tuning,
                  stats, stats_reset, write_matrix_market)
from .server import Server  # noqa: F401
