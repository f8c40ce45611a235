"""GB300-native visual matrix ordering (VMO): CUDA library for sm_103a behind a
C-ABI (include/vmo.h) with a thin Python binding (``vmo``)."""
from . import server, vmo  # noqa: F401
from .vmo import (Hypergraph, Params, VmoError, batch_layout, batch_order, default_params, init_coords,  # noqa: F401
                  kmeans, load, stats, stats_reset)
from .server import Server  # noqa: F401
