"""GB300-native patch-AMR wave propagation (ForestClaw's hot path, arXiv 1703.03116).

All numerical work runs in the CUDA library ``libfc.so`` (include/fc.h); this
package only marshals arguments to it.  Importing it loads the library and
fails loudly when it has not been built -- there is no CPU fallback.
"""
from . import _lib
from ._lib import BRICK, F32, F64, PERIODIC, SPHERE, WALLS, Desc, FcError, load
from .forest import (Forest, initial_forest, layout_check, layout_neighbours, layout_reflux,
                     layout_regrid, make_desc, set_allocator, torch_allocator, uniform_leaves)

load()

__all__ = ["Forest", "Desc", "FcError", "make_desc", "initial_forest", "uniform_leaves",
           "layout_check", "layout_neighbours", "layout_reflux", "layout_regrid", "set_allocator",
           "torch_allocator", "F32", "F64", "WALLS", "PERIODIC", "SPHERE", "BRICK"]


def launch_count(reset: bool = False) -> int:
    """Kernel launches this library issued on the calling thread."""
    return int(load().fc_launch_count(1 if reset else 0))
