"""GB300 (sm_103a) exact sparse multivariate polynomial product.

The compute lives in libpolymul.so (CUDA kernels behind the C-ABI of
include/polymul.h); this package is its thin Python binding.  Importing the
package loads nothing; the first call loads the library and raises if it is
missing.
"""

from ._native import (  # noqa: F401
    BatchPlan,
    Plan,
    autotune,
    grid,
    batch_autotune,
    Server,
    batch_polymul,
    batch_workspace,
    PolymulError,
    Product,
    PROBE_SYMBOLS,
    SYMBOLS,
    lib,
    out_bound,
    pack,
    polymul,
    polymul_noalloc,
    polymul_range,
    polymul_ws,
    probe_lib,
    probe_mac,
    probe_oprate,
    shard_bounds,
    split_cumulative,
    unpack,
    workspace_size,
)

__all__ = ["BatchPlan", "Plan", "autotune", "grid", "batch_autotune", "Server", "batch_polymul", "batch_workspace", "polymul", "polymul_noalloc", "polymul_range", "shard_bounds", "split_cumulative", "polymul_ws", "workspace_size", "unpack", "pack", "out_bound", "probe_lib", "probe_mac", "probe_oprate", "PolymulError", "Product", "lib", "SYMBOLS", "PROBE_SYMBOLS"]
