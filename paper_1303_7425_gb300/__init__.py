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
    batch_autotune,
    Server,
    batch_polymul,
    batch_workspace,
    PolymulError,
    Product,
    SYMBOLS,
    lib,
    out_bound,
    pack,
    polymul,
    polymul_noalloc,
    probe_mac,
    unpack,
)

__all__ = ["BatchPlan", "Plan", "autotune", "batch_autotune", "Server", "batch_polymul", "batch_workspace", "polymul", "polymul_noalloc", "unpack", "pack", "out_bound", "probe_mac", "PolymulError", "Product", "lib", "SYMBOLS"]
