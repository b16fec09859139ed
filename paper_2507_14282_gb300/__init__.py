"""GB300-native faux-shock hybrid particle-in-cell engine.

The compute path is the CUDA library ``libfs.so`` (C ABI in include/fs.h);
this package is its thin Python binding (:mod:`.fs`) plus the in-tree build
(:mod:`.build`).
"""
from .fs import FauxShock, FsError, params_default  # noqa: F401
