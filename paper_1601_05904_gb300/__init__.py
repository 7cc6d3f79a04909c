"""GB300-native AIDW interpolation with even-grid kNN (arXiv 1601.05904).

The compute path is the CUDA library ``libaidw.so`` (sources in ``csrc/``,
C-ABI in ``include/aidw.h``); ``binding`` wraps its entry points with the
same names.  Importing this package does not load the library; ``load()``
does, and raises if it has not been built.
"""
from . import inputs  # noqa: F401


def load():
    from . import binding
    return binding.load()
