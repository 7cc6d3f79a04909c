"""GB300-native AIDW interpolation with even-grid kNN (arXiv 1601.05904).

The compute path is the CUDA library ``libaidw.so`` (sources in ``csrc/``,
C ABI in ``include/aidw.h``); ``binding`` wraps its entry points under the
same names.  Importing this package does not load the library: ``load()``
does, and raises if it has not been built.  Attribute access such as
``paper_1601_05904_gb300.aidw_interpolate`` resolves to the binding.
"""
from . import inputs  # noqa: F401


def load():
    from . import binding
    return binding.load()


def __getattr__(name):
    if name.startswith("aidw_") or name in ("Params", "Grid", "AidwError", "interpolate_host",
                                            "BatchJob", "BatchPlan", "AIDW_FP32_COMP",
                                            "AIDW_FP64_PLAIN", "STAGES"):
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
