"""GB300 (sm_103a) implementation of the per-frame path of "Dynamic Diffuse
Global Illumination Resampling" (arXiv 2108.05263).

* ``csrc/``   -- CUDA kernels and the C ABI of ``libddgi.so`` (``include/ddgi.h``)
* ``build``   -- in-tree nvcc build of ``libddgi.so``
* ``ddgi``    -- ctypes binding with the ABI's names (imports torch)
"""
from . import build  # noqa: F401

__all__ = ["build", "load"]


def load():
    """Import the binding and load the built library (raises if not built)."""
    from . import ddgi
    ddgi.load()
    return ddgi
