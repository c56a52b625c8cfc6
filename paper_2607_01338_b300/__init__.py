"""B300-native (sm_103a) IRIS-SO synthetic-observation library.

The CUDA library ``libirt.so`` (C ABI in include/irt.h) renders PPV cubes of a
molecular line plus dust continuum from 3-D gas fields, and the gradients of a
cube loss with respect to density, temperature and velocity.  This package is
its Python binding: ``binding`` mirrors the C ABI, ``api`` wraps it for
PyTorch tensors and streams.  The library is loaded on first use of any of
the names below (so that ``paper_2607_01338_b300.build`` can run before it
exists); a missing library raises ImportError, there is no fallback.
"""
import importlib

_BINDING = ("irt_create_grid", "irt_forward_ppv", "irt_adjoint_ppv", "irt_destroy",
            "irt_grid_stats", "irt_launch_count", "IrtError", "LIB_PATH")
_API = ("COMPONENTS", "Grid", "LevelTable", "RenderConfig", "RenderPPV", "ForwardGraph", "adjoint",
        "alloc_cubes", "beam_convolve", "forward", "forward_batch", "forward_lines",
        "latitude_mean",
        "render_ppv")

__all__ = list(_BINDING + _API)


def __getattr__(name):
    if name in _BINDING:
        return getattr(importlib.import_module(".binding", __name__), name)
    if name in _API:
        return getattr(importlib.import_module(".api", __name__), name)
    raise AttributeError(name)
