"""GB300 (sm_103a) library for the third-order unstructured WENO residual (arXiv 1712.08317).

The compute path is libweno3.so (C ABI in include/weno3.h): a host C++ mesh
builder and FP64 least-squares precompute, and CUDA kernels for the cell
reconstruction, the face flux and the gather fused with the RK3 stage.
This package only marshals arguments to it; there is no CPU fallback, and
loading fails loudly if the library cannot be built or opened.
"""
from ._build import build  # noqa: F401


def __getattr__(name):
    if name in ("Mesh", "Solver", "split_fp32", "params_struct"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
