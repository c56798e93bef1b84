"""GB300 (sm_103a) implementation of the DDLR preconditioner of Li & Saad,
"Low-rank correction methods for algebraic domain decomposition
preconditioners": batched level-scheduled local solves, E/E^T products,
low-rank corrections (DDLR-1, DDLR-2), GPU Lanczos and PCG, behind the C ABI
of include/ddlr.h.  This package is the Python binding of that library.
"""
from .ddlr import DDLR, DdlrError, EXPORTS, Server, load, options  # noqa: F401
from .build import build  # noqa: F401
