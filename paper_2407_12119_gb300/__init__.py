"""GB300 (sm_103a) hot path of the ETX4VELO GNN track finder.

``etx`` is the ctypes binding of ``libetx.so`` (C ABI in include/etx.h);
``build`` compiles the library in-tree with nvcc.
"""
from . import etx  # noqa: F401
from .etx import Context, EtxError  # noqa: F401
