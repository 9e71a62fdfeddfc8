import ctypes
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Reuse freed heap memory instead of returning it to the OS: fresh pages are
# slow to fault in on some hosts and the oracle allocates large temporaries.
try:
    _libc = ctypes.CDLL("libc.so.6")
    _libc.mallopt(-3, 1 << 30)       # M_MMAP_THRESHOLD
    _libc.mallopt(-1, 2 ** 31 - 1)   # M_TRIM_THRESHOLD
    _libc.mallopt(-2, 256 << 20)     # M_TOP_PAD
except OSError:
    pass


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libetx.so")
