"""GB300-native PIFS fractal-encoding hot path (range-domain search + decode).

The compute lives in libfic.so (CUDA for sm_103a, C ABI in include/fic.h);
``fic`` is a thin ctypes binding of it.
"""
from . import fic  # noqa: F401
from .fic import (FIC_SEARCH_AUTO, FIC_SEARCH_SIMT, FIC_SEARCH_TC, MAP_DTYPE, FicError, counts,  # noqa: F401
                  decode, encode, encode_workspace_size, maps_to_numpy, params)
