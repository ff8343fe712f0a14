"""GB300-native off-tree edge recovery of pdGRASS (parallel density-aware
graph spectral sparsification, arXiv 2508.20403).

The hot path is the CUDA library built from csrc/ (C ABI: include/pdgrass.h);
`binding` marshals numpy / torch arguments into it.
"""
from .binding import (BatchSparsifier, Options, PdgError, Sparsifier, default_options, load,  # noqa: F401
                      status_string)
