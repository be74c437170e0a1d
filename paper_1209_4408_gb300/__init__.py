"""GB300-native Game of Life generation step (B3/S23, eight neighbours,
wrap-around board) for arxiv 1209.4408.

The work runs in ``libgol.so``: hand-written CUDA kernels for sm_103a behind
the C ABI declared in ``include/gol.h``.  This package is the thin Python
binding (``gol``), the continuous-batching request loop (``serve``) and the
autotuner (``autotune``).  Importing it loads the library and raises if it
has not been built: there is no CPU path.
"""
from .gol import *  # noqa: F401,F403
from .gol import load as _load

_load()
from . import autotune as _autotune  # noqa: E402

_autotune.load_shipped()
