"""FP64 CPU oracle of the PVG renderer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2311_18561_gb300``) and never imports it.

``pvg_oracle.c`` holds the arithmetic (time evaluation, projection, SH
colour, brute-force and culled compositing, exact reverse mode); this module
only marshals numpy arrays through ctypes.  ``binning.py`` holds the integer
side (tile keys, stable sort, tile ranges) written with numpy.
"""
from .oracle import (  # noqa: F401
    DEFAULT_OPTS, build, load, num_threads, preprocess, render, render_bwd,
    sh_basis, time_eval, cam_array,
)
