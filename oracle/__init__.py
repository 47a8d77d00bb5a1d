"""FP64 CPU oracle of the PVG renderer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2311_18561_gb300``) and never imports it.

``pvg_oracle.c`` holds the arithmetic (time evaluation, projection, SH
colour, brute-force and culled compositing, the extra v_bar / rho /
semantic channels, exact reverse mode); this module
only marshals numpy arrays through ctypes.  ``binning.py`` holds the integer
side (tile keys, stable sort, tile ranges) written with numpy; ``loss.py``
the photometric loss (1 - lambda_r) L1 + lambda_r L_ssim and its gradient,
in numpy FP64.
"""
from .oracle import (  # noqa: F401
    DEFAULT_OPTS, FEAT_RHO, FEAT_SEM, FEAT_VBAR, build, cam_array, feat_count, load,
    num_threads, preprocess, render, render_bwd, sh_basis, time_eval,
)
