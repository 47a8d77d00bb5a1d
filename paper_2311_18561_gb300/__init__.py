"""GB300-native PVG rasterizer (time-conditioned, differentiable).

The CUDA library behind ``include/pvg.h`` is loaded lazily on first use
(``paper_2311_18561_gb300.abi``); importing the package itself loads
nothing, so the seeded input generators (``synth``) can be used without it.
"""
