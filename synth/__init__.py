"""Seeded synthetic scenes for the PackUV-GS render step.

This module produces inputs only: atlases of Gaussian attributes, occupancy
and dynamic bitmasks, and camera views.  It holds none of the render step's
arithmetic (no activation, projection, colour, binning or compositing), so
both the CUDA library and the CPU oracle can consume its output without
sharing any method code.
"""

from .scenes import (  # noqa: F401
    View,
    Scene,
    CONFIG_NAMES,
    make_scene,
    config_scene,
    look_at,
    random_target,
    motion_flow,
    actor_sphere,
    pack_bits,
    channel_count,
)
