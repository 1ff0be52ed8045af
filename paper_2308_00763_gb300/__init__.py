"""GB300-native (sm_103a) per-frame SIR particle-filter step for video object tracking.

The compute path is the CUDA library built from ``csrc/`` (see ``include/pf.h`` for the
C ABI); :mod:`.binding` marshals arguments to it and exposes the same entry-point names.
:mod:`.synth` generates the seeded synthetic tracking videos used as inputs.
"""
from .binding import *  # noqa: F401,F403
from .binding import Batch, Filter, make_config  # noqa: F401

__version__ = "0.1.0"
