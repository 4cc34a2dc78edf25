"""Seeded synthetic stereo inputs (no stereo-method arithmetic)."""
from .stereo import *  # noqa: F401,F403
from .stereo import batch_sizes_uneven  # noqa: F401
