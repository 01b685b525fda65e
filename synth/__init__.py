"""Seeded synthetic inputs (frames, crops, random weights and score maps)."""
from .scenes import *  # noqa: F401,F403
from .scenes import __all__  # noqa: F401
