"""Seeded synthetic inputs (rooms, ray-cast depth, poses) for tests and benchmarks."""
from .scenes import *  # noqa: F401,F403
