"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This package only builds inputs: grid axes, velocity values at grid nodes and
particle start positions.  It holds none of the advection method's arithmetic
(no cell search, no interpolation, no time stepping), so the FP64 oracle and the
CUDA path can both read the same inputs without sharing any of the method.
"""
from .fields import *  # noqa: F401,F403
from .particles import *  # noqa: F401,F403
