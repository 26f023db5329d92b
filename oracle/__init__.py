"""FP64 CPU oracle of the particle-advection step (test infrastructure only).

Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
may import this package.  The CUDA library never does.
"""
from .oracle import (  # noqa: F401
    ALIVE, OOB_HORIZ, OOB_DEPTH, NAN, DELETED, BROWNIAN, SINK, SETTLE, AGE, SAMPLE, EULER, RK4,
    RKF45, rkf45_trial,
    LINEAR, NEAREST, build, lib, Field, Kernel, run, sample, sample_tracer, velocity, locate,
    locate_lon,
    wrap_lon, philox4x32_10, normal_pair, quantise, dequantise,
)
