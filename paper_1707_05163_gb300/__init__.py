"""GB300-native particle advection (Parcels method, arXiv 1707.05163).

The compute path is the CUDA library ``_build/libparcels_gb.so`` behind the C
ABI in ``include/parcels_gb.h``; this package only marshals arguments to it.
"""
from .api import (MLP, FieldSet, Kernel, ParticleSet, displacement, execute_batch,  # noqa: F401
                  surrogate_apply, surrogate_features, surrogate_run)
from ._native import PGError, load  # noqa: F401
from . import build as _build_module  # noqa: F401
