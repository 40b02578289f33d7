"""GB300-native batched acoustic modelling, adjoint and FWI gradient.

Python front end of libwave (``include/wave.h``): the binding in ``wave.py``
keeps the C names; ``synth`` draws seeded synthetic inputs.
"""
from .wave import (Grid, WaveError, STORE_BF16, STORE_CHECKPOINT, STORE_FP32, wave_adjoint,  # noqa: F401
                   wave_checkpoint_schedule, wave_courant_limit, wave_forward, wave_gradient, wave_ricker,
                   wave_workspace_size)
