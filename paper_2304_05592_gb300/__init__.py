"""GB300-native batched acoustic modelling, adjoint and FWI gradient.

Python front end of libwave (``include/wave.h``): the binding in ``wave.py``
keeps the C names; ``synth`` draws seeded synthetic inputs.
"""
from .wave import (Grid, WaveError, STORE_BF16, STORE_CHECKPOINT, STORE_FP32, WRT_SLOWNESS2,  # noqa: F401
                   WRT_VELOCITY, wave_adjoint, wave_autotune, wave_born, wave_checkpoint_schedule,
                   wave_courant_limit, wave_forward, wave_gradient, wave_jacobian_adjoint, wave_ricker,
                   wave_workspace_size)
