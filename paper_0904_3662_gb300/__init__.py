"""libahfgpu: GB300 (sm_103a) kernels for AHF's per-halo unbinding stage.

The compute path is the C ABI in include/ahf.h, implemented in csrc/ and
built into libahfgpu.so; `ahf` is its thin ctypes binding and `synth` the
seeded input generator.
"""
from . import ahf  # noqa: F401
from .ahf import (AHFError, Context, Params, Particles, halo_array,  # noqa: F401
                  halos_from_population, load_library, params_for,
                  particles_from_population, results_to_numpy)
