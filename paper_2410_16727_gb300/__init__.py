"""GB300-native seed-parallel trajectory optimisation (the motion-optimiser hot
path that DiffusionSeeder seeds): CUDA kernels for sm_103a behind the C ABI in
include/dseed.h, a thin ctypes binding (binding.py), a user API (api.py) and the
seeded synthetic workloads (inputs.py).  Importing the package loads nothing;
binding.load() loads libdseed.so and raises if it has not been built."""
__all__ = ["inputs", "binding", "api", "build"]
