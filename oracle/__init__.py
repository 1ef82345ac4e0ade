"""FP64 CPU oracle for the seed-parallel trajectory optimisation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
import this package.  It wraps ``dseed_oracle.c`` (plain C, double precision,
built with the host compiler) through ctypes and shares no code with the CUDA
path.  See the header of ``dseed_oracle.c`` for what is computed and how each
part is pinned.
"""
from .oracle import (  # noqa: F401
    build, load, Oracle, fk_frames, flange_pose, esdf_build, esdf_lookup, num_threads, set_num_threads,
    lbfgs_quadratic, success_thresholds,
)
