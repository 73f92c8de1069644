"""GB300-native (sm_103a) hot path of RKHS-BA: correspondence-free multi-frame
bundle adjustment of semantic point clouds (arXiv 2403.01254).

The CUDA library ``librkhsba.so`` (C ABI in include/rkhsba.h) does all the
work; ``rkhsba`` is its ctypes binding.  Importing this package does not
touch the GPU; loading the library fails loudly when it cannot be built.
"""
from .rkhsba import (Problem, RkhsbaError, Server, load, make_params, rkhsba_create,  # noqa: F401
                     rkhsba_create_device, rkhsba_destroy, rkhsba_edge_pairs, rkhsba_eval,
                     rkhsba_get_state, rkhsba_info, rkhsba_iterate, rkhsba_launch_count,
                     rkhsba_rebuild, rkhsba_set_poses_device, rkhsba_solve, rkhsba_profile,
                     EXPORTS)

__all__ = ["Problem", "Server", "RkhsbaError", "load", "make_params", "EXPORTS"]
