"""GB300 (sm_103a) ORCA crowd-simulation step: hand-written CUDA behind a C ABI.

The compute path is liborca_gb300.so (csrc/); ``abi`` is its ctypes binding and
``scenarios`` the seeded synthetic crowds.  Build with ``build.build()``.
"""
from . import scenarios  # noqa: F401
from .abi import (OrcaError, OrcaSim, load_library, make_params, orca_create,  # noqa: F401
                  orca_destroy, orca_get_cells, orca_get_counters, orca_get_neighbors,
                  orca_get_state, orca_last_error, orca_num_agents, orca_set_agents,
                  orca_status_string, orca_step, orca_sync, orca_workspace_size)

__all__ = ["scenarios", "OrcaSim", "OrcaError", "load_library", "make_params"]
