"""GB300-native (sm_103a) matrix logarithm by inverse scaling and squaring
with computation-graph polynomials (Jarlebring, Sastre, Ibanez, arXiv
2401.10089).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/logm.h``); this package is its thin Python binding.
"""
from .api import (LogmFunction, Ragged, get_tuning, logm, logm_backward, logm_backward_workspace_size,
                  logm_context_size, logm_execute, logm_execute_host, logm_graph_eval, logm_host_workspace_size,
                  logm_plan, logm_sqrt, logm_version, logm_workspace_size, set_tuning)

__all__ = ["LogmFunction", "Ragged", "get_tuning", "logm", "logm_backward", "logm_backward_workspace_size",
           "logm_context_size", "logm_execute", "logm_execute_host", "logm_graph_eval", "logm_host_workspace_size",
           "logm_plan", "logm_sqrt", "logm_version", "logm_workspace_size", "set_tuning"]
