"""B300-native (sm_103a) dynamic-circuit MPS simulator: the DMRG-style compression step,
mid-circuit measurement / collapse / classically controlled gates and the multi-path
branch ensemble of "Tensor Network Simulation of Dynamic Circuits", behind the C ABI
``libdcs`` (include/dcs.h).  ``Simulator`` is the Python binding of that ABI."""
from .sim import (DCSError, Simulator, bits_of, encode_ops, mps_to_dense,  # noqa: F401
                  topk_select_global)

__all__ = ["Simulator", "DCSError", "bits_of", "encode_ops", "mps_to_dense",
           "topk_select_global"]
