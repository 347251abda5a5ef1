"""GB300-native sliced tensor-network contraction (libtnc) and its Python binding.

The compute path is the C-ABI library ``libtnc.so`` (CUDA for sm_103a plus a
C++ host planner); ``Network`` marshals arguments to it. PyTorch only provides
device memory and streams. There is no CPU fallback: if the library is
missing, importing the binding raises.
"""

from ._lib import (Network, TNCError, FP32, SPLIT_TF32, SPLIT_BF16, SPLIT_BF16X2, SPLIT_FP16X2, contract_many, tune_table, lib_path,
                   load_library, peak_probe, worklist_many)

__all__ = ["Network", "TNCError", "contract_many", "tune_table", "FP32", "SPLIT_TF32", "SPLIT_BF16", "SPLIT_BF16X2", "SPLIT_FP16X2",
           "lib_path", "load_library", "peak_probe", "worklist_many"]
