"""Dense MTTKRP and CP-ALS on one GB300 GPU (sm_103a), after "Shared-Memory
Parallelization of MTTKRP for Dense Tensors" (Hayashi, Ballard, Jiang, Tobia).

The compute lives in ``lib/libmttkrp.so`` (CUDA kernels behind the C ABI of
``include/mttkrp.h``); this package is its thin torch binding.
"""
from .api import (ALS, ALGOS, BatchedMTTKRP, mttkrp_batched, PRECISIONS, CPLoss, Workspace, cp_gradient, cp_loss, cp_residual,
                  default_workspace, ffma_probe, gram, gram_hadamard_solve, khatri_rao, multi_ttv, mttkrp,
                  mttkrp_all, mttkrp_sym, norm2, pack_symmetric, sym_packed_dims, partial_mttkrp, partial_mttkrp_split, split_tensor)
from ._lib import MtkError, load

__all__ = ["ALS", "ALGOS", "BatchedMTTKRP", "mttkrp_batched", "PRECISIONS", "CPLoss", "Workspace", "cp_gradient", "cp_loss",
           "cp_residual", "default_workspace", "ffma_probe", "gram", "gram_hadamard_solve", "khatri_rao",
           "multi_ttv", "mttkrp", "mttkrp_all", "mttkrp_sym", "norm2", "pack_symmetric", "sym_packed_dims", "partial_mttkrp", "partial_mttkrp_split", "split_tensor", "MtkError", "load"]
