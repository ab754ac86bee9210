"""GB300-native ADMoM non-negative CP factorization (Liavas & Sidiropoulos, arXiv 1409.2383).

The compute path is ``libntf.so`` (hand-written CUDA for sm_103a behind the C ABI of
``include/ntf.h``); :mod:`paper_1409_2383_gb300.ntf` is its thin Python binding.
"""
from .ntf import (NTF_BF16, NTF_F32, NTF_KR_AUX, NTF_KR_PRIMAL, NTF_RHO_ADAPTIVE, NTF_RHO_FIXED,
                  NTF_RHO_TRACE, Context, NTFError, Params, default_params, lib, to_bf16,
                  zeros_state)

__all__ = ["Context", "NTFError", "Params", "default_params", "lib", "to_bf16", "zeros_state",
           "NTF_F32", "NTF_BF16", "NTF_KR_PRIMAL", "NTF_KR_AUX", "NTF_RHO_ADAPTIVE",
           "NTF_RHO_TRACE", "NTF_RHO_FIXED"]
