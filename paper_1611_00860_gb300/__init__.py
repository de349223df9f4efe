"""GB300-native runtime for HPVM's hierarchical dataflow graphs (arXiv
1611.00860): the sgemm example graph lowered to hand-written sm_103a kernels
behind the C-ABI of ``include/hpvm.h``.

Importing the package loads the CUDA library; it fails with ImportError when
the library has not been built (there is no CPU path).
"""
from . import _lib  # noqa: F401  (loads libhpvm_gb300.so or raises)
from ._lib import (  # noqa: F401
    HPVM_TIER_BF16,
    HPVM_TIER_BF16X3,
    HPVM_TIER_BF16X6,
    HPVM_TIER_FP32,
    HPVM_TIER_FP32_DFG,
    HPVM_TIER_FP8,
    HpvmError,
)
from .sgemm import SgemmDFG, build_sgemm_graph, make_args  # noqa: F401

TIERS = {
    "fp32_dfg": HPVM_TIER_FP32_DFG,
    "fp32": HPVM_TIER_FP32,
    "bf16x3": HPVM_TIER_BF16X3,
    "bf16x6": HPVM_TIER_BF16X6,
    "bf16": HPVM_TIER_BF16,
    "fp8": HPVM_TIER_FP8,
}
