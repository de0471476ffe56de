"""B300 batched-einsum engine (arxiv 2601.12220 method, sm_103a kernels).

The engine lives in the C-ABI library libbe.so (include/be.h); this package
is its thin Python binding.  Importing it loads the library and fails loudly
if it has not been built (``python paper_2601_12220_b300/build.py``).
"""
from .binding import (  # noqa: F401
    BEError, Batch, Canon, Config, Server, Context, Einsum, execute, execute_host, graph_check, identify, lib,
    make_config, peak_probe, plan_strategy, tune, tune_batch, raise_kernel, identify_kernel,
    OK, EPARSE, EINVALID, ESHAPE, EDTYPE, ETOOMANY, ENOTFOUND, EDB, EBUDGET, ETIMEOUT, ECUDA,
    EUNSUPPORTED, EARG, I8, I32, I64, F16, F32, F64, C64, C128, BF16, STRAT_AUTO, STRAT_GENERIC,
    STRAT_ELEMENT, STRAT_DENSE_SPLIT, PREC_FP64, PREC_SPLIT, SIGMA_INDEX, SIGMA_ARG, SIGMA_ROW, SIGMA_POS,
    KERNEL_ELEMENT, KERNEL_GENERIC, KERNEL_DENSE_GEMM, KERNEL_SPLIT, KERNEL_PERSISTENT,
)

lib()
