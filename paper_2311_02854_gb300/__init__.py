"""Python binding of libdmrg (two-site ab initio DMRG hot path on GB300).

Argument marshalling only: every computation runs in the library's CUDA
kernels behind the C-ABI declared in ``include/dmrg.h``.  Device buffers are
passed as raw pointers (``torch.Tensor.data_ptr()`` or an int); the library
never sees torch types.  Importing does not require a GPU; creating a plan
does, and fails loudly if ``libdmrg.so`` has not been built.
"""
from ._lib import (DMRG_BF16, DMRG_BF16X3, DMRG_BF16X6, DMRG_FP64, DMRG_FP64_TC, DMRG_PRECOND_JACOBI, DMRG_PRECOND_MLP,  # noqa: F401
                   DMRGError, Options, Plan, Stats, extrapolate, grouped_gemm, grouped_gemm_noalloc, lib,
                   lib_path, noalloc_scratch_bytes, selftest_wait, version)
