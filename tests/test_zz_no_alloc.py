"""The allocation-free GEMM entry point (be_gemm_split_noalloc).

Some callers cannot let a library allocate device memory: they keep every
device byte in their own pool or budget, where an unexpected cudaMalloc could
fail or go unaccounted and a cudaFree could synchronize the device.  This entry
point serves them by keeping its scratch in a fixed array inside the library.

The test calls it through the C ABI twice in a row (different shapes and
data, so the second call must not see the first call's leftovers) and checks
each result against the existing entry point (be_execute on the dense split
strategy, whose scratch the context allocates) within the split-precision
tolerance used by the other tests, |a - b| <= 1e-6 * S with S the absolute
contraction.  It also checks that a problem too large for the fixed array is
refused.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

import paper_2601_12220_b300 as be  # noqa: E402

DEV = "cuda:0"


def noalloc(A, B, C, stream):
    M, K = A.shape
    N = B.shape[1]
    return be.lib().be_gemm_split_noalloc(
        ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()), B.stride(0),
        ctypes.c_void_p(C.data_ptr()), C.stride(0), M, N, K, ctypes.c_void_p(stream.cuda_stream))


def existing(ctx, A, B):
    M, K = A.shape
    N = B.shape[1]
    e = be.Einsum(f"ik,kj->ij | A,B ; A:f64[{M},{K}] ; B:f64[{K},{N}]")
    C = torch.empty((M, N), dtype=torch.float64, device=DEV)
    be.execute(ctx, e, {"A": A, "B": B}, [C], precision=be.PREC_SPLIT, cfg=be.make_config(be.STRAT_DENSE_SPLIT))
    return C


def test_noalloc_matches_existing_entry_point_twice():
    ctx = be.Context(None, device=0)
    stream = torch.cuda.current_stream()
    g = np.random.default_rng(11)
    for M, N, K in [(300, 257, 1000), (129, 64, 3000)]:
        A = torch.from_numpy(g.standard_normal((M, K))).to(DEV)
        B = torch.from_numpy(g.standard_normal((K, N))).to(DEV)
        C = torch.full((M, N), float("nan"), dtype=torch.float64, device=DEV)
        rc = noalloc(A, B, C, stream)
        assert rc == be.OK, be.lib().be_last_error().decode()
        ref = existing(ctx, A, B)
        torch.cuda.synchronize()
        S = (A.abs() @ B.abs()).cpu().numpy()
        diff = np.abs(C.cpu().numpy() - ref.cpu().numpy())
        assert np.all(np.isfinite(diff))
        assert np.all(diff <= 1e-6 * S), diff.max()


def test_noalloc_rejects_oversize():
    A = torch.zeros((1024, 4096), dtype=torch.float64, device=DEV)
    B = torch.zeros((4096, 1024), dtype=torch.float64, device=DEV)
    C = torch.zeros((1024, 1024), dtype=torch.float64, device=DEV)
    rc = noalloc(A, B, C, torch.cuda.current_stream())
    assert rc == be.ETOOMANY
    assert "bytes of scratch" in be.lib().be_last_error().decode()
