"""The allocation-free GEMM entry point (be_gemm_split_noalloc).

Some callers cannot let a library allocate device memory: they keep every
device byte in their own pool or budget, where an unexpected cudaMalloc could
fail or go unaccounted and a cudaFree could synchronize the device.  This entry
point serves them by keeping its scratch in a fixed array inside the library.

The test calls it through the C ABI twice in a row (different shapes and
data, so the second call must not see the first call's leftovers) and checks
each result against the existing entry point (be_execute on the dense split
strategy, whose scratch the context allocates): both run the same kernels,
so the results must agree bit for bit, and the first is also held to the
split-precision tolerance |C - AB| <= 1e-6 * S against the FP64 oracle (S the
absolute contraction).  It also checks that a call after the warm-up leaves
the device's free memory unchanged, that K = 0 gives zeros, that short row
strides and oversize problems are refused, and that the status word reads
BE_OK.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

import paper_2601_12220_b300 as be  # noqa: E402
from oracle import evaluate as ev  # noqa: E402

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


def noalloc_status():
    v = ctypes.c_int32(-1)
    assert be.lib().be_gemm_split_noalloc_status(ctypes.byref(v)) == be.OK
    return v.value


def test_noalloc_matches_existing_entry_point_twice():
    ctx = be.Context(None, device=0)
    stream = torch.cuda.current_stream()
    g = np.random.default_rng(11)
    for call, (M, N, K) in enumerate([(300, 257, 1000), (129, 64, 3000)]):
        An, Bn = g.standard_normal((M, K)), g.standard_normal((K, N))
        A, B = torch.from_numpy(An).to(DEV), torch.from_numpy(Bn).to(DEV)
        C = torch.full((M, N), float("nan"), dtype=torch.float64, device=DEV)
        rc = noalloc(A, B, C, stream)
        assert rc == be.OK, be.lib().be_last_error().decode()
        ref = existing(ctx, A, B)
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, ref.cpu().numpy())
        if call == 0:
            r, S = ev.evaluate(f"ik,kj->ij | A,B ; A:f64[{M},{K}] ; B:f64[{K},{N}]", dict(A=An, B=Bn))[0]
            assert np.all(np.abs(got - r) <= 1e-6 * S)
    assert noalloc_status() == be.OK


def test_noalloc_allocates_nothing_after_warmup():
    stream = torch.cuda.current_stream()
    g = np.random.default_rng(12)
    A = torch.from_numpy(g.standard_normal((256, 512))).to(DEV)
    B = torch.from_numpy(g.standard_normal((512, 384))).to(DEV)
    C = torch.empty((256, 384), dtype=torch.float64, device=DEV)
    assert noalloc(A, B, C, stream) == be.OK      # warm-up: the array's address is looked up here
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    C2 = torch.empty_like(C)
    free1 = torch.cuda.mem_get_info()[0]
    assert noalloc(A, B, C2, stream) == be.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1
    assert free1 <= free0
    assert torch.equal(C, C2)


def test_noalloc_k0_and_argument_errors():
    stream = torch.cuda.current_stream()
    A = torch.zeros((64, 0), dtype=torch.float64, device=DEV)
    B = torch.zeros((0, 48), dtype=torch.float64, device=DEV)
    C = torch.full((64, 48), float("nan"), dtype=torch.float64, device=DEV)
    lib = be.lib()
    rc = lib.be_gemm_split_noalloc(None, 0, None, 48, ctypes.c_void_p(C.data_ptr()), 48, 64, 48, 0,
                                   ctypes.c_void_p(stream.cuda_stream))
    assert rc == be.OK, lib.be_last_error().decode()
    torch.cuda.synchronize()
    assert torch.all(C == 0.0)
    A = torch.zeros((64, 32), dtype=torch.float64, device=DEV)
    B = torch.zeros((32, 48), dtype=torch.float64, device=DEV)
    rc = lib.be_gemm_split_noalloc(ctypes.c_void_p(A.data_ptr()), 16, ctypes.c_void_p(B.data_ptr()), 48,
                                   ctypes.c_void_p(C.data_ptr()), 48, 64, 48, 32, ctypes.c_void_p(stream.cuda_stream))
    assert rc == be.EARG
    rc = lib.be_gemm_split_noalloc(ctypes.c_void_p(A.data_ptr()), 32, ctypes.c_void_p(B.data_ptr()), 48,
                                   ctypes.c_void_p(C.data_ptr()), 40, 64, 48, 32, ctypes.c_void_p(stream.cuda_stream))
    assert rc == be.EARG
    assert lib.be_gemm_split_noalloc_status(None) == be.EARG


def test_noalloc_rejects_oversize():
    A = torch.zeros((1024, 8192), dtype=torch.float64, device=DEV)
    B = torch.zeros((8192, 1024), dtype=torch.float64, device=DEV)
    C = torch.zeros((1024, 1024), dtype=torch.float64, device=DEV)
    rc = noalloc(A, B, C, torch.cuda.current_stream())
    assert rc == be.ETOOMANY
    assert "bytes of scratch" in be.lib().be_last_error().decode()
