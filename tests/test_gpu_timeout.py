"""Failure detection on the tensor-core kernels and on the dependency waits
of factored batch steps, tested without a GPU fault.

A context's wait limit (be_ctx_set_wait_limit) of a hundred SM cycles makes
the pipeline waits of the element strategy's digit-split GEMM and of the
dense split GEMM run out on purpose: the first wait on data that is still
being produced (a TMA copy from HBM, a tile of digits) gives up, the CTA
stops issuing, lets its issued MMAs and copies complete, frees its tensor
memory and leaves BE_ETIMEOUT in the context's status word.  The context
stays usable: the next call with the default limit gives correct results
and status BE_OK.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

import paper_2601_12220_b300 as be  # noqa: E402
from oracle import evaluate as ev  # noqa: E402
import workloads as W  # noqa: E402

DEV = "cuda:0"


def _dg(ctx, E, cfg):
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    e = be.Einsum(text)
    outs = [torch.full((E, 35), float("nan"), dtype=torch.float64, device=DEV) for _ in range(3)]
    be.execute(ctx, e, {k: torch.from_numpy(v).to(DEV) for k, v in arrs.items()}, outs, cfg=cfg)
    torch.cuda.synchronize()
    return text, arrs, [o.cpu().numpy() for o in outs]


def test_element_tc_wait_runs_out_then_recovers():
    ctx = be.Context(None, device=0)
    tc = be.make_config(be.STRAT_ELEMENT, (0, 0, 3))
    assert ctx.status() == be.OK
    ctx.set_wait_limit(100)
    _dg(ctx, 40000, tc)
    assert ctx.status() == be.ETIMEOUT
    assert ctx.status() == be.OK            # read and cleared
    ctx.set_wait_limit(0)
    text, arrs, got = _dg(ctx, 3000, tc)
    assert ctx.status() == be.OK
    ref = ev.evaluate(text, arrs)
    for x in range(3):
        r, S = ref[x]
        assert np.all(np.abs(got[x] - r) <= 1e-12 * S)


def _dense(ctx, M, N, K, seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((M, K))
    B = g.standard_normal((K, N))
    e = be.Einsum(f"ik,kj->ij | A,B ; A:f64[{M},{K}] ; B:f64[{K},{N}]")
    C = torch.full((M, N), float("nan"), dtype=torch.float64, device=DEV)
    be.execute(ctx, e, {"A": torch.from_numpy(A).to(DEV), "B": torch.from_numpy(B).to(DEV)}, [C],
               precision=be.PREC_SPLIT, cfg=be.make_config(be.STRAT_DENSE_SPLIT))
    torch.cuda.synchronize()
    return A, B, C.cpu().numpy()


def test_dense_wait_runs_out_then_recovers():
    ctx = be.Context(None, device=0)
    ctx.set_wait_limit(100)
    _dense(ctx, 512, 512, 4096, 1)
    assert ctx.status() == be.ETIMEOUT
    ctx.set_wait_limit(0)
    A, B, C = _dense(ctx, 300, 257, 1000, 2)
    assert ctx.status() == be.OK
    S = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - A @ B) <= 1e-6 * S)


def test_wait_limit_rejects_negative():
    ctx = be.Context(None, device=0)
    with pytest.raises(be.BEError) as exc:
        ctx.set_wait_limit(-1)
    assert exc.value.code == be.EARG


def test_peak_probe_rates_plausible():
    """The FP64 and FP32 FMA-chain probes report rates between a tenth of and
    twice the nominal B300 figures (1.25 and about 77 TFLOP/s), FP32 far above
    FP64."""
    f64 = be.peak_probe("fp64", reps=3)
    f32 = be.peak_probe("fp32", reps=3)
    assert 0.1 * 1.25 < f64 < 2 * 1.25
    assert 0.1 * 77 < f32 < 2 * 77
    assert f32 > 10 * f64


def _chain_batch(ctx, seed):
    """A batch with one factored instance ('ab,bc,cd,de->ae', three steps
    deep): its later steps wait for the earlier ones inside the launch."""
    g = np.random.default_rng(seed)
    shapes = {"P": (32, 48), "Q": (48, 40), "R": (40, 36), "T": (36, 24)}   # the oracle's nest stays small
    arrs = {k: g.standard_normal(v) for k, v in shapes.items()}
    text = "ab,bc,cd,de->ae | P,Q,R,T ; " + " ; ".join(f"{k}:f64[{v[0]},{v[1]}]" for k, v in shapes.items())
    e = be.Einsum(text)
    out = [torch.full(e.out_shape, float("nan"), dtype=torch.float64, device=DEV)]
    b = be.Batch(ctx, [(e, {k: torch.from_numpy(v).to(DEV) for k, v in arrs.items()}, out)])
    assert b.factored()["instances"] == 1 and b.factored()["phases"] == 3
    return b, text, arrs, out


def test_factored_step_wait_runs_out_then_recovers():
    """A wait limit of a hundred SM cycles, in force when a factored batch is
    created, makes its dependency waits run out while the earlier steps are
    still running: BE_ETIMEOUT in the context's status word, the waiting
    tiles skipped (and still counted, so that nothing waits for them).  A
    batch created afterwards with the default limit is correct."""
    ctx = be.Context(None, device=0)
    ctx.set_wait_limit(100)
    b, _, _, _ = _chain_batch(ctx, 3)
    b.run()
    torch.cuda.synchronize()
    assert ctx.status() == be.ETIMEOUT
    assert ctx.status() == be.OK
    ctx.set_wait_limit(0)
    b, text, arrs, out = _chain_batch(ctx, 4)
    b.run()
    torch.cuda.synchronize()
    assert ctx.status() == be.OK
    (r, S), = ev.evaluate(text, arrs)
    assert np.all(np.abs(out[0].cpu().numpy() - r) <= 1e-12 * S)
