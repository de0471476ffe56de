"""Persistent multi-instance executor (be_batch_*) on the GPU.

Every output has one owner and a fixed evaluation order, so the batch must
reproduce BE_STRAT_GENERIC on each instance alone bit for bit; a sample is
also checked against the FP64 oracle with the tolerances of test_gpu_parity.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

import paper_2601_12220_b300 as be  # noqa: E402
from oracle import evaluate as ev  # noqa: E402
import workloads as W  # noqa: E402

DEV = "cuda:0"


def make_items(n, seed, **caps):
    g = np.random.default_rng(seed)
    items, meta = [], []
    for _ in range(n):
        inst = W.mix_instance(g, **caps)
        text = W.instance_spec(inst)
        arrs = W.instance_arrays(inst, g)
        e = be.Einsum(text)
        dt = torch.float64 if e.out_dtype == be.F64 else torch.float32
        bufs = {k: torch.from_numpy(v).to(DEV) for k, v in arrs.items()}
        outs = [torch.full(e.out_shape, float("nan"), dtype=dt, device=DEV) for _ in range(e.b)]
        items.append((e, bufs, outs))
        meta.append((inst, text, arrs))
    return items, meta


def generic_alone(e, bufs):
    dt = torch.float64 if e.out_dtype == be.F64 else torch.float32
    outs = [torch.empty(e.out_shape, dtype=dt, device=DEV) for _ in range(e.b)]
    be.execute(None, e, bufs, outs, cfg=be.make_config(be.STRAT_GENERIC))
    return outs


def test_batch_bitwise_equals_generic_and_oracle():
    items, meta = make_items(40, 7, lo_exp=1.0, hi_exp=5.0, max_operand=1 << 16, max_flops=1 << 22)
    ctx = be.Context(None, device=0)
    b = be.Batch(ctx, items)
    info = b.info()
    assert info["rows"] == sum(e.b for e, _, _ in items)
    b.run()
    torch.cuda.synchronize()
    for (e, bufs, outs), (inst, text, arrs) in zip(items, meta):
        alone = generic_alone(e, bufs)
        torch.cuda.synchronize()
        for o, a in zip(outs, alone):
            assert torch.equal(o, a)
    # oracle on a sample of instances
    for (e, bufs, outs), (inst, text, arrs) in list(zip(items, meta))[:12]:
        ref = ev.evaluate(text, arrs)
        K = 1 + math.prod(v for c, v in inst.lens.items() if c not in inst.out) + len(inst.ins)
        tol = 1e-12 if inst.dtype == "f64" else max(K * 2.0 ** -24 / (1 - K * 2.0 ** -24), 1e-6)
        for r in range(e.b):
            got = outs[r].cpu().numpy().astype(np.float64)
            assert np.all(np.abs(got - ref[r][0]) <= tol * ref[r][1])


def test_batch_replay_sees_new_contents():
    items, meta = make_items(10, 9, lo_exp=1.0, hi_exp=4.0, max_operand=1 << 14, max_flops=1 << 20)
    b = be.Batch(None, items, be.make_config(tile=(128, 12, 2)))
    b.run()
    torch.cuda.synchronize()
    first = [[o.clone() for o in outs] for _, _, outs in items]
    b.run()
    torch.cuda.synchronize()
    for (_, _, outs), f in zip(items, first):
        for o, a in zip(outs, f):
            assert torch.equal(o, a)
    for _, bufs, _ in items:
        for t in bufs.values():
            t.mul_(2)
    b.run()
    torch.cuda.synchronize()
    for e, bufs, outs in items:
        alone = generic_alone(e, bufs)
        torch.cuda.synchronize()
        for o, a in zip(outs, alone):
            assert torch.equal(o, a)


def test_batch_functional_instances():
    E = 500
    D, G, a, bb = W.dg_gradient(E=E)
    dg = be.Einsum(W.dg_gradient_spec(E=E))
    dg_bufs = {k: torch.from_numpy(v).to(DEV) for k, v in dict(D=D, G=G, a=a, b=bb).items()}
    dg_outs = [torch.empty((E, 35), dtype=torch.float64, device=DEV) for _ in range(3)]
    A = torch.from_numpy(np.random.default_rng(1).standard_normal((40, 30))).to(DEV)
    B = torch.from_numpy(np.random.default_rng(2).standard_normal((30, 50))).to(DEV)
    aff = be.Einsum("ik,kj->ij | P,Q ; A:f64[40,30] ; B:f64[30,50] ; P(i,k) := $a1*A[i,k]+$b1 ; "
                    "Q(k,j) := $a2*B[k,j]+$b2")
    aff_out = [torch.empty((40, 50), dtype=torch.float64, device=DEV)]
    sc = (0.5, -1.25, 2.0, 0.75)
    b = be.Batch(None, [(dg, dg_bufs, dg_outs), (aff, {"A": A, "B": B}, aff_out, sc)])
    b.run()
    torch.cuda.synchronize()
    ref = ev.evaluate(W.dg_gradient_spec(E=E), dict(D=D, G=G, a=a, b=bb))
    for x in range(3):
        assert np.all(np.abs(dg_outs[x].cpu().numpy() - ref[x][0]) <= 1e-12 * ref[x][1])
    alone = [torch.empty_like(aff_out[0])]
    be.execute(None, aff, {"A": A, "B": B}, alone, scalars=sc, cfg=be.make_config(be.STRAT_GENERIC))
    torch.cuda.synchronize()
    assert torch.equal(alone[0], aff_out[0])


def test_empty_batch_and_empty_rows():
    b = be.Batch(None, [])
    b.run()
    e = be.Einsum("ij->i | A ; A:f64[0,3]")
    b = be.Batch(None, [(e, {"A": torch.zeros((0, 3), dtype=torch.float64, device=DEV)},
                         [torch.zeros((0,), dtype=torch.float64, device=DEV)])])
    b.run()
    torch.cuda.synchronize()
    assert b.info()["tiles"] == 0


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_gemm_tiles_same_bits_at_any_tile_side(dt):
    """Two-operand rows run as GEMM tiles.  The persistent executor uses the
    default side (32 for FP64, 64 for FP32) while a lone launch of a small
    row picks a smaller one to fill the SMs; every output still sums its
    terms in increasing k, so the bits agree."""
    g = np.random.default_rng(3)
    tdt = torch.float64 if dt == "f64" else torch.float32
    specs = [("ik,kj->ij", (70, 33), (33, 90)), ("ki,kj->ij", (40, 64), (40, 33)),
             ("ijcd,cdab->ijab", (5, 9, 6, 7), (6, 7, 8, 5)), ("ik,kj->ij", (600, 40), (40, 700))]
    items = []
    for text, sa, sb in specs:
        spec = f"{text} | A,B ; A:{dt}[{','.join(map(str, sa))}] ; B:{dt}[{','.join(map(str, sb))}]"
        e = be.Einsum(spec)
        bufs = {"A": torch.from_numpy(g.standard_normal(sa)).to(tdt).to(DEV),
                "B": torch.from_numpy(g.standard_normal(sb)).to(tdt).to(DEV)}
        items.append((e, bufs, [torch.full(e.out_shape, float("nan"), dtype=tdt, device=DEV)]))
    ctx = be.Context(None, device=0)
    be.Batch(ctx, items).run()
    torch.cuda.synchronize()
    for e, bufs, outs in items:
        alone = generic_alone(e, bufs)
        torch.cuda.synchronize()
        assert torch.equal(outs[0], alone[0])
