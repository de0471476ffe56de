"""GPU parity of the dense split-precision strategy (tcgen05) vs the FP64 oracle.

Split-precision tolerance: |got - ref| <= 1e-6 * S componentwise (S the
absolute contraction).  A priori the split keeps about 24 bits of each
operand in three BF16 parts, drops the products below the third level
(about 2^-23 relative), loses at most 2^-23 of the leading accumulator per
MMA between drains (4 MMAs at the default drain interval) and sums the
drains with Kahan's compensation; the measured error is reported
alongside.  Small-integer inputs (|x| <= 3) are exact in the first BF16
part and in every partial sum, so those cases must match bit for bit.
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


@pytest.fixture(scope="module")
def ctx():
    return be.Context(None, device=0)


def run_split(ctx, text, arrs):
    e = be.Einsum(text)
    assert be.plan_strategy(ctx, e, precision=be.PREC_SPLIT) == be.STRAT_DENSE_SPLIT
    outs = [torch.full(e.out_shape, float("nan"), dtype=torch.float64, device=DEV) for _ in range(e.b)]
    be.execute(ctx, e, {k: torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for k, v in arrs.items()}, outs,
               precision=be.PREC_SPLIT)
    assert ctx.status() == be.OK
    return [o.cpu().numpy() for o in outs]


def rel_err(got, ref, S):
    d = np.abs(got - ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(S > 0, d / S, np.where(d == 0, 0.0, np.inf))
    return r


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (1, 1, 1), (129, 5, 65), (200, 300, 1000), (256, 128, 4096),
                                   (64, 257, 2049)])
def test_gemm_shapes(ctx, M, N, K):
    g = np.random.default_rng(M * 7 + N * 3 + K)
    A, B = g.standard_normal((M, K)), g.standard_normal((K, N))
    text = f"ik,kj->ij | A,B ; A:f64[{M},{K}] ; B:f64[{K},{N}]"
    got, = run_split(ctx, text, dict(A=A, B=B))
    (ref, S), = ev.evaluate(text, dict(A=A, B=B))
    r = rel_err(got, ref, S)
    assert r.max() <= 1e-6, r.max()


def test_integers_bit_exact(ctx):
    g = np.random.default_rng(1)
    M, N, K = 300, 200, 3000
    A = g.integers(-3, 4, size=(M, K)).astype(np.float64)
    B = g.integers(-3, 4, size=(K, N)).astype(np.float64)
    text = f"ik,kj->ij | A,B ; A:f64[{M},{K}] ; B:f64[{K},{N}]"
    got, = run_split(ctx, text, dict(A=A, B=B))
    assert np.array_equal(got, A @ B)


def test_wide_dynamic_range(ctx):
    """Rows and columns spanning many binades: rows inside [2^-26, 2^40)
    take the fixed scale, the others their own power-of-two scale."""
    g = np.random.default_rng(2)
    M, N, K = 130, 140, 700
    A = g.standard_normal((M, K)) * np.exp2(g.integers(-40, 40, size=(M, 1)))
    B = g.standard_normal((K, N)) * np.exp2(g.integers(-40, 40, size=(1, N)))
    text = f"ik,kj->ij | A,B ; A:f64[{M},{K}] ; B:f64[{K},{N}]"
    got, = run_split(ctx, text, dict(A=A, B=B))
    (ref, S), = ev.evaluate(text, dict(A=A, B=B))
    assert rel_err(got, ref, S).max() <= 1e-6


def test_chem_reduced(ctx):
    """Workload 3 shape at v=16, o=8: 'abef,efij->abij', b=4, shared efij."""
    As, T = W.chem_dense(v=16, o=8)
    arrs = {f"A{k}": A for k, A in enumerate(As)} | {"T": T}
    text = W.chem_dense_spec(v=16, o=8)
    got = run_split(ctx, text, arrs)
    ref = ev.evaluate(text, arrs)
    for k in range(4):
        assert rel_err(got[k], ref[k][0], ref[k][1]).max() <= 1e-6


def test_swapped_operand_roles(ctx):
    """'kj,ik->ij' puts the free letters of the second operand first: the
    plan takes the second operand as A and the first as B (C = A B with the
    roles swapped); within 1e-6 S of the oracle."""
    g = np.random.default_rng(9)
    A, B = g.standard_normal((30, 20)), g.standard_normal((20, 40))
    text = "kj,ik->ij | B,A ; A:f64[30,20] ; B:f64[20,40]"
    got, = run_split(ctx, text, dict(A=A, B=B))
    (ref, S), = ev.evaluate(text, dict(A=A, B=B))
    assert rel_err(got, ref, S).max() <= 1e-6


def test_interleaved_output_rejected_then_generic(ctx):
    """'abk,kc->acb' interleaves the two operands' free letters in the output:
    not a plain GEMM layout; AUTO falls back to the generic kernel."""
    e = be.Einsum("abk,kc->acb | A,B ; A:f64[6,5,20] ; B:f64[20,7]")
    assert be.plan_strategy(ctx, e, precision=be.PREC_SPLIT) == be.STRAT_GENERIC
    with pytest.raises(be.BEError) as ex:
        be.plan_strategy(ctx, e, be.make_config(be.STRAT_DENSE_SPLIT), precision=be.PREC_SPLIT)
    assert ex.value.code == be.EUNSUPPORTED


def test_needs_context():
    e = be.Einsum("ik,kj->ij | A,B ; A:f64[8,8] ; B:f64[8,8]")
    t = torch.zeros((8, 8), dtype=torch.float64, device=DEV)
    with pytest.raises(be.BEError) as ex:
        be.execute(None, e, {"A": t, "B": t}, [torch.empty_like(t)], precision=be.PREC_SPLIT,
                   cfg=be.make_config(be.STRAT_DENSE_SPLIT))
    assert ex.value.code == be.EARG


def test_chem_full_size_sampled(ctx):
    """Workload 3 at full size (v=128, o=32, b=4): 4096 sampled entries per
    row against the oracle, plus the error statistics."""
    As, T = W.chem_dense()
    arrs = {f"A{k}": A for k, A in enumerate(As)} | {"T": T}
    text = W.chem_dense_spec()
    got = run_split(ctx, text, arrs)
    g = np.random.default_rng(0)
    n_out = 128 * 128 * 32 * 32
    sel = np.unique(np.concatenate([g.integers(0, n_out, 4096), [0, n_out - 1]]))
    ref = ev.evaluate(text, arrs, sel=sel)
    worst = 0.0
    for k in range(4):
        r = rel_err(got[k].reshape(-1)[sel], ref[k][0], ref[k][1])
        worst = max(worst, r.max())
    print(f"split-precision max error / S over samples: {worst:.3e}")
    assert worst <= 1e-6


def run_split_sc(ctx, text, arrs, scalars=()):
    e = be.Einsum(text)
    assert be.plan_strategy(ctx, e, precision=be.PREC_SPLIT) == be.STRAT_DENSE_SPLIT
    outs = [torch.full(e.out_shape, float("nan"), dtype=torch.float64, device=DEV) for _ in range(e.b)]
    be.execute(ctx, e, {k: torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for k, v in arrs.items()}, outs,
               precision=be.PREC_SPLIT, scalars=scalars)
    assert ctx.status() == be.OK
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("M,N,K", [(300, 260, 200), (129, 5, 65), (256, 384, 2048)])
def test_affine_producers_runtime_scalars(ctx, M, N, K):
    """(alpha1 A + beta1)(alpha2 B + beta2) with runtime scalars, fused into
    the split of both operands."""
    g = np.random.default_rng(M + N + K)
    A, B = g.standard_normal((M, K)), g.standard_normal((K, N))
    text = (f"ik,kj->ij | P,Q ; A:f64[{M},{K}] ; B:f64[{K},{N}] ; P(i,k) := $a1*A[i,k]+$b1 ; "
            f"Q(k,j) := $a2*B[k,j]+$b2")
    sc = (0.5, -1.25, 2.0, 0.75)
    got, = run_split_sc(ctx, text, dict(A=A, B=B), sc)
    (ref, S), = ev.evaluate(text, dict(A=A, B=B), scalars=dict(a1=sc[0], b1=sc[1], a2=sc[2], b2=sc[3]))
    assert rel_err(got, ref, S).max() <= 1e-6


def test_affine_tccg_shape_literals(ctx):
    """A TCCG-shaped contraction 'abcd,cdef->abef' (M = ab, K = cd, N = ef)
    with literal coefficients, a subtraction and a division by a constant,
    two rows sharing the second operand."""
    g = np.random.default_rng(5)
    a, b, c, d, e_, f = 12, 20, 9, 30, 14, 10
    A0, A1 = g.standard_normal((a, b, c, d)), g.standard_normal((a, b, c, d))
    B = g.standard_normal((c, d, e_, f))
    text = (f"abcd,cdef->abef | P0,Q | P1,Q ; A0:f64[{a},{b},{c},{d}] ; A1:f64[{a},{b},{c},{d}] ; "
            f"B:f64[{c},{d},{e_},{f}] ; P0(a,b,c,d) := 0.5*A0[a,b,c,d] - 2.0 ; "
            f"P1(a,b,c,d) := -(A1[a,b,c,d] + 1.5) ; Q(c,d,e,f) := B[c,d,e,f]/4.0 + 0.25")
    arrs = dict(A0=A0, A1=A1, B=B)
    got = run_split_sc(ctx, text, arrs)
    ref = ev.evaluate(text, arrs)
    for k in range(2):
        assert rel_err(got[k], ref[k][0], ref[k][1]).max() <= 1e-6


def test_affine_integers_bit_exact(ctx):
    """Small-integer operands and integer coefficients stay exact in every
    TF32 part and partial sum: bit-exact against the oracle."""
    g = np.random.default_rng(9)
    M, N, K = 200, 150, 1500
    A = g.integers(-3, 4, (M, K)).astype(np.float64)
    B = g.integers(-3, 4, (K, N)).astype(np.float64)
    text = (f"ik,kj->ij | P,Q ; A:f64[{M},{K}] ; B:f64[{K},{N}] ; P(i,k) := 2*A[i,k]-1 ; "
            f"Q(k,j) := $s*B[k,j]+$t")
    got, = run_split_sc(ctx, text, dict(A=A, B=B), (-2.0, 3.0))
    (ref, S), = ev.evaluate(text, dict(A=A, B=B), scalars=dict(s=-2.0, t=3.0))
    assert np.array_equal(got, ref)


def test_rows_outside_the_fixed_scale_window(ctx):
    """Rows whose largest entry lies far outside [2^-26, 2^40) (2^-300,
    2^-60, 2^60, 2^300) are split again with their own scale; columns of B
    at 2^+-200.  Every output within 1e-6 S."""
    g = np.random.default_rng(5)
    M, N, K = 8, 6, 200
    A = g.standard_normal((M, K)) * np.exp2(np.array([-300, -60, -27, 0, 39, 41, 60, 300], dtype=float))[:, None]
    B = g.standard_normal((K, N)) * np.exp2(np.array([-200, -20, 0, 0, 20, 200], dtype=float))[None, :]
    text = f"ik,kj->ij | A,B ; A:f64[{M},{K}] ; B:f64[{K},{N}]"
    got, = run_split(ctx, text, dict(A=A, B=B))
    (ref, S), = ev.evaluate(text, dict(A=A, B=B))
    assert rel_err(got, ref, S).max() <= 1e-6


@pytest.mark.parametrize("hdrain", [2, 4])
def test_longer_drain_intervals(ctx, hdrain):
    """Drain intervals of 2 and 4 k-blocks (faster, with a looser a-priori
    bound) on N(0,1) data: the measured error stays far inside 1e-6 S."""
    g = np.random.default_rng(6 + hdrain)
    M, N, K = 256, 256, 2048
    A, B = g.standard_normal((M, K)), g.standard_normal((K, N))
    text = f"ik,kj->ij | A,B ; A:f64[{M},{K}] ; B:f64[{K},{N}]"
    e = be.Einsum(text)
    outs = [torch.full(e.out_shape, float("nan"), dtype=torch.float64, device=DEV)]
    be.execute(ctx, e, {"A": torch.from_numpy(A).to(DEV), "B": torch.from_numpy(B).to(DEV)}, outs,
               cfg=be.make_config(be.STRAT_DENSE_SPLIT, (0, 0, hdrain)), precision=be.PREC_SPLIT)
    assert ctx.status() == be.OK
    (ref, S), = ev.evaluate(text, dict(A=A, B=B))
    assert rel_err(outs[0].cpu().numpy(), ref, S).max() <= 1e-7
