"""Tensor-core variant of the element strategy (digit-split GEMM on tcgen05)
against the FP64 oracle, |got - ref| <= 1e-12 * S componentwise (S the
oracle's absolute contraction), and bit for bit on integer-valued inputs.

The cases walk the kernel's shape logic: ragged tiles of 128 elements, one
to several column blocks (two 16-column halves of 16 / R values of i each),
K = NJ from 1 to 40 (one to three MMA K-steps), every fused
producer kind, R from 1 to 4, and elements whose magnitudes differ by many
orders (per-element scaling of the digits).
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
TC = be.make_config(be.STRAT_ELEMENT, (0, 0, 3))
DF = be.make_config(be.STRAT_ELEMENT, (0, 0, 2))


def run(text, arrs, cfg=TC):
    e = be.Einsum(text)
    outs = [torch.full(e.out_shape, float("nan"), dtype=torch.float64, device=DEV) for _ in range(e.b)]
    bufs = {k: torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for k, v in arrs.items()}
    be.execute(None, e, bufs, outs, cfg=cfg)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def check(text, arrs, cfg=TC, tol=1e-12):
    got = run(text, arrs, cfg)
    ref = ev.evaluate(text, arrs)
    for k, g in enumerate(got):
        r, S = ref[k]
        assert np.all(np.isfinite(g))
        err = np.abs(g - r)
        assert np.all(err <= tol * S), f"row {k}: worst err/S {np.max(err / np.maximum(S, 1e-300)):.3e}"
    return got, ref


@pytest.mark.parametrize("E", [1, 127, 128, 129, 1000, 4099])
def test_dg_ragged_tiles(E):
    D, G, a, b = W.dg_gradient(E=E)
    check(W.dg_gradient_spec(E=E), dict(D=D, G=G, a=a, b=b))


@pytest.mark.parametrize("ndof", [4, 10, 20, 35])
def test_dg_polynomial_orders(ndof):
    """P1..P4 tetrahedra: K = 4..35, one to three column blocks of 12 i."""
    E = 700
    D, G, a, b = W.dg_gradient(E=E, ndof=ndof)
    check(W.dg_gradient_spec(E=E, ndof=ndof), dict(D=D, G=G, a=a, b=b))


def test_dg_p5_falls_back():
    """P5 (56 dofs) needs more shared D planes than fit: the default takes
    the double-float variant, a forced tensor-core run is refused."""
    E = 300
    D, G, a, b = W.dg_gradient(E=E, ndof=56)
    text = W.dg_gradient_spec(E=E, ndof=56)
    check(text, dict(D=D, G=G, a=a, b=b), be.make_config(be.STRAT_ELEMENT))
    with pytest.raises(be.BEError) as exc:
        run(text, dict(D=D, G=G, a=a, b=b), TC)
    assert exc.value.code == be.EUNSUPPORTED


@pytest.mark.parametrize("producer", ["a[e,j]", "sin(a[e,j])*b[e,j]", "a[e,j]*b[e,j]"])
def test_producer_kinds(producer):
    E = 515
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E, producer=producer)
    if producer == "a[e,j]":   # b is then not referenced: declare only what is used
        text = text.replace(f" ; b:f64[{E},35]", "")
        arrs.pop("b")
    check(text, arrs)


@pytest.mark.parametrize("dim", [1, 2, 4])
def test_dimensions(dim):
    """R = dim terms per output (R = 1, 2, 4 need no column padding)."""
    E = 300
    D, G, a, b = W.dg_gradient(E=E, ndof=20, dim=dim)
    check(W.dg_gradient_spec(E=E, ndof=20, dim=dim), dict(D=D, G=G, a=a, b=b))


@pytest.mark.parametrize("NI,NJ", [(50, 40), (1, 1), (64, 17)])
def test_plain_operator(NI, NJ):
    """'ij,ej->ei' (R = 1, no geometric factor): one or two blocks of 32 i,
    K from 1 to 40 (one to three MMA K-steps)."""
    E = 333
    g = np.random.default_rng(NI * 100 + NJ)
    D = g.standard_normal((NI, NJ))
    u = g.standard_normal((E, NJ))
    check(f"ij,ej->ei | D,U ; D:f64[{NI},{NJ}] ; U:f64[{E},{NJ}]", dict(D=D, U=u))


@pytest.mark.parametrize("ndof", [4, 10])
def test_many_tiles_per_cta_one_block(ndof):
    """E = 150000 gives every CTA several tiles; with one column block per
    tile the producer runs furthest ahead of the epilogue."""
    E = 150000
    D, G, a, b = W.dg_gradient(E=E, ndof=ndof)
    check(W.dg_gradient_spec(E=E, ndof=ndof), dict(D=D, G=G, a=a, b=b))


def test_integers_bit_exact():
    E = 777
    D, G, a, b = W.dg_gradient(E=E, ints=True)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E, producer="a[e,j]*b[e,j]")
    got = run(text, arrs)
    ref = ev.evaluate(text, arrs)
    for x in range(3):
        assert np.array_equal(got[x], ref[x][0])


def test_wide_magnitude_range():
    """Elements scaled by 2^-60 .. 2^60 and rows of D by 2^-30 .. 2^30: the
    digits are scaled per element and per row of D."""
    E = 640
    D, G, a, b = W.dg_gradient(E=E)
    g = np.random.default_rng(77)
    b = b * np.exp2(g.integers(-60, 61, size=(E, 1)).astype(np.float64))
    D = D * np.exp2(g.integers(-30, 31, size=(3, 35, 1)).astype(np.float64))
    check(W.dg_gradient_spec(E=E), dict(D=D, G=G, a=a, b=b))


def test_sparse_rows_componentwise():
    """Rows of u with one large entry and the rest 1e-9 smaller, rows of D
    likewise, and elements that are all zero.  The digits share one scale
    per row, so many outputs here cannot be certified by the per-output
    check; those elements are recomputed in FP64 and every output still
    meets the componentwise 1e-12 * S.  All-zero elements are exact zeros."""
    E = 256
    D, G, a, b = W.dg_gradient(E=E)
    b = b.copy()
    b[::3, 1:] *= 1e-9
    b[1::7] = 0.0
    D = D.copy()
    D[:, ::2, 1:] *= 1e-9
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    got, _ = check(text, arrs)
    for x in range(3):
        assert np.all(got[x][1::7] == 0.0)
    check(text, arrs, DF)


@pytest.mark.parametrize("seed", [0, 1])
def test_random_wide_range_entries(seed):
    """Every entry of b (hence u) and of D scaled by its own 2^U, U uniform
    in [-40, 40]: the worst case for shared digit scales.  The default path
    meets 1e-12 * S componentwise on every output."""
    E = 1500
    D, G, a, b = W.dg_gradient(E=E)
    g = np.random.default_rng(500 + seed)
    b = b * np.exp2(g.integers(-40, 41, size=b.shape).astype(np.float64))
    D = D * np.exp2(g.integers(-40, 41, size=D.shape).astype(np.float64))
    check(W.dg_gradient_spec(E=E), dict(D=D, G=G, a=a, b=b))
    check(W.dg_gradient_spec(E=E), dict(D=D, G=G, a=a, b=b), be.make_config(be.STRAT_ELEMENT))


def test_cancelling_outputs():
    """Outputs that cancel almost exactly (G and D chosen so that
    sum_r g_r t_r is tiny against S).  The check bounds the error against
    sum_r |g_r| |t_r| <= S, not against |R|, so these outputs are certified
    without recomputation, and they meet 1e-12 * S."""
    E = 512
    D, G, a, b = W.dg_gradient(E=E)
    G = G.copy()
    G[:, 2, :] = 0.0
    G[:, 1, :] = -G[:, 0, :]
    D = D.copy()
    D[1] = D[0] * (1.0 + 2.0 ** -40)
    check(W.dg_gradient_spec(E=E), dict(D=D, G=G, a=a, b=b))


def test_matches_double_float_variant():
    E = 2000
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    tc, ref = check(text, arrs, TC)
    dfv, _ = check(text, arrs, DF)
    for x in range(3):
        assert np.all(np.abs(tc[x] - dfv[x]) <= 2e-12 * ref[x][1])


def test_default_is_tensor_core_and_unsupported_shape_is_refused():
    E = 64
    D, G, a, b = W.dg_gradient(E=E)
    text = W.dg_gradient_spec(E=E)
    dflt = run(text, dict(D=D, G=G, a=a, b=b), be.make_config(be.STRAT_ELEMENT))
    tc = run(text, dict(D=D, G=G, a=a, b=b), TC)
    for x in range(3):
        assert np.array_equal(dflt[x], tc[x])
    # K = 65 is beyond the exact-level bound
    g = np.random.default_rng(3)
    e = be.Einsum(f"ij,ej->ei | D,U ; D:f64[8,65] ; U:f64[{E},65]")
    out = [torch.empty((E, 8), dtype=torch.float64, device=DEV)]
    bufs = {"D": torch.from_numpy(g.standard_normal((8, 65))).to(DEV),
            "U": torch.from_numpy(g.standard_normal((E, 65))).to(DEV)}
    with pytest.raises(be.BEError) as exc:
        be.execute(None, e, bufs, out, cfg=TC)
    assert exc.value.code == be.EUNSUPPORTED
    be.execute(None, e, bufs, out)   # the default takes another strategy
    torch.cuda.synchronize()


def test_out_of_range_operands_take_the_tested_path():
    """Sine arguments beyond 2^20 and operands below 2^-70 fail the batch
    range test, so their batches run the tested producer (FP64 sine and
    conversion through FP64); neighbouring batches keep the fast one."""
    E = 700
    D, G, a, b = W.dg_gradient(E=E)
    a, b = a.copy(), b.copy()
    a[5, 3] = 3.0e6
    a[100, :] *= 2.0 ** 25
    a[400, 0] = -2.0 ** 21
    b[200, 7] = 2.0 ** -80
    b[300, :] = 0.0
    check(W.dg_gradient_spec(E=E), dict(D=D, G=G, a=a, b=b))
