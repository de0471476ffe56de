"""Stacked form of the element strategy (DG local divergence and face mass)
against the FP64 oracle: |got - ref| <= 1e-12 * S componentwise for the
FP64-pipe, double-float and tensor-core variants (the last for contracted
extents up to 64), bit for bit on integer inputs.

The divergence 'xre,rij,xej->ei' reads the field through a select producer
F(x,e,j) := x==0 ? u : (x==1 ? v : w); the face mass 'fe,ifj,fej->ei' has
the face letter f in all three operands.  The cases cover P1..P4 (contracted
extents 12..105), ragged element tiles, b = 1..8 rows with their own fields
and a shared operator, and a plain three-index field buffer.
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
FP64 = be.make_config(be.STRAT_ELEMENT, (0, 0, 1))
DF = be.make_config(be.STRAT_ELEMENT, (0, 0, 2))
TC = be.make_config(be.STRAT_ELEMENT, (0, 0, 3))


def run(text, arrs, cfg=None):
    e = be.Einsum(text)
    outs = [torch.full(e.out_shape, float("nan"), dtype=torch.float64, device=DEV) for _ in range(e.b)]
    bufs = {k: torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for k, v in arrs.items()}
    be.execute(None, e, bufs, outs, cfg=cfg)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def check(text, arrs, cfg=None, tol=1e-12):
    got = run(text, arrs, cfg)
    ref = ev.evaluate(text, arrs)
    for k, g in enumerate(got):
        r, S = ref[k]
        assert np.all(np.isfinite(g))
        err = np.abs(g - r)
        assert np.all(err <= tol * S), f"row {k}: worst err/S {np.max(err / np.maximum(S, 1e-300)):.3e}"
    return got


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("cfg", [None, DF, FP64, TC], ids=["default", "df", "fp64", "tc"])
def test_divergence_orders(order, cfg):
    E = 777
    D, data = W.dg_divergence(E=E, order=order, rows=1)
    text, arrs = W.dg_divergence_spec(E=E, order=order, rows=1), W.dg_divergence_arrays(D, data)
    if cfg is TC and order == 4:                 # K = 3 x 35 = 105 > 64
        with pytest.raises(be.BEError) as exc:
            run(text, arrs, TC)
        assert exc.value.code == be.EUNSUPPORTED
        return
    check(text, arrs, cfg)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("cfg", [None, DF, FP64, TC], ids=["default", "df", "fp64", "tc"])
def test_face_mass_orders(order, cfg):
    """K = 4 NF = 12, 24, 40, 60: every order fits the tensor-core variant
    (P4 with one buffer of u's digit planes)."""
    E = 777
    M, data = W.face_mass(E=E, order=order, rows=1)
    check(W.face_mass_spec(E=E, order=order, rows=1), W.face_mass_arrays(M, data), cfg)


@pytest.mark.parametrize("rows", [2, 8])
def test_batched_rows(rows):
    """b rows with their own metric terms and fields share D; the tile
    shrinks until the eight produced operands fit shared memory."""
    E = 1000
    D, data = W.dg_divergence(E=E, order=4, rows=rows)
    check(W.dg_divergence_spec(E=E, order=4, rows=rows), W.dg_divergence_arrays(D, data))
    M, fd = W.face_mass(E=E, order=3, rows=rows)
    check(W.face_mass_spec(E=E, order=3, rows=rows), W.face_mass_arrays(M, fd))


@pytest.mark.parametrize("E", [1, 5, 32, 33, 4099])
def test_ragged_elements(E):
    D, data = W.dg_divergence(E=E, order=2, rows=1)
    check(W.dg_divergence_spec(E=E, order=2, rows=1), W.dg_divergence_arrays(D, data))


@pytest.mark.parametrize("cfg", [DF, FP64, TC], ids=["df", "fp64", "tc"])
def test_integers_bit_exact(cfg):
    E = 500
    D, data = W.dg_divergence(E=E, order=3, rows=2, ints=True)
    text = W.dg_divergence_spec(E=E, order=3, rows=2)
    arrs = W.dg_divergence_arrays(D, data)
    got = run(text, arrs, cfg)
    ref = ev.evaluate(text, arrs)
    for k in range(2):
        assert np.array_equal(got[k], ref[k][0])
    M, fd = W.face_mass(E=E, order=4, rows=1, ints=True)
    text = W.face_mass_spec(E=E, order=4, rows=1)
    arrs = W.face_mass_arrays(M, fd)
    assert np.array_equal(run(text, arrs, cfg)[0], ev.evaluate(text, arrs)[0][0])


def test_plain_field_buffer():
    """The field as one buffer F[x,e,j] (no select) and J with its letters
    in another order: the same stacked form."""
    E, N = 300, 10
    g = np.random.default_rng(11)
    D = g.standard_normal((3, N, N))
    F = g.standard_normal((3, E, N))
    J = g.standard_normal((E, 3, 3))
    text = f"erx,rij,xej->ei | J,D,F ; J:f64[{E},3,3] ; D:f64[3,{N},{N}] ; F:f64[3,{E},{N}]"
    check(text, dict(J=J, D=D, F=F))


@pytest.mark.parametrize("rows", [1, 3, 8])
def test_tensor_core_groups_and_shared_rows(rows):
    """Tensor-core variant with several producer groups (each row its own
    fields: the tiles run over groups x element tiles) and with rows that
    repeat a group (the same fields: one value written to both rows)."""
    E = 1000
    M, fd = W.face_mass(E=E, order=4, rows=rows)
    check(W.face_mass_spec(E=E, order=4, rows=rows), W.face_mass_arrays(M, fd), TC)
    D, data = W.dg_divergence(E=E, order=3, rows=rows)
    text = W.dg_divergence_spec(E=E, order=3, rows=rows)
    arrs = W.dg_divergence_arrays(D, data)
    check(text, arrs, TC)
    # the first row twice: one group, two rows
    rows_part, decls = text.split(" ; ", 1)
    head, rows_text = rows_part.split(" | ", 1)
    first = rows_text.split(" | ")[0]
    check(f"{head} | {first} | {rows_text} ; {decls}", arrs, TC)


def test_tensor_core_wide_range_and_zero_elements():
    """Fields spanning many decades (most elements cannot be certified and
    are recomputed in FP64 at the end of their tile), elements whose fields
    are all zero (exact zeros) and metric terms of 2^+-40: every output
    within 1e-12 * S."""
    E = 640
    g = np.random.default_rng(5)
    D, data = W.dg_divergence(E=E, order=3, rows=1)
    arrs = W.dg_divergence_arrays(D, data)
    arrs = {k: v.copy() for k, v in arrs.items()}
    fields = [k for k, v in arrs.items() if v.ndim == 2 and v.shape[0] == E]
    for k in fields:
        arrs[k][::3] *= np.exp2(g.integers(-40, 41, size=arrs[k][::3].shape))
        arrs[k][5::11] = 0.0
    text = W.dg_divergence_spec(E=E, order=3, rows=1)
    got = check(text, arrs, TC)
    M, fd = W.face_mass(E=E, order=2, rows=1)
    marr = {k: v.copy() for k, v in W.face_mass_arrays(M, fd).items()}
    marr["U0"] *= np.exp2(g.integers(-40, 41, size=marr["U0"].shape))   # U[f, e, j]
    marr["U0"][:, 7::13] = 0.0
    check(W.face_mass_spec(E=E, order=2, rows=1), marr, TC)
    assert np.all(np.isfinite(got[0]))


def test_tensor_core_variant_refuses_long_contractions():
    """The divergence at P4 contracts K = 105 > 64 values: the tensor-core
    variant refuses it (the default for the stacked form is the double-float
    kernel)."""
    E = 64
    D, data = W.dg_divergence(E=E, order=4, rows=1)
    with pytest.raises(be.BEError) as exc:
        run(W.dg_divergence_spec(E=E, order=4, rows=1), W.dg_divergence_arrays(D, data), TC)
    assert exc.value.code == be.EUNSUPPORTED
