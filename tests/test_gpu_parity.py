"""GPU parity: the CUDA path through the C ABI vs the FP64 oracle.

Tolerances (componentwise, against the oracle's absolute contraction S):
  FP64 paths       |got - ref| <= 1e-12 * S
  FP32-output path |got - ref| <= max(gamma_K(2^-24), 1e-6) * S,
                   gamma_K = K u / (1 - K u), K = contracted terms + operands
Integer-valued inputs make every correct evaluation order exact, so those
cases are compared bit for bit.
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


def to_dev(arrs):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for k, v in arrs.items()}


def run(text, arrs, cfg=None, scalars=(), precision=be.PREC_FP64, ctx=None):
    e = be.Einsum(text)
    dt = torch.float64 if e.out_dtype == be.F64 else torch.float32
    outs = [torch.full(e.out_shape, float("nan"), dtype=dt, device=DEV) for _ in range(e.b)]
    be.execute(ctx, e, to_dev(arrs), outs, cfg=cfg, scalars=scalars, precision=precision)
    torch.cuda.synchronize()
    return [o.cpu().numpy().astype(np.float64) for o in outs], e


def assert_close(got, ref, S, tol):
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    bound = tol * S
    bad = err > bound
    if bad.any():
        k = np.argmax(err - bound)
        raise AssertionError(f"{bad.sum()} entries off; worst err {err.flat[k]:.3e} vs bound {bound.flat[k]:.3e}")


def gamma(K, u=2.0 ** -24):
    return K * u / (1 - K * u)


# ------------------------------------------------------------- element strategy

@pytest.mark.parametrize("strategy", [be.STRAT_AUTO, be.STRAT_ELEMENT, be.STRAT_GENERIC])
def test_fem_action_full(strategy):
    D, us = W.fem_action()
    arrs = {"D": D, **{f"u{k}": u for k, u in enumerate(us)}}
    text = W.fem_action_spec()
    got, e = run(text, arrs, cfg=be.make_config(strategy))
    ref = ev.evaluate(text, arrs)
    for k in range(4):
        assert_close(got[k], ref[k][0], ref[k][1], 1e-12)


def test_fem_action_integers_bit_exact():
    D, us = W.fem_action(ints=True)
    arrs = {"D": D, **{f"u{k}": u for k, u in enumerate(us)}}
    text = W.fem_action_spec()
    for strategy in (be.STRAT_ELEMENT, be.STRAT_GENERIC):
        got, _ = run(text, arrs, cfg=be.make_config(strategy))
        ref = ev.evaluate(text, arrs)
        for k in range(4):
            assert np.array_equal(got[k], ref[k][0])


@pytest.mark.parametrize("E", [1, 31, 33, 1000, 4099])
def test_dg_gradient_ragged(E):
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    assert be.plan_strategy(None, be.Einsum(text)) == be.STRAT_ELEMENT
    got, _ = run(text, arrs)
    ref = ev.evaluate(text, arrs)
    for x in range(3):
        assert_close(got[x], ref[x][0], ref[x][1], 1e-12)


def test_dg_gradient_integers_bit_exact():
    E = 777
    D, G, a, b = W.dg_gradient(E=E, ints=True)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E, producer="a[e,j]*b[e,j]")
    for strategy in (be.STRAT_ELEMENT, be.STRAT_GENERIC):
        got, _ = run(text, arrs, cfg=be.make_config(strategy))
        ref = ev.evaluate(text, arrs)
        for x in range(3):
            assert np.array_equal(got[x], ref[x][0])


def test_dg_gradient_fp64_pipe_variant():
    E = 1001
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    got, _ = run(text, arrs, cfg=be.make_config(be.STRAT_ELEMENT, (32, 256, 1)))
    ref = ev.evaluate(text, arrs)
    for x in range(3):
        assert_close(got[x], ref[x][0], ref[x][1], 1e-12)


@pytest.mark.parametrize("variant", [2, 3])
def test_df_sine_matches_fp64_sin(variant):
    """The fused producer sin(a) * b with b = 1 through an identity operator
    returns the double-float sine itself; compare with CUDA's FP64 sin.  The
    arguments reach 2^19.9, where the quadrant must come from x in FP64 (a
    float image of x can be a quadrant off there).  Variant 2 is the
    double-float kernel, 3 the tensor-core kernel."""
    E, N = 6144, 35
    g = np.random.default_rng(12)
    a = np.concatenate([g.standard_normal((E // 3, N)) * 3, g.uniform(-1e4, 1e4, (E // 3, N)),
                        g.uniform(2.0 ** 18, 2.0 ** 19.9, (E // 3, N)) * g.choice([-1.0, 1.0], (E // 3, N))])
    a[0, :5] = [0.0, np.pi, -np.pi / 2, 1e-30, 2.0 ** 19]
    text = (f"ij,ej->ei | D,U ; D:f64[{N},{N}] ; a:f64[{E},{N}] ; b:f64[{E},{N}] ; "
            f"U(e,j) := sin(a[e,j])*b[e,j]")
    got, _ = run(text, dict(D=np.eye(N), a=a, b=np.ones((E, N))), cfg=be.make_config(be.STRAT_ELEMENT, (0, 0, variant)))
    ref = torch.sin(torch.from_numpy(a).to(DEV)).cpu().numpy()
    # double-float carries about 46-48 significant bits
    assert np.max(np.abs(got[0] - ref)) <= 1e-14


@pytest.mark.parametrize("tile", [8, 32, 64])
def test_dg_gradient_tiles(tile):
    E = 2048 + 17
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    got, _ = run(text, arrs, cfg=be.make_config(be.STRAT_ELEMENT, (tile, 256)))
    ref = ev.evaluate(text, arrs)
    for x in range(3):
        assert_close(got[x], ref[x][0], ref[x][1], 1e-12)


def test_dg_gradient_full_size_sampled():
    """E = 262144, the benchmark's launch configuration; sampled outputs per
    row against the oracle evaluated one by one."""
    E = 262144
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    got, _ = run(text, arrs)
    g = np.random.default_rng(0)
    sel = np.unique(np.concatenate([g.integers(0, E * 35, 4096), [0, E * 35 - 1]]))
    ref = ev.evaluate(text, arrs, sel=sel)
    for x in range(3):
        assert_close(got[x].reshape(-1)[sel], ref[x][0], ref[x][1], 1e-12)


# ------------------------------------------------------------- generic strategy

@pytest.mark.parametrize("k", range(24))
def test_uneven_mix_notations(k):
    g = np.random.default_rng(100 + k)
    inst = W.mix_instance(g, lo_exp=1.0, hi_exp=3.5, max_operand=1 << 14, max_flops=1 << 22)
    text = W.instance_spec(inst)
    arrs = W.instance_arrays(inst, g)
    got, e = run(text, arrs)
    ref = ev.evaluate(text, arrs)
    K = 1 + math.prod(v for c, v in inst.lens.items() if c not in inst.out) + len(inst.ins)
    tol = 1e-12 if inst.dtype == "f64" else max(gamma(K), 1e-6)
    for r in range(e.b):
        assert_close(got[r], ref[r][0], ref[r][1], tol)


def test_producers_generic():
    rng = np.random.default_rng(8)
    E, N = 300, 10
    u, v, w = (rng.standard_normal((E, N)) for _ in range(3))
    J = rng.standard_normal((3, 3, E))
    D = rng.standard_normal((3, N, N))
    text = (f"xre,rij,xej->ei | J,D,F ; J:f64[3,3,{E}] ; D:f64[3,{N},{N}] ; u:f64[{E},{N}] ; "
            f"v:f64[{E},{N}] ; w:f64[{E},{N}] ; F(x,e,j):f64[3,{E},{N}] := x==0 ? u[e,j] : (x==1 ? v[e,j] : w[e,j])")
    arrs = dict(J=J, D=D, u=u, v=v, w=w)
    got, _ = run(text, arrs)
    ref = ev.evaluate(text, arrs)
    assert_close(got[0], ref[0][0], ref[0][1], 1e-12)
    # affine producers with runtime scalars, (alpha1 A + beta1)(alpha2 B + beta2)
    A = rng.standard_normal((40, 30))
    B = rng.standard_normal((30, 50))
    text = ("ik,kj->ij | P,Q ; A:f64[40,30] ; B:f64[30,50] ; P(i,k) := $a1*A[i,k]+$b1 ; "
            "Q(k,j) := $a2*B[k,j]+$b2")
    sc = (0.5, -1.25, 2.0, 0.75)
    got, _ = run(text, dict(A=A, B=B), scalars=sc)
    ref = ev.evaluate(text, dict(A=A, B=B), scalars=dict(a1=sc[0], b1=sc[1], a2=sc[2], b2=sc[3]))
    assert_close(got[0], ref[0][0], ref[0][1], 1e-12)


def test_feinsum_listing(golden):
    text = golden("einsum_examples.json")["feinsum_listing"]["spec"]
    rng = np.random.default_rng(3)
    arrs = dict(P=rng.standard_normal((96, 4)), Q=rng.standard_normal(4), R=rng.standard_normal(4))
    got, _ = run(text, arrs)
    ref = ev.evaluate(text, arrs)
    for r in range(2):
        assert_close(got[r], ref[r][0], ref[r][1], 1e-12)


def test_strided_views():
    rng = np.random.default_rng(4)
    D = torch.from_numpy(rng.standard_normal((35, 35))).to(DEV)
    U = torch.from_numpy(rng.standard_normal((35, 500))).to(DEV)
    e = be.Einsum("ij,ej->ei | D,U ; D:f64[35,35] ; U:f64[500,35]")
    out = torch.empty((500, 35), dtype=torch.float64, device=DEV)
    for strategy in (be.STRAT_ELEMENT, be.STRAT_GENERIC):
        be.execute(None, e, {"D": D.t(), "U": U.t()}, [out], cfg=be.make_config(strategy))
        torch.cuda.synchronize()
        ref, S = ev.einsum_f64("ei", ["ij", "ej"], [D.t().cpu().numpy(), U.t().cpu().numpy()])
        assert_close(out.cpu().numpy(), ref, S, 1e-12)


def test_edge_cases():
    # empty contracted axis -> zeros
    got, _ = run("ij->i | A ; A:f64[5,0]", {"A": np.zeros((5, 0))})
    assert np.array_equal(got[0], np.zeros(5))
    # scalar output (full contraction) of a diagonal
    rng = np.random.default_rng(5)
    A = rng.standard_normal((7, 7))
    got, _ = run("ii-> | A ; A:f64[7,7]", {"A": A})
    ref, S = ev.einsum_f64("", ["ii"], [A])
    assert_close(got[0], ref, S, 1e-12)
    # empty element axis
    D, G, a, b = W.dg_gradient(E=0)
    got, _ = run(W.dg_gradient_spec(E=0), dict(D=D, G=G, a=a, b=b))
    assert got[0].shape == (0, 35)


def test_execute_host_matches_device():
    E = 5000
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    e = be.Einsum(text)
    ctx = be.Context(None, device=0)
    outs = [np.empty((E, 35)) for _ in range(3)]
    be.execute_host(ctx, e, arrs, outs)
    dev, _ = run(text, arrs)
    for x in range(3):
        assert np.array_equal(outs[x], dev[x])


@pytest.mark.parametrize("E", [60001, 100000])
def test_execute_host_chunked_matches_device(E):
    """Above 64 MB the host path streams element chunks through three
    streams; every chunk's results equal the device run bit for bit."""
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    ctx = be.Context(None, device=0)
    outs = [np.full((E, 35), np.nan) for _ in range(3)]
    be.execute_host(ctx, be.Einsum(text), arrs, outs)
    dev, _ = run(text, arrs)
    for x in range(3):
        assert np.array_equal(outs[x], dev[x])


def test_execute_host_unchunkable_layout_and_stacked_form():
    """A field stored with the element letter inside (not outermost) keeps
    the one-piece host path; the stacked divergence form streams in chunks."""
    E, N = 300000, 35
    g = np.random.default_rng(4)
    U = g.standard_normal((N, E))
    Dm = g.standard_normal((N, N))
    text = f"je,ij->ei | U,D ; U:f64[{N},{E}] ; D:f64[{N},{N}]"
    ctx = be.Context(None, device=0)
    out = [np.full((E, N), np.nan)]
    be.execute_host(ctx, be.Einsum(text), dict(U=U, D=Dm), out)
    dev, _ = run(text, dict(U=U, D=Dm))
    assert np.array_equal(out[0], dev[0])
    D, data = W.dg_divergence(E=100000, order=4, rows=1)
    arrs = W.dg_divergence_arrays(D, data)
    text = W.dg_divergence_spec(E=100000, order=4, rows=1)
    out = [np.full((100000, 35), np.nan)]
    be.execute_host(ctx, be.Einsum(text), arrs, out)
    dev, _ = run(text, arrs)
    assert np.array_equal(out[0], dev[0])


def test_deterministic():
    E = 3001
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    first, _ = run(text, arrs)
    for _ in range(3):
        again, _ = run(text, arrs)
        for x in range(3):
            assert np.array_equal(first[x], again[x])


def test_lookup_transfer_same_bits():
    """A config stored under the normal form and applied to a renamed,
    permuted copy gives the same bits as on the original (transfer, Alg. 2)."""
    E = 2000
    D, G, a, b = W.dg_gradient(E=E)
    arrs = dict(D=D, G=G, a=a, b=b)
    text = W.dg_gradient_spec(E=E)
    ctx = be.Context(None, device=0)
    e = be.Einsum(text)
    ctx.record(e.canonicalize(), be.make_config(be.STRAT_ELEMENT, (16, 128)), 1e-3)
    got, _ = run(text, arrs, ctx=ctx)
    rows = " | ".join(f"D,G{x},U" for x in (2, 1, 0))
    decls = text.split(";", 1)[1]
    text2 = f"pqs,ep,es->eq | {rows} ;" + decls.replace("G[e,r,", "G[e,p,").replace("(e,r)", "(e,p)") \
        .replace("(e,j)", "(e,s)").replace("a[e,j]", "a[e,s]").replace("b[e,j]", "b[e,s]")
    e2 = be.Einsum(text2)
    assert e2.canonicalize().key == e.canonicalize().key
    got2, _ = run(text2, arrs, ctx=ctx)
    for x in range(3):
        assert np.array_equal(got[x], got2[2 - x])


@pytest.mark.parametrize("share", [1, 10, 17, 0], ids=["df", "mixed", "fp64", "default"])
def test_small_operator_kernel_fp64_share(share):
    """Small operators (NI, NJ <= 8) run one element per thread, a share of
    the elements as FP64 multiply-adds and the rest in double-float
    (tile[3] = 1 + sixteenths on the FP64 pipe): FEM action (4 x 4, four
    fields), a P1-sized gradient (R = 3 with G and the sine producer) and a
    7 x 7 operator, with element counts that leave ragged blocks."""
    cfg = be.make_config(be.STRAT_ELEMENT, (0, 0, 2, share))
    E = 5003
    D, us = W.fem_action(E=E)
    text = W.fem_action_spec(E=E)
    arrs = {"D": D, **{f"u{k}": u for k, u in enumerate(us)}}
    got, _ = run(text, arrs, cfg=cfg)
    for k, (r, S) in enumerate(ev.evaluate(text, arrs)):
        assert_close(got[k], r, S, 1e-12)
    for ndof in (4, 7):
        E = 3001
        D, G, a, b = W.dg_gradient(E=E, ndof=ndof)
        text = W.dg_gradient_spec(E=E, ndof=ndof)
        arrs = dict(D=D, G=G, a=a, b=b)
        got, _ = run(text, arrs, cfg=cfg)
        for k, (r, S) in enumerate(ev.evaluate(text, arrs)):
            assert_close(got[k], r, S, 1e-12)


GEN = be.make_config(be.STRAT_GENERIC)


@pytest.mark.parametrize("text_fmt,shapes", [
    # mode 0 for a 100-term contraction with 40000 outputs (thread per output
    # up to 512 terms once there are 32768 outputs)
    ("ik,kj,k->ij", {"A": (200, 100), "B": (100, 200), "C": (100,)}),
    # mode 0 (contraction < 64), one and two contracted letters
    ("ij,j->i", {"A": (70, 9), "B": (9,)}),
    ("ijk,jk->i", {"A": (50, 3, 5), "B": (3, 5)}),
    # mode 1 (warp per output), ragged chunks (1000 = 32 * 31 + 8)
    ("ik,kj->ij", {"A": (33, 1000), "B": (1000, 17)}),
    # mode 2 (CTA per output), four contracted letters
    ("iabcd,abcd->i", {"A": (5, 9, 10, 11, 23), "B": (9, 10, 11, 23)}),
    # a medium contraction: a CTA per output when there are few outputs (15),
    # a warp per output when there are many (1088)
    ("ik,kj->ij", {"A": (3, 3001), "B": (3001, 5)}),
    ("ik,kj->ij", {"A": (34, 2500), "B": (2500, 32)}),
    # three operands, the innermost contracted letter shorter than a chunk
    ("ab,bc,cd->ad", {"A": (7, 300), "B": (300, 9), "C": (9, 6)}),
    # lanes sharing the runs of the innermost letter: a warp over 5 runs of
    # 160; 8 CTA groups of 32 lanes over 12 runs of 300; 2 groups of 128
    # lanes over 2 runs of 1100 (ragged last passes)
    ("ijk,jk->i", {"A": (1100, 5, 160), "B": (5, 160)}),
    ("ijk,jk->i", {"A": (10, 12, 300), "B": (12, 300)}),
    ("ijk,jk->i", {"A": (6, 2, 1100), "B": (2, 1100)}),
    # operands the innermost contracted letter does not move multiply each
    # run's sum once: one (triple product), two (the isomorphism example),
    # none with two operands, and two beside a fully hoisted one
    ("ik,kl,lj->ij", {"A": (9, 40), "B": (40, 70), "C": (70, 11)}),
    ("ijk,ik,ij,ij->i", {"A": (30, 40, 50), "B": (30, 50), "C": (30, 40), "D": (30, 40)}),
    ("ij,ik->i", {"A": (50, 60), "B": (50, 70)}),
    ("il,j,k,i->i", {"A": (25, 33), "B": (7,), "C": (9,), "D": (25,)}),
    # operands no contracted letter moves multiply the sum once (hoisted):
    # one, two, and the third of Fig. 1's operands
    ("ij,j,i->i", {"A": (45, 700), "B": (700,), "C": (45,)}),
    ("ij,i,j,i->i", {"A": (20, 90), "B": (20,), "C": (90,), "D": (20,)}),
    ("mnj,mni,kli->ijkl", {"A": (9, 11, 5), "B": (9, 11, 6), "C": (4, 3, 6)}),
    # four operands, no contracted letter; and an empty contraction
    ("ij,ij,i,j->ij", {"A": (40, 30), "B": (40, 30), "C": (40,), "D": (30,)}),
    ("ik,kj->ij", {"A": (6, 0), "B": (0, 7)}),
])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_generic_running_offsets(text_fmt, shapes, dt):
    """Rows of plain views take the generic evaluator's running-offset path in
    all three modes; results match the oracle (FP32 within its gamma bound)."""
    g = np.random.default_rng(len(text_fmt) + 7)
    names = list(shapes)
    arrs = {n: g.standard_normal(sh).astype(np.float32 if dt == "f32" else np.float64) for n, sh in shapes.items()}
    decl = " ; ".join(f"{n}:{dt}[{','.join(str(d) for d in sh)}]" for n, sh in shapes.items())
    text = f"{text_fmt} | {','.join(names)} ; {decl}"
    got, e = run(text, arrs, cfg=GEN)
    ref, S = ev.evaluate(text, arrs)[0]
    ins, out = text_fmt.split("->")
    lens = {c: d for op, n in zip(ins.split(","), names) for c, d in zip(op, shapes[n])}
    K = int(np.prod([lens[c] for c in lens if c not in out])) if any(c not in out for c in lens) else 1
    u = 2.0 ** -24
    tol = 1e-12 if dt == "f64" else max(K * u / (1 - K * u), 1e-6)    # gamma_K for FP32 accumulation
    assert got[0].shape == ref.shape
    assert np.all(np.abs(got[0] - ref) <= tol * S)


@pytest.mark.parametrize("text_fmt,shapes", [
    # ragged M, N and K (K = 33: slices of 16, 16 and 1)
    ("ik,kj->ij", {"A": (70, 33), "B": (33, 90)}),
    # the first operand holds the output's second letter
    ("kj,ik->ij", {"A": (20, 48), "B": (65, 20)}),
    # several letters per role, K-major and N-major loads
    ("ijcd,cdab->ijab", {"A": (5, 9, 6, 7), "B": (6, 7, 8, 5)}),
    ("ki,kj->ij", {"A": (40, 64), "B": (40, 33)}),
    ("ik,jk->ij", {"A": (100, 24), "B": (37, 24)}),
    # a batch letter in both operands and the output
    ("bik,bkj->bij", {"A": (3, 40, 20), "B": (3, 20, 50)}),
    # a contracted letter only one operand has
    ("ikl,kj->ij", {"A": (33, 9, 4), "B": (9, 40)}),
    # Fig. 1's notation: the third operand, which no contracted letter moves,
    # multiplies each finished sum of the first two
    ("mnj,mni,kli->ijkl", {"A": (9, 11, 40), "B": (9, 11, 36), "C": (2, 3, 36)}),
])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_generic_gemm_tiles(text_fmt, shapes, dt):
    """Two-operand rows with large enough M, N and K run as 64 x 64 GEMM
    tiles staged in shared memory; each output sums its terms in increasing
    k, so the oracle bound is gamma_K (FP32) or 1e-12 (FP64)."""
    g = np.random.default_rng(len(text_fmt) + 11)
    names = list(shapes)
    arrs = {n: g.standard_normal(sh).astype(np.float32 if dt == "f32" else np.float64) for n, sh in shapes.items()}
    decl = " ; ".join(f"{n}:{dt}[{','.join(str(d) for d in sh)}]" for n, sh in shapes.items())
    text = f"{text_fmt} | {','.join(names)} ; {decl}"
    got, e = run(text, arrs, cfg=GEN)
    ref, S = ev.evaluate(text, arrs)[0]
    ins, out = text_fmt.split("->")
    lens = {c: d for op, n in zip(ins.split(","), names) for c, d in zip(op, shapes[n])}
    K = int(np.prod([lens[c] for c in lens if c not in out]))
    assert_close(got[0], ref, S, 1e-12 if dt == "f64" else max(gamma(K), 1e-6))
