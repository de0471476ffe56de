"""Persistent multi-instance executor (be_batch_*) on the GPU.

Every output has one owner and a fixed evaluation order, so with factoring
off (stage_mask bit 1) the batch must reproduce BE_STRAT_GENERIC on each
instance alone bit for bit; a sample is also checked against the FP64
oracle with the tolerances of test_gpu_parity.  Factored instances (the
same sum as a sequence of two-operand einsums) are checked against the
oracle and for bitwise-identical replays.
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
NO_FACTOR = be.make_config(stage_mask=2)       # every generic instance on its loop nest


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


def default_alone(ctx, e, bufs):
    dt = torch.float64 if e.out_dtype == be.F64 else torch.float32
    outs = [torch.empty(e.out_shape, dtype=dt, device=DEV) for _ in range(e.b)]
    be.execute(ctx, e, bufs, outs)
    return outs


def test_batch_bitwise_equals_generic_and_oracle():
    """Generic instances match BE_STRAT_GENERIC alone bit for bit; the
    element-shaped FP64 instances of the mix take the element strategy and
    match be_execute's default (the same kernel) bit for bit."""
    items, meta = make_items(40, 7, lo_exp=1.0, hi_exp=5.0, max_operand=1 << 16, max_flops=1 << 22)
    ctx = be.Context(None, device=0)
    b = be.Batch(ctx, items, NO_FACTOR)
    kinds = b.kinds()
    n_el = sum(1 for e, _, _ in items if be.plan_strategy(ctx, e) == be.STRAT_ELEMENT)
    assert kinds["element"] == n_el and kinds["dense"] == 0 and kinds["generic"] == len(items) - n_el
    info = b.info()
    assert info["rows"] == sum(e.b for e, _, _ in items if be.plan_strategy(ctx, e) != be.STRAT_ELEMENT)
    b.run()
    torch.cuda.synchronize()
    for (e, bufs, outs), (inst, text, arrs) in zip(items, meta):
        if be.plan_strategy(ctx, e) == be.STRAT_ELEMENT:
            alone = default_alone(ctx, e, bufs)
        else:
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
    b = be.Batch(None, items, be.make_config(tile=(128, 12, 2), stage_mask=2))
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
        if be.plan_strategy(None, e) == be.STRAT_ELEMENT:
            alone = default_alone(None, e, bufs)
        else:
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
    be.Batch(ctx, items, NO_FACTOR).run()
    torch.cuda.synchronize()
    for e, bufs, outs in items:
        alone = generic_alone(e, bufs)
        torch.cuda.synchronize()
        assert torch.equal(outs[0], alone[0])


def test_mixed_kind_batch():
    """One graph with all three strategies: element-shaped FP64 instances
    (FEM action, DG gradient P4 on the tensor-core element kernel), dense
    FP64 GEMM-form instances on the split-precision tensor-core path
    (cfg.split = 1) and generic instances.  Each result equals be_execute
    with the same strategy alone, bit for bit, and the oracle within the
    strategy's tolerance (1e-12 S; 1e-6 S for the split path; FP32 rows
    max(gamma_K, 1e-6) S)."""
    g = np.random.default_rng(31)
    items, meta, kind = [], [], []

    def add(text, arrs, k):
        e = be.Einsum(text)
        dt = torch.float64 if e.out_dtype == be.F64 else torch.float32
        bufs = {n: torch.from_numpy(v).to(DEV) for n, v in arrs.items()}
        outs = [torch.full(e.out_shape, float("nan"), dtype=dt, device=DEV) for _ in range(e.b)]
        items.append((e, bufs, outs))
        meta.append((text, arrs))
        kind.append(k)

    # element: FEM action b = 4 and the DG gradient P4
    D = g.uniform(-1, 1, (4, 4))
    us = {f"u{k}": g.uniform(-1, 1, (3000, 4)) for k in range(4)}
    add("ij,ej->ei | " + " | ".join(f"D,u{k}" for k in range(4)) + " ; D:f64[4,4] ; " +
        " ; ".join(f"u{k}:f64[3000,4]" for k in range(4)), dict(D=D, **us), "element")
    Dg, G, a, bb = W.dg_gradient(E=2500)
    add(W.dg_gradient_spec(E=2500), dict(D=Dg, G=G, a=a, b=bb), "element")
    # dense: FP64 matmul and the cluster form, above 2^20 multiply-adds
    A, B = g.standard_normal((256, 192)), g.standard_normal((192, 320))
    add("ik,kj->ij | A,B ; A:f64[256,192] ; B:f64[192,320]", dict(A=A, B=B), "dense")
    T, V = g.standard_normal((12, 12, 16, 16)), g.standard_normal((16, 16, 12, 12))
    add("ijcd,cdab->ijab | T,V | T,W ; T:f64[12,12,16,16] ; V:f64[16,16,12,12] ; W:f64[16,16,12,12]",
        dict(T=T, V=V, W=g.standard_normal((16, 16, 12, 12))), "dense")
    # generic: the mix
    gi, gm = make_items(12, 8, lo_exp=1.0, hi_exp=4.0, max_operand=1 << 14, max_flops=1 << 18)
    for it, m in zip(gi, gm):
        e = it[0]
        if be.plan_strategy(None, e) == be.STRAT_ELEMENT:
            continue
        items.append(it)
        meta.append((m[1], m[2]))
        kind.append("generic")
    ctx = be.Context(None, device=0)
    batch = be.Batch(ctx, items, be.make_config(split=1, stage_mask=2))
    k = batch.kinds()
    assert k == {"generic": kind.count("generic"), "element": 2, "dense": 2}
    batch.run()
    torch.cuda.synchronize()
    for (e, bufs, outs), (text, arrs), kd in zip(items, meta, kind):
        if kd == "element":
            alone = default_alone(ctx, e, bufs)
        elif kd == "dense":
            dt = torch.float64
            alone = [torch.empty(e.out_shape, dtype=dt, device=DEV) for _ in range(e.b)]
            be.execute(ctx, e, bufs, alone, precision=be.PREC_SPLIT, cfg=be.make_config(be.STRAT_DENSE_SPLIT))
        else:
            alone = generic_alone(e, bufs)
        torch.cuda.synchronize()
        for o, a_ in zip(outs, alone):
            assert torch.equal(o, a_), (kd, text[:60])
        if kd == "generic":
            continue                      # bitwise the generic strategy, checked against the oracle above
        ref = ev.evaluate(text, arrs)
        tol = 1e-6 if kd == "dense" else 1e-12
        for o, (r, S) in zip(outs, ref):
            assert np.all(np.abs(o.cpu().numpy() - r) <= tol * S), (kd, text[:60])
    assert ctx.status() == be.OK


def test_tune_batch_records_under_batch_key(tmp_path):
    """be_tune_batch times the launch-shape candidates of a batch and records
    them under the batch key; a batch created without a configuration then
    uses the best record -- also when the same instances are listed in
    another order (the key is built from their sorted canonical keys)."""
    items, _ = make_items(16, 12, lo_exp=2.0, hi_exp=6.0, max_operand=1 << 16, max_flops=1 << 22)
    ctx = be.Context(str(tmp_path / "db.txt"), device=0)
    best, sec, n = be.tune_batch(ctx, items, reps=2)
    assert n in (9, 18) and sec > 0
    assert best.tile[0] in (128, 256) and best.tile[1] in (18, 20, 22) and best.tile[2] in (2, 3, 4)
    assert ctx.db_size() == 1
    tuned = be.Batch(ctx, items)
    ref = be.Batch(None, items, best)
    assert tuned.info() == ref.info()
    rev = be.Batch(ctx, list(reversed(items)))
    assert rev.info() == ref.info()
    # resume: a fresh context reading the same file finds the record
    ctx2 = be.Context(str(tmp_path / "db.txt"), device=0)
    assert be.Batch(ctx2, items).info() == ref.info()


FACTOR_SPECS = [
    # (spec without declarations, shapes per buffer, dtype, factored?)
    ("ik,kl,lj->ij | A,B,C | A,D,C", {"A": (40, 50), "B": (50, 60), "C": (60, 30), "D": (50, 60)}, True),
    ("mnj,mni,kli->ijkl | A,B,C", {"A": (9, 11, 7), "B": (9, 11, 6), "C": (5, 4, 6)}, True),
    ("ij,kl,jl->ik | A,B,C", {"A": (30, 40), "B": (20, 50), "C": (40, 50)}, True),
    ("xre,rij,xej->ei | F,D,U", {"F": (3, 3, 200), "D": (3, 20, 20), "U": (3, 200, 20)}, True),
    ("ab,bc,cd,de->ae | P,Q,R,T", {"P": (16, 24), "Q": (24, 32), "R": (32, 20), "T": (20, 12)}, True),
    ("iij,jk,kl->il | A,B,C", {"A": (12, 12, 30), "B": (30, 25), "C": (25, 14)}, True),
    ("ijk,ik,ij,ij->i | A,B,C,D", {"A": (6, 7, 8), "B": (6, 8), "C": (6, 7), "D": (6, 7)}, True),
    ("ij,j->i | A,x", {"A": (30, 40), "x": (40,)}, False),
    ("ij,ik->i | A,B | C,B", {"A": (20, 30), "B": (20, 25), "C": (20, 30)}, True),
    ("ijl,jk,kl->il | A,B,C", {"A": (10, 12, 9), "B": (12, 14), "C": (14, 9)}, True),
]


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_factored_instances_match_the_oracle(dt):
    """Instances whose best pairwise order cuts the loop nest's multiply-adds
    at least 1.5 times run as two-operand steps over intermediates, in phases
    (the 4-operand chain is 3 steps deep), waiting in one launch for the
    steps they read: every output within the
    precision's tolerance of the FP64 oracle (1e-12 S; FP32 max(gamma_K,
    1e-6) S), replays bitwise identical, and the same batch with factoring
    off still equals the generic strategy alone bit for bit."""
    g = np.random.default_rng(41)
    tdt = torch.float64 if dt == "f64" else torch.float32
    items, meta = [], []
    for spec, shapes, _ in FACTOR_SPECS:
        decl = " ; ".join(f"{k}:{dt}[{','.join(map(str, v))}]" for k, v in shapes.items())
        text = f"{spec} ; {decl}"
        arrs = {k: g.standard_normal(v).astype(np.float32 if dt == "f32" else np.float64) for k, v in shapes.items()}
        e = be.Einsum(text)
        bufs = {k: torch.from_numpy(v).to(DEV) for k, v in arrs.items()}
        outs = [torch.full(e.out_shape, float("nan"), dtype=tdt, device=DEV) for _ in range(e.b)]
        items.append((e, bufs, outs))
        meta.append((text, arrs))
    b = be.Batch(None, items)
    f = b.factored()
    # the divergence form is element-shaped in FP64 and takes that strategy
    assert f["instances"] == sum(1 for s, (e, _, _) in zip(FACTOR_SPECS, items)
                                 if s[2] and be.plan_strategy(None, e) != be.STRAT_ELEMENT)
    assert f["phases"] >= 3 and f["workspace_bytes"] > 0
    b.run()
    torch.cuda.synchronize()
    first = [[o.clone() for o in outs] for _, _, outs in items]
    b.run()
    torch.cuda.synchronize()
    for (e, bufs, outs), fst, (text, arrs) in zip(items, first, meta):
        for o, a in zip(outs, fst):
            assert torch.equal(o, a)
        ref = ev.evaluate(text, arrs)
        tol = 1e-12
        if dt == "f32":
            # gamma_K of the whole contraction: K = contracted terms + operands
            notation, row0 = text.split("|")[0], text.split("|")[1].split(";")[0]
            lhs, out = notation.strip().split("->")
            lens = {}
            for letters, name in zip(lhs.split(","), row0.strip().split(",")):
                lens.update(zip(letters, arrs[name.strip()].shape))
            K = math.prod(v for c, v in lens.items() if c not in out) + len(lhs.split(","))
            tol = max(K * 2.0 ** -24 / (1 - K * 2.0 ** -24), 1e-6)
        for k, (r, S) in enumerate(ref):
            got = outs[k].cpu().numpy().astype(np.float64)
            assert np.all(np.abs(got - r) <= tol * S), text[:40]
    off = be.Batch(None, items, NO_FACTOR)
    assert off.factored()["instances"] == 0 and off.factored()["phases"] == 1
    off.run()
    torch.cuda.synchronize()
    for e, bufs, outs in items:
        if be.plan_strategy(None, e) == be.STRAT_ELEMENT:
            alone = default_alone(None, e, bufs)
        else:
            alone = generic_alone(e, bufs)
        torch.cuda.synchronize()
        for o, a in zip(outs, alone):
            assert torch.equal(o, a)


DENSE_FACTOR_SPECS = [
    # (spec without declarations, shapes per buffer); sizes make the first
    # pairwise order unique and its GEMM step at least 2^23 multiply-adds
    # face mass with 128 output dofs (beyond the element strategy's
    # operators): the operator's contracted letters (f, j) are contiguous
    ("fe,ifj,fej->ei | J,M,U | K,M,V", {"J": (4, 1024), "M": (128, 4, 32), "U": (4, 1024, 32),
                                         "K": (4, 1024), "V": (4, 1024, 32)}),
    # DG gradient with 96 output dofs: D[r, i, j] puts i between the
    # contracted r and j, so D is first copied into an (i, r, j) layout
    ("rij,er,ej->ei | D,G,U", {"D": (3, 96, 48), "G": (2048, 3), "U": (2048, 48)}),
    # triple product: the first step's result is the GEMM's A operand
    ("ik,kl,lj->ij | A,B,C", {"A": (128, 64), "B": (64, 64), "C": (64, 1024)}),
]


def test_dense_routed_factored_instances():
    """With split >= 2, factored FP64 instances of two steps whose last step
    is a GEMM of at least 2^23 multiply-adds run on a dense branch: the first
    step (and a permuted copy of the operator where its layout does not
    flatten) as generic launches, the GEMM in split precision.  Every output
    within 1e-6 S of the FP64 oracle, replays bitwise identical; with split
    off the same instances are factored in the persistent launch and meet
    1e-12 S."""
    g = np.random.default_rng(43)
    items, meta = [], []
    for spec, shapes in DENSE_FACTOR_SPECS:
        decl = " ; ".join(f"{k}:f64[{','.join(map(str, v))}]" for k, v in shapes.items())
        text = f"{spec} ; {decl}"
        arrs = {k: g.standard_normal(v) for k, v in shapes.items()}
        e = be.Einsum(text)
        bufs = {k: torch.from_numpy(v).to(DEV) for k, v in arrs.items()}
        outs = [torch.full(e.out_shape, float("nan"), dtype=torch.float64, device=DEV) for _ in range(e.b)]
        items.append((e, bufs, outs))
        meta.append((text, arrs))
    refs = [ev.evaluate(text, arrs) for text, arrs in meta]
    ctx = be.Context(None, device=0)
    b = be.Batch(ctx, items, be.make_config(split=2))
    assert [b.instance_kind(k) for k in range(len(items))] == ["dense factored"] * len(items)
    one = be.Batch(ctx, items, be.make_config(split=1))       # the route is off at split = 1
    assert [one.instance_kind(k) for k in range(len(items))] == ["factored"] * len(items)
    one.close()
    assert b.kinds()["dense"] == len(items) and b.factored()["instances"] == 0
    b.run()
    torch.cuda.synchronize()
    first = [[o.clone() for o in outs] for _, _, outs in items]
    b.run()
    torch.cuda.synchronize()
    assert ctx.status() == be.OK
    for (e, _, outs), fst, ref, (text, _) in zip(items, first, refs, meta):
        for k, (r, S) in enumerate(ref):
            assert torch.equal(outs[k], fst[k])
            got = outs[k].cpu().numpy()
            assert np.all(np.abs(got - r) <= 1e-6 * S), text[:30]
    off = be.Batch(ctx, items, be.make_config(split=0))
    assert [off.instance_kind(k) for k in range(len(items))] == ["factored"] * len(items)
    off.run()
    torch.cuda.synchronize()
    for (e, _, outs), ref, (text, _) in zip(items, refs, meta):
        for k, (r, S) in enumerate(ref):
            assert np.all(np.abs(outs[k].cpu().numpy() - r) <= 1e-12 * S), text[:30]
    with pytest.raises(be.BEError):
        b.instance_kind(len(items))
