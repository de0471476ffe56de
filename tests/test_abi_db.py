"""Tuning database keyed by the normal form (CPU only).

Every isomorphic copy must retrieve the same stored config (the key is the
normal form), different classes never share a record, the file persists
and resumes, and a corrupt file is reported as BE_EDB.
"""
import os

import pytest

import paper_2601_12220_b300 as be
import workloads as W


def fem_copy(g):
    r = W.relabel("ei", ["ij", "ej"], [["D", f"u{k}"] for k in range(4)], g)
    lens = {r.rename["i"]: 4, r.rename["j"]: 4, r.rename["e"]: 4096}
    decl = {}
    for row in r.rows:
        for p, a in enumerate(row):
            decl[a] = ",".join(str(lens[c]) for c in r.ins[p])
    return be.Einsum(f"{','.join(r.ins)}->{r.out} | " + " | ".join(",".join(x) for x in r.rows) + " ; " +
                     " ; ".join(f"{a}:f64[{s}]" for a, s in decl.items()))


def test_record_lookup_transfer(tmp_path):
    db = str(tmp_path / "tune.db")
    ctx = be.Context(db, device_name="test-device", device=-1)
    base = be.Einsum(W.fem_action_spec())
    cb = base.canonicalize()
    assert ctx.lookup(cb) is None
    cfg = be.make_config(be.STRAT_ELEMENT, (128, 256), stages=2, stage_mask=0b10, vec=2)
    ctx.record(cb, cfg, 2e-6)
    ctx.record(cb, be.make_config(be.STRAT_GENERIC), 5e-6)     # slower: must not win
    g = W.rng(1, 5)
    for _ in range(50):
        c = fem_copy(g).canonicalize()
        got, sec = ctx.lookup(c)
        assert got.as_tuple() == cfg.as_tuple() and sec == 2e-6
    # another precision mode and another class do not match
    assert ctx.lookup(cb, be.PREC_SPLIT) is None
    other = be.Einsum("ij,ej->ie | D,u ; D:f64[4,4] ; u:f64[4096,4]").canonicalize()
    assert ctx.lookup(other) is None
    ctx.close()
    # resume from the file
    ctx2 = be.Context(db, device_name="test-device", device=-1)
    assert ctx2.db_size() == 1
    assert ctx2.lookup(cb)[0].as_tuple() == cfg.as_tuple()
    # a different device name is a different key
    ctx3 = be.Context(db, device_name="other", device=-1)
    assert ctx3.lookup(cb) is None


def test_corrupt_db(tmp_path):
    p = tmp_path / "bad.db"
    p.write_text("be1:1;1;a->a;3;A0;float64\tdev\t0\tnot numbers\t1.0\n")
    with pytest.raises(be.BEError) as ex:
        be.Context(str(p), device_name="dev", device=-1)
    assert ex.value.code == be.EDB
    p.write_text("garbage line\n")
    with pytest.raises(be.BEError) as ex:
        be.Context(str(p), device_name="dev", device=-1)
    assert ex.value.code == be.EDB


def test_in_memory_db():
    ctx = be.Context(None, device_name="mem", device=-1)
    c = be.Einsum("ij,j->i | A,B | A,C ; A:f64[96,4] ; B:f64[4] ; C:f64[4]").canonicalize()
    ctx.record(c, be.make_config(be.STRAT_GENERIC, (32,)), 1.0)
    assert ctx.db_size() == 1
    assert ctx.lookup(c)[0].tile[0] == 32


def test_plan_strategy_uses_db(tmp_path):
    ctx = be.Context(None, device_name="dev", device=-1)
    e = be.Einsum(W.dg_gradient_spec(E=1024))
    assert be.plan_strategy(ctx, e) == be.STRAT_ELEMENT
    ctx.record(e.canonicalize(), be.make_config(be.STRAT_GENERIC), 1.0)
    assert be.plan_strategy(ctx, e) == be.STRAT_GENERIC
    # a forced strategy that does not fit is rejected
    mm = be.Einsum("ik,kj->ij | A,B ; A:f64[8,100] ; B:f64[100,100]")
    with pytest.raises(be.BEError) as ex:
        be.plan_strategy(None, mm, be.make_config(be.STRAT_ELEMENT))
    assert ex.value.code == be.EUNSUPPORTED


@pytest.mark.parametrize("order", [1, 4])
def test_plan_strategy_stacked_element_form(order):
    """The DG divergence (select producer over x) and the face mass plan as
    the element strategy's stacked form; letters summed outside the
    operator, or two stacking letters, do not."""
    for text in (W.dg_divergence_spec(E=1000, order=order, rows=3), W.face_mass_spec(E=1000, order=order, rows=2)):
        assert be.plan_strategy(None, be.Einsum(text)) == be.STRAT_ELEMENT
    # y is summed in A and B but also appears nowhere in D: two stacking letters
    two = be.Einsum("xye,ij,xyej->ei | A,D,B ; A:f64[2,2,50] ; D:f64[6,6] ; B:f64[2,2,50,6]")
    assert be.plan_strategy(None, two) == be.STRAT_GENERIC
    # a letter of A alone (summed outside the operator)
    lone = be.Einsum("ze,ij,ej->ei | A,D,B ; A:f64[3,50] ; D:f64[6,6] ; B:f64[50,6]")
    assert be.plan_strategy(None, lone) == be.STRAT_GENERIC


def test_plan_dense_affine_producers():
    """Operands that are affine in one buffer reference plan as the dense
    split strategy; other producers do not."""
    ok = ["P(i,k) := $a*A[i,k]+$b", "P(i,k) := 2.0*A[i,k]-1.0", "P(i,k) := -(A[i,k]/3.0)", "P(i,k) := ($a+1)*A[i,k]"]
    bad = ["P(i,k) := A[i,k]*A[i,k]", "P(i,k) := sin(A[i,k])", "P(i,k) := 1.0/A[i,k]", "P(i,k) := A[i,k]+i"]
    for body in ok + bad:
        e = be.Einsum(f"ik,kj->ij | P,B ; A:f64[64,48] ; B:f64[48,40] ; {body}")
        want = be.STRAT_DENSE_SPLIT if body in ok else be.STRAT_GENERIC
        assert be.plan_strategy(None, e, precision=be.PREC_SPLIT) == want, body


def test_batch_records_load(tmp_path):
    """Records of tuned batches (keys "batch1:<n>:<hash of the instances'
    canonical keys>") are read back from the database file like einsum
    records; other prefixes are refused."""
    p = tmp_path / "b.db"
    p.write_text("batch1:16:00ff00ff00ff00ff\tdev\t0\t0 256 20 4 0 0 0 0 1\t2.5e-03\n"
                 "batch1:16:00ff00ff00ff00ff\tdev\t0\t0 128 18 2 0 0 0 0 1\t3.5e-03\n")
    ctx = be.Context(str(p), device_name="dev", device=-1)
    assert ctx.db_size() == 1
    p.write_text("tune:16:00ff\tdev\t0\t0 256 20 4 0 0 0 0 1\t2.5e-03\n")
    with pytest.raises(be.BEError) as ex:
        be.Context(str(p), device_name="dev", device=-1)
    assert ex.value.code == be.EDB
