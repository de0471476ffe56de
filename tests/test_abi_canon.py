"""Canonicalization through the C ABI vs the brute-force oracle (CPU only).

Normal forms and token vectors must match the oracle bit for bit; the
induced graph must satisfy the compliance conditions of Appendix B.2 and
have the node count of the Eq. for N^IDG.
"""
import itertools

import numpy as np
import pytest

import paper_2601_12220_b300 as be
from oracle import canon as C
import workloads as W
from test_oracle_canon import corpus, _be

SHORT = {"float64": "f64", "float32": "f32", "float16": "f16", "bfloat16": "bf16", "int32": "i32",
         "int64": "i64", "int8": "i8"}


def spec_of(e: C.BE) -> str:
    args = []
    for r in e.rows:
        for a in r:
            if a not in args:
                args.append(a)
    rows = " | ".join(",".join(r) for r in e.rows)
    decls = " ; ".join(f"{a}:{SHORT[e.dtype(a)]}[{','.join(map(str, e.shape(a)))}]" for a in args)
    return f"{','.join(''.join(s) for s in e.ins)}->{''.join(e.out)} | {rows} ; {decls}"


def test_exports_every_declared_symbol():
    import re
    import os
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "be.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char \*)\s*\**\s*(be_\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations found"
    L = be.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(be.binding.EXPORTS)


def test_golden_canonical_example(golden):
    g = golden("canonical_example.json")
    for d in g["einsums"]:
        e = be.Einsum(spec_of(_be(d)))
        assert e.canonicalize().key == g["key"]


@pytest.mark.parametrize("name", ["isomorphic_einsums.json", "isomorphic_batched.json", "fig1.json"])
def test_golden_isomorphic_pairs(golden, name):
    g = golden(name)
    e1, e2 = _be(g["e1"]), _be(g["e2"])
    k1 = be.Einsum(spec_of(e1)).canonicalize().key
    k2 = be.Einsum(spec_of(e2)).canonicalize().key
    assert k1 == k2 == C.canonicalize(e1).key


def test_keys_and_tokens_match_oracle_on_corpus():
    es = corpus(21, 60)
    for e in es:
        c = be.Einsum(spec_of(e)).canonicalize()
        o = C.canonicalize(e, all_index_bijections=False)
        assert c.key == o.key, spec_of(e)
        assert c.tokens == o.tokens


def test_iff_on_corpus():
    es = corpus(23, 30)
    keys = [be.Einsum(spec_of(e)).canonicalize().key for e in es]
    for a, b in itertools.combinations(range(len(es)), 2):
        if (es[a].b, es[a].n) != (es[b].b, es[b].n):
            assert keys[a] != keys[b]
            continue
        assert (keys[a] == keys[b]) == (C.isomorphic(es[a], es[b]) is not None)


def test_idempotence_and_sigma_reconstruct():
    for e in corpus(25, 25):
        ee = be.Einsum(spec_of(e))
        c = ee.canonicalize()
        # C(C(e)) = C(e): re-parse the printed form
        o = C.canonicalize(e, all_index_bijections=False)
        ce = be.Einsum(spec_of(o.form)).canonicalize()
        assert ce.key == c.key
        # sigma maps: canonical symbols -> user symbols rebuild e exactly
        f = o.form
        sI = {chr(ord("a") + k): c.sigma(be.SIGMA_INDEX, k) for k in range(len(C.index_lengths(f)))}
        nargs = len({a for r in f.rows for a in r})
        sA = {f"A{k}": c.sigma(be.SIGMA_ARG, k) for k in range(nargs)}
        si = [int(c.sigma(be.SIGMA_ROW, q)) for q in range(f.b)]
        sj = [int(c.sigma(be.SIGMA_POS, p)) for p in range(f.n)]
        rebuilt = C.apply_sigma(C.Canon(c.key, f, sI, sA, si, sj, c.tokens))
        assert rebuilt == e


def test_fem_200_copies():
    ins, out = ["ij", "ej"], "ei"
    rows = [["D", f"u{k}"] for k in range(4)]
    g = W.rng(1, 77)
    keys = set()
    for _ in range(200):
        r = W.relabel(out, ins, rows, g)
        lens = {r.rename["i"]: 4, r.rename["j"]: 4, r.rename["e"]: 4096}
        decl = {}
        for row in r.rows:
            for p, a in enumerate(row):
                decl[a] = ",".join(str(lens[c]) for c in r.ins[p])
        text = f"{','.join(r.ins)}->{r.out} | " + " | ".join(",".join(x) for x in r.rows) + " ; " + \
            " ; ".join(f"{a}:f64[{s}]" for a, s in decl.items())
        keys.add(be.Einsum(text).canonicalize().key)
    assert keys == {"be1:4;2;ab->ac,bc;4096,4,4;A0,A1/A2,A1/A3,A1/A4,A1;float64,float64,float64,float64,float64"}


def test_functional_and_idealized_share_a_form():
    """The DG gradient with u = sin(a)*b and G slices has the same normal form
    as its idealized version (every lambda a plain row-major buffer)."""
    E = 1000
    f = be.Einsum(W.dg_gradient_spec(E=E))
    ideal = be.Einsum(f"rij,er,ej->ei | D,G0,U | D,G1,U | D,G2,U ; D:f64[3,35,35] ; G0:f64[{E},3] ; "
                      f"G1:f64[{E},3] ; G2:f64[{E},3] ; U:f64[{E},35]")
    assert f.canonicalize().key == ideal.canonicalize().key


def test_identify_alg2(golden):
    g = golden("isomorphic_batched.json")
    e1, e2 = (be.Einsum(spec_of(_be(g[k]))) for k in ("e1", "e2"))
    m = be.identify(e1, e2)
    # every symbol of e1 is mapped; applying the map to e1 yields an einsum with e2's normal form
    assert set(m) == {"i", "j", "k", "A", "B", "C", "D"}
    assert m["A"] == "P" and m["i"] == "i"
    other = be.Einsum("ij,jk->ik | A,B ; A:f64[5,5] ; B:f64[5,5]")
    with pytest.raises(be.BEError) as ex:
        be.identify(e1, other)
    assert ex.value.code == be.EINVALID


def test_graph_node_counts_and_compliance(golden):
    g = golden("einsum_examples.json")
    e = be.Einsum("ik,ij->i | A,B ; A:f64[72,18] ; B:f64[72,18]")
    cols, eds = e.induced_graph()
    assert len(cols) == g["induced_graph"]["nodes"] == 18
    assert be.graph_check(cols, eds) == 0
    f = be.Einsum(W.fem_action_spec())
    assert len(f.induced_graph()[0]) == g["fem_config_graph"]["nodes"] == 37
    for ee in corpus(31, 20):
        cols, eds = be.Einsum(spec_of(ee)).induced_graph()
        assert be.graph_check(cols, eds) == 0


def test_graph_check_detects_violations():
    e = be.Einsum("ik,ij->i | A,B ; A:f64[72,18] ; B:f64[72,18]")
    cols, eds = e.induced_graph()
    # C2: an argument node with a successor
    bad = np.vstack([eds, [[0, 1]]])
    assert be.graph_check(cols, bad) == 2
    # C1: a colour outside 1..9
    c2 = cols.copy()
    c2[0] = 12
    assert be.graph_check(c2, eds) == 1
    # C8: drop one predecessor of an input access node
    acc = int(np.where(cols == 3)[0][0])
    drop = [k for k, (a, b) in enumerate(eds) if b == acc and cols[a] == 6][0]
    assert be.graph_check(cols, np.delete(eds, drop, axis=0)) == 8
    # C21: break the dim tournament
    dims = np.where(cols == 9)[0]
    k = [i for i, (a, b) in enumerate(eds) if a == dims[0] and b == dims[1]][0]
    assert be.graph_check(cols, np.delete(eds, k, axis=0)) in (18, 21)


@pytest.mark.parametrize("text,code", [
    ("ij,jk", be.EPARSE),
    ("ij,jk->ik | A ; A:f64[2,2]", be.EINVALID),
    ("ij,jk->iz | A,B ; A:f64[2,2] ; B:f64[2,2]", be.EINVALID),
    ("ij,jk->ii | A,B ; A:f64[2,2] ; B:f64[2,2]", be.EINVALID),
    ("ij,jk->ik | A,B ; A:f64[2,3] ; B:f64[2,2]", be.ESHAPE),
    ("ij,jk->ik | A,B ; A:f64[2,2] ; B:f64[2]", be.EINVALID),
    ("ij,jk->ik | A,B ; A:q64[2,2] ; B:f64[2,2]", be.EDTYPE),
    ("ij,jk->ik | A,C ; A:f64[2,2] ; B:f64[2,2]", be.EINVALID),
    (",ij->ij | s,A ; s:f64[] ; A:f64[2,2]", be.EUNSUPPORTED),
    ("->", be.EINVALID),
    ("ij->i | U ; a:f64[3,4] ; U(i,j) := sin(a[i,j]) *", be.EPARSE),
])
def test_parse_errors(text, code):
    with pytest.raises(be.BEError) as ex:
        be.Einsum(text)
    assert ex.value.code == code


def test_canonicalize_latency_sub_ms():
    import time
    e = be.Einsum(W.dg_gradient_spec())
    t = time.perf_counter()
    for _ in range(200):
        e.canonicalize()
    dt = (time.perf_counter() - t) / 200
    assert dt < 1e-3, dt
