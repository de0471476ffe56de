"""Pins of the brute-force canonicalizer and isomorphism judge (CPU only).

The oracle's C_lex and its direct isomorphism search are pinned against the
paper's worked examples and against each other on random tiny corpora (the
iff-property of a canonicalization function), plus idempotence and the
reconstruction of e from C(e) and the sigma maps.
"""
import itertools

import numpy as np
import pytest

from oracle import canon as C
import workloads as W


def _be(d, length=None):
    lhs, out = d["notation"].split("->")
    ins = lhs.split(",")
    if "shapes" in d:
        shapes = d["shapes"]
    else:
        shapes = {}
        for r in d["rows"]:
            for p, a in enumerate(r):
                shapes[a] = [length or d.get("length") or d.get("n")] * len(ins[p])
    return C.make(out, ins, d["rows"], shapes, d.get("dtype", "float64"))


# ---------------------------------------------------------------- golden


def test_paper_canonical_example(golden):
    g = golden("canonical_example.json")
    e1, e2 = (_be(d) for d in g["einsums"])
    c1, c2 = C.canonicalize(e1), C.canonicalize(e2)
    assert c1.key == g["key"] and c2.key == g["key"]
    want = _be(g["canonical"])
    assert c1.form == want and c2.form == want


def test_paper_isomorphic_einsums(golden):
    g = golden("isomorphic_einsums.json")
    e1, e2 = _be(g["e1"]), _be(g["e2"])
    w = C.isomorphic(e1, e2)
    assert w is not None
    # the paper's maps are a valid witness: check them against the definition
    sj = [x - 1 for x in g["sigma_j"]]
    sI, sA = g["sigma_I"], g["sigma_A"]
    for j in range(e1.n):
        assert list(e1.ins[j]) == [sI[c] for c in e2.ins[sj[j]]]
        assert sA[e2.rows[0][sj[j]]] == e1.rows[0][j]
    assert C.canonicalize(e1).key == C.canonicalize(e2).key


def test_paper_isomorphic_batched(golden):
    g = golden("isomorphic_batched.json")
    e1, e2 = _be(g["e1"]), _be(g["e2"])
    si = [x - 1 for x in g["sigma_i"]]
    sj = [x - 1 for x in g["sigma_j"]]
    sI, sA = g["sigma_I"], g["sigma_A"]
    for j in range(e1.n):
        assert list(e1.ins[j]) == [sI[c] for c in e2.ins[sj[j]]]
    for i in range(e1.b):
        for j in range(e1.n):
            assert sA[e2.rows[si[i]][sj[j]]] == e1.rows[i][j]
    assert C.isomorphic(e1, e2) is not None
    assert C.canonicalize(e1).key == C.canonicalize(e2).key


def test_paper_fig1(golden):
    g = golden("fig1.json")
    e1, e2 = _be(g["e1"]), _be(g["e2"])
    # the figure's substitution maps e1's symbols to e2's; check it directly
    ren, args = g["index_e1_to_e2"], g["args_e1_to_e2"]
    assert "".join(ren[c] for c in e1.out) == "".join(e2.out)
    opmap = [x - 1 for x in g["operands_e1_to_e2"]]
    rowmap = [x - 1 for x in g["rows_e1_to_e2"]]
    for j in range(e1.n):
        assert "".join(ren[c] for c in e1.ins[j]) == "".join(e2.ins[opmap[j]])
    for i in range(e1.b):
        for j in range(e1.n):
            assert args[e1.rows[i][j]] == e2.rows[rowmap[i]][opmap[j]]
    assert C.isomorphic(e1, e2) is not None
    assert C.canonicalize(e1).key == C.canonicalize(e2).key


def test_paper_examples_non_isomorphic():
    mm = C.make("ij", ["ik", "kj"], [["A", "B"]], {"A": (10, 4), "B": (4, 10)}, "float64")
    mt = C.make("ij", ["ik", "jk"], [["A", "B"]], {"A": (10, 4), "B": (10, 4)}, "float64")
    assert C.isomorphic(mm, mt) is None
    assert C.canonicalize(mm).key != C.canonicalize(mt).key
    # sharing pattern matters: [[A,B],[A,C]] vs [[A,B],[C,D]]
    sh = C.make("i", ["ij", "j"], [["A", "B"], ["A", "C"]], {"A": (96, 4), "B": (4,), "C": (4,)}, "float64")
    ns = C.make("i", ["ij", "j"], [["A", "B"], ["D", "C"]], {"A": (96, 4), "B": (4,), "C": (4,), "D": (96, 4)}, "float64")
    assert C.isomorphic(sh, ns) is None
    assert C.canonicalize(sh).key != C.canonicalize(ns).key
    # dtype matters
    f32 = C.make("i", ["ij", "j"], [["A", "B"]], {"A": (96, 4), "B": (4,)}, {"A": "float32", "B": "float64"})
    f64 = C.make("i", ["ij", "j"], [["A", "B"]], {"A": (96, 4), "B": (4,)}, "float64")
    assert C.canonicalize(f32).key != C.canonicalize(f64).key


# ------------------------------------------------------- random corpora


def random_be(g: np.random.Generator):
    b = int(g.integers(1, 4))
    n = int(g.integers(1, 4))
    nidx = int(g.integers(1, 5))
    letters = "pqrstuvw"[:nidx]
    lens = {c: int(g.integers(2, 4)) for c in letters}
    ins = []
    for _ in range(n):
        k = int(g.integers(1, 4))
        ins.append("".join(letters[int(g.integers(nidx))] for _ in range(k)))
    used = sorted(set("".join(ins)))
    nout = int(g.integers(0, len(used) + 1))
    out = "".join(g.permutation(used)[:nout])
    rows, shapes, dtypes, pool = [], {}, {}, []
    for _ in range(b):
        row = []
        for p in range(n):
            shp = tuple(lens[c] for c in ins[p])
            cands = [a for a in pool if shapes[a] == shp]
            if cands and g.random() < 0.4:
                a = cands[int(g.integers(len(cands)))]
            else:
                a = f"X{len(pool)}"
                pool.append(a)
                shapes[a] = shp
                dtypes[a] = "float64" if g.random() < 0.7 else "float32"
            row.append(a)
        rows.append(row)
    return C.make(out, ins, rows, shapes, dtypes)


def relabel_be(e, g):
    r = W.relabel("".join(e.out), ["".join(s) for s in e.ins], [list(x) for x in e.rows], g)
    perm = {a: f"Y{k}" for k, a in enumerate(g.permutation(sorted({a for x in e.rows for a in x})))}
    rows = [[perm[a] for a in row] for row in r.rows]
    return C.make(r.out, r.ins, rows, {perm[a]: s for a, s in e.shapes}, {perm[a]: d for a, d in e.dtypes})


def mutate_be(e, g):
    """A small random edit that may or may not change the class."""
    kind = int(g.integers(3))
    rows = [list(r) for r in e.rows]
    dtypes = dict(e.dtypes)
    shapes = dict(e.shapes)
    if kind == 0:
        a = sorted(dtypes)[int(g.integers(len(dtypes)))]
        dtypes[a] = "float32" if dtypes[a] == "float64" else "float64"
    elif kind == 1 and e.b > 1:
        # replace one occurrence by a fresh argument of the same shape
        i, j = int(g.integers(e.b)), int(g.integers(e.n))
        shapes["Z"] = shapes[rows[i][j]]
        dtypes["Z"] = dtypes[rows[i][j]]
        rows[i][j] = "Z"
    else:
        ins = ["".join(s) for s in e.ins]
        j = int(g.integers(e.n))
        ins[j] = ins[j][::-1]
        shapes = {}
        lens = C.index_lengths(e)
        for r in rows:
            for p, a in enumerate(r):
                shapes[a] = tuple(lens[c] for c in ins[p])
        try:
            return C.make(e.out, ins, rows, shapes, dtypes)
        except C.CanonError:
            return e
    try:
        return C.make(e.out, e.ins, rows, shapes, dtypes)
    except C.CanonError:
        return e


def corpus(seed, n_base):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(n_base):
        e = random_be(g)
        out += [e, relabel_be(e, g), mutate_be(e, g), relabel_be(mutate_be(e, g), g)]
    return out


def test_iff_key_equality_vs_isomorphism():
    es = corpus(7, 40)
    keys = [C.canonicalize(e).key for e in es]
    buckets = {}
    for k, e in enumerate(es):
        buckets.setdefault((e.b, e.n, len(e.out), len(C.index_lengths(e))), []).append(k)
    n_iso = n_non = 0
    for idx in buckets.values():
        for a, b in itertools.combinations(idx, 2):
            iso = C.isomorphic(es[a], es[b]) is not None
            assert iso == (keys[a] == keys[b]), (es[a], es[b])
            n_iso += iso
            n_non += not iso
    assert n_iso > 30 and n_non > 30


def test_first_appearance_equals_full_enumeration():
    for e in corpus(11, 15):
        assert C.canonicalize(e, True).tokens == C.canonicalize(e, False).tokens


def test_idempotence_and_reconstruction():
    for e in corpus(3, 20):
        c = C.canonicalize(e)
        assert C.canonicalize(c.form).form == c.form            # C(C(e)) = C(e)
        assert C.apply_sigma(c) == e                            # sigma maps C(e) back to e


def test_fem_200_copies_one_key():
    """Workload 1: 200 copies under random renames, row permutations and
    operand swaps all give one normal form."""
    ins, out = ["ij", "ej"], "ei"
    rows = [["D", f"u{k}"] for k in range(4)]
    shapes = {"D": (4, 4), **{f"u{k}": (4096, 4) for k in range(4)}}
    base = C.make(out, ins, rows, shapes, "float64")
    key = C.canonicalize(base).key
    g = W.rng(1, 99)
    for _ in range(200):
        r = W.relabel(out, ins, rows, g)
        e = C.make(r.out, r.ins, r.rows, shapes, "float64")
        assert C.canonicalize(e, all_index_bijections=False).key == key
    assert key == "be1:4;2;ab->ac,bc;4096,4,4;A0,A1/A2,A1/A3,A1/A4,A1;float64,float64,float64,float64,float64"


def test_planted_mistake_is_caught(monkeypatch):
    """Dropping the length part of T (a plausible slip) must make the iff
    test fail on the corpus: the pins are sensitive to it."""
    orig = C._tokens

    def no_lengths(e, lens, row_perm, op_perm, idx_id):
        T, order = orig(e, lens, row_perm, op_perm, idx_id)
        k = 3 + len(e.out) + sum(1 + len(e.ins[p]) for p in op_perm)
        return T[:k] + T[k + len(lens):], order
    monkeypatch.setattr(C, "_tokens", no_lengths)
    e1 = C.make("i", ["ij"], [["A"]], {"A": (3, 2)}, "float64")
    e2 = C.make("i", ["ij"], [["A"]], {"A": (3, 3)}, "float64")
    assert C.isomorphic(e1, e2) is None
    assert C.canonicalize(e1).key.split(";")[0:3] == C.canonicalize(e2).key.split(";")[0:3]
    assert C.canonicalize(e1).tokens == C.canonicalize(e2).tokens      # mistake collapses classes


def test_26_indices():
    letters = "abcdefghijklmnopqrstuvwxyz"
    e = C.make("", [letters], [["A"]], {"A": (1,) * 26}, "float64")
    assert C.canonicalize(e, all_index_bijections=False).key.startswith("be1:1;1;->abcdefghijklmnopqrstuvwxyz;")
