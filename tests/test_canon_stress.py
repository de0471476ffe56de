"""Canonicalizer stress: the engine's normal form (be_canonicalize through
the C ABI) against the brute-force oracle on more than 10^4 random tiny
batched einsums, bit for bit in the key text and the token vector.

Besides the general random generator, a high-symmetry generator builds the
inputs where a pruning slip in the search would show: every index of one
length (so arguments can be shared across positions), rows repeated
verbatim or with their arguments permuted, a small argument pool shared by
all rows and positions, and repeated-index patterns (diagonals such as
'pp', transposed pairs such as 'pq,qp').  Each einsum is also presented
under a random renaming, row permutation and operand permutation, which
must give the same key.  A subset is checked against the oracle's full
enumeration of index bijections (no first-appearance shortcut), and the
iff-property (equal keys <=> isomorphic by the definition's direct search)
is checked pairwise on a symmetric corpus.
"""
import itertools

import numpy as np
import pytest

import paper_2601_12220_b300 as be
from oracle import canon as C
from test_abi_canon import spec_of
from test_oracle_canon import random_be, relabel_be


def symmetric_be(g: np.random.Generator) -> C.BE:
    b = int(g.integers(2, 5))
    n = int(g.integers(1, 4))
    nidx = int(g.integers(1, 4))
    letters = "pqrs"[:nidx]
    L = int(g.integers(2, 4))
    pats = []
    for _ in range(n):
        k = int(g.integers(1, 3))
        if k == 2 and g.random() < 0.3:
            c = letters[int(g.integers(nidx))]
            pats.append(c + c)                                   # diagonal
        elif k == 2 and pats and len(pats[-1]) == 2 and g.random() < 0.5:
            pats.append(pats[-1][::-1])                          # transposed pair
        else:
            pats.append("".join(letters[int(g.integers(nidx))] for _ in range(k)))
    used = sorted(set("".join(pats)))
    nout = int(g.integers(0, len(used) + 1))
    out = "".join(g.permutation(used)[:nout])
    pool = [f"S{k}" for k in range(int(g.integers(1, 4)))]
    rows = []
    for i in range(b):
        if rows and g.random() < 0.4:
            rows.append(list(rows[int(g.integers(len(rows)))]))        # verbatim repeat
        elif rows and g.random() < 0.3:
            r = list(rows[int(g.integers(len(rows)))])
            rows.append([r[k] for k in g.permutation(len(r))])         # arguments permuted
        else:
            rows.append([pool[int(g.integers(len(pool)))] if g.random() < 0.7 else f"F{i}_{p}" for p in range(n)])
    shapes, dtypes = {}, {}
    for r in rows:
        for p, a in enumerate(r):
            shapes[a] = (L,) * len(pats[p])
            dtypes.setdefault(a, "float64" if g.random() < 0.85 else "float32")
    return C.make(out, pats, rows, shapes, dtypes)


def _valid(gen, g):
    while True:
        try:
            e = gen(g)
            C.validate(e)
            return e
        except C.CanonError:
            continue


def stress_corpus(seed, n):
    g = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        e = _valid(symmetric_be if g.random() < 0.6 else random_be, g)
        out += [e, relabel_be(e, g)]
    return out[:n]


def test_keys_and_tokens_match_oracle_10k():
    es = stress_corpus(2024, 12000)
    for k in range(0, len(es), 2):
        e, r = es[k], es[k + 1]
        o = C.canonicalize(e, all_index_bijections=False)
        ce = be.Einsum(spec_of(e)).canonicalize()
        cr = be.Einsum(spec_of(r)).canonicalize()
        assert ce.key == o.key, spec_of(e)
        assert ce.tokens == o.tokens, spec_of(e)
        assert cr.key == o.key, (spec_of(e), spec_of(r))


def test_full_index_enumeration_subset():
    for e in stress_corpus(77, 1500):
        o = C.canonicalize(e, all_index_bijections=True)
        assert be.Einsum(spec_of(e)).canonicalize().key == o.key, spec_of(e)


def test_iff_on_symmetric_corpus():
    g = np.random.default_rng(5)
    es = [_valid(symmetric_be, g) for _ in range(150)]
    es += [relabel_be(e, g) for e in es[:75]]
    keys = [be.Einsum(spec_of(e)).canonicalize().key for e in es]
    buckets = {}
    for k, e in enumerate(es):
        buckets.setdefault((e.b, e.n, len(e.out), len(C.index_lengths(e))), []).append(k)
    n_iso = n_non = 0
    for idx in buckets.values():
        for a, b in itertools.combinations(idx, 2):
            iso = C.isomorphic(es[a], es[b]) is not None
            assert iso == (keys[a] == keys[b]), (spec_of(es[a]), spec_of(es[b]))
            n_iso += iso
            n_non += not iso
    assert n_iso >= 75 and n_non > 100
