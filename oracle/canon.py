"""Brute-force canonical form and isomorphism judge -- test infrastructure only.

Definitions followed
  * Batched einsum (b, n, I_out, (I_in,j), ((A^{i,j}))) -- Sec. "Batched
    Einstein Summation", Def. of a batched einsum.
  * Batched-einsum isomorphism via sigma^i, sigma^j, sigma^I, sigma^A --
    Sec. "Isomorphic Batched Einstein Summations", Def. of batched einsum
    isomorphism.  Reading taken for the per-row argument condition: for all
    rows i and positions j, sigma^A(A'^{sigma^i(i), sigma^j(j)}) = A^{i,j}
    with sigma^A a bijection A^all(e2) -> A^all(e1) that preserves shape and
    dtype (this is the reading under which the paper's worked example of
    isomorphic batched einsums checks out).
  * Canonicalization function C with e ~ e' <=> C(e) = C(e') -- Sec. "A
    Canonical form for Batched Einsums", Def. of a canonicalization
    function.  The paper's own C depends on the graph canonizer it calls, so
    the exact normal form is fixed here as C_lex:

      T(e) = [b, n, |I_out|, ids(I_out), |I_in,1|, ids(I_in,1), ...,
              |I_in,n|, ids(I_in,n), len(id 0..N_index-1),
              arg(1,1..n), ..., arg(b,1..n), DtypeRank(arg 0..N_arg-1)]

    and C_lex(e) is the relabeling with lexicographically smallest T over
    all row permutations sigma^i, operand permutations sigma^j and index
    bijections sigma^I; arguments are numbered by first appearance in
    row-major order.  Index name k is the k-th letter, argument name k is
    "A<k>" (the naming of the paper's canonical-form example).
    DtypeRank is the table of the induced-graph appendix (int8 1 ... complex128
    8); bfloat16, absent from the paper, is given rank 9.

The brute force here enumerates every sigma^i, sigma^j and (optionally) every
index bijection sigma^I, so it does not rely on the fact that
first-appearance index numbering minimizes the index part.

Parity: pinned by the paper's worked examples (tests/golden/), by
idempotence, by the iff-property against the direct isomorphism search on
random tiny corpora, and by reconstruction of e from C(e) and sigma.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

DTYPE_RANK = {"int8": 1, "int32": 2, "int64": 3, "float16": 4, "float32": 5,
              "float64": 6, "complex64": 7, "complex128": 8, "bfloat16": 9}
LETTERS = "abcdefghijklmnopqrstuvwxyz"


class CanonError(ValueError):
    pass


@dataclass(frozen=True)
class BE:
    """A batched einsum with concrete argument shapes and dtypes."""
    out: tuple
    ins: tuple
    rows: tuple
    shapes: tuple      # sorted ((arg, shape), ...)
    dtypes: tuple      # sorted ((arg, dtype), ...)

    @property
    def b(self):
        return len(self.rows)

    @property
    def n(self):
        return len(self.ins)

    def shape(self, a):
        return dict(self.shapes)[a]

    def dtype(self, a):
        return dict(self.dtypes)[a]


def make(out, ins, rows, shapes, dtypes) -> BE:
    """Build and validate a batched einsum (soundness rules of Sec.
    "Preliminaries" for every row)."""
    out = tuple(out)
    ins = tuple(tuple(s) for s in ins)
    rows = tuple(tuple(r) for r in rows)
    args = {a for r in rows for a in r}
    shapes = {a: tuple(shapes[a]) for a in args}
    if isinstance(dtypes, str):
        dtypes = {a: dtypes for a in args}
    dtypes = {a: dtypes[a] for a in args}
    e = BE(out, ins, rows, tuple(sorted(shapes.items())), tuple(sorted(dtypes.items())))
    validate(e)
    return e


def validate(e: BE):
    if e.n == 0:
        raise CanonError("n = 0")
    if e.b == 0:
        raise CanonError("b = 0")
    if len(set(e.out)) != len(e.out):
        raise CanonError("repeated output index")
    all_idx = set().union(*[set(s) for s in e.ins])
    if len(all_idx) > 26:
        raise CanonError("more than 26 indices")
    if not set(e.out) <= all_idx:
        raise CanonError("output index not in any input")
    lens = {}
    for r in e.rows:
        if len(r) != e.n:
            raise CanonError("row arity")
        for j, a in enumerate(r):
            shp = e.shape(a)
            if len(shp) != len(e.ins[j]):
                raise CanonError(f"Dim({a}) != |I_in,{j}|")
            for c, L in zip(e.ins[j], shp):
                if lens.setdefault(c, L) != L:
                    raise CanonError(f"length of {c} inconsistent")
    return lens


def index_lengths(e: BE) -> dict:
    return validate(e)


def _tokens(e, lens, row_perm, op_perm, idx_id):
    """T of the einsum obtained by taking rows in ``row_perm`` order, operands
    in ``op_perm`` order and numbering indices by ``idx_id``; arguments are
    numbered by first appearance.  Returns (T, arg_order)."""
    T = [e.b, e.n, len(e.out)] + [idx_id[c] for c in e.out]
    for p in op_perm:
        T.append(len(e.ins[p]))
        T.extend(idx_id[c] for c in e.ins[p])
    by_id = sorted(idx_id, key=idx_id.get)
    T.extend(lens[c] for c in by_id)
    names = {}
    for q in row_perm:
        for p in op_perm:
            a = e.rows[q][p]
            if a not in names:
                names[a] = len(names)
            T.append(names[a])
    order = sorted(names, key=names.get)
    T.extend(DTYPE_RANK[e.dtype(a)] for a in order)
    return T, order


def _first_appearance(e, op_perm):
    ids = {}
    for c in list(e.out) + [c for p in op_perm for c in e.ins[p]]:
        if c not in ids:
            ids[c] = len(ids)
    return ids


@dataclass
class Canon:
    key: str
    form: BE            # the canonical batched einsum (letters a.., args A0..)
    sigma_I: dict       # canonical letter -> user letter
    sigma_A: dict       # canonical arg name -> user arg name
    sigma_i: list       # canonical row q -> user row
    sigma_j: list       # canonical position p -> user position
    tokens: list


def canonicalize(e: BE, all_index_bijections: bool = True) -> Canon:
    """C_lex(e) by exhaustive search over S_b x S_n (x S_{N_index})."""
    lens = index_lengths(e)
    letters = sorted(lens)
    best = None
    for op_perm in itertools.permutations(range(e.n)):
        if all_index_bijections:
            cands = (dict(zip(letters, perm)) for perm in itertools.permutations(range(len(letters))))
        else:
            cands = [_first_appearance(e, op_perm)]
        for idx_id in cands:
            for row_perm in itertools.permutations(range(e.b)):
                T, order = _tokens(e, lens, row_perm, op_perm, idx_id)
                if best is None or T < best[0]:
                    best = (T, order, row_perm, op_perm, dict(idx_id))
    T, order, row_perm, op_perm, idx_id = best
    inv_idx = {v: k for k, v in idx_id.items()}
    sigma_I = {LETTERS[k]: inv_idx[k] for k in range(len(letters))}
    arg_name = {a: f"A{k}" for k, a in enumerate(order)}
    sigma_A = {v: k for k, v in arg_name.items()}
    to_canon = {u: c for c, u in sigma_I.items()}
    form = make(
        [to_canon[c] for c in e.out],
        [[to_canon[c] for c in e.ins[p]] for p in op_perm],
        [[arg_name[e.rows[q][p]] for p in op_perm] for q in row_perm],
        {arg_name[a]: e.shape(a) for a in order},
        {arg_name[a]: e.dtype(a) for a in order},
    )
    return Canon(key_text(form), form, sigma_I, sigma_A, list(row_perm), list(op_perm), T)


def key_text(f: BE) -> str:
    """Printed normal form:
    be1:<b>;<n>;<out>-><in1>,...;<lengths by index>;<rows A0,A1/...>;<dtypes by arg>
    """
    lens = index_lengths(f)
    letters = sorted(lens)
    args = sorted({a for r in f.rows for a in r}, key=lambda s: int(s[1:]))
    return "be1:{};{};{}->{};{};{};{}".format(
        f.b, f.n, "".join(f.out), ",".join("".join(s) for s in f.ins),
        ",".join(str(lens[c]) for c in letters),
        "/".join(",".join(r) for r in f.rows),
        ",".join(f.dtype(a) for a in args))


def apply_sigma(c: Canon) -> BE:
    """Rebuild the user's einsum from C(e) and the sigma maps (the maps send
    canonical symbols to the user's, as Alg. 1 returns them)."""
    f = c.form
    b, n = f.b, f.n
    inv_i = [None] * b
    for q, u in enumerate(c.sigma_i):
        inv_i[u] = q
    inv_j = [None] * n
    for p, u in enumerate(c.sigma_j):
        inv_j[u] = p
    out = [c.sigma_I[x] for x in f.out]
    ins = [[c.sigma_I[x] for x in f.ins[inv_j[u]]] for u in range(n)]
    rows = [[c.sigma_A[f.rows[inv_i[ur]][inv_j[u]]] for u in range(n)] for ur in range(b)]
    shapes = {c.sigma_A[a]: s for a, s in f.shapes}
    dtypes = {c.sigma_A[a]: d for a, d in f.dtypes}
    return make(out, ins, rows, shapes, dtypes)


def isomorphic(e1: BE, e2: BE):
    """Direct search for (sigma^i, sigma^j, sigma^I, sigma^A) per the
    definition of batched-einsum isomorphism.  sigma^I : I^all(e2) -> I^all(e1),
    sigma^A : A^all(e2) -> A^all(e1).  Returns the witness or None."""
    if (e1.b, e1.n, len(e1.out)) != (e2.b, e2.n, len(e2.out)):
        return None
    l1, l2 = index_lengths(e1), index_lengths(e2)
    if len(l1) != len(l2):
        return None
    if [len(s) for s in e1.ins] and sorted(len(s) for s in e1.ins) != sorted(len(s) for s in e2.ins):
        return None
    idx2 = sorted(l2)
    idx1 = sorted(l1)
    for sj in itertools.permutations(range(e1.n)):
        if any(len(e1.ins[j]) != len(e2.ins[sj[j]]) for j in range(e1.n)):
            continue
        for img in itertools.permutations(idx1):
            sI = dict(zip(idx2, img))
            if any(sI[c2] != c1 for c1, c2 in zip(e1.out, e2.out)):
                continue
            ok = all(e1.ins[j][d] == sI[e2.ins[sj[j]][d]]
                     for j in range(e1.n) for d in range(len(e1.ins[j])))
            if not ok:
                continue
            for si in itertools.permutations(range(e1.b)):
                sA = {}
                good = True
                for i in range(e1.b):
                    for j in range(e1.n):
                        a2 = e2.rows[si[i]][sj[j]]
                        a1 = e1.rows[i][j]
                        if sA.setdefault(a2, a1) != a1:
                            good = False
                            break
                    if not good:
                        break
                if not good or len(set(sA.values())) != len(sA):
                    continue
                if any(e2.shape(a2) != e1.shape(a1) or e2.dtype(a2) != e1.dtype(a1)
                       for a2, a1 in sA.items()):
                    continue
                return {"sigma_i": si, "sigma_j": sj, "sigma_I": sI, "sigma_A": sA}
    return None


def from_spec_text(notation: str, rows, shapes, dtypes) -> BE:
    lhs, out = notation.replace(" ", "").split("->")
    return make(out, lhs.split(","), rows, shapes, dtypes)
