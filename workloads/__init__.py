"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and random relabelings.  It holds none
of the batched-einsum arithmetic (no contraction, no canonicalization), so
both the oracle under ``oracle/`` and the CUDA path may take their inputs
from here without sharing any of the method's code.

Every generator uses numpy's PCG64 with a fixed base seed per workload plus a
per-tensor offset, so a given (workload, size) always yields the same arrays.

Workload shapes follow the paper's FEM / DG / chemistry examples:
  * FEM action  'ij,ej->ei', b=4, D 4x4 shared, E=4096 (Sec. "Batched
    Einstein Summation", the hot-loop example, and the motivating
    FEM operator of the introduction).
  * DG local gradient split per derivative direction x, P4 tetrahedron
    (35 dofs), E=262144 elements, u = sin(a)*b fused into the operand load
    (Sec. "Batched einsums in DG-FEM Operators", local gradient tuple and
    the gradient kernel pattern of Appendix C).
  * Chemistry-style dense contraction 'abef,efij->abij' with v=128, o=32
    (the cluster-operator form quoted in the introduction).
  * An uneven mix drawn from twelve notations that appear in the paper.
"""
from __future__ import annotations

import itertools
import math
import string
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1000

# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------


def rng(workload: int, offset: int = 0) -> np.random.Generator:
    """PCG64 stream for tensor ``offset`` of workload ``workload``."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + workload, offset]))


def uniform(workload, offset, shape, lo=-1.0, hi=1.0):
    return rng(workload, offset).uniform(lo, hi, size=shape)


def normal(workload, offset, shape):
    return rng(workload, offset).standard_normal(size=shape)


def small_ints(workload, offset, shape, lo=-3, hi=3):
    """Integer-valued float64 entries in [lo, hi]: products and sums of these
    stay exact in FP64, so any correct evaluation order gives the same bits."""
    return rng(workload, offset).integers(lo, hi + 1, size=shape).astype(np.float64)


# --------------------------------------------------------------------------
# Workload 1: FEM action 'ij,ej->ei'
# --------------------------------------------------------------------------

FEM_SPEC_NOTATION = "ij,ej->ei"


def fem_action(E: int = 4096, ndof: int = 4, b: int = 4, ints: bool = False):
    """Shared reference matrix D (ndof x ndof) and b field arrays u_k (E x ndof),
    all uniform[-1, 1] (or small integers when ``ints``)."""
    gen = small_ints if ints else uniform
    D = gen(1, 0, (ndof, ndof))
    us = [gen(1, 1 + k, (E, ndof)) for k in range(b)]
    return D, us


def fem_action_spec(E: int = 4096, ndof: int = 4, b: int = 4) -> str:
    rows = " | ".join(f"D,u{k}" for k in range(b))
    decls = " ; ".join([f"D:f64[{ndof},{ndof}]"] + [f"u{k}:f64[{E},{ndof}]" for k in range(b)])
    return f"{FEM_SPEC_NOTATION} | {rows} ; {decls}"


# --------------------------------------------------------------------------
# Workload 2: DG local gradient with a functional field operand
# --------------------------------------------------------------------------


def dg_gradient(E: int = 262144, ndof: int = 35, dim: int = 3, ints: bool = False):
    """D[r,i,j] (dim x ndof x ndof), geometric factors G[e,r,x] (E x dim x dim),
    fields a, b (E x ndof); all N(0,1) in FP64 (small integers when ``ints``;
    the fused producer then stays exact only if it has no transcendental)."""
    if ints:
        D = small_ints(2, 0, (dim, ndof, ndof))
        G = small_ints(2, 1, (E, dim, dim))
        a = small_ints(2, 2, (E, ndof))
        b = small_ints(2, 3, (E, ndof))
    else:
        D = normal(2, 0, (dim, ndof, ndof))
        G = normal(2, 1, (E, dim, dim))
        a = normal(2, 2, (E, ndof))
        b = normal(2, 3, (E, ndof))
    return D, G, a, b


def dg_gradient_spec(E: int = 262144, ndof: int = 35, dim: int = 3, producer: str = "sin(a[e,j])*b[e,j]") -> str:
    """Text of the DG gradient batched einsum: row x computes
    R_x[e,i] = sum_{r,j} D[r,i,j] * G[e,r,x] * U[e,j] with U the fused field."""
    rows = " | ".join(f"D,G{x},U" for x in range(dim))
    decls = [f"D:f64[{dim},{ndof},{ndof}]", f"G:f64[{E},{dim},{dim}]",
             f"a:f64[{E},{ndof}]", f"b:f64[{E},{ndof}]"]
    decls += [f"G{x}(e,r) := G[e,r,{x}]" for x in range(dim)]
    decls += [f"U(e,j) := {producer}"]
    return f"rij,er,ej->ei | {rows} ; " + " ; ".join(decls)


# --------------------------------------------------------------------------
# DG local divergence and face mass: b einsums sharing the operator
# --------------------------------------------------------------------------


def tet_dofs(order: int) -> int:
    """Nodal dofs of a Pk tetrahedron, (k+1)(k+2)(k+3)/6."""
    return (order + 1) * (order + 2) * (order + 3) // 6


def tri_dofs(order: int) -> int:
    """Nodal dofs of a Pk triangle (one face of the tetrahedron), (k+1)(k+2)/2."""
    return (order + 1) * (order + 2) // 2


def dg_divergence(E: int = 100000, order: int = 4, rows: int = 1, ints: bool = False):
    """Shared D[r,i,j] (3 x N x N) and per row k the metric terms J_k[x,r,e]
    (3 x 3 x E) and the vector field's components u_k, v_k, w_k (E x N),
    N = tet_dofs(order); N(0,1) FP64, or small integers when ``ints``."""
    N = tet_dofs(order)
    f = small_ints if ints else normal
    D = f(6, 0, (3, N, N))
    data = []
    for k in range(rows):
        data.append(dict(J=f(6, 1 + 4 * k, (3, 3, E)), u=f(6, 2 + 4 * k, (E, N)),
                         v=f(6, 3 + 4 * k, (E, N)), w=f(6, 4 + 4 * k, (E, N))))
    return D, data


def dg_divergence_spec(E: int = 100000, order: int = 4, rows: int = 1) -> str:
    """Text of the DG local divergence, one einsum per field:
    R_k[e,i] = sum_{x,r,j} J_k[x,r,e] D[r,i,j] F_k[x,e,j], with F_k selecting
    the component u_k, v_k or w_k by x."""
    N = tet_dofs(order)
    decls = [f"D:f64[3,{N},{N}]"]
    for k in range(rows):
        decls += [f"J{k}:f64[3,3,{E}]", f"u{k}:f64[{E},{N}]", f"v{k}:f64[{E},{N}]", f"w{k}:f64[{E},{N}]",
                  f"F{k}(x,e,j):f64[3,{E},{N}] := x==0 ? u{k}[e,j] : (x==1 ? v{k}[e,j] : w{k}[e,j])"]
    body = " | ".join(f"J{k},D,F{k}" for k in range(rows))
    return f"xre,rij,xej->ei | {body} ; " + " ; ".join(decls)


def dg_divergence_arrays(D, data) -> dict:
    arrs = {"D": D}
    for k, d in enumerate(data):
        for name in ("J", "u", "v", "w"):
            arrs[f"{name}{k}"] = d[name]
    return arrs


def face_mass(E: int = 100000, order: int = 4, rows: int = 1, ints: bool = False):
    """Shared face lift M[i,f,j] (N x 4 x NF) and per row k the face
    Jacobians J_k[f,e] (4 x E) and face values U_k[f,e,j] (4 x E x NF),
    N = tet_dofs(order), NF = tri_dofs(order); N(0,1) FP64 or small ints."""
    N, NF = tet_dofs(order), tri_dofs(order)
    f = small_ints if ints else normal
    M = f(7, 0, (N, 4, NF))
    data = [dict(J=f(7, 1 + 2 * k, (4, E)), U=f(7, 2 + 2 * k, (4, E, NF))) for k in range(rows)]
    return M, data


def face_mass_spec(E: int = 100000, order: int = 4, rows: int = 1) -> str:
    """Text of the face mass term R_k[e,i] = sum_{f,j} J_k[f,e] M[i,f,j] U_k[f,e,j]."""
    N, NF = tet_dofs(order), tri_dofs(order)
    decls = [f"M:f64[{N},4,{NF}]"]
    for k in range(rows):
        decls += [f"J{k}:f64[4,{E}]", f"U{k}:f64[4,{E},{NF}]"]
    body = " | ".join(f"J{k},M,U{k}" for k in range(rows))
    return f"fe,ifj,fej->ei | {body} ; " + " ; ".join(decls)


def face_mass_arrays(M, data) -> dict:
    arrs = {"M": M}
    for k, d in enumerate(data):
        arrs[f"J{k}"] = d["J"]
        arrs[f"U{k}"] = d["U"]
    return arrs


# --------------------------------------------------------------------------
# Workload 3: dense chemistry-style contraction 'abef,efij->abij'
# --------------------------------------------------------------------------


def _decay(n1, n2):
    g1 = np.arange(n1)[:, None]
    g2 = np.arange(n2)[None, :]
    return np.abs(g1 - g2).astype(np.float64)


def chem_dense(v: int = 128, o: int = 32, b: int = 4, ints: bool = False):
    """A_k[a,b,e,f] = N(0,1)*exp(-(|a-e|+|b-f|)/8) (v^4 each, k=1..b) and the
    shared T[e,f,i,j] = N(0,1)*exp(-(|e-i|+|f-j|)/8) (v^2 o^2).  "Index gap"
    is read as the L1 distance between the paired indices.  With ``ints`` the
    entries are small integers instead (exactly representable in FP16)."""
    if ints:
        As = [small_ints(3, 1 + k, (v, v, v, v)) for k in range(b)]
        T = small_ints(3, 0, (v, v, o, o))
        return As, T
    dae = _decay(v, v)                      # |a-e|
    w4 = np.exp(-(dae[:, None, :, None] + dae[None, :, None, :]) / 8.0)
    As = []
    for k in range(b):
        A = normal(3, 1 + k, (v, v, v, v))
        A *= w4
        As.append(A)
    dei = _decay(v, o)
    wT = np.exp(-(dei[:, None, :, None] + dei[None, :, None, :]) / 8.0)
    T = normal(3, 0, (v, v, o, o)) * wT
    return As, T


def chem_dense_spec(v: int = 128, o: int = 32, b: int = 4) -> str:
    rows = " | ".join(f"A{k},T" for k in range(b))
    decls = [f"A{k}:f64[{v},{v},{v},{v}]" for k in range(b)] + [f"T:f64[{v},{v},{o},{o}]"]
    return f"abef,efij->abij | {rows} ; " + " ; ".join(decls)


# --------------------------------------------------------------------------
# Random relabelings (index renames, row permutations, operand swaps)
# --------------------------------------------------------------------------


@dataclass
class Relabeled:
    out: str
    ins: list
    rows: list
    row_perm: list          # new row q is old row row_perm[q]
    op_perm: list           # new operand p is old operand op_perm[p]
    rename: dict            # old letter -> new letter


def relabel(out: str, ins, rows, gen: np.random.Generator, arg_rename=None) -> Relabeled:
    """Apply a random injective index rename into a..z, a random row
    permutation and a random operand permutation (the same for all rows)."""
    letters = sorted(set(out).union(*[set(s) for s in ins]))
    targets = gen.permutation(list(string.ascii_lowercase))[: len(letters)]
    rename = {c: str(t) for c, t in zip(letters, targets)}
    b, n = len(rows), len(ins)
    row_perm = [int(x) for x in gen.permutation(b)]
    op_perm = [int(x) for x in gen.permutation(n)]
    new_out = "".join(rename[c] for c in out)
    new_ins = ["".join(rename[c] for c in ins[p]) for p in op_perm]
    ar = arg_rename or (lambda a: a)
    new_rows = [[ar(rows[q][p]) for p in op_perm] for q in row_perm]
    return Relabeled(new_out, new_ins, new_rows, row_perm, op_perm, rename)


# --------------------------------------------------------------------------
# Notations of the uneven mix (all appear in the paper)
# --------------------------------------------------------------------------

# (name, notation).  Sources: matmul example; matvec of the transform-writer
# listing; FEM action; DG gradient / divergence / face mass tuples; the
# batched triple product; the Fig. 1 contraction; the canonical-form
# example; the isomorphic-batched example; the two cluster contractions of
# the introduction.
MIX_NOTATIONS = [
    ("matmul", "ik,kj->ij"),
    ("matvec", "ij,j->i"),
    ("fem_action", "ij,ej->ei"),
    ("dg_gradient", "rij,er,ej->ei"),
    ("dg_divergence", "xre,rij,xej->ei"),
    ("face_mass", "fe,ifj,fej->ei"),
    ("triple_product", "ik,kl,lj->ij"),
    ("fig1", "mnj,mni,kli->ijkl"),
    ("canon_example", "ij,ik->i"),
    ("iso_example", "ijk,ik,ij,ij->i"),
    ("cluster", "ijcd,cdab->ijab"),
    ("tensor_train", "ij,kl,jl->ik"),
]


def _flops(out, ins, lens):
    idx = set(out).union(*[set(s) for s in ins])
    vol = 1
    for c in idx:
        vol *= lens[c]
    return 2 * vol * max(1, len(ins) - 1) if len(ins) > 1 else vol


@dataclass
class Instance:
    name: str
    out: str
    ins: list
    rows: list
    shapes: dict
    dtype: str
    lens: dict
    row_perm: list = field(default_factory=list)
    op_perm: list = field(default_factory=list)


def mix_instance(gen: np.random.Generator, lo_exp=3.0, hi_exp=12.0,
                 max_operand=1 << 22, max_flops=1 << 30, max_tries=1000) -> Instance:
    """One instance of the uneven mix: a notation picked uniformly, index
    lengths round(2^U(lo,hi)); while an operand is too large or the
    instance's flop count exceeds the cap, every exponent is shrunk by 10 %
    toward lo; dtype f64 or f32 with p = 1/2;
    b in {1..4} with the first operand shared by all rows; then a random
    rename and row / operand permutation."""
    name, notation = MIX_NOTATIONS[int(gen.integers(len(MIX_NOTATIONS)))]
    lhs, out = notation.split("->")
    ins = lhs.split(",")
    letters = sorted(set(out).union(*[set(s) for s in ins]))
    u = {c: gen.uniform(lo_exp, hi_exp) for c in letters}
    for _ in range(max_tries):
        lens = {c: int(round(2.0 ** u[c])) for c in letters}
        sizes = [math.prod(lens[c] for c in s) for s in ins] + [math.prod(lens[c] for c in out)]
        if max(sizes) <= max_operand and _flops(out, ins, lens) <= max_flops:
            break
        # over a cap: shrink every exponent toward the lower end and retry
        u = {c: lo_exp + 0.9 * (v - lo_exp) for c, v in u.items()}
    else:
        raise RuntimeError("could not draw an instance under the caps")
    dtype = "f64" if gen.random() < 0.5 else "f32"
    b = int(gen.integers(1, 5))
    rows = []
    for q in range(b):
        rows.append(["X0"] + [f"X{p}_{q}" for p in range(1, len(ins))])
    r = relabel(out, ins, rows, gen)
    shapes = {}
    for row in r.rows:
        for p, a in enumerate(row):
            shapes[a] = tuple(lens[c] for c in _inv_letters(r.ins[p], r.rename))
    new_lens = {r.rename[c]: lens[c] for c in letters}
    return Instance(name, r.out, r.ins, r.rows, shapes, dtype, new_lens, r.row_perm, r.op_perm)


def _inv_letters(s, rename):
    inv = {v: k for k, v in rename.items()}
    return [inv[c] for c in s]


def instance_spec(inst: Instance) -> str:
    rows = " | ".join(",".join(r) for r in inst.rows)
    seen = []
    for r in inst.rows:
        for a in r:
            if a not in seen:
                seen.append(a)
    decls = [f"{a}:{inst.dtype}[{','.join(str(x) for x in inst.shapes[a])}]" for a in seen]
    return f"{','.join(inst.ins)}->{inst.out} | {rows} ; " + " ; ".join(decls)


def instance_arrays(inst: Instance, gen: np.random.Generator, ints: bool = False):
    """Arrays for every distinct argument of ``inst`` in first-appearance order."""
    seen = []
    for r in inst.rows:
        for a in r:
            if a not in seen:
                seen.append(a)
    out = {}
    dt = np.float64 if inst.dtype == "f64" else np.float32
    for a in seen:
        if ints:
            x = gen.integers(-2, 3, size=inst.shapes[a]).astype(dt)
        else:
            x = gen.uniform(-1.0, 1.0, size=inst.shapes[a]).astype(dt)
        out[a] = x
    return out


def poisson_arrivals(rate: float, duration: float, seed_offset: int = 0):
    """Arrival times (seconds) of a Poisson stream (workload 5)."""
    g = rng(5, seed_offset)
    t, ts = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= duration:
            return np.asarray(ts)
        ts.append(t)


def all_permutations(n):
    return list(itertools.permutations(range(n)))
