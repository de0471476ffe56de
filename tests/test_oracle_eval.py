"""Pins of the FP64 oracle evaluator (CPU only).

Each check ties the oracle to something other than itself: numpy's einsum
and matmul on integer-valued inputs (exact), pure-Python brute force on tiny
inputs, the paper's worked examples, closed forms for the producer listings,
and special cases (trace, empty axis, outer product).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import evaluate as ev
import workloads as W


def brute(out, ins, ops):
    """Pure-Python definition of Eq. (1) for tiny inputs."""
    lens = {}
    for s, A in zip(ins, ops):
        for c, L in zip(s, A.shape):
            lens[c] = L
    letters = sorted(lens)
    con = [c for c in letters if c not in out]
    R = np.zeros(tuple(lens[c] for c in out))
    for ov in itertools.product(*[range(lens[c]) for c in out]):
        acc = 0.0
        for cv in itertools.product(*[range(lens[c]) for c in con]):
            env = dict(zip(out, ov)) | dict(zip(con, cv))
            p = 1.0
            for s, A in zip(ins, ops):
                p *= A[tuple(env[c] for c in s)]
            acc += p
        R[ov] = acc
    return R


@pytest.mark.parametrize("notation", [
    "ik,kj->ij", "ij,j->i", "ij,ej->ei", "rij,er,ej->ei", "xre,rij,xej->ei",
    "fe,ifj,fej->ei", "ik,kl,lj->ij", "mnj,mni,kli->ijkl", "ij,ik->i",
    "ijk,ik,ij,ij->i", "ijcd,cdab->ijab", "ij,kl,jl->ik", "ii->i", "ii->", "ij->", "i,j->ij",
])
def test_integer_inputs_match_numpy_exactly(notation):
    lhs, out = notation.split("->")
    ins = lhs.split(",")
    g = np.random.default_rng(5)
    lens = {c: int(g.integers(1, 6)) for c in set("".join(ins))}
    ops = [g.integers(-3, 4, size=tuple(lens[c] for c in s)).astype(np.float64) for s in ins]
    R, S = ev.einsum_f64(out, ins, ops)
    assert np.array_equal(R, np.einsum(notation, *ops))
    assert np.array_equal(S, np.einsum(notation, *[np.abs(A) for A in ops]))
    assert np.array_equal(R, brute(out, ins, ops))


def test_random_inputs_match_bruteforce():
    g = np.random.default_rng(9)
    for notation in ["ik,kj->ij", "rij,er,ej->ei", "mnj,mni,kli->ijkl"]:
        lhs, out = notation.split("->")
        ins = lhs.split(",")
        lens = {c: int(g.integers(2, 5)) for c in set("".join(ins))}
        ops = [g.standard_normal(tuple(lens[c] for c in s)) for s in ins]
        R, _ = ev.einsum_f64(out, ins, ops)
        np.testing.assert_allclose(R, brute(out, ins, ops), rtol=1e-13, atol=1e-13)


def test_paper_matmul_example(golden):
    g = golden("einsum_examples.json")["matmul"]
    rng = np.random.default_rng(1)
    A = rng.integers(-5, 6, size=g["shapes"]["A"]).astype(np.float64)
    B = rng.integers(-5, 6, size=g["shapes"]["B"]).astype(np.float64)
    R, _ = ev.einsum_f64("ij", ["ik", "kj"], [A, B])
    assert R.shape == tuple(g["out_shape"])
    assert np.array_equal(R, A @ B)


def test_paper_triple_product(golden):
    g = golden("einsum_examples.json")["triple_product"]
    rng = np.random.default_rng(2)
    n = g["n"]
    arrs = {k: rng.integers(-3, 4, size=(n, n)).astype(np.float64) for k in "ABCD"}
    spec = "ik,kl,lj->ij | A,B,C | B,C,D ; " + " ; ".join(f"{k}:f64[{n},{n}]" for k in "ABCD")
    (R1, _), (R2, _) = ev.evaluate(spec, arrs)
    assert np.array_equal(R1, arrs["A"] @ arrs["B"] @ arrs["C"])
    assert np.array_equal(R2, arrs["B"] @ arrs["C"] @ arrs["D"])


def test_feinsum_listing_closed_form(golden):
    """y1 = sum_j P^2 (3 cos Q + 5), y2 = sum_j P^2 sin R; with Q = 0 and
    R = pi/2 these are 8 * rowsum(P^2) and rowsum(P^2)."""
    spec = golden("einsum_examples.json")["feinsum_listing"]["spec"]
    P = np.arange(96 * 4, dtype=np.float64).reshape(96, 4) % 7 - 3
    (y1, _), (y2, _) = ev.evaluate(spec, {"P": P, "Q": np.zeros(4), "R": np.full(4, math.pi / 2)})
    assert np.array_equal(y1, 8.0 * (P * P).sum(1))
    assert np.array_equal(y2, (P * P).sum(1))


def test_fused_equals_materialized_fem_operator():
    """FEM operator of the introduction: y = D sin(q) as a functional einsum
    equals materialize-then-contract (the BLAS GEMV route)."""
    rng = np.random.default_rng(4)
    D = rng.standard_normal((20, 30))
    q = rng.standard_normal(30)
    spec = "ij,j->i | D,X ; D:f64[20,30] ; q:f64[30] ; X(j) := sin(q[j])"
    (y, _), = ev.evaluate(spec, {"D": D, "q": q})
    q1 = np.array([math.sin(v) for v in q])
    np.testing.assert_allclose(y, D @ q1, rtol=1e-14, atol=1e-14)


def test_dg_gradient_spec_small():
    E = 17
    D, G, a, b = W.dg_gradient(E=E, ndof=10, dim=3)
    res = ev.evaluate(W.dg_gradient_spec(E=E, ndof=10, dim=3), dict(D=D, G=G, a=a, b=b))
    U = np.sin(a) * b
    for x in range(3):
        ref = np.einsum("rij,er,ej->ei", D, G[:, :, x], U)
        np.testing.assert_allclose(res[x][0], ref, rtol=1e-12, atol=1e-12)


def test_select_producer_divergence_listing():
    """Local divergence listing: f(x,e,j) selects u, v or w by x."""
    rng = np.random.default_rng(8)
    E, N = 5, 4
    u, v, w = (rng.integers(-3, 4, size=(E, N)).astype(np.float64) for _ in range(3))
    J = rng.integers(-3, 4, size=(3, 3, E)).astype(np.float64)
    D = rng.integers(-3, 4, size=(3, N, N)).astype(np.float64)
    spec = (f"xre,rij,xej->ei | J,D,F ; J:f64[3,3,{E}] ; D:f64[3,{N},{N}] ; u:f64[{E},{N}] ; "
            f"v:f64[{E},{N}] ; w:f64[{E},{N}] ; F(x,e,j):f64[3,{E},{N}] := x==0 ? u[e,j] : (x==1 ? v[e,j] : w[e,j])")
    (R, _), = ev.evaluate(spec, dict(J=J, D=D, u=u, v=v, w=w))
    F = np.stack([u, v, w])
    assert np.array_equal(R, np.einsum("xre,rij,xej->ei", J, D, F))


def test_empty_axis_and_sampling():
    R, S = ev.einsum_f64("i", ["ij"], [np.zeros((3, 0))])
    assert np.array_equal(R, np.zeros(3)) and np.array_equal(S, np.zeros(3))
    g = np.random.default_rng(0)
    A, B = g.standard_normal((7, 5)), g.standard_normal((5, 9))
    full, _ = ev.einsum_f64("ij", ["ik", "kj"], [A, B])
    sel = np.array([0, 8, 62, 17])
    part, _ = ev.einsum_f64("ij", ["ik", "kj"], [A, B], sel=sel)
    assert np.array_equal(part, full.reshape(-1)[sel])


def test_planted_mistake_in_odometer_is_caught():
    """A transposed operand (a plausible slip) fails the numpy pin."""
    g = np.random.default_rng(3)
    A = g.integers(-3, 4, size=(3, 4)).astype(np.float64)
    B = g.integers(-3, 4, size=(4, 5)).astype(np.float64)
    R, _ = ev.einsum_f64("ij", ["ik", "kj"], [A, B])
    slip, _ = ev.einsum_f64("ij", ["ki", "kj"], [A.T.copy(), B])   # same math, other layout
    assert np.array_equal(R, slip)
    bad, _ = ev.einsum_f64("ij", ["ik", "kj"], [A, B[::-1].copy()])
    assert not np.array_equal(bad, np.einsum("ik,kj->ij", A, B))
