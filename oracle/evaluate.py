"""FP64 oracle evaluation of (functional) batched einsums -- test infrastructure only.

For each row i of a batched einsum the oracle computes
    R_i[I_out] = sum over non-output indices of prod_k M(A^{i,k})(I_in,k)
(Def. "Functional Batched Einstein Summation"), by first materialising every
lambda operand M(A) over its whole domain dom(A) in FP64 and then running the
nested loops of einsum_ref.c.  Materialising a lambda yields exactly the
values the definition evaluates at each index tuple, so this is the
definition written out, not a reordering of it.

Transcendentals use the host libm through einsum_ref.c.  Narrower inputs are
upcast to FP64 exactly before contracting.

Parity: see einsum_ref.c; the producer evaluation is pinned by hand-computed
values in tests/test_oracle_eval.py (the FEM operator of the introduction and
the matvec listing of the Feinsum section).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import spec as S

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile einsum_ref.c with gcc (-O2 -fopenmp, plain loops)."""
    src = os.path.join(_HERE, "einsum_ref.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_einsum_f64.restype = ctypes.c_int
            L.oracle_einsum_f64.argtypes = [
                ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                ctypes.POINTER(ctypes.c_void_p),
                ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                ctypes.c_void_p, ctypes.c_void_p]
            for nm in ("oracle_sin", "oracle_cos", "oracle_exp"):
                f = getattr(L, nm)
                f.restype = None
                f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            L.oracle_set_threads.restype = ctypes.c_int
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def set_threads(n: int) -> int:
    return lib().oracle_set_threads(int(n))


def _libm(name, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    getattr(lib(), "oracle_" + name)(x.size, x.ctypes.data, y.ctypes.data)
    return y


def einsum_f64(out: str, ins, operands, sel=None):
    """Evaluate one einsum; returns (R, S) with S the absolute contraction.
    ``sel``: optional flat row-major output positions to evaluate."""
    letters = sorted(set(out).union(*[set(s) for s in ins]) if ins else set(out))
    ids = {c: k for k, c in enumerate(letters)}
    lens = {}
    for s, A in zip(ins, operands):
        if A.ndim != len(s):
            raise ValueError("operand rank differs from its index list")
        for c, L in zip(s, A.shape):
            if lens.setdefault(c, L) != L:
                raise ValueError(f"inconsistent length for {c}")
    ops = [np.ascontiguousarray(A, dtype=np.float64) for A in operands]
    len_arr = (ctypes.c_int64 * max(1, len(letters)))(*[lens[c] for c in letters])
    out_arr = (ctypes.c_int * max(1, len(out)))(*[ids[c] for c in out])
    ndim = (ctypes.c_int * len(ops))(*[len(s) for s in ins])
    flat = [ids[c] for s in ins for c in s]
    ids_arr = (ctypes.c_int * max(1, len(flat)))(*flat)
    ptrs = (ctypes.c_void_p * len(ops))(*[A.ctypes.data for A in ops])
    out_shape = tuple(lens[c] for c in out)
    if sel is None:
        R = np.empty(out_shape, dtype=np.float64)
        Sv = np.empty(out_shape, dtype=np.float64)
        nsel, selp = 0, None
    else:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        R = np.empty(sel.shape, dtype=np.float64)
        Sv = np.empty(sel.shape, dtype=np.float64)
        nsel, selp = sel.size, sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    rc = lib().oracle_einsum_f64(len(letters), len_arr, len(out), out_arr, len(ops), ndim, ids_arr,
                                 ptrs, nsel, selp, R.ctypes.data, Sv.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_einsum_f64 failed ({rc})")
    return R, Sv


def _eval_node(node, grids, buffers, scalars):
    op = node.op
    if op == "num":
        return np.float64(node.val)
    if op == "scalar":
        return np.float64(scalars[node.val])
    if op == "param":
        return grids[node.val].astype(np.float64)
    if op == "ref":
        A = np.asarray(buffers[node.val], dtype=np.float64)
        idx = tuple(grids[s] if isinstance(s, str) else s for s in node.kids)
        return A[idx]
    k = [_eval_node(c, grids, buffers, scalars) for c in node.kids]
    if op == "neg":
        return -k[0]
    if op == "add":
        return k[0] + k[1]
    if op == "sub":
        return k[0] - k[1]
    if op == "mul":
        return k[0] * k[1]
    if op == "div":
        return k[0] / k[1]
    if op == "eq":
        return (k[0] == k[1])
    if op == "ne":
        return (k[0] != k[1])
    if op == "select":
        return np.where(k[0], k[1], k[2])
    if op == "call":
        x = np.broadcast_to(k[0], next(iter(grids.values())).shape) if grids else np.asarray(k[0])
        if node.val == "abs":
            return np.abs(x)
        return _libm(node.val, x)
    raise ValueError(op)


def materialize(sp: S.Spec, name: str, buffers, scalars=None) -> np.ndarray:
    """Values of the operand ``name`` over its whole domain, FP64."""
    if name in sp.buffers:
        return np.asarray(buffers[name], dtype=np.float64)
    f = sp.functionals[name]
    shape = sp.arg_shapes[name]
    grids = dict(zip(f.params, np.indices(shape))) if shape else {}
    v = _eval_node(f.expr, grids, buffers, scalars or {})
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), shape)
    # the lambda's result type: round through it when narrower than FP64
    dt = sp.arg_dtypes[name]
    if dt == "float32":
        v = v.astype(np.float32).astype(np.float64)
    return np.ascontiguousarray(v)


def evaluate(text: str, buffers, scalars=None, sel=None, rows=None):
    """Per row i: (R_i, S_i).  ``sel``: optional flat output positions
    (same for every row); ``rows``: optional subset of rows."""
    sp = S.parse(text)
    cache = {}
    res = []
    for i, row in enumerate(sp.rows):
        if rows is not None and i not in rows:
            res.append(None)
            continue
        ops = []
        for a in row:
            if a not in cache:
                cache[a] = materialize(sp, a, buffers, scalars)
            ops.append(cache[a])
        res.append(einsum_f64(sp.out, sp.ins, ops, sel))
    return res
