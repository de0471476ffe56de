"""Independent reader of the textual batched-einsum spec (oracle side).

Test infrastructure only.  This reader shares no code with the C++ parser of
the product path; both implement the same small grammar:

    spec  := notation ('|' row)+ (';' decl)*
    notation := idx (',' idx)* '->' idx          idx := [a-z]*
    row   := name (',' name)*                     (n names, one per operand)
    decl  := name ':' dtype '[' int (',' int)* ']'           a buffer
           | name '(' p (',' p)* ')' [':' dtype ['[' dims ']']] ':=' expr
    expr  := c-like expression over +,-,*,/, unary -, sin/cos/exp/abs,
             numbers, $scalars, lambda params, buffer refs  name[sub, ...]
             with sub a lambda param or an integer, and  p==k ? x : y

A row names idealized arguments; a name declared with ':=' is a functional
operand, i.e. a lambda over its domain (Def. "Functional Batched Einstein
Summation"); a buffer named directly in a row is the identity lambda of an
idealized functional batched einsum (Def. "Idealized Functional Batched
Einsum").  Index letters are a..z (grammar of an index, Sec.
"Preliminaries").
"""
from __future__ import annotations

import re
from dataclasses import dataclass, field

DTYPE_NAMES = {
    "i8": "int8", "i32": "int32", "i64": "int64", "f16": "float16",
    "f32": "float32", "f64": "float64", "c64": "complex64",
    "c128": "complex128", "bf16": "bfloat16",
}
for _v in list(DTYPE_NAMES.values()):
    DTYPE_NAMES[_v] = _v


class SpecError(ValueError):
    pass


@dataclass
class Node:
    op: str                 # num, scalar, param, ref, neg, add, sub, mul, div, call, select, eq
    val: object = None
    kids: list = field(default_factory=list)


@dataclass
class Functional:
    name: str
    params: list
    expr: Node
    dtype: str | None
    shape: tuple | None


@dataclass
class Spec:
    out: str
    ins: list
    rows: list
    buffers: dict          # name -> (dtype, shape)
    functionals: dict      # name -> Functional
    arg_shapes: dict = field(default_factory=dict)
    arg_dtypes: dict = field(default_factory=dict)


_TOKEN = re.compile(r"\s*(?:(\d+\.\d*(?:[eE][-+]?\d+)?|\d+(?:[eE][-+]?\d+)?|\.\d+(?:[eE][-+]?\d+)?)|(\$?[A-Za-z_][A-Za-z_0-9]*)|(==|!=|[-+*/()\[\],?:]))")


def _tokens(s):
    pos, out = 0, []
    s = s.strip()
    while pos < len(s):
        m = _TOKEN.match(s, pos)
        if not m or m.end() == pos:
            raise SpecError(f"bad token at {s[pos:pos + 10]!r}")
        out.append(m.group(1) or m.group(2) or m.group(3))
        pos = m.end()
    return out


class _P:
    def __init__(self, toks):
        self.t, self.i = toks, 0

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else None

    def take(self, want=None):
        tok = self.peek()
        if tok is None or (want is not None and tok != want):
            raise SpecError(f"expected {want!r}, got {tok!r}")
        self.i += 1
        return tok

    def expr(self):
        c = self.cmp()
        if self.peek() == "?":
            self.take("?")
            a = self.expr()
            self.take(":")
            b = self.expr()
            return Node("select", kids=[c, a, b])
        return c

    def cmp(self):
        a = self.add()
        if self.peek() in ("==", "!="):
            op = self.take()
            b = self.add()
            return Node("eq" if op == "==" else "ne", kids=[a, b])
        return a

    def add(self):
        a = self.mul()
        while self.peek() in ("+", "-"):
            op = self.take()
            a = Node("add" if op == "+" else "sub", kids=[a, self.mul()])
        return a

    def mul(self):
        a = self.unary()
        while self.peek() in ("*", "/"):
            op = self.take()
            a = Node("mul" if op == "*" else "div", kids=[a, self.unary()])
        return a

    def unary(self):
        if self.peek() == "-":
            self.take()
            return Node("neg", kids=[self.unary()])
        if self.peek() == "+":
            self.take()
            return self.unary()
        return self.primary()

    def primary(self):
        tok = self.take()
        if tok == "(":
            e = self.expr()
            self.take(")")
            return e
        if re.fullmatch(r"[\d.].*", tok):
            return Node("num", float(tok))
        if tok.startswith("$"):
            return Node("scalar", tok[1:])
        if self.peek() == "(":
            self.take("(")
            a = self.expr()
            self.take(")")
            if tok not in ("sin", "cos", "exp", "abs"):
                raise SpecError(f"unknown function {tok}")
            return Node("call", tok, [a])
        if self.peek() == "[":
            self.take("[")
            subs = []
            while True:
                s = self.take()
                if re.fullmatch(r"\d+", s):
                    subs.append(int(s))
                elif re.fullmatch(r"[A-Za-z_]\w*", s):
                    subs.append(s)
                else:
                    raise SpecError(f"bad subscript {s}")
                if self.peek() == ",":
                    self.take(",")
                    continue
                self.take("]")
                break
            return Node("ref", tok, subs)
        return Node("param", tok)


def parse_expr(text: str) -> Node:
    p = _P(_tokens(text))
    e = p.expr()
    if p.peek() is not None:
        raise SpecError(f"trailing input {p.peek()!r}")
    return e


_DECL_BUF = re.compile(r"^([A-Za-z_]\w*)\s*:\s*(\w+)\s*\[([\d,\s]*)\]$")
_DECL_FUN = re.compile(r"^([A-Za-z_]\w*)\s*\(([^)]*)\)\s*(?::\s*(\w+)\s*(?:\[([\d,\s]*)\])?)?\s*:=\s*(.+)$")


def _dims(s):
    s = s.strip()
    return tuple(int(x) for x in s.split(",")) if s else ()


def _refs(node, acc):
    if node.op == "ref":
        acc.append(node)
        return acc
    for k in node.kids:
        _refs(k, acc)
    return acc


def parse(text: str) -> Spec:
    parts = [p.strip() for p in text.split(";")]
    head = [p.strip() for p in parts[0].split("|")]
    notation = head[0].replace(" ", "")
    if "->" not in notation:
        raise SpecError("missing '->'")
    lhs, out = notation.split("->")
    ins = lhs.split(",") if lhs else []
    for s in ins + [out]:
        if not re.fullmatch(r"[a-z]*", s):
            raise SpecError(f"bad index list {s!r}")
    if len(set(out)) != len(out):
        raise SpecError("repeated output index")
    rows = [[x.strip() for x in r.split(",")] for r in head[1:]]
    if not rows:
        raise SpecError("no rows")
    for r in rows:
        if len(r) != len(ins):
            raise SpecError("row arity differs from the notation")
    buffers, functionals = {}, {}
    for d in parts[1:]:
        if not d:
            continue
        m = _DECL_BUF.match(d)
        if m:
            buffers[m.group(1)] = (DTYPE_NAMES[m.group(2)], _dims(m.group(3)))
            continue
        m = _DECL_FUN.match(d)
        if m:
            params = [p.strip() for p in m.group(2).split(",") if p.strip()]
            dt = DTYPE_NAMES[m.group(3)] if m.group(3) else None
            shp = _dims(m.group(4)) if m.group(4) is not None else None
            functionals[m.group(1)] = Functional(m.group(1), params, parse_expr(m.group(5)), dt, shp)
            continue
        raise SpecError(f"bad declaration {d!r}")
    spec = Spec(out, ins, rows, buffers, functionals)
    _type(spec)
    return spec


_RANK = {"int8": 1, "int32": 2, "int64": 3, "float16": 4, "float32": 5,
         "float64": 6, "complex64": 7, "complex128": 8, "bfloat16": 9}


# promotion order for the result type of a lambda operand without an
# explicit annotation (the paper leaves it open; this is our reading)
_PROMOTE = ["int8", "int32", "int64", "bfloat16", "float16", "float32",
            "float64", "complex64", "complex128"]


def _type(spec: Spec):
    for r in spec.rows:
        for a in r:
            if a in spec.functionals:
                f = spec.functionals[a]
                refs = _refs(f.expr, [])
                shape = list(f.shape) if f.shape is not None else [None] * len(f.params)
                if len(shape) != len(f.params):
                    raise SpecError(f"{a}: shape rank differs from its parameters")
                for ref in refs:
                    if ref.val not in spec.buffers:
                        raise SpecError(f"{a}: unknown buffer {ref.val}")
                    bshape = spec.buffers[ref.val][1]
                    if len(bshape) != len(ref.kids):
                        raise SpecError(f"{a}: wrong subscript count for {ref.val}")
                    for pos, s in enumerate(ref.kids):
                        if isinstance(s, str):
                            k = f.params.index(s)
                            if shape[k] is None:
                                shape[k] = bshape[pos]
                            elif shape[k] != bshape[pos]:
                                raise SpecError(f"{a}: inconsistent extent of {s}")
                if any(x is None for x in shape):
                    raise SpecError(f"{a}: cannot infer the extent of every parameter")
                spec.arg_shapes[a] = tuple(shape)
                if f.dtype:
                    spec.arg_dtypes[a] = f.dtype
                else:
                    dts = [spec.buffers[r.val][0] for r in refs] or ["float64"]
                    spec.arg_dtypes[a] = max(dts, key=_PROMOTE.index)
            elif a in spec.buffers:
                spec.arg_dtypes[a], spec.arg_shapes[a] = spec.buffers[a]
            else:
                raise SpecError(f"undeclared argument {a}")
