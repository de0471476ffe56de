"""Thin ctypes binding of the engine's C ABI (include/be.h).

Argument marshalling only: every step (parse, canonicalize, lookup,
evaluation) runs inside libbe.so.  Device buffers are torch tensors (torch
provides device memory and streams); host buffers for ``execute_host`` are
numpy arrays.  The library is loaded from this package's directory and an
ImportError is raised if it has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbe.so")

OK, EPARSE, EINVALID, ESHAPE, EDTYPE, ETOOMANY, ENOTFOUND, EDB, EBUDGET, ETIMEOUT, ECUDA, EUNSUPPORTED, EARG = range(13)
I8, I32, I64, F16, F32, F64, C64, C128, BF16 = 1, 2, 3, 4, 5, 6, 7, 8, 9
STRAT_AUTO, STRAT_GENERIC, STRAT_ELEMENT, STRAT_DENSE_SPLIT = 0, 1, 2, 3
PREC_FP64, PREC_SPLIT = 0, 1
SIGMA_INDEX, SIGMA_ARG, SIGMA_ROW, SIGMA_POS = 0, 1, 2, 3
STATUS_NAMES = {0: "BE_OK", 1: "BE_EPARSE", 2: "BE_EINVALID", 3: "BE_ESHAPE", 4: "BE_EDTYPE",
                5: "BE_ETOOMANY", 6: "BE_ENOTFOUND", 7: "BE_EDB", 8: "BE_EBUDGET", 9: "BE_ETIMEOUT",
                10: "BE_ECUDA", 11: "BE_EUNSUPPORTED", 12: "BE_EARG"}

# every symbol include/be.h declares
EXPORTS = [
    "be_version", "be_last_error", "be_parse", "be_free_einsum", "be_einsum_info", "be_einsum_out_shape",
    "be_einsum_buffer", "be_canonicalize", "be_free_canon", "be_canon_key", "be_canon_sigma",
    "be_canon_tokens", "be_induced_graph", "be_graph_check", "be_identify", "be_ctx_create",
    "be_ctx_destroy", "be_lookup", "be_record", "be_db_size", "be_execute", "be_execute_host",
    "be_plan_strategy", "be_status", "be_ctx_set_timing", "be_ctx_timing", "be_gemm_split_noalloc",
    "be_gemm_split_noalloc_status", "be_ctx_set_wait_limit", "be_peak_probe",
    "be_batch_create", "be_batch_run", "be_batch_info", "be_batch_kinds", "be_batch_instance_kind", "be_batch_factored", "be_batch_destroy", "be_tune", "be_tune_batch",
    "be_server_create", "be_server_submit", "be_server_wait", "be_server_drain", "be_server_stats",
    "be_server_reset_stats", "be_server_trace", "be_server_destroy", "be_raise", "be_raised_name", "be_record_facts",
    "be_load_transforms",
]
KERNEL_ELEMENT, KERNEL_GENERIC, KERNEL_DENSE_GEMM, KERNEL_SPLIT, KERNEL_PERSISTENT = 0, 1, 2, 3, 4


class BEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int32), ("tile", ctypes.c_int32 * 4), ("stages", ctypes.c_int32),
                ("stage_mask", ctypes.c_uint32), ("vec", ctypes.c_int32), ("split", ctypes.c_int32)]

    def as_tuple(self):
        return (self.strategy, tuple(self.tile), self.stages, self.stage_mask, self.vec, self.split)


def make_config(strategy=0, tile=(0, 0, 0, 0), stages=0, stage_mask=0, vec=0, split=0) -> Config:
    c = Config()
    c.strategy = strategy
    for k in range(4):
        c.tile[k] = tile[k] if k < len(tile) else 0
    c.stages, c.stage_mask, c.vec, c.split = stages, stage_mask, vec, split
    return c


class Buf(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("strides", ctypes.POINTER(ctypes.c_int64)),
                ("ndim", ctypes.c_int32), ("dtype", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with python paper_2601_12220_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        P = ctypes.POINTER
        sig = {
            "be_version": (ctypes.c_int, []),
            "be_last_error": (ctypes.c_char_p, []),
            "be_parse": (ctypes.c_int, [ctypes.c_char_p, P(vp)]),
            "be_free_einsum": (None, [vp]),
            "be_einsum_info": (ctypes.c_int, [vp] + [P(i32)] * 7),
            "be_einsum_out_shape": (ctypes.c_int, [vp, P(i64)]),
            "be_einsum_buffer": (ctypes.c_int, [vp, i32, ctypes.c_char_p, sz, P(sz), P(i32), P(i32), P(i64)]),
            "be_canonicalize": (ctypes.c_int, [vp, P(vp)]),
            "be_free_canon": (None, [vp]),
            "be_canon_key": (ctypes.c_int, [vp, ctypes.c_char_p, sz, P(sz)]),
            "be_canon_sigma": (ctypes.c_int, [vp, i32, i32, ctypes.c_char_p, sz, P(sz)]),
            "be_canon_tokens": (ctypes.c_int, [vp, P(i64), sz, P(sz)]),
            "be_induced_graph": (ctypes.c_int, [vp, P(i32), P(i32), i32, P(i32), i64, P(i64)]),
            "be_graph_check": (ctypes.c_int, [i32, P(i32), P(i32), i64, P(i32)]),
            "be_identify": (ctypes.c_int, [vp, vp, ctypes.c_char_p, sz, P(sz)]),
            "be_raise": (ctypes.c_int, [ctypes.c_char_p, P(vp)]),
            "be_record_facts": (ctypes.c_int, [vp, vp, P(Config), i32, i32, i32, P(ctypes.c_double)]),
            "be_load_transforms": (ctypes.c_int, [vp, ctypes.c_char_p, i32, i32, P(i32)]),
            "be_raised_name": (ctypes.c_int, [vp, i32, i32, ctypes.c_char_p, sz, P(sz)]),
            "be_ctx_create": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_char_p, i32, sz, P(vp)]),
            "be_ctx_destroy": (None, [vp]),
            "be_lookup": (ctypes.c_int, [vp, vp, i32, P(Config), P(ctypes.c_double)]),
            "be_record": (ctypes.c_int, [vp, vp, i32, P(Config), ctypes.c_double]),
            "be_db_size": (ctypes.c_int, [vp, P(i64)]),
            "be_execute": (ctypes.c_int, [vp, vp, P(Config), i32, P(Buf), i32, P(Buf), i32,
                                          P(ctypes.c_double), i32, vp]),
            "be_execute_host": (ctypes.c_int, [vp, vp, P(Config), i32, P(Buf), i32, P(Buf), i32,
                                               P(ctypes.c_double), i32, vp]),
            "be_plan_strategy": (ctypes.c_int, [vp, vp, P(Config), i32, P(i32)]),
            "be_status": (ctypes.c_int, [vp, P(i32)]),
            "be_ctx_set_timing": (ctypes.c_int, [vp, i32]),
            "be_gemm_split_noalloc": (ctypes.c_int, [vp, i64, vp, i64, vp, i64, i64, i64, i64, vp]),
            "be_gemm_split_noalloc_status": (ctypes.c_int, [P(i32)]),
            "be_ctx_set_wait_limit": (ctypes.c_int, [vp, i64]),
            "be_peak_probe": (ctypes.c_int, [i32, i32, P(ctypes.c_double)]),
            "be_batch_create": (ctypes.c_int, [vp, i32, P(vp), P(P(Buf)), P(i32), P(P(Buf)), P(i32),
                                               P(P(ctypes.c_double)), P(i32), P(Config), P(vp)]),
            "be_batch_run": (ctypes.c_int, [vp, vp]),
            "be_batch_info": (ctypes.c_int, [vp, P(i64), P(i64), P(ctypes.c_double)]),
            "be_batch_kinds": (ctypes.c_int, [vp, P(i32), P(i32), P(i32)]),
            "be_batch_instance_kind": (ctypes.c_int, [vp, i32, P(i32)]),
            "be_batch_factored": (ctypes.c_int, [vp, P(i32), P(i32), P(i64)]),
            "be_tune_batch": (ctypes.c_int, [vp, i32, P(vp), P(P(Buf)), P(i32), P(P(Buf)), P(i32),
                                             P(P(ctypes.c_double)), P(i32), P(Config), i32, vp, P(Config),
                                             P(ctypes.c_double), P(i32)]),
            "be_batch_destroy": (None, [vp]),
            "be_server_create": (ctypes.c_int, [vp, i32, i32, sz, P(vp)]),
            "be_server_submit": (ctypes.c_int, [vp, vp, P(Buf), i32, P(Buf), i32, P(ctypes.c_double), i32, P(i64)]),
            "be_server_wait": (ctypes.c_int, [vp, i64, ctypes.c_double, P(i32), P(ctypes.c_double)]),
            "be_server_drain": (ctypes.c_int, [vp, ctypes.c_double]),
            "be_server_stats": (ctypes.c_int, [vp, P(i64), P(i64), P(ctypes.c_double), P(ctypes.c_double),
                                               P(ctypes.c_double), P(sz), P(i64)]),
            "be_server_reset_stats": (ctypes.c_int, [vp]),
            "be_server_trace": (ctypes.c_int, [vp, P(ctypes.c_double), i64, P(i64)]),
            "be_server_destroy": (None, [vp]),
            "be_tune": (ctypes.c_int, [vp, vp, i32, P(Buf), i32, P(Buf), i32, P(ctypes.c_double), i32, i32, i32,
                                       ctypes.c_double, i32, vp, P(Config), P(ctypes.c_double), P(i32)]),
            "be_ctx_timing": (ctypes.c_int, [vp, i32, P(i64), P(ctypes.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != OK:
        raise BEError(code, lib().be_last_error().decode())


def _string(fn, *args):
    need = ctypes.c_size_t(0)
    fn(*args, None, 0, ctypes.byref(need))
    buf = ctypes.create_string_buffer(need.value)
    check(fn(*args, buf, need.value, ctypes.byref(need)))
    return buf.value.decode()


# ---------------------------------------------------------------- IR

# parse text -> the metadata of its handle (counts, output shape, buffer
# declarations), a function of the text alone: a text parsed again (a
# repeated request) still runs be_parse but skips the queries
_META: dict = {}
_META_MAX = 4096


def _describe(h):
    v = [ctypes.c_int32() for _ in range(7)]
    check(lib().be_einsum_info(h, *[ctypes.byref(x) for x in v]))
    info = tuple(x.value for x in v)
    out_ndim = info[5]
    shp = (ctypes.c_int64 * max(1, out_ndim))()
    check(lib().be_einsum_out_shape(h, shp))
    buffers = []
    for k in range(info[2]):
        dt, nd = ctypes.c_int32(), ctypes.c_int32()
        s = (ctypes.c_int64 * 26)()
        need = ctypes.c_size_t(0)
        lib().be_einsum_buffer(h, k, None, 0, ctypes.byref(need), None, None, None)
        nm = ctypes.create_string_buffer(need.value)
        check(lib().be_einsum_buffer(h, k, nm, need.value, ctypes.byref(need), ctypes.byref(dt),
                                     ctypes.byref(nd), s))
        buffers.append((nm.value.decode(), dt.value, tuple(s[d] for d in range(nd.value))))
    return info, tuple(shp[k] for k in range(out_ndim)), tuple(buffers)


class Einsum:
    """be_parse handle (or, through raise_kernel, a be_raise handle)."""

    def __init__(self, text: str, _handle=None):
        if _handle is None:
            h = ctypes.c_void_p()
            check(lib().be_parse(text.encode(), ctypes.byref(h)))
            meta = _META.get(text)
            if meta is None:
                meta = _describe(h)
                if len(_META) >= _META_MAX:
                    _META.clear()
                _META[text] = meta
        else:
            h = _handle
            meta = _describe(h)
        self._h = h
        self.text = text
        info, self.out_shape, self.buffers = meta
        self.b, self.n, self.n_buffers, self.n_args, self.n_scalars, self.out_ndim, self.out_dtype = info

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.be_free_einsum(self._h)
            self._h = None

    def canonicalize(self) -> "Canon":
        return Canon(self)

    def induced_graph(self):
        n, ne = ctypes.c_int32(), ctypes.c_int64()
        check(lib().be_induced_graph(self._h, ctypes.byref(n), None, 0, None, 0, ctypes.byref(ne)))
        cols = (ctypes.c_int32 * max(1, n.value))()
        eds = (ctypes.c_int32 * max(2, 2 * ne.value))()
        check(lib().be_induced_graph(self._h, ctypes.byref(n), cols, n.value, eds, ne.value, ctypes.byref(ne)))
        colors = np.array(cols[:n.value], dtype=np.int32)
        edges = np.array(eds[:2 * ne.value], dtype=np.int32).reshape(-1, 2)
        return colors, edges


RAISED_SPEC, RAISED_LOOP, RAISED_OUTPUT = 0, 1, 2


def raise_kernel(kernel: str) -> Einsum:
    """be_raise: the functional batched einsum a loop-nest kernel computes.
    The result carries ``loop_names`` (index letter -> loop name) and
    ``outputs`` (row -> output array); ``text`` is the raised be_parse text."""
    h = ctypes.c_void_p()
    check(lib().be_raise(kernel.encode(), ctypes.byref(h)))
    spec = _string(lib().be_raised_name, h, RAISED_SPEC, 0)
    e = Einsum(spec, _handle=h)
    e.kernel = kernel
    e.loop_names = {}
    k = 0
    while True:
        need = ctypes.c_size_t(0)
        if lib().be_raised_name(h, RAISED_LOOP, k, None, 0, ctypes.byref(need)) != OK:
            break
        e.loop_names[chr(ord("a") + k)] = _string(lib().be_raised_name, h, RAISED_LOOP, k)
        k += 1
    e.outputs = [_string(lib().be_raised_name, h, RAISED_OUTPUT, r) for r in range(e.b)]
    return e


def identify_kernel(ref: "Einsum", kernel: "Einsum") -> dict:
    """Alg. 2 against a raised kernel: ref's index letters and argument names
    -> the kernel's loop names and argument names."""
    pairs = [kv.split("=") for kv in _string(lib().be_identify, ref.handle, kernel.handle).split(";") if kv]
    names = getattr(kernel, "loop_names", {})
    n_idx = len(names)                 # be_identify lists the indices first
    return {k: (names.get(v, v) if q < n_idx else v) for q, (k, v) in enumerate(pairs)}


def graph_check(colors, edges) -> int:
    colors = np.ascontiguousarray(colors, dtype=np.int32)
    edges = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1)
    failed = ctypes.c_int32()
    check(lib().be_graph_check(len(colors), colors.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               edges.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(edges) // 2,
                               ctypes.byref(failed)))
    return failed.value


class Canon:
    """be_canonicalize handle: C(e), its printed key and the sigma maps."""

    def __init__(self, e: Einsum):
        h = ctypes.c_void_p()
        check(lib().be_canonicalize(e.handle, ctypes.byref(h)))
        self._h = h
        self._key = None
        self._tokens = None

    @property
    def handle(self):
        return self._h

    @property
    def key(self) -> str:
        """The normal form's printed key (read from the handle on first use)."""
        if self._key is None:
            self._key = _string(lib().be_canon_key, self._h)
        return self._key

    @property
    def tokens(self) -> list:
        """The normal form's token vector (read from the handle on first use)."""
        if self._tokens is None:
            n = ctypes.c_size_t()
            lib().be_canon_tokens(self._h, None, 0, ctypes.byref(n))
            t = (ctypes.c_int64 * max(1, n.value))()
            check(lib().be_canon_tokens(self._h, t, n.value, ctypes.byref(n)))
            self._tokens = list(t[:n.value])
        return self._tokens

    def sigma(self, kind: int, k: int) -> str:
        return _string(lib().be_canon_sigma, self._h, kind, k)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.be_free_canon(self._h)
            self._h = None


def identify(ref: Einsum, target: Einsum) -> dict:
    """Alg. 2: ref's names -> target's names (BEError if the forms differ)."""
    s = _string(lib().be_identify, ref.handle, target.handle)
    return dict(kv.split("=") for kv in s.split(";") if kv)


# ---------------------------------------------------------------- context / DB

class Context:
    def __init__(self, db_path=None, device_name=None, device=0, hbm_budget=0):
        h = ctypes.c_void_p()
        check(lib().be_ctx_create(db_path.encode() if db_path else None,
                                  device_name.encode() if device_name else None, device, hbm_budget,
                                  ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def lookup(self, canon: Canon, precision=PREC_FP64):
        c = Config()
        sec = ctypes.c_double()
        code = lib().be_lookup(self._h, canon.handle, precision, ctypes.byref(c), ctypes.byref(sec))
        if code == ENOTFOUND:
            return None
        check(code)
        return c, sec.value

    def record(self, canon: Canon, cfg: Config, seconds: float, precision=PREC_FP64):
        check(lib().be_record(self._h, canon.handle, precision, ctypes.byref(cfg), seconds))

    def record_facts(self, ref: "Einsum", cfg: Config, precision=PREC_FP64, warmup=3, reps=10) -> float:
        """Time cfg on synthetic operands of ref's shapes and store it under
        ref's normal form; returns the seconds per run."""
        sec = ctypes.c_double()
        check(lib().be_record_facts(self._h, ref.handle, ctypes.byref(cfg), precision, warmup, reps,
                                    ctypes.byref(sec)))
        return sec.value

    def load_transforms(self, text: str, warmup=3, reps=10) -> int:
        """Register a transform library (lines '<reference> => <config>');
        returns the number of registrations recorded."""
        n = ctypes.c_int32()
        check(lib().be_load_transforms(self._h, text.encode(), warmup, reps, ctypes.byref(n)))
        return n.value

    def db_size(self) -> int:
        n = ctypes.c_int64()
        check(lib().be_db_size(self._h, ctypes.byref(n)))
        return n.value

    def status(self) -> int:
        """Wait for the device and read (and clear) the device status word."""
        v = ctypes.c_int32()
        check(lib().be_status(self._h, ctypes.byref(v)))
        return v.value

    def set_timing(self, enable=True):
        check(lib().be_ctx_set_timing(self._h, 1 if enable else 0))

    def set_wait_limit(self, cycles: int = 0):
        """Limit (SM cycles) of the tensor-core kernels' pipeline waits; 0 = default."""
        check(lib().be_ctx_set_wait_limit(self._h, int(cycles)))

    def timing(self, kernel: int):
        """(launches, total ms) of kernel id since the last read."""
        n, ms = ctypes.c_int64(), ctypes.c_double()
        check(lib().be_ctx_timing(self._h, kernel, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.be_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


# ---------------------------------------------------------------- execution

_TORCH_DT = None


def _torch_dtype_code(t):
    global _TORCH_DT
    if _TORCH_DT is None:
        import torch
        _TORCH_DT = {torch.float64: F64, torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16,
                     torch.int32: I32, torch.int64: I64, torch.int8: I8}
    return _TORCH_DT[t.dtype]


_NP_DT = {np.dtype(np.float64): F64, np.dtype(np.float32): F32, np.dtype(np.float16): F16,
          np.dtype(np.int32): I32, np.dtype(np.int64): I64, np.dtype(np.int8): I8}


def _bufs_torch(tensors, keep, dense_only=False):
    arr = (Buf * max(1, len(tensors)))()
    for k, t in enumerate(tensors):
        arr[k].ptr = t.data_ptr()
        arr[k].ndim = t.dim()
        arr[k].dtype = _torch_dtype_code(t)
        if not dense_only and not t.is_contiguous():
            st = (ctypes.c_int64 * max(1, t.dim()))(*t.stride())
            keep.append(st)
            arr[k].strides = st
        else:
            arr[k].strides = None
    return arr


def _scalars(vals):
    vals = list(vals or [])
    return (ctypes.c_double * max(1, len(vals)))(*vals), len(vals)


def _order(e: Einsum, bufs):
    if isinstance(bufs, dict):
        return [bufs[name] for name, _, _ in e.buffers]
    return list(bufs)


def execute(ctx, e: Einsum, bufs, outs, cfg: Config | None = None, precision=PREC_FP64, scalars=(),
            stream=None):
    """Evaluate every row of e on the GPU.  bufs: dict name -> tensor or a
    list in declaration order; outs: one tensor per row; stream: a
    torch.cuda.Stream (default: the current stream)."""
    import torch
    keep = []
    bl = _order(e, bufs)
    if len(bl) != len(e.buffers):
        raise BEError(EARG, f"expected {len(e.buffers)} buffers, got {len(bl)}")
    for t, (name, _, shape) in zip(bl, e.buffers):
        if tuple(t.shape) != shape or not t.is_cuda:
            raise BEError(ESHAPE, f"buffer {name}: expected a CUDA tensor of shape {shape}, got {tuple(t.shape)}")
    for t in outs:
        if tuple(t.shape) != e.out_shape or not t.is_cuda or not t.is_contiguous():
            raise BEError(ESHAPE, f"outputs must be dense CUDA tensors of shape {e.out_shape}")
    bi = _bufs_torch(bl, keep)
    bo = _bufs_torch(outs, keep, dense_only=True)
    sc, ns = _scalars(scalars)
    if stream is None:
        stream = torch.cuda.current_stream()
    check(lib().be_execute(ctx.handle if ctx else None, e.handle, ctypes.byref(cfg) if cfg else None, precision,
                           bi, len(bl), bo, len(outs), sc, ns, ctypes.c_void_p(stream.cuda_stream)))


def execute_host(ctx, e: Einsum, bufs, outs, cfg: Config | None = None, precision=PREC_FP64, scalars=(),
                 stream=None):
    """As execute, with dense host numpy arrays; blocks until done."""
    bl = [np.ascontiguousarray(x) for x in _order(e, bufs)]
    for x, (name, _, shape) in zip(bl, e.buffers):
        if tuple(x.shape) != shape:
            raise BEError(ESHAPE, f"buffer {name}: expected shape {shape}, got {tuple(x.shape)}")
    for x in outs:
        if tuple(x.shape) != e.out_shape:
            raise BEError(ESHAPE, f"outputs must have shape {e.out_shape}")
    arr = (Buf * max(1, len(bl)))()
    for k, x in enumerate(bl):
        arr[k].ptr, arr[k].ndim, arr[k].dtype, arr[k].strides = x.ctypes.data, x.ndim, _NP_DT[x.dtype], None
    oarr = (Buf * max(1, len(outs)))()
    for k, x in enumerate(outs):
        assert x.flags.c_contiguous
        oarr[k].ptr, oarr[k].ndim, oarr[k].dtype, oarr[k].strides = x.ctypes.data, x.ndim, _NP_DT[x.dtype], None
    sc, ns = _scalars(scalars)
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    check(lib().be_execute_host(ctx.handle, e.handle, ctypes.byref(cfg) if cfg else None, precision, arr, len(bl),
                                oarr, len(outs), sc, ns, s))


def tune(ctx, e: Einsum, bufs, outs, precision=PREC_FP64, scalars=(), warmup=2, min_reps=5, min_seconds=0.0,
         force=False, stream=None):
    """Autotune e on these buffers; returns (best Config, seconds, configs timed)."""
    import torch
    keep = []
    bl = _order(e, bufs)
    bi = _bufs_torch(bl, keep)
    bo = _bufs_torch(outs, keep, dense_only=True)
    sc, ns = _scalars(scalars)
    if stream is None:
        stream = torch.cuda.current_stream()
    best, sec, n = Config(), ctypes.c_double(), ctypes.c_int32()
    check(lib().be_tune(ctx.handle, e.handle, precision, bi, len(bl), bo, len(outs), sc, ns, warmup, min_reps,
                        min_seconds, 1 if force else 0, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(best),
                        ctypes.byref(sec), ctypes.byref(n)))
    return best, sec.value, n.value


class Server:
    """Serving loop with continuous batching (native worker thread + streams)."""

    def __init__(self, ctx, precision=PREC_FP64, n_streams=8, hbm_budget=0):
        h = ctypes.c_void_p()
        check(lib().be_server_create(ctx.handle if ctx else None, precision, n_streams, hbm_budget,
                                     ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def prepare(self, e: Einsum, bufs, outs, scalars=()):
        """Marshal a request once; the returned object can be submitted many times."""
        keep = []
        bl = _order(e, bufs)
        bi = _bufs_torch(bl, keep)
        bo = _bufs_torch(outs, keep, dense_only=True)
        sc, ns = _scalars(scalars)
        return (e, bi, len(bl), bo, len(outs), sc, ns, keep, bl, outs)

    def submit(self, req) -> int:
        e, bi, nb, bo, no, sc, ns = req[:7]
        i = ctypes.c_int64()
        check(lib().be_server_submit(self._h, e.handle, bi, nb, bo, no, sc, ns, ctypes.byref(i)))
        self._keep[i.value] = req
        return i.value

    def wait(self, rid: int, timeout=-1.0):
        st, lat = ctypes.c_int32(), ctypes.c_double()
        check(lib().be_server_wait(self._h, rid, timeout, ctypes.byref(st), ctypes.byref(lat)))
        self._keep.pop(rid, None)
        return st.value, lat.value

    def drain(self, timeout=-1.0):
        check(lib().be_server_drain(self._h, timeout))
        self._keep.clear()

    def stats(self):
        c, f = ctypes.c_int64(), ctypes.c_int64()
        p50, p99, thr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        pk, mi = ctypes.c_size_t(), ctypes.c_int64()
        check(lib().be_server_stats(self._h, ctypes.byref(c), ctypes.byref(f), ctypes.byref(p50), ctypes.byref(p99),
                                    ctypes.byref(thr), ctypes.byref(pk), ctypes.byref(mi)))
        return {"completed": c.value, "failed": f.value, "p50_s": p50.value, "p99_s": p99.value,
                "throughput": thr.value, "peak_bytes": pk.value, "max_inflight": mi.value}

    def trace(self):
        """Completed requests since the last reset: array of rows (id, submit,
        admit, launched, done, stream), seconds."""
        n = ctypes.c_int64()
        check(lib().be_server_trace(self._h, None, 0, ctypes.byref(n)))
        rows = (ctypes.c_double * (6 * max(1, n.value)))()
        check(lib().be_server_trace(self._h, rows, n.value, ctypes.byref(n)))
        return np.frombuffer(rows, dtype=np.float64)[: 6 * n.value].reshape(-1, 6).copy()

    def reset_stats(self):
        check(lib().be_server_reset_stats(self._h))

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.be_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def _batch_arrays(items):
    """C arrays of be_batch_create / be_tune_batch for (einsum, buffers,
    outputs[, scalars]) items, and the objects they borrow."""
    keep = []
    n = len(items)
    es = (ctypes.c_void_p * max(1, n))()
    bptr = (ctypes.POINTER(Buf) * max(1, n))()
    optr = (ctypes.POINTER(Buf) * max(1, n))()
    nb = (ctypes.c_int32 * max(1, n))()
    no = (ctypes.c_int32 * max(1, n))()
    sptr = (ctypes.POINTER(ctypes.c_double) * max(1, n))()
    ns = (ctypes.c_int32 * max(1, n))()
    for k, item in enumerate(items):
        e, bufs, outs = item[0], item[1], item[2]
        scal = item[3] if len(item) > 3 else ()
        bl = _order(e, bufs)
        for t, (name, _, shape) in zip(bl, e.buffers):
            if tuple(t.shape) != shape or not t.is_cuda:
                raise BEError(ESHAPE, f"instance {k} buffer {name}: expected shape {shape}")
        for t in outs:
            if tuple(t.shape) != e.out_shape or not t.is_contiguous():
                raise BEError(ESHAPE, f"instance {k}: outputs must be dense of shape {e.out_shape}")
        bi = _bufs_torch(bl, keep)
        bo = _bufs_torch(outs, keep, dense_only=True)
        sc, nsc = _scalars(scal)
        keep += [bi, bo, sc, e, bl, outs]
        es[k] = e.handle.value
        bptr[k] = ctypes.cast(bi, ctypes.POINTER(Buf))
        optr[k] = ctypes.cast(bo, ctypes.POINTER(Buf))
        nb[k], no[k], ns[k] = len(bl), len(outs), nsc
        sptr[k] = ctypes.cast(sc, ctypes.POINTER(ctypes.c_double))
    return (es, bptr, nb, optr, no, sptr, ns), keep


class Batch:
    """Multi-instance executor over many (einsum, buffers, outputs) instances,
    replayed as one CUDA graph per run: generic instances as tiles of one
    persistent launch, element-shaped and (with cfg.split >= 1) dense FP64
    instances on their own strategies in concurrent graph branches."""

    def __init__(self, ctx, items, cfg: Config | None = None):
        arrays, keep = _batch_arrays(items)
        es, bptr, nb, optr, no, sptr, ns = arrays
        n = len(items)
        h = ctypes.c_void_p()
        check(lib().be_batch_create(ctx.handle if ctx else None, n, es, bptr, nb, optr, no, sptr, ns,
                                    ctypes.byref(cfg) if cfg else None, ctypes.byref(h)))
        self._h = h
        self._keep = keep

    def run(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        check(lib().be_batch_run(self._h, ctypes.c_void_p(stream.cuda_stream)))

    def info(self):
        r, t, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        check(lib().be_batch_info(self._h, ctypes.byref(r), ctypes.byref(t), ctypes.byref(w)))
        return {"rows": r.value, "tiles": t.value, "terms": w.value}

    def kinds(self):
        """Instances per strategy: {"generic": g, "element": m, "dense": d}."""
        g, m, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().be_batch_kinds(self._h, ctypes.byref(g), ctypes.byref(m), ctypes.byref(d)))
        return {"generic": g.value, "element": m.value, "dense": d.value}

    INSTANCE_KINDS = ("loop nest", "element", "dense", "factored", "dense factored")

    def instance_kind(self, k: int) -> str:
        """How instance k is evaluated: one of INSTANCE_KINDS ("dense" and
        "dense factored" run in split precision)."""
        v = ctypes.c_int32()
        check(lib().be_batch_instance_kind(self._h, k, ctypes.byref(v)))
        return self.INSTANCE_KINDS[v.value]

    def factored(self):
        """Factored instances, persistent launches (phases) per run and bytes of
        the intermediates' workspace."""
        n, q, w = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        check(lib().be_batch_factored(self._h, ctypes.byref(n), ctypes.byref(q), ctypes.byref(w)))
        return {"instances": n.value, "phases": q.value, "workspace_bytes": w.value}

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.be_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def tune_batch(ctx, items, base: Config | None = None, reps=5, stream=None):
    """be_tune_batch: time the batch's launch-shape candidates, record them
    under the batch key; returns (best Config, seconds, candidates timed)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    (es, bptr, nb, optr, no, sptr, ns), keep = _batch_arrays(items)
    best, sec, n = Config(), ctypes.c_double(), ctypes.c_int32()
    check(lib().be_tune_batch(ctx.handle, len(items), es, bptr, nb, optr, no, sptr, ns,
                              ctypes.byref(base) if base else None, int(reps), ctypes.c_void_p(stream.cuda_stream),
                              ctypes.byref(best), ctypes.byref(sec), ctypes.byref(n)))
    del keep
    return best, sec.value, n.value


def peak_probe(kind: str, reps=5) -> float:
    """Measured peak of the FP64 ("fp64") or FP32 ("fp32") pipe, TFLOP/s."""
    v = ctypes.c_double()
    check(lib().be_peak_probe({"fp64": 0, "fp32": 1}[kind], int(reps), ctypes.byref(v)))
    return v.value


def plan_strategy(ctx, e: Einsum, cfg: Config | None = None, precision=PREC_FP64) -> int:
    s = ctypes.c_int32()
    check(lib().be_plan_strategy(ctx.handle if ctx else None, e.handle, ctypes.byref(cfg) if cfg else None,
                                 precision, ctypes.byref(s)))
    return s.value
