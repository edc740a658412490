"""FP64 CPU oracle for application DAGs -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The library path never does: it shares no code,
header, table or helper with the CUDA executor.

``oracle.c`` holds the arithmetic (see its header for the definitions and the
passages of the paper they follow).  This module compiles it with gcc (no
fused multiply-add contraction, so x86 and Arm hosts give identical bits),
marshals workload descriptions into its structs, and returns numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

from synth import BF16, F32, np_storage_dtype

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPS = {"gemm": 0, "add": 1, "softmax": 2, "unary": 3}
ACTS = {"none": 0, "relu": 1, "gelu": 2}
DT = {F32: 0, BF16: 1}
ERRORS = {0: "OK", 1: "EINVAL", 2: "ECYCLE", 3: "ESHAPE", 4: "EDTYPE", 5: "EMULTIWRITER", 6: "ENOMEM"}


class Buf(C.Structure):
    _fields_ = [("rows", C.c_int32), ("cols", C.c_int32), ("dtype", C.c_int32),
                ("view_of", C.c_int32), ("col_offset", C.c_int32)]


class Nd(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32), ("bias", C.c_int32),
                ("out", C.c_int32), ("trans_b", C.c_int32), ("act", C.c_int32), ("batch", C.c_int32),
                ("scale", C.c_double)]


class Tile(C.Structure):
    _fields_ = [("node", C.c_int32), ("r0", C.c_int32), ("r1", C.c_int32), ("c0", C.c_int32),
                ("c1", C.c_int32)]


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"oracle: {ERRORS.get(code, code)} {what}")


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, plain C99, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        compile_source(_SRC, tmp)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_source(src: str, out: str) -> None:
    """gcc, plain C99, no fused multiply-add contraction (x86 and Arm agree)."""
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-D_DEFAULT_SOURCE", src, "-o", out, "-lm"])


def load(path: str):
    """Open a compiled oracle library and declare its entry points.  ``lib()``
    uses the build of ``oracle.c``; the mutation tests load deliberately broken
    copies through here."""
    L = C.CDLL(path)
    P = C.POINTER
    L.or_f64_to_bf16.argtypes = [C.c_double]
    L.or_f64_to_bf16.restype = C.c_uint16
    L.or_validate.argtypes = [P(Buf), C.c_int, P(Nd), C.c_int]
    L.or_topo_order.argtypes = [P(Buf), C.c_int, P(Nd), C.c_int, P(C.c_int32)]
    L.or_is_topological.argtypes = [P(Buf), P(Nd), C.c_int, P(C.c_int32)]
    L.or_run.argtypes = [P(Buf), C.c_int, P(Nd), C.c_int, P(C.c_void_p), P(C.c_int32)]
    L.or_run_node.argtypes = [P(Buf), C.c_int, P(Nd), C.c_int, P(C.c_void_p), C.c_int,
                              C.c_int64, C.c_int64]
    L.or_run_tiles.argtypes = [P(Buf), C.c_int, P(Nd), C.c_int, P(C.c_void_p), P(Tile), C.c_int,
                               P(C.c_int32)]
    L.or_make_tiles.argtypes = [P(Buf), P(Nd), C.c_int, C.c_int, C.c_int, P(Tile), C.c_int]
    L.or_tile_deps.argtypes = [P(Buf), P(Nd), P(Tile), C.c_int, P(C.c_int32), C.c_int]
    L.or_check_trace.argtypes = [P(Buf), C.c_int, P(Nd), C.c_int, P(Tile), C.c_int,
                                 P(C.c_uint32), P(C.c_uint32), P(C.c_int32), P(C.c_int32)]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


# ---------------------------------------------------------------------------
def _structs(w):
    bufs = (Buf * len(w.buffers))()
    for i, b in enumerate(w.buffers):
        bufs[i] = Buf(b.rows, b.cols, DT[b.dtype], b.view_of, b.col_offset)
    nodes = (Nd * max(1, len(w.nodes)))()
    for i, n in enumerate(w.nodes):
        nodes[i] = Nd(OPS[n.op], n.a, n.b, n.bias, n.out, n.trans_b, ACTS[n.act], n.batch, float(n.scale))
    return bufs, nodes


def f64_to_bf16(x: float) -> int:
    return int(lib().or_f64_to_bf16(float(x)))


def validate(w) -> int:
    bufs, nodes = _structs(w)
    return int(lib().or_validate(bufs, len(w.buffers), nodes, len(w.nodes)))


def topo_order(w) -> List[int]:
    bufs, nodes = _structs(w)
    out = (C.c_int32 * max(1, len(w.nodes)))()
    rc = lib().or_topo_order(bufs, len(w.buffers), nodes, len(w.nodes), out)
    if rc:
        raise OracleError(rc, "topo_order")
    return list(out[: len(w.nodes)])


def is_topological(w, order: Sequence[int]) -> bool:
    bufs, nodes = _structs(w)
    o = (C.c_int32 * max(1, len(order)))(*order)
    return bool(lib().or_is_topological(bufs, nodes, len(w.nodes), o))


def _storage(w, inputs: Dict[int, np.ndarray], poison: bool):
    """Allocate dense storage for every root buffer; copy inputs; poison the rest with NaN."""
    store = {}
    for i, b in enumerate(w.buffers):
        if b.view_of >= 0:
            continue
        dt = np_storage_dtype(b.dtype)
        if i in inputs:
            a = np.ascontiguousarray(inputs[i], dtype=dt).reshape(b.rows, b.cols).copy()
        elif poison:
            a = np.full((b.rows, b.cols), np.nan, np.float32) if b.dtype == F32 else \
                np.full((b.rows, b.cols), 0x7FC0, np.uint16)
        else:
            a = np.zeros((b.rows, b.cols), dt)
        store[i] = a
    ptrs = (C.c_void_p * len(w.buffers))()
    for i in range(len(w.buffers)):
        ptrs[i] = store[i].ctypes.data if i in store else None
    return store, ptrs


def run(w, inputs: Dict[int, np.ndarray], order: Optional[Sequence[int]] = None,
        poison: bool = True) -> Dict[int, np.ndarray]:
    """Execute the DAG in topological order; returns every root buffer (storage dtype)."""
    bufs, nodes = _structs(w)
    store, ptrs = _storage(w, inputs, poison)
    o = None if order is None else (C.c_int32 * max(1, len(order)))(*order)
    rc = lib().or_run(bufs, len(w.buffers), nodes, len(w.nodes), ptrs, o)
    if rc:
        raise OracleError(rc, w.name)
    return store


def view(w, store: Dict[int, np.ndarray], bid: int) -> np.ndarray:
    """The (rows x cols) array of buffer `bid`, resolving column-slice views."""
    b = w.buffers[bid]
    if b.view_of < 0:
        return store[bid]
    return store[b.view_of][:, b.col_offset:b.col_offset + b.cols]


def run_node_rows(w, store: Dict[int, np.ndarray], k: int, r0: int, r1: int) -> None:
    """Run rows [r0, r1) of kernel k in place on `store` (bounded CPU samples)."""
    bufs, nodes = _structs(w)
    ptrs = (C.c_void_p * len(w.buffers))()
    for i in range(len(w.buffers)):
        ptrs[i] = store[i].ctypes.data if i in store else None
    rc = lib().or_run_node(bufs, len(w.buffers), nodes, len(w.nodes), ptrs, k, r0, r1)
    if rc:
        raise OracleError(rc, "run_node")


def make_tiles(w, bm: int, bn: int) -> np.ndarray:
    """The oracle's own plain tiling: returns an (n, 5) int array of (node, r0, r1, c0, c1)."""
    bufs, nodes = _structs(w)
    cap = 1 << 20
    t = (Tile * cap)()
    n = lib().or_make_tiles(bufs, nodes, len(w.nodes), bm, bn, t, cap)
    if n < 0:
        raise OracleError(1, "too many tiles")
    return np.array([(x.node, x.r0, x.r1, x.c0, x.c1) for x in t[:n]], dtype=np.int32).reshape(-1, 5)


def _tiles(tiles) -> "C.Array":
    tiles = np.asarray(tiles, dtype=np.int32).reshape(-1, 5)
    arr = (Tile * max(1, len(tiles)))()
    for i, r in enumerate(tiles):
        arr[i] = Tile(*[int(v) for v in r])
    return arr


def tile_deps(w, tiles) -> List[tuple]:
    """Edges (u, v): tile v reads a region tile u writes."""
    bufs, nodes = _structs(w)
    t = _tiles(tiles)
    nt = len(np.asarray(tiles).reshape(-1, 5))
    cap = max(16, nt * nt)
    e = (C.c_int32 * (2 * cap))()
    k = lib().or_tile_deps(bufs, nodes, t, nt, e, cap)
    if k < 0:
        raise OracleError(1, "tile_deps cap")
    return [(e[2 * i], e[2 * i + 1]) for i in range(k)]


def run_tiles(w, inputs: Dict[int, np.ndarray], tiles, order: Optional[Sequence[int]] = None) -> Dict[int, np.ndarray]:
    """Tiled simulator on NaN-poisoned storage; tiles run in `order`."""
    bufs, nodes = _structs(w)
    store, ptrs = _storage(w, inputs, poison=True)
    t = _tiles(tiles)
    nt = len(np.asarray(tiles).reshape(-1, 5))
    o = None if order is None else (C.c_int32 * max(1, nt))(*order)
    rc = lib().or_run_tiles(bufs, len(w.buffers), nodes, len(w.nodes), ptrs, t, nt, o)
    if rc:
        raise OracleError(rc, "run_tiles")
    return store


def check_trace(w, tiles, start, end):
    """Legality of an observed tile execution (see or_check_trace): (code, bad_u, bad_v)."""
    bufs, nodes = _structs(w)
    t = _tiles(tiles)
    nt = len(np.asarray(tiles).reshape(-1, 5))
    s = np.ascontiguousarray(start, dtype=np.uint32)
    e = np.ascontiguousarray(end, dtype=np.uint32)
    bu, bv = C.c_int32(-1), C.c_int32(-1)
    rc = lib().or_check_trace(bufs, len(w.buffers), nodes, len(w.nodes), t, nt,
                              s.ctypes.data_as(C.POINTER(C.c_uint32)), e.ctypes.data_as(C.POINTER(C.c_uint32)),
                              C.byref(bu), C.byref(bv))
    return int(rc), int(bu.value), int(bv.value)


def rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    """Normwise infinity-relative error max|g - r| / max|r| (both widened to f64)."""
    g = np.asarray(got, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    den = max(float(np.max(np.abs(r))) if r.size else 0.0, 1e-30)
    return float(np.max(np.abs(g - r))) / den if r.size else 0.0
