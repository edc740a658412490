"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module is deliberately free of the DAG method's arithmetic: it only draws
numbers, rounds them once to the storage dtype of a buffer, and describes the
shape of a workload (which buffers exist, which node reads which buffer).  Both
the FP64 oracle (``oracle/``) and the GPU library receive exactly the arrays
produced here, so any difference between them comes from the computation.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser published
by Vigna).  Stream element ``i`` of seed ``s`` is ``mix(s + (i+1)*0x9E3779B97F4A7C15)``.
Uniform in [-1,1): ``(u >> 11) * 2**-53 * 2 - 1``.  Normal: Box-Muller on two
consecutive uniforms in (0,1].
"""
from __future__ import annotations

import ctypes as _C
import os as _os
import subprocess as _sp
import threading as _th

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

F32 = "f32"
BF16 = "bf16"
DTYPES = (F32, BF16)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Elements ``offset .. offset+n-1`` of the SplitMix64 stream of ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """float64 array, uniform on [lo, hi) from the 53 high bits of each draw."""
    n = int(np.prod(shape))
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (lo + (hi - lo) * u).reshape(shape)


def normal(seed: int, shape, std: float = 1.0) -> np.ndarray:
    """float64 array, N(0, std^2) by Box-Muller (cosine branch) on pairs of draws."""
    n = int(np.prod(shape))
    r = splitmix64(seed, 2 * n)
    u1 = ((r[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0,1]
    u2 = (r[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return (std * z).reshape(shape)


def f32_to_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even); uint16 bits."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32)
    lsb = (b >> np.uint32(16)) & np.uint32(1)
    r = (b + np.uint32(0x7FFF) + lsb) >> np.uint32(16)
    return r.astype(np.uint16)


def bf16_bits_to_f32(h: np.ndarray) -> np.ndarray:
    """Widen bfloat16 bit patterns (uint16) to float32 exactly."""
    return (np.asarray(h, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def to_storage(x: np.ndarray, dtype: str) -> np.ndarray:
    """Store a float64 draw in a buffer dtype: float32 array, or uint16 bf16 bits.

    Inputs are rounded f64 -> f32 -> bf16; this is a property of the input
    recipe only (both sides read the same stored bits).
    """
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    if dtype == F32:
        return x32
    if dtype == BF16:
        return f32_to_bf16_bits(x32)
    raise ValueError(f"unknown dtype {dtype!r}")


def storage_to_f64(a: np.ndarray, dtype: str) -> np.ndarray:
    """Widen a stored buffer to float64 (exact)."""
    if dtype == F32:
        return np.asarray(a, dtype=np.float32).astype(np.float64)
    if dtype == BF16:
        return bf16_bits_to_f32(a).astype(np.float64)
    raise ValueError(f"unknown dtype {dtype!r}")


def np_storage_dtype(dtype: str):
    return np.float32 if dtype == F32 else np.uint16


# ---------------------------------------------------------------------------
# fast fill (C, multithreaded) with the same definitions, straight to storage
# ---------------------------------------------------------------------------
_HERE = _os.path.dirname(_os.path.abspath(__file__))
_GEN_SRC = _os.path.join(_HERE, "_gen.c")
_GEN_LIB = _os.path.join(_HERE, "_build", "libsynthgen.so")
_gen = None
_gen_lock = _th.Lock()


def build(force: bool = False) -> str:
    _os.makedirs(_os.path.dirname(_GEN_LIB), exist_ok=True)
    if force or not _os.path.exists(_GEN_LIB) or _os.path.getmtime(_GEN_LIB) < _os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + f".{_os.getpid()}.tmp"
        _sp.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", _GEN_SRC,
                        "-o", tmp, "-lm"])
        _os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _lib():
    global _gen
    with _gen_lock:
        if _gen is None:
            L = _C.CDLL(build())
            L.synth_fill.argtypes = [_C.c_int, _C.c_uint64, _C.c_double, _C.c_double, _C.c_int64, _C.c_int,
                                     _C.c_void_p, _C.c_int]
            L.synth_fill.restype = _C.c_int
            _gen = L
    return _gen


def fill(kind: str, seed: int, shape, dtype: str, a: float, b: float = 0.0) -> np.ndarray:
    """Storage array (f32, or bf16 bits) of uniform(lo=a, hi=b) or normal(std=a) draws."""
    n = int(np.prod(shape))
    out = np.empty(n, np_storage_dtype(dtype))
    _lib().synth_fill(0 if kind == "uniform" else 1, seed & 0xFFFFFFFFFFFFFFFF, float(a), float(b), n,
                      1 if dtype == BF16 else 0, out.ctypes.data, min(32, _os.cpu_count() or 1))
    return out.reshape(shape)
