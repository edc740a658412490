"""Convenience layer over the C ABI: build the ABI structs from a workload
description and move numpy arrays in and out.  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
from typing import Dict, Optional

import numpy as np

from . import _binding as abi

_DT = {"f32": abi.DAG_F32, "bf16": abi.DAG_BF16}
_OP = {"gemm": abi.DAG_OP_GEMM, "add": abi.DAG_OP_ADD, "softmax": abi.DAG_OP_SOFTMAX, "unary": abi.DAG_OP_UNARY}
_ACT = {"none": abi.DAG_ACT_NONE, "relu": abi.DAG_ACT_RELU, "gelu": abi.DAG_ACT_GELU}


def _np_dtype(dt: str):
    return np.float32 if dt == "f32" else np.uint16


def describe(w, resident_inputs: bool = False, streamed=None):
    """(nodes, edges, buffers) ABI structs for a workload with .buffers/.nodes.

    Inputs are streamed (uploaded each submit) unless `resident_inputs`, or
    unless their id is not in `streamed` when that set is given.
    """
    bufs = []
    for i, b in enumerate(w.buffers):
        flags = 0
        if b.role == "input":
            flags |= abi.DAG_BUF_INPUT
            if resident_inputs or (streamed is not None and i not in streamed):
                flags |= abi.DAG_BUF_RESIDENT
        if b.role == "output":
            flags |= abi.DAG_BUF_OUTPUT
        bufs.append(abi.dag_buffer_desc(b.rows, b.cols, _DT[b.dtype], flags, b.view_of, b.col_offset))
    nodes = []
    for n in w.nodes:
        nodes.append(abi.dag_node_desc(_OP[n.op], n.a, n.b, n.bias, n.out, n.trans_b, _ACT[n.act],
                                       float(n.scale), n.batch, getattr(n, "component", 0)))
    edges = [abi.dag_edge(*e) for e in getattr(w, "edges", [])]  # optional explicit k_i,b_r -> k_j,b_s
    return nodes, edges, bufs


def options(**kw) -> abi.dag_options:
    o = abi.dag_options()
    costs = kw.pop("node_cost_us", None)
    for k, v in kw.items():
        setattr(o, k, v)
    if costs is not None:
        arr = (C.c_float * len(costs))(*[float(c) for c in costs])
        o.node_cost_us = C.cast(arr, C.POINTER(C.c_float))
        o._keep = arr  # keep alive with the struct
    return o


class Dag:
    """One created DAG on the current CUDA device."""

    def __init__(self, w, opts: Optional[abi.dag_options] = None, resident_inputs: bool = False, streamed=None,
                 _handle=None):
        self.w = w
        self._opts = opts
        if _handle is None:
            nodes, edges, bufs = describe(w, resident_inputs, streamed)
            _handle = abi.dag_create(nodes, edges, bufs, opts)
        self.h = _handle
        self._keep: Dict[int, np.ndarray] = {}
        self._pinned = []

    @classmethod
    def batch(cls, workloads, opts: Optional[abi.dag_options] = None, resident_inputs: bool = False,
              streamed=None):
        """Many DAGs in one plan and one persistent launch (dag_batch_create).
        Buffer ids (also in `streamed`) follow synth.workloads.concat(workloads)."""
        from synth.workloads import concat
        items, off = [], 0
        for w in workloads:
            local = None if streamed is None else {i - off for i in streamed if off <= i < off + len(w.buffers)}
            nodes, _, bufs = describe(w, resident_inputs, local)
            items.append((nodes, bufs))
            off += len(w.buffers)
        h = abi.dag_batch_create(items, opts)
        return cls(concat(workloads), opts, _handle=h)

    # -- data -------------------------------------------------------------
    def set_inputs(self, inputs: Dict[int, np.ndarray], pinned: bool = False) -> None:
        for bid, arr in inputs.items():
            b = self.w.buffers[bid]
            a = np.ascontiguousarray(arr, dtype=_np_dtype(b.dtype)).reshape(b.rows, b.cols)
            if pinned:
                p = abi.dag_host_alloc(a.nbytes)
                self._pinned.append(p)
                dst = np.ctypeslib.as_array((C.c_uint8 * a.nbytes).from_address(p))
                dst[:] = a.view(np.uint8).reshape(-1)
                abi.dag_set_input(self.h, bid, p)
                self._keep[bid] = dst
            else:
                self._keep[bid] = a
                abi.dag_set_input(self.h, bid, a.ctypes.data)

    def clear_input(self, bid: int) -> None:
        """Forget the host pointer; the device copy stays (later submits reuse it)."""
        abi.dag_set_input(self.h, bid, None)

    def output(self, bid: int) -> np.ndarray:
        b = self.w.buffers[bid]
        out = np.empty((b.rows, b.cols), _np_dtype(b.dtype))
        abi.dag_get_output(self.h, bid, out.ctypes.data)
        return out

    # -- execution ----------------------------------------------------------
    def submit(self, stream: int = 0) -> None:
        abi.dag_submit(self.h, stream)

    def submit_coarse(self, stream: int = 0) -> None:
        abi.dag_submit_coarse(self.h, stream)

    def wait(self, timeout_ns: int = 30_000_000_000) -> int:
        return abi.dag_wait(self.h, timeout_ns)

    def run(self, coarse: bool = False) -> None:
        (self.submit_coarse if coarse else self.submit)()
        abi.check(self.wait(), "dag_wait")

    def run_cq(self, n_queues: int = 1, components: int = abi.DAG_TC_WHOLE, fifo: int = 0, times: bool = False):
        """The paper's Alg. 1 on CUDA streams (dag_submit_cq), synchronous.
        Returns the dag_cq_result, plus per-kernel (start_us, end_us) arrays
        when times is set."""
        r, ts, te = abi.dag_submit_cq(self.h, n_queues, components, fifo, 0, len(self.w.nodes) if times else 0)
        return (r, ts, te) if times else r

    def trace(self):
        return abi.dag_trace_get(self.h)

    def write_cq_chrome_trace(self, path: str, n_queues: int = 1, components: int = abi.DAG_TC_WHOLE,
                              fifo: int = 0):
        """Run the paper's Alg. 1 on streams (run_cq) and write each kernel's
        window as a Chrome trace-event file, one process per task component
        (the Gantt view of the paper's §5).  Returns the dag_cq_result."""
        import json
        from .trace import kernel_windows_trace
        r, ts, te = self.run_cq(n_queues=n_queues, components=components, fifo=fifo, times=True)
        n = len(self.w.nodes)
        if components == abi.DAG_TC_GIVEN:
            groups = [getattr(x, "component", 0) for x in self.w.nodes]
        elif components == abi.DAG_TC_WHOLE:
            groups = [0] * n
        else:
            groups = list(range(n))
        names = [x.name or f"{x.op}{i}" for i, x in enumerate(self.w.nodes)]
        with open(path, "w") as f:
            json.dump(kernel_windows_trace(ts, te, names, groups), f)
        return r

    def write_chrome_trace(self, path: str) -> None:
        """The last traced submit as a Chrome trace-event file (a Gantt chart per
        SM; needs options(trace=1)).  See trace.py."""
        from .trace import write_chrome_trace
        names = [n.name or f"{n.op}{i}" for i, n in enumerate(self.w.nodes)]
        write_chrome_trace(path, self.trace(), names)

    def tiles(self):
        return abi.dag_tiles_get(self.h)

    def fusion(self):
        return abi.dag_fusion_get(self.h)

    def merges(self):
        """(leader, column offset) per kernel: sibling GEMMs the planner merged."""
        return abi.dag_merge_get(self.h)

    def plan(self):
        return abi.dag_plan_get(self.h)

    def close(self) -> None:
        if self.h:
            abi.dag_destroy(self.h)
            self.h = None
        for p in self._pinned:
            abi.dag_host_free(p)
        self._pinned = []
        self._keep = {}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
