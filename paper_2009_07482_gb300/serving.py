"""Serving layer over dag_server_*: model descriptors from workloads and host
buffers for requests.  Argument marshalling only; admission, launch and
completion run in the library's native serving loop."""
from __future__ import annotations

import ctypes as C
from typing import Dict, List, Optional

import numpy as np

from . import _binding as abi
from .dag import _np_dtype, describe, options


def activation_ids(w) -> List[int]:
    """Inputs that are not GEMM weights or biases: the per-request data."""
    weights = {n.b for n in w.nodes if n.op == "gemm"} | {n.bias for n in w.nodes if n.op == "gemm" and n.bias >= 0}
    return [i for i in w.input_ids() if i not in weights]


class Server:
    def __init__(self, workloads, weights: List[Dict[int, np.ndarray]], max_slots: int = 32,
                 hbm_reserve_bytes: int = 0, node_costs: Optional[List[Optional[List[float]]]] = None, opts=None):
        self.w = list(workloads)
        self._keep = []
        models = []
        for k, w in enumerate(self.w):
            acts = set(activation_ids(w))
            nodes, _, bufs = describe(w, streamed=acts)
            wptr = [0] * len(w.buffers)
            for i, a in weights[k].items():
                if i in acts:
                    continue
                b = w.buffers[i]
                a = np.ascontiguousarray(a, dtype=_np_dtype(b.dtype)).reshape(b.rows, b.cols)
                self._keep.append(a)
                wptr[i] = a.ctypes.data
            costs = node_costs[k] if node_costs else None
            models.append((nodes, bufs, wptr, costs))
        self.s = abi.dag_server_create(models, max_slots, hbm_reserve_bytes, opts)
        self.acts = [sorted(activation_ids(w)) for w in self.w]
        self.outs = [w.output_ids() for w in self.w]

    def set_default_io(self, model: int, inputs: Dict[int, np.ndarray]):
        """Pinned default request buffers of a model (used by the simulation)."""
        w = self.w[model]
        ins, outs = [], []
        for i in self.acts[model]:
            a = np.ascontiguousarray(inputs[i])
            p = abi.dag_host_alloc(a.nbytes)
            C.memmove(p, a.ctypes.data, a.nbytes)
            self._keep.append(("pinned", p))
            ins.append(p)
        for i in self.outs[model]:
            b = w.buffers[i]
            p = abi.dag_host_alloc(b.rows * b.cols * (4 if b.dtype == "f32" else 2))
            self._keep.append(("pinned", p))
            outs.append(p)
        abi.dag_server_set_io(self.s, model, ins, outs)

    def submit(self, model: int, inputs: Dict[int, np.ndarray]):
        """Queue one request; returns (ticket, output arrays filled on completion)."""
        w = self.w[model]
        ins = []
        for i in self.acts[model]:
            a = np.ascontiguousarray(inputs[i], dtype=_np_dtype(w.buffers[i].dtype))
            self._keep.append(a)
            ins.append(a.ctypes.data)
        outs = {i: np.empty((w.buffers[i].rows, w.buffers[i].cols), _np_dtype(w.buffers[i].dtype))
                for i in self.outs[model]}
        self._keep.extend(outs.values())
        t = abi.dag_server_submit(self.s, model, ins, [outs[i].ctypes.data for i in self.outs[model]])
        return t, outs

    def close(self):
        if self.s:
            abi.dag_server_destroy(self.s)
            self.s = None
        for k in self._keep:
            if isinstance(k, tuple) and k[0] == "pinned":
                abi.dag_host_free(k[1])
        self._keep = []
