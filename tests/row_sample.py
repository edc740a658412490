"""Row-sampled oracle checks at full workload sizes.

In the MLP, fork-join and random layered DAGs every kernel is row-wise: row i
of a kernel's output depends on row i of its row-space inputs (GEMM A,
elementwise and softmax inputs) and on whole weight operands (GEMM B, bias).
So the oracle run on the same DAG with only rows R of every row-space buffer
gives rows R of every output exactly as the full DAG defines them."""
import dataclasses

import numpy as np

import oracle


def row_space(w):
    weights = set()
    for n in w.nodes:
        if n.op == "gemm":
            weights.add(n.b)
            if n.bias >= 0:
                weights.add(n.bias)
    rs = set()
    for i, b in enumerate(w.buffers):
        if b.role != "input" or i not in weights:
            rs.add(i)
    assert not (rs & weights), "a buffer is both a weight and row-space"
    assert all(n.batch == 1 for n in w.nodes if n.op == "gemm"), "batched GEMMs are not row-wise"
    return rs


def oracle_rows(w, inputs, rows):
    """Oracle store of the row subset; rows index every row-space buffer."""
    rs = row_space(w)
    ws = w.clone()
    for i in rs:
        ws.buffers[i] = dataclasses.replace(ws.buffers[i], rows=len(rows))
    sub = {i: (a[rows] if i in rs else a) for i, a in inputs.items()}
    return ws, oracle.run(ws, sub)
