"""Shared helpers of the GPU tests: run a workload through the C ABI and
compare every computed buffer with the FP64 oracle."""
import numpy as np

import oracle
from tests import trace_check
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag
from synth import BF16, F32, storage_to_f64

# per-buffer normwise tolerances: max|g - r| / max|r|
TOL = {F32: 1e-5, BF16: 2e-2}


def bf16_tainted(w):
    """Buffers whose stored values depend on bf16 arithmetic: a buffer stored
    as bf16 (rounded once where it is written, f32 -> bf16 on the device and
    f64 -> bf16 in the oracle, which can differ by one bf16 ulp), the output
    of a GEMM with bf16 operands (f32 accumulation of bf16 products), and
    everything written downstream of either.  Input buffers are exact on both
    sides as stored, so they taint nothing.  A parent buffer written through
    column-slice views is tainted when any of its views is."""
    tainted = set()
    views = {}
    for i, b in enumerate(w.buffers):
        if b.view_of >= 0:
            views.setdefault(b.view_of, []).append(i)

    def reads(bid):
        return bid in tainted or any(v in tainted for v in views.get(bid, ()))

    order = _topo(w)
    for k in order:
        n = w.nodes[k]
        t = (w.buffers[n.out].dtype == BF16
             or (n.op == "gemm" and w.buffers[n.a].dtype == BF16)
             or any(reads(x) for x in (n.a, n.b, n.bias) if x >= 0))
        if t:
            tainted.add(n.out)
    for parent, vs in views.items():
        if any(v in tainted for v in vs):
            tainted.add(parent)
    return tainted


def _topo(w):
    """Node ids in an order where every writer precedes its readers."""
    writer = {}
    for k, n in enumerate(w.nodes):
        writer[n.out] = k
        if w.buffers[n.out].view_of >= 0:
            writer.setdefault(("parent", w.buffers[n.out].view_of), []).append(k)
    deps = []
    for n in w.nodes:
        d = set()
        for x in (n.a, n.b, n.bias):
            if x < 0:
                continue
            if x in writer:
                d.add(writer[x])
            d.update(writer.get(("parent", x), ()))
        deps.append(d)
    done, order = set(), []
    pending = list(range(len(w.nodes)))
    while pending:
        rest = []
        for k in pending:
            if deps[k] <= done:
                done.add(k)
                order.append(k)
            else:
                rest.append(k)
        assert len(rest) < len(pending), "cyclic workload"
        pending = rest
    return order


_TAINT_CACHE = {}


def node_tolerance(w, bid):
    """Per-buffer tolerance: bf16's (2e-2) for a buffer whose values depend on
    bf16 arithmetic (see bf16_tainted), f32's (1e-5) for every other buffer,
    also inside a batch that holds bf16 DAGs beside f32 ones."""
    key = id(w)
    hit = _TAINT_CACHE.get(key)
    if hit is None or hit[0] is not w:
        hit = (w, bf16_tainted(w))
        _TAINT_CACHE[key] = hit
    return TOL[BF16] if bid in hit[1] or w.buffers[bid].dtype == BF16 else TOL[F32]


def written_buffers(w, fused=None):
    """Buffers the DAG's kernels write.  With the library's fusion map
    (kernel -> the kernel whose tiles compute it, or -1), a buffer that one
    kernel of a fused group writes and another of the group reads is never
    written."""
    outs = {n.out for n in w.nodes}
    groups = {}
    for v, h in enumerate(fused or []):
        if h >= 0:
            groups.setdefault(h, {h}).add(v)
    for g in groups.values():
        for x in g:
            for y in g:
                if x != y and w.nodes[y].out in (w.nodes[x].a, w.nodes[x].b):
                    outs.discard(w.nodes[y].out)
    return sorted(outs)


def run_gpu(w, inputs, coarse=False, opts=None, resident=False, keep=False):
    d = Dag(w, opts, resident_inputs=resident)
    d.set_inputs(inputs)
    d.run(coarse=coarse)
    outs = {b: d.output(b) for b in written_buffers(w, d.fusion())}
    if keep:
        return d, outs
    d.close()
    return outs


def compare(w, got, ref_store, bids=None):
    """{buffer: rel_err}; raises AssertionError above tolerance."""
    errs = {}
    for b in bids or sorted(got):
        dt = w.buffers[b].dtype
        g = storage_to_f64(got[b], dt)
        r = storage_to_f64(oracle.view(w, ref_store, b), dt)
        assert np.all(np.isfinite(g)), f"buffer {b} ({w.buffers[b].name}) has non-finite values"
        e = oracle.rel_err(g, r)
        errs[b] = e
        tol = node_tolerance(w, b)
        assert e <= tol, f"buffer {b} ({w.buffers[b].name}): rel err {e:.3e} > {tol}"
    return errs


def check_trace(w, d):
    recs = d.trace()
    trace_check.check(w, [(r.node, r.r0, r.r1, r.c0, r.c1) for r in recs], [r.split for r in recs],
                      [r.start_ticket for r in recs], [r.end_ticket for r in recs], d.fusion(), d.merges())
    return recs


def bits_equal(a, b):
    return all(np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)) for k in a)
