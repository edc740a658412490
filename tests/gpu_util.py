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


def node_tolerance(w, bid):
    """bf16 tolerance for anything downstream of a bf16 GEMM, else f32's."""
    for n in w.nodes:
        if n.op == "gemm" and w.buffers[n.a].dtype == BF16:
            return TOL[BF16]
    return TOL[w.buffers[bid].dtype] if w.buffers[bid].dtype == BF16 else TOL[F32]


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
                      [r.start_ticket for r in recs], [r.end_ticket for r in recs], d.fusion())
    return recs


def bits_equal(a, b):
    return all(np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)) for k in a)
