"""Epilogue fusion, host side: which elementwise kernels the planner runs
inside a GEMM epilogue, and the trace check that a fused tile's epilogue
waited for its other operands (a planted mistake must be caught)."""
import numpy as np
import pytest

from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300 import dag as dagmod
from synth import BF16, F32
from synth.workloads import Workload, branchy_mlp, fork_join
from tests import trace_check


def _fusion(w, **opt):
    n, e, b = dagmod.describe(w, resident_inputs=True)
    return abi.dag_fusion_host(n, e, b, dagmod.options(**opt))


def _names(w, fused):
    return {w.nodes[v].name: w.nodes[h].name for v, h in enumerate(fused) if h >= 0}


ALL = abi.DAG_FUSE_ALL


def test_branchy_mlp_add_tree_fuses_into_the_last_branch_layers():
    # with adds fused: add0_0 = fc0_2 + fc1_2 and then add1_0 = add0_0 + add0_1
    # run in fc0_2's epilogue; add0_1 = fc2_2 + fc3_2 in fc2_2's.  By default
    # (no fusion) and with activations only, nothing fuses.
    for dt in (BF16, F32):
        w = branchy_mlp(dt, batch=256, width=512, hidden=1024, out=256)
        assert _names(w, _fusion(w, fuse=ALL)) == {"add0_0": "fc0_2", "add1_0": "fc0_2", "add0_1": "fc2_2"}
        assert all(h < 0 for h in _fusion(w))
        assert all(h < 0 for h in _fusion(w, fuse=abi.DAG_FUSE_ACT))
    # f32 GEMMs on the SM cores have their own epilogue: nothing fuses
    w = branchy_mlp(F32, batch=256, width=512, hidden=1024, out=256)
    assert all(h < 0 for h in _fusion(w, fuse=ALL, f32_gemm=abi.DAG_F32_GEMM_SIMT))


def test_fork_join_add_fuses_into_the_first_branch():
    w = fork_join(256)
    assert _names(w, _fusion(w, fuse=ALL)) == {"K3": "K1"}


def _gemm(w, M, N, K, out_role="inter", out_dt=BF16, dt=BF16, seed=0):
    A = w.buf(M, K, dt, "input", ("uniform", seed + 1))
    B = w.buf(K, N, dt, "input", ("uniform", seed + 2))
    C = w.buf(M, N, out_dt, out_role)
    return w.node("gemm", A, C, b=B), C


def test_fusion_rules():
    # a GEMM output that is also read by another kernel, or is a DAG output,
    # or is read through a view, stays in memory
    fa = dict(fuse=ALL)
    w = Workload("two_readers")
    g, C = _gemm(w, 128, 128, 64)
    w.node("unary", C, w.buf(128, 128, F32, "output"), act="relu")
    w.node("unary", C, w.buf(128, 128, F32, "output"), act="gelu")
    assert all(h < 0 for h in _fusion(w, **fa))
    w = Workload("gemm_output_is_a_sink")
    g, C = _gemm(w, 128, 128, 64, out_role="output")
    w.node("unary", C, w.buf(128, 128, F32, "output"), act="relu")
    assert all(h < 0 for h in _fusion(w, **fa))
    w = Workload("read_through_a_view")
    g, C = _gemm(w, 128, 128, 64)
    V = w.buf(128, 64, BF16, "inter", view_of=C, col_offset=64)
    w.node("unary", V, w.buf(128, 64, F32, "output"), act="relu")
    assert all(h < 0 for h in _fusion(w, **fa))
    # x + x reads the GEMM output twice: not fused
    w = Workload("self_add")
    g, C = _gemm(w, 128, 128, 64)
    w.node("add", C, w.buf(128, 128, F32, "output"), b=C)
    assert all(h < 0 for h in _fusion(w, **fa))
    # a softmax is row-wide: not fused; an activation then an add: both, in order
    w = Workload("chain")
    g, C = _gemm(w, 128, 128, 64)
    S = w.buf(128, 128, BF16)
    u = w.node("unary", C, S, act="gelu")
    X = w.buf(128, 128, F32, "input", ("uniform", 9))
    T = w.buf(128, 128, F32)
    a = w.node("add", X, T, b=S)
    w.node("softmax", T, w.buf(128, 128, F32, "output"))
    assert _fusion(w, **fa) == [-1, g, g, -1]
    assert _fusion(w, fuse=abi.DAG_FUSE_ACT) == [-1, g, -1, -1]   # activations only
    assert _fusion(w) == [-1, -1, -1, -1]                         # default: none
    # at most two kernels per GEMM
    w = Workload("long_chain")
    g, C = _gemm(w, 128, 128, 64)
    prev = C
    for i in range(4):
        nxt = w.buf(128, 128, BF16, "output" if i == 3 else "inter")
        w.node("unary", prev, nxt, act="relu")
        prev = nxt
    assert _fusion(w, **fa) == [-1, g, g, -1, -1]


def _serial_tickets(t):
    start = np.arange(len(t), dtype=np.int64) * 2
    return start, start + 1


def test_trace_check_catches_an_epilogue_that_did_not_wait():
    """Queue order is legal; moving the tile that produces a fused add's other
    operand after the fused tile that reads it must be reported."""
    w = fork_join(256)
    n, e, b = dagmod.describe(w, resident_inputs=True)
    opts = dagmod.options(tile_override=64, fuse=ALL)
    t, _ = abi.dag_plan_host(n, e, b, opts, 148)
    fused = abi.dag_fusion_host(n, e, b, opts)
    start, end = _serial_tickets(t)
    trace_check.check(w, t[:, :5], t[:, 5] >> 16, start, end, fused)
    k1 = [i for i in range(len(t)) if t[i, 0] == 1]       # K1 tiles: they also compute K3 = C1 + C2
    k2 = [i for i in range(len(t)) if t[i, 0] == 2]       # K2 tiles write C2
    i = k1[0]
    j = next(j for j in k2 if t[j, 1] == t[i, 1] and t[j, 3] == t[i, 3])  # the K2 tile of the same region
    late_start, late_end = start.copy(), end.copy()
    late_start[j], late_end[j] = start[i] + 10 ** 6, end[i] + 10 ** 6
    with pytest.raises(AssertionError):
        trace_check.check(w, t[:, :5], t[:, 5] >> 16, late_start, late_end, fused)
    # without the fusion map the trace is not even complete (K3 has no tiles)
    with pytest.raises(AssertionError):
        trace_check.check(w, t[:, :5], t[:, 5] >> 16, start, end)


def _split_plan():
    """The branchy MLP's host plan: its last GEMM is split in K (partials store
    sums, a finishing partial adds them and writes the region)."""
    w = branchy_mlp(BF16)
    n, e, b = dagmod.describe(w, resident_inputs=True)
    t, _ = abi.dag_plan_host(n, e, b, None, 148)
    split = t[:, 5] >> 16
    S, idx = split & 0xFF, split >> 8
    assert (S > 1).any()
    start = np.arange(len(t), dtype=np.int64) * 2    # tiles one at a time, in queue order
    return w, t, split, S, idx, start


def test_trace_check_split_k_violations_are_caught():
    w, t, split, S, idx, start = _split_plan()
    trace_check.check(w, t[:, :5], split, start, start + 1)          # legal
    fin = np.nonzero((S > 1) & (idx == S - 1))[0][0]
    region = tuple(t[fin, [0, 1, 3]])
    part = next(i for i in np.nonzero((S > 1) & (idx < S - 1))[0] if tuple(t[i, [0, 1, 3]]) == region)
    # (1) the finishing partial starts before a partial of its region has ended
    s1, e1 = start.copy(), start + 1
    s1[fin], e1[fin] = e1[part] - 1, e1[part] + 1
    with pytest.raises(AssertionError, match="ends after its finishing tile"):
        trace_check.check(w, t[:, :5], split, s1, e1)
    # (2) a partial starts before a tile producing its A rows has released them
    node = w.nodes[t[part, 0]]
    pa = next(v for v, x in enumerate(w.nodes) if x.out == node.a)
    prod = [i for i in range(len(t)) if t[i, 0] == pa and t[i, 1] < t[part, 2] and t[part, 1] < t[i, 2]]
    assert prod
    s2, e2 = start.copy(), start + 1
    s2[part] = e2[prod[-1]] - 1
    assert s2[part] < e2[part]
    with pytest.raises(AssertionError, match="illegal trace"):
        trace_check.check(w, t[:, :5], split, s2, e2)
