"""The C ABI on the host (no GPU): the library loads and exports every
declared entry point; validation; the paper's §3 classification example; and
the planner's queue order checked by the oracle's independent trace checker."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300 import dag as dagmod
from synth import BF16, F32
from synth.workloads import Workload, branchy_mlp, encoder_block, fork_join, random_layered
from tests import trace_check
from tests.conftest import ROOT, load_golden


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2009_07482_gb300 import build
    build.build()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(dag_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert "dag_create" in names and "dag_submit" in names and "dag_wait" in names and "dag_destroy" in names
    L = abi.lib()
    for n in names:
        assert hasattr(L, n), n
    assert abi.last_error() == ""


def _analysis_of_golden():
    g = load_golden("paper_fig_platform_dag.json")
    bid = {n: i for i, n in enumerate(g["buffers"])}
    kid = {k: i for i, k in enumerate(g["kernels"])}
    bufs = [abi.dag_buffer_desc(4, 4, abi.DAG_F32, abi.DAG_BUF_INPUT if n in g["inputs"] else 0, -1, 0)
            for n in g["buffers"]]
    ops = {"add": abi.DAG_OP_ADD, "unary": abi.DAG_OP_UNARY}
    nodes = [abi.dag_node_desc(ops[k["op"]], bid[k["a"]], bid[k["b"]] if "b" in k else -1, -1, bid[k["out"]],
                               0, 0, 1.0, 1, k["component"]) for k in g["kernels"].values()]
    return g, bid, kid, abi.dag_analyze(nodes, [], bufs)


def test_classification_matches_paper_worked_example():
    g, bid, kid, a = _analysis_of_golden()
    T = [kid[k] for k in ("k0", "k1", "k2", "k3", "k4")]
    front = {k for k in g["kernels"] if kid[k] in T and a["cls"][kid[k]] & 1}
    end = {k for k in g["kernels"] if kid[k] in T and a["cls"][kid[k]] & 2}
    inn = {k for k in g["kernels"] if kid[k] in T and a["cls"][kid[k]] & 4}
    assert front == set(g["expect"]["FRONT"])
    assert end == set(g["expect"]["END"])
    assert inn == set(g["expect"]["IN"])
    got_intra = {(s, d, b) for s, b, d, _, inter in a["edges"] if not inter}
    got_inter = {(s, d, b) for s, b, d, _, inter in a["edges"] if inter}
    assert got_intra == {(kid[s], kid[d], bid[b]) for s, d, b in g["expect"]["intra"]}
    assert got_inter == {(kid[s], kid[d], bid[b]) for s, d, b in g["expect"]["inter"]}
    iso = {(b, k) for k, b, w, i in a["copies"] if k in T and w and i}
    assert iso == {(bid[b], kid[k]) for b, k in g["expect"]["isolated_writes_in_T"]}
    # every other kernel-buffer dependency of T is a dependent copy
    dep = [(k, b, w) for k, b, w, i in a["copies"] if k in T and not i]
    assert len(dep) == len([c for c in a["copies"] if c[0] in T]) - 2


def test_fork_join_single_component_classification():
    w = fork_join(8)
    n, e, b = dagmod.describe(w)
    a = abi.dag_analyze(n, e, b)
    assert a["cls"] == [1, 4, 4, 2]        # K0 FRONT, K1/K2 IN, K3 END
    assert a["topo"] == [0, 1, 2, 3]
    assert all(inter == 0 for *_, inter in a["edges"])


def _codes(w):
    n, e, b = dagmod.describe(w)
    try:
        abi.dag_analyze(n, e, b)
        return 0
    except abi.DagError as ex:
        return ex.status


def test_validation_codes_agree_with_oracle():
    cases = []
    w = Workload("cycle")
    a = w.buf(4, 4, F32, "input", ("uniform", 1))
    b0, b1 = w.buf(4, 4), w.buf(4, 4)
    w.node("gemm", a, b0, b=b1)
    w.node("gemm", a, b1, b=b0)
    cases.append((w, abi.DAG_ECYCLE))
    w = Workload("two writers")
    a = w.buf(4, 4, F32, "input", ("uniform", 1))
    o = w.buf(4, 4)
    w.node("unary", a, o)
    w.node("unary", a, o)
    cases.append((w, abi.DAG_EMULTIWRITER))
    w = Workload("in place")
    a = w.buf(4, 4, F32, "input", ("uniform", 1))
    o = w.buf(4, 4)
    w.node("unary", a, o)
    w.node("unary", o, o)
    cases.append((w, abi.DAG_EMULTIWRITER))
    w = Workload("shape")
    a = w.buf(4, 5, F32, "input", ("uniform", 1))
    b = w.buf(4, 5, F32, "input", ("uniform", 2))
    w.node("gemm", a, w.buf(4, 5), b=b)
    cases.append((w, abi.DAG_ESHAPE))
    w = Workload("mixed dtypes")
    a = w.buf(4, 4, F32, "input", ("uniform", 1))
    b = w.buf(4, 4, BF16, "input", ("uniform", 2))
    w.node("gemm", a, w.buf(4, 4), b=b)
    cases.append((w, abi.DAG_EDTYPE))
    w = Workload("writes an input")
    a = w.buf(4, 4, F32, "input", ("uniform", 1))
    b = w.buf(4, 4, F32, "input", ("uniform", 2))
    w.node("unary", a, b)
    cases.append((w, abi.DAG_EMULTIWRITER))
    w = Workload("reads unwritten")
    a = w.buf(4, 4)
    w.node("unary", a, w.buf(4, 4))
    cases.append((w, abi.DAG_EINVAL))
    for w, code in cases:
        assert _codes(w) == code, w.name
    # the oracle's own validation agrees where it has the same notion
    assert oracle.validate(cases[1][0]) == 5 and oracle.validate(cases[3][0]) == 3


def test_edges_must_be_implied():
    w = fork_join(8)
    n, _, b = dagmod.describe(w)
    good = [abi.dag_edge(0, 4, 1, 4), abi.dag_edge(1, 5, 3, 5)]
    abi.dag_analyze(n, good, b)
    with pytest.raises(abi.DagError) as ex:
        abi.dag_analyze(n, [abi.dag_edge(1, 5, 2, 5)], b)   # K2 does not read C1
    assert ex.value.status == abi.DAG_EINVAL


PLAN_CASES = [
    ("fork_join_256", lambda: fork_join(256)),
    ("fork_join_ragged", lambda: fork_join(200)),
    ("mlp_bf16", lambda: branchy_mlp(BF16)),
    ("mlp_f32", lambda: branchy_mlp(F32)),
    ("encoder", lambda: encoder_block()),
    ("encoder_small", lambda: encoder_block(batch=2, seq=64, d_model=128, heads=4, d_head=32, ffn=256)),
] + [(f"random_{s}", (lambda s=s: random_layered(1000 + s))) for s in range(6)]


@pytest.mark.parametrize("name,make", PLAN_CASES, ids=[c[0] for c in PLAN_CASES])
@pytest.mark.parametrize("n_sm", [148, 7])
def test_queue_order_is_a_legal_schedule(name, make, n_sm):
    """Running tiles one by one in queue order must be dependency-legal by the
    oracle's own region analysis: the persistent kernel's deadlock freedom
    rests on this (every tile a CTA waits on was claimed earlier)."""
    w = make()
    n, e, b = dagmod.describe(w, resident_inputs=True)
    for sched in (abi.DAG_SCHED_RANK_MODEL, abi.DAG_SCHED_FIFO):
        opts = dagmod.options(scheduler=sched)
        t, info = abi.dag_plan_host(n, e, b, opts, n_sm)
        assert info.n_tiles == len(t) > 0
        start = np.arange(len(t), dtype=np.uint32) * 2
        trace_check.check(w, t[:, :5], t[:, 5] >> 16, start, start + 1, abi.dag_fusion_host(n, e, b, opts),
                          abi.dag_merge_host(n, b, opts))


def test_plan_algorithmic_totals():
    w = branchy_mlp(BF16)
    n, e, b = dagmod.describe(w, resident_inputs=True)
    _, info = abi.dag_plan_host(n, e, b, None, 148)
    assert info.flops == pytest.approx(sum(w.node_flops(k) for k, x in enumerate(w.nodes) if x.op == "gemm"))
    assert info.flops == pytest.approx(64.42450944e9)
    assert info.bytes == pytest.approx(sum(w.node_bytes(k) for k in range(len(w.nodes))))


def _f32_gemm_with_views(a_off):
    """An f32 GEMM whose A is a column slice starting at column a_off of a
    wider buffer, and a second GEMM on a plain buffer."""
    w = Workload("f32_views")
    P = w.buf(256, 96 + 8, F32, "input", ("uniform", 1))
    A = w.buf(256, 96, F32, "inter", view_of=P, col_offset=a_off)
    B = w.buf(96, 200, F32, "input", ("uniform", 2))
    C = w.buf(256, 200, F32, "output")
    w.node("gemm", A, C, b=B)
    X = w.buf(300, 64, F32, "input", ("uniform", 3))
    D = w.buf(300, 200, F32, "output")
    w.node("gemm", X, D, b=w.buf(64, 200, F32, "input", ("uniform", 4)))
    return w


@pytest.mark.parametrize("a_off,mode", [(0, 0), (4, 0), (1, 0), (0, 1), (0, 2)])
def test_f32_gemm_tile_kind(a_off, mode):
    """f32 GEMMs take the tensor-core 3 x TF32 tiles unless an operand view
    does not start on a 16-byte boundary or SIMT is asked for; then the SIMT
    FFMA shapes (64/128 rows x 64/128 columns).  With B read K-major (here:
    resident weights kept transposed) and N > 64 the tiles are 128 x 128 or
    128 x 256 (the wide form) when the level has tiles enough for the SMs
    (planned here for a 4-SM GPU), else -- and always under
    DAG_F32_GEMM_TENSOR_NARROW -- 128 x 64."""
    w = _f32_gemm_with_views(a_off)
    n, e, b = dagmod.describe(w, resident_inputs=True)
    t, _ = abi.dag_plan_host(n, e, b, dagmod.options(f32_gemm=mode), 4)
    # the same level on a full GPU with a short K loop: twice as many 128 x 64 tiles
    t_full, _ = abi.dag_plan_host(n, e, b, dagmod.options(f32_gemm=mode), 148)
    if mode == 0 and a_off % 4 == 0:
        assert ((t_full[:, 5] & 0xFFFF) == 64).all()
    for node, want_tc in ((0, mode != 1 and a_off % 4 == 0), (1, mode != 1)):
        mine = t[t[:, 0] == node]
        rows = mine[:, 2] - mine[:, 1]
        cols = mine[:, 4] - mine[:, 3]
        if want_tc and mode == 2:
            assert (mine[:, 5] == 64).all()
            assert rows.max() == 128 and cols.max() == 64
        elif want_tc:
            bn = int(mine[0, 5])
            assert bn in (128, 256) and ((mine[:, 5] & 0xFFFF) == bn).all()
            assert rows.max() == 128 and cols.max() <= bn
        else:
            assert set(mine[:, 5].tolist()) <= {0, 1, 2}


def _noalloc_status(bufs, ptrs, pitch):
    nodes = [abi.dag_node_desc(abi.DAG_OP_ADD, 0, 1, -1, 2, 0, 0, 1.0, 1, 0)]
    return abi.dag_run_noalloc(nodes, bufs, ptrs, pitch, None, 0)


@pytest.mark.parametrize("seed", [6000, 6001, 6002])
def test_split_k_only_where_the_tile_form_runs_a_share_of_k(seed):
    """Split K is planned for bf16 tiles and the wide f32 form, whose device
    loops take their share of the K blocks; the 128 x 64 f32 tiles and the
    SIMT f32 tiles always run the whole K loop, so a plan never splits them
    (a split there would sum S whole-K products)."""
    for w in (random_layered(seed, 8, 24, 4, sizes=(64, 128, 256, 512, 1024)), fork_join(256)):
        for res in (False, True):
            n, e, b = dagmod.describe(w, resident_inputs=res)
            t, _ = abi.dag_plan_host(n, e, b, dagmod.options(), 152)
            for row in t:
                node = w.nodes[int(row[0])]
                split = int(row[5]) >> 16
                if node.op != "gemm" or not split:
                    continue
                bf16 = w.buffers[node.a].dtype == BF16
                assert bf16 or (int(row[5]) & 0xFFFF) in (128, 256), (w.name, int(row[0]), int(row[5]) & 0xFFFF)


def test_sibling_gemms_merge_into_one_plan_gemm():
    """The planner merges GEMMs that read one A with private resident weights
    (the encoder's Q/K/V projections of every head: one GEMM of 3072 columns,
    192 tiles of 128 x 256 for 768 of 128 x 64) -- and leaves them alone under
    merge = 1 or keep_layout = 1, with streamed weights, with outputs the
    caller reads back, and across task components.  The plan's algorithmic
    work is the DAG's own either way."""
    w = encoder_block()
    n, e, b = dagmod.describe(w, resident_inputs=True)
    lead, off = abi.dag_merge_host(n, b, dagmod.options())
    proj = [v for v, x in enumerate(w.nodes) if x.name.startswith("proj_")]
    assert {lead[v] for v in proj} == {proj[0]} and sorted(off[v] for v in proj) == list(range(0, 3072, 64))
    assert all(lead[v] < 0 for v in range(len(w.nodes)) if v not in proj)
    t, info = abi.dag_plan_host(n, e, b, dagmod.options(), 148)
    t1, info1 = abi.dag_plan_host(n, e, b, dagmod.options(merge=1), 148)
    mine = t[t[:, 0] == proj[0]]
    assert len(mine) == 192 and set((mine[:, 5] & 0xFFFF).tolist()) == {256} and mine[:, 4].max() == 3072
    assert not any(int(r[0]) in proj[1:] for r in t)
    assert len(t1) - len(t) == 768 - 192 and (info.flops, info.bytes) == (info1.flops, info1.bytes)
    for o in (dagmod.options(merge=1), dagmod.options(keep_layout=1)):
        assert all(x < 0 for x in abi.dag_merge_host(n, b, o)[0])
    n2, _, b2 = dagmod.describe(w)  # weights streamed every submit
    assert all(x < 0 for x in abi.dag_merge_host(n2, b2, dagmod.options())[0])
    # three siblings per component, one of them read back by the caller
    w3 = Workload("siblings")
    X = w3.buf(512, 256, BF16, "input", ("uniform", 1))
    for comp in range(2):
        for i in range(3):
            W = w3.buf(256, 64, BF16, "input", ("uniform", 10 + 3 * comp + i))
            O = w3.buf(512, 64, BF16, "output" if (comp, i) == (1, 2) else "inter")
            w3.node("gemm", X, O, b=W, component=comp)
            if (comp, i) != (1, 2):
                w3.node("unary", O, w3.buf(512, 64, BF16, "output"), act="relu", component=comp)
    n3, _, b3 = dagmod.describe(w3, resident_inputs=True)
    lead3, off3 = abi.dag_merge_host(n3, b3, dagmod.options())
    g = [v for v, x in enumerate(w3.nodes) if x.op == "gemm"]
    assert [lead3[v] for v in g] == [g[0], g[0], g[0], g[3], g[3], -1]
    assert [off3[v] for v in g] == [0, 64, 128, 0, 64, 0]


def test_trace_checker_sees_a_merged_tile_as_its_siblings_shares():
    """A merged GEMM's tile stands for its siblings' shares of its columns:
    the queue order passes only with the merge map given (without it the
    siblings' regions are never written); a tile reading a projection that
    starts before the merged tiles holding its columns have ended fails, and
    so does a trace missing one merged tile."""
    w = encoder_block(batch=2, seq=64, d_model=128, heads=4, d_head=32, ffn=256)
    n, e, b = dagmod.describe(w, resident_inputs=True)
    opts = dagmod.options()
    t, _ = abi.dag_plan_host(n, e, b, opts, 148)
    fused, merges = abi.dag_fusion_host(n, e, b, opts), abi.dag_merge_host(n, b, opts)
    proj = [v for v, x in enumerate(w.nodes) if x.name.startswith("proj_")]
    L = merges[0][proj[0]]
    assert L >= 0 and all(merges[0][v] == L for v in proj)
    start = np.arange(len(t), dtype=np.int64) * 2 + 2
    args = (t[:, :5], t[:, 5] >> 16)
    trace_check.check(w, *args, start, start + 1, fused, merges)
    with pytest.raises(AssertionError, match="illegal trace"):
        trace_check.check(w, *args, start, start + 1, fused, None)
    outs = {w.nodes[v].out for v in proj}
    readers = {v for v, x in enumerate(w.nodes) if x.op == "gemm" and ({x.a, x.b} & outs) and v not in proj}
    c = next(i for i, r in enumerate(t) if int(r[0]) in readers)
    early = start.copy()
    early[c] = 0                   # before every merged projection tile has ended
    with pytest.raises(AssertionError, match="illegal trace"):
        trace_check.check(w, *args, early, start + 1, fused, merges)
    keep = np.ones(len(t), bool)
    keep[np.nonzero(t[:, 0] == L)[0][0]] = False
    with pytest.raises(AssertionError, match="illegal trace"):
        trace_check.check(w, t[keep, :5], t[keep, 5] >> 16, start[keep], start[keep] + 1, fused, merges)


def test_no_alloc_rejects_overlapping_root_buffers():
    """dag_run_noalloc: two root buffers sharing device memory (an output
    placed on an input, or rows of one falling inside another) are rejected
    with DAG_EINVAL before any device call; interleaved buffers whose rows
    never meet, and disjoint ones, pass this check (and then, with no GPU
    here, stop at the device query with DAG_EDEVICE)."""
    f32 = abi.DAG_F32
    bufs = [abi.dag_buffer_desc(4, 16, f32, abi.DAG_BUF_INPUT, -1, 0),
            abi.dag_buffer_desc(4, 16, f32, abi.DAG_BUF_INPUT, -1, 0),
            abi.dag_buffer_desc(4, 16, f32, abi.DAG_BUF_OUTPUT, -1, 0)]
    base = 1 << 30
    # the output on top of the first input
    assert _noalloc_status(bufs, [base, base + 4096, base], [16, 16, 16]) == abi.DAG_EINVAL
    assert "overlap" in abi.last_error()
    # the output starting inside the second input's last row
    assert _noalloc_status(bufs, [base, base + 4096, base + 4096 + 3 * 64 + 32], [16, 16, 16]) == abi.DAG_EINVAL
    # three buffers interleaved column-wise in one allocation of pitch 48: rows never meet
    assert _noalloc_status(bufs, [base, base + 64, base + 128], [48, 48, 48]) == abi.DAG_EDEVICE
    # the same, but the second one 16 bytes too wide for its slot
    wide = list(bufs)
    wide[1] = abi.dag_buffer_desc(4, 20, f32, abi.DAG_BUF_INPUT, -1, 0)
    assert _noalloc_status(wide, [base, base + 64, base + 128], [48, 48, 48]) == abi.DAG_EINVAL
    # disjoint
    assert _noalloc_status(bufs, [base, base + 4096, base + 8192], [16, 16, 16]) == abi.DAG_EDEVICE
