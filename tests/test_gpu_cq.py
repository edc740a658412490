"""The paper's own fine-grained form (§4.B, Alg. 1; the clustering scheme of
§5) on CUDA streams (dag_submit_cq): the same tiles as the persistent
executor, so the same bits; dependency-legal kernel times; one component at a
time on the device; the callback count the component partition implies."""
import numpy as np
import pytest

import oracle
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag, options
from synth import BF16, F32
from synth.workloads import Workload, branchy_mlp, encoder_block, fork_join, random_layered, transformer_heads
from tests.gpu_util import bits_equal, compare, written_buffers

pytestmark = pytest.mark.gpu

SLACK_US = 1.0  # CUDA event timestamps: ~0.5 us resolution


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _outputs(d, w):
    return {b: d.output(b) for b in written_buffers(w, d.fusion())}


def _preds(w):
    """Kernel predecessors by buffer overlap (producer of any read region)."""
    root = lambda b: w.buffers[b].view_of if w.buffers[b].view_of >= 0 else b
    span = lambda b: (w.buffers[b].col_offset, w.buffers[b].col_offset + w.buffers[b].cols)
    pred = [set() for _ in w.nodes]
    for v, n in enumerate(w.nodes):
        for b in (n.a, n.b, n.bias):
            if b < 0:
                continue
            for u, m in enumerate(w.nodes):
                if u != v and root(m.out) == root(b):
                    (a0, a1), (b0, b1) = span(m.out), span(b)
                    if a0 < b1 and b0 < a1:
                        pred[v].add(u)
    return pred


CASES = [
    ("fork_join_f32", lambda: fork_join(200)),
    ("mlp_bf16_small", lambda: branchy_mlp(BF16, batch=96, width=256, hidden=384, out=128)),
    ("encoder_small", lambda: encoder_block(batch=2, seq=64, d_model=128, heads=4, d_head=32, ffn=256)),
    ("heads4_b128", lambda: transformer_heads(4, 128)),
    ("random_1004", lambda: random_layered(1004)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_cq_same_bits_as_persistent_and_legal_times(name, make):
    w = make()
    ins = w.make_inputs()
    d = Dag(w, options(), resident_inputs=True)
    d.set_inputs(ins)
    d.run()
    base = _outputs(d, w)
    errs = compare(w, base, oracle.run(w, ins))
    assert errs
    pred = _preds(w)
    n_sinks = sum(1 for v in range(len(w.nodes)) if not any(v in p for p in pred))
    for mode, q in [(abi.DAG_TC_WHOLE, 1), (abi.DAG_TC_WHOLE, 3), (abi.DAG_TC_PER_KERNEL, 1),
                    (abi.DAG_TC_GIVEN, 2)]:
        r, ts, te = d.run_cq(n_queues=q, components=mode, times=True)
        assert bits_equal(base, _outputs(d, w)), (mode, q)
        # kernel v starts after every predecessor ended
        for v, ps in enumerate(pred):
            for u in ps:
                assert ts[v] >= te[u] - SLACK_US, (mode, q, u, v, te[u], ts[v])
        assert (te >= ts).all()
        assert r.device_us >= te.max() - SLACK_US
        if mode == abi.DAG_TC_PER_KERNEL:
            assert r.n_components == len(w.nodes) and r.n_callbacks == len(w.nodes)
            # one component (= kernel) at a time holds the device
            order = np.argsort(ts, kind="stable")
            for a, b in zip(order[:-1], order[1:]):
                assert ts[b] >= te[a] - SLACK_US
        elif mode == abi.DAG_TC_WHOLE:
            assert r.n_components == 1 and r.n_callbacks == n_sinks and r.gap_us == 0.0
    d.close()


def test_cq_heads_one_component_at_a_time():
    """The clustering partition of §5 (one task component per head): heads
    run one after another on the one device, each over its own queues."""
    H = 4
    w = transformer_heads(H, 128)
    d = Dag(w, options(), resident_inputs=True)
    d.set_inputs(w.make_inputs())
    r, ts, te = d.run_cq(n_queues=3, components=abi.DAG_TC_GIVEN, times=True)
    assert r.n_components == H and r.n_callbacks == H  # one END kernel (cw) per head
    spans = sorted((ts[[i for i, n in enumerate(w.nodes) if n.component == h]].min(),
                    te[[i for i, n in enumerate(w.nodes) if n.component == h]].max()) for h in range(H))
    for (a0, a1), (b0, b1) in zip(spans[:-1], spans[1:]):
        assert b0 >= a1 - SLACK_US
    assert r.gap_us >= 0.0 and r.host_us > 0.0
    d.close()


def test_cq_streamed_inputs_are_uploaded_on_their_queues():
    w = fork_join(128)
    streamed = set(w.input_ids())
    d = Dag(w, options(), streamed=streamed)
    for seed in (1, 2):
        ins = {b: np.ascontiguousarray(a * (1.0 + seed)).astype(a.dtype) for b, a in w.make_inputs().items()}
        d.set_inputs(ins)
        d.run_cq(n_queues=2, components=abi.DAG_TC_PER_KERNEL)
        compare(w, _outputs(d, w), oracle.run(w, ins))
    d.close()


def test_cq_rejects_a_cyclic_partition():
    """a -> b -> c with a and c in one component and b in another: the
    component graph has a cycle, so Alg. 1 could never dispatch either."""
    w = Workload("cyc")
    X = w.buf(64, 64, F32, "input", ("uniform", 1))
    Y = w.buf(64, 64, F32, "inter")
    Zb = w.buf(64, 64, F32, "inter")
    O = w.buf(64, 64, F32, "output")
    w.node("unary", X, Y, act="relu", component=0)
    w.node("unary", Y, Zb, act="relu", component=1)
    w.node("unary", Zb, O, act="relu", component=0)
    d = Dag(w, options(), resident_inputs=True)
    d.set_inputs(w.make_inputs())
    with pytest.raises(RuntimeError, match="cycle"):
        d.run_cq(n_queues=1, components=abi.DAG_TC_GIVEN)
    d.run()  # the handle stays usable
    d.close()


@pytest.mark.parametrize("name,sym", [("fork_join.json", {"N": 192}), ("transformer_head.json", {"beta": 128})])
def test_spec_files_run_on_both_executors(name, sym):
    """A JSON specification (paper §4.A) runs as written: its explicit edges
    pass dag_create's check, its cq and tc drive Alg. 1 on streams, and both
    executors match the oracle with the same bits."""
    import os
    from paper_2009_07482_gb300 import spec
    from tests.conftest import ROOT
    sd = spec.load(os.path.join(ROOT, "paper_2009_07482_gb300", "specs", name), sym)
    w = sd.to_workload()
    ins = w.make_inputs()
    d = Dag(w, options(trace=1), resident_inputs=True)
    d.set_inputs(ins)
    d.run()
    base = _outputs(d, w)
    compare(w, base, oracle.run(w, ins))
    r = d.run_cq(n_queues=sd.queues, components=abi.DAG_TC_GIVEN)
    assert r.n_components == len(set(n.component for n in sd.nodes))
    assert bits_equal(base, _outputs(d, w))
    d.close()


def test_setup_cq_follows_the_papers_worked_example():
    """The paper's DAG of §3 (component T = {k0..k4}, fed by {k5, k6} and
    feeding {k7, k8}) with three command queues: setup_cq sends k0..k4 to
    q0, q1, q2, q0, q1 (§4.B, its example of Fig. 'dispatch'; round-robin over
    the component's own queues, in dispatch order), and the results match the
    oracle and the persistent executor bit for bit."""
    from tests.conftest import load_golden
    g = load_golden("paper_fig_platform_dag.json")
    w = Workload("paper_platform_dag")
    bid = {}
    sinks = {"y7", "y8"}
    for i, nme in enumerate(g["buffers"]):
        role = "input" if nme in g["inputs"] else "output" if nme in sinks else "inter"
        bid[nme] = w.buf(192, 256, F32, role, ("uniform", 300 + i) if role == "input" else None, nme)
    kid = {}
    for k, spec in g["kernels"].items():
        kw = {"b": bid[spec["b"]]} if "b" in spec else {"act": "relu"}
        kid[k] = w.node(spec["op"], bid[spec["a"]], bid[spec["out"]], name=k, component=spec["component"], **kw)
    ins = w.make_inputs()
    d = Dag(w, options(), resident_inputs=False)
    try:
        d.set_inputs(ins)
        d.run()
        fine = _outputs(d, w)
        r, _, _, q = abi.dag_submit_cq(d.h, n_queues=g["setup_cq"]["n_queues"], components=abi.DAG_TC_GIVEN,
                                       n_nodes=len(w.nodes), queues=True)
        assert r.n_components == 3
        cq = _outputs(d, w)
    finally:
        d.close()
    assert {k: int(q[kid[k]]) for k in g["setup_cq"]["queue"]} == g["setup_cq"]["queue"]
    compare(w, fine, oracle.run(w, ins))
    assert bits_equal(fine, cq)
