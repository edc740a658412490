"""The JSON specification frontend (paper §4.A): the example specifications
describe the same DAGs as the built-in workloads (same oracle bits), symbols
resolve from defaults and overrides, the paper's transpose kernel fuses into
the consuming matmul, and malformed specifications are rejected."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300 import dag as dagmod
from paper_2009_07482_gb300 import spec
from synth.workloads import fork_join, transformer_heads
from tests.conftest import ROOT

SPECS = os.path.join(ROOT, "paper_2009_07482_gb300", "specs")


def _load(name, **sym):
    return spec.load(os.path.join(SPECS, name), sym)


def _raw(name):
    with open(os.path.join(SPECS, name)) as f:
        return json.load(f)


def test_evaluate_symbolic_sizes():
    s = {"M": 6, "N": 4}
    assert spec.evaluate("M*N", s) == 24
    assert spec.evaluate("(M + 2) // 4 * N", s) == 8
    assert spec.evaluate("2**N - M", s) == 10
    assert spec.evaluate(128, s) == 128
    assert spec.evaluate("M / 2", s) == 3
    for bad in ("M / 4", "Q*2", "__import__('os').getcwd()", "M if N else 1", "[M]", "", True):
        with pytest.raises(spec.SpecError):
            spec.evaluate(bad, s)


def test_fork_join_spec_is_the_fork_join_dag():
    d = _load("fork_join.json")
    ref = fork_join(256)
    assert [n.op for n in d.nodes] == [n.op for n in ref.nodes]
    assert [(d.buffers[n.out].rows, d.buffers[n.out].cols) for n in d.nodes] == \
           [(ref.buffers[n.out].rows, ref.buffers[n.out].cols) for n in ref.nodes]
    # the same arrays in, the same oracle bits out
    w = d.to_workload()
    rins = ref.make_inputs()
    name_of = {"k0.arg0": "A0", "k0.arg1": "B0", "k1.arg1": "B1", "k2.arg1": "B2"}
    rid = {b.name: i for i, b in enumerate(ref.buffers)}
    ins = {i: rins[rid[name_of[w.buffers[i].name]]] for i in w.input_ids()}
    got = oracle.run(w, ins)[w.output_ids()[0]]
    want = oracle.run(ref, rins)[ref.output_ids()[0]]
    assert np.array_equal(np.asarray(got), np.asarray(want))
    # explicit edges pass the library's check (each is implied by the buffers)
    n, e, b = dagmod.describe(w, resident_inputs=True)
    assert len(e) == 4
    t, info = abi.dag_plan_host(n, e, b, None, 148)
    assert info.n_tiles == len(t) > 0


def test_symbols_override_defaults():
    d = _load("fork_join.json", N=96)
    assert {(b.rows, b.cols) for b in d.buffers} == {(96, 96)}
    assert d.queues == 2 and d.symbols == {"N": 96}


def test_transpose_fuses_into_the_consuming_matmul():
    d = _load("transformer_head.json", beta=64)
    assert len(d.nodes) == 7 and 3 not in d.kernel_of_node  # kernel 3 is the transpose
    qk = d.nodes[d.kernel_of_node.index(4)]
    assert qk.op == "gemm" and qk.trans_b == 1
    assert qk.b == d.nodes[d.kernel_of_node.index(1)].out  # reads K itself, K-major
    # same oracle bits as the built-in one-head DAG
    ref = transformer_heads(1, 64)
    w = d.to_workload()
    rins = ref.make_inputs()
    rid = {b.name: i for i, b in enumerate(ref.buffers)}
    name_of = {"k0.arg0": "X", "k1.arg0": "X", "k2.arg0": "X", "k0.arg1": "Wq0", "k1.arg1": "Wk0",
               "k2.arg1": "Wv0", "k7.arg1": "Wh0"}
    ins = {i: rins[rid[name_of[w.buffers[i].name]]] for i in w.input_ids()}
    got = oracle.run(w, ins)[w.output_ids()[0]]
    want = oracle.run(ref, rins)[ref.output_ids()[0]]
    assert np.array_equal(np.asarray(got), np.asarray(want))
    n, e, b = dagmod.describe(w, resident_inputs=True)
    abi.dag_plan_host(n, e, b, None, 148)


def test_task_components_from_tc():
    s = _raw("fork_join.json")
    s["tc"] = [[0], [1, 2], [3]]
    d = spec.loads(json.dumps(s))
    assert [n.component for n in d.nodes] == [0, 1, 1, 2]


def _broken(mutate):
    s = _raw("fork_join.json")
    mutate(s)
    with pytest.raises(spec.SpecError):
        spec.loads(json.dumps(s))


def test_malformed_specifications_are_rejected():
    _broken(lambda s: s["kernels"][3].update(ioBuffers=[{"type": "float", "size": "N*N", "pos": 3}]))
    _broken(lambda s: s["kernels"][1].update(dev="cpu"))
    _broken(lambda s: s["kernels"][2].update(name="conv2d"))
    _broken(lambda s: s["kernels"][0]["outputBuffers"][0].update(size="N*N+1"))      # size vs role
    _broken(lambda s: s["kernels"][0]["inputBuffers"][0].update(size="N*N/3"))       # not an integer
    _broken(lambda s: s.update(edges=s["edges"] + ["3,2 -> 1,1"]))                   # a cycle
    _broken(lambda s: s.update(edges=s["edges"] + ["2,2 -> 3,0"]))                   # two producers
    _broken(lambda s: s.update(edges=["0,1 -> 1,0"]))                                # not an output
    _broken(lambda s: s.update(edges=["0,2 -> 1,2"]))                                # not an input
    _broken(lambda s: s.update(edges=["0,2 - 1,0"]))                                 # syntax
    _broken(lambda s: s.update(tc=[[0, 1], [2]]))                                    # kernel 3 missing
    _broken(lambda s: s.update(tc=[[0, 1, 2, 3], [1]]))                              # kernel 1 twice
    _broken(lambda s: s.update(cq={"gpu": 0}))


def test_transpose_must_feed_a_matmul_b_operand():
    s = _raw("transformer_head.json")
    s["edges"] = [e for e in s["edges"] if e != "3,1 -> 4,1"] + ["3,1 -> 5,0"]
    s["edges"] = [e for e in s["edges"] if e != "4,2 -> 5,0"]
    with pytest.raises(spec.SpecError):
        spec.loads(json.dumps(s), {"beta": 32})
