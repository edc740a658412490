"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times (persistent executor, resident inputs), checked against the
FP64 oracle on sampled rows (row-wise DAGs) or sampled sequences (encoder),
plus the tile-trace legality of the whole execution."""
import numpy as np
import pytest

import oracle
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag, options
from synth import BF16, F32, storage_to_f64
from synth.workloads import branchy_mlp, concat, encoder_block, fork_join, random_batch, random_layered
from tests.gpu_util import bits_equal, check_trace, compare, node_tolerance, run_gpu, written_buffers
from tests import trace_check
from tests.row_sample import oracle_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _check_rows(w, ins, got, rows, bids):
    ws, ref = oracle_rows(w, ins, rows)
    for b in bids:
        dt = w.buffers[b].dtype
        g = storage_to_f64(got[b][rows], dt)
        r = storage_to_f64(oracle.view(ws, ref, b), dt)
        e = oracle.rel_err(g, r)
        assert e <= node_tolerance(w, b), f"{w.name} buffer {b}: rel err {e:.3e}"


@pytest.mark.parametrize("dt,rows", [(BF16, [0, 1, 127, 128, 255, 300, 510, 511]), (F32, [0, 200, 511])])
def test_branchy_mlp_full_size(dt, rows):
    w = branchy_mlp(dt)
    ins = w.make_inputs()
    d = Dag(w, options(trace=1), resident_inputs=True)
    d.set_inputs(ins)
    d.run()
    outs = {b: d.output(b) for b in w.output_ids()}
    inter = [i for i, b in enumerate(w.buffers) if b.name in ("h0_0", "sum1_0", "L1")]
    outs.update({b: d.output(b) for b in inter})
    _check_rows(w, ins, outs, np.array(rows), list(outs))
    check_trace(w, d)
    d.close()


def test_fork_join_full_size():
    w = fork_join(256)
    ins = w.make_inputs()
    d = Dag(w, options(trace=1), resident_inputs=True)
    d.set_inputs(ins)
    d.run()
    compare(w, {b: d.output(b) for b in written_buffers(w, d.fusion())}, oracle.run(w, ins))
    check_trace(w, d)
    d.close()


def test_encoder_full_size_sampled_sequences():
    w = encoder_block()
    ins = w.make_inputs()
    d = Dag(w, options(trace=1), resident_inputs=True)
    d.set_inputs(ins)
    d.run()
    Y = w.output_ids()[0]
    y = d.output(Y)
    check_trace(w, d)
    d.close()
    X = w.input_ids()[0]
    for s in (0, 5):
        w1 = encoder_block(batch=1)       # same weights: same seeds, drawn in the same order
        ins1 = w1.make_inputs()
        ins1[w1.input_ids()[0]] = ins[X][256 * s: 256 * (s + 1)]
        ref = oracle.run(w1, ins1)
        e = oracle.rel_err(storage_to_f64(y[256 * s: 256 * (s + 1)], F32), storage_to_f64(ref[w1.output_ids()[0]], F32))
        assert e <= 2e-2, (s, e)


def test_batched_random_dags_full_size():
    """256 random layered DAGs in one persistent launch replayed from a CUDA
    graph; six DAGs checked row-sampled against the oracle, and the trace of
    those DAGs checked for legality."""
    ws = random_batch(256)
    offs = np.cumsum([0] + [len(w.buffers) for w in ws])
    noffs = np.cumsum([0] + [len(w.nodes) for w in ws])
    d = Dag.batch(ws, options(trace=1, use_graph=1), resident_inputs=True)
    full_ins = {}
    for k, w in enumerate(ws):
        for i, a in w.make_inputs().items():
            full_ins[int(offs[k]) + i] = a
    d.set_inputs(full_ins)
    d.run()
    d.run()   # a replay of the captured graph
    recs = d.trace()
    fusion = d.fusion()
    lead, moff = d.merges()
    rows = np.array([0, 31, 63])
    for k in (0, 1, 17, 100, 200, 255):
        w = ws[k]
        ins = {i: full_ins[int(offs[k]) + i] for i in w.input_ids()}
        got = {b: d.output(int(offs[k]) + b) for b in w.output_ids()}
        _check_rows(w, ins, got, rows, list(got))
        sub = [r for r in recs if noffs[k] <= r.node < noffs[k + 1]]
        tiles = np.array([(r.node - noffs[k], r.r0, r.r1, r.c0, r.c1) for r in sub], np.int32)
        fused = [h - noffs[k] if h >= 0 else -1 for h in fusion[noffs[k]:noffs[k + 1]]]
        merged = ([h - noffs[k] if h >= 0 else -1 for h in lead[noffs[k]:noffs[k + 1]]], moff[noffs[k]:noffs[k + 1]])
        trace_check.check(w, tiles, [r.split for r in sub], [r.start_ticket for r in sub],
                          [r.end_ticket for r in sub], fused, merged)
    d.close()


def test_batch_of_small_dags_matches_oracle_and_graph_replay():
    ws = [random_layered(2000 + i, 6, 24, 4, sizes=(64, 128, 256)) for i in range(12)]
    ws += [fork_join(128, seed=3), encoder_block(batch=2, seq=64, d_model=128, heads=4, d_head=32, ffn=256, seed=4)]
    w = concat(ws)
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    outs = {}
    for graph in (0, 1):
        d = Dag.batch(ws, options(trace=1, use_graph=graph))
        d.set_inputs(ins)
        for _ in range(2):
            d.run()
        got = {b: d.output(b) for b in written_buffers(w, d.fusion())}
        compare(w, got, ref)
        check_trace(w, d)
        outs[graph] = got
        d.close()
    assert bits_equal(outs[0], outs[1])


def test_autotuner_picks_a_measured_plan():
    w = branchy_mlp(BF16, batch=256, width=512, hidden=1024, out=256, seed=8)
    ins = w.make_inputs()
    d = Dag(w, options(autotune=1), resident_inputs=True)
    info = d.plan()
    assert info.tuned_us > 0 and info.tile_override in (0, 128, 256)
    d.set_inputs(ins)
    d.run()
    compare(w, {b: d.output(b) for b in written_buffers(w, d.fusion())}, oracle.run(w, ins))
    d.close()
