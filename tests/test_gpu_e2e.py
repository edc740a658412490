"""The end-to-end path the benchmark's e2e figure times: activations streamed
from pinned host memory on the upload streams every submit (the paper's
isolated writes, §3), the persistent launch, and every sink read back into
registered pinned host memory on a copy stream after the launch (isolated
reads, §3; the readback after each END kernel of Alg. 1).  Several submits in
a row with new activations each time: every registered sink must equal the
FP64 oracle on that submit's inputs (per-buffer normwise tolerance) and, bit
for bit, what dag_get_output reads from the device afterwards."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag, options
from paper_2009_07482_gb300.serving import activation_ids
from synth import storage_to_f64
from synth.workloads import branchy_mlp, encoder_block, fork_join
from tests.gpu_util import node_tolerance
from tests.row_sample import oracle_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _pinned_view(p, b):
    n = b.rows * b.cols
    if b.dtype == "f32":
        return np.ctypeslib.as_array((C.c_float * n).from_address(p)).reshape(b.rows, b.cols)
    return np.ctypeslib.as_array((C.c_uint16 * n).from_address(p)).reshape(b.rows, b.cols)


def _run_e2e(w, submits, rows=None):
    """`submits` submits through the C ABI with streamed activations and
    registered readbacks; returns [(inputs, {sink: host copy})] per submit,
    and the dag_get_output of the last one."""
    X_ids = activation_ids(w)
    base = w.make_inputs()
    d = Dag(w, options(), streamed=set(X_ids))
    d.set_inputs({k: v for k, v in base.items() if k not in X_ids})   # resident weights
    xin = {}
    for i in X_ids:
        b = w.buffers[i]
        p = abi.dag_host_alloc(b.rows * b.cols * (4 if b.dtype == "f32" else 2))
        xin[i] = (p, _pinned_view(p, b))
        abi.dag_set_input(d.h, i, p)
    yout = {}
    for Y in w.output_ids():
        b = w.buffers[Y]
        p = abi.dag_host_alloc(b.rows * b.cols * (4 if b.dtype == "f32" else 2))
        yout[Y] = (p, _pinned_view(p, b))
        yout[Y][1].fill(0xFFFF if b.dtype != "f32" else np.nan)
        abi.dag_set_output(d.h, Y, p)
    runs = []
    try:
        for s in range(submits):
            ins = dict(base)
            for i in X_ids:
                b = w.buffers[i]
                a = synth.fill("uniform", 70_000 + 97 * s + i, (b.rows, b.cols), b.dtype, -1.0, 1.0)
                xin[i][1][:] = a
                ins[i] = a
            d.submit()
            abi.check(d.wait(), "dag_wait")
            runs.append((ins, {Y: v.copy() for Y, (p, v) in yout.items()}))
        dev = {Y: d.output(Y) for Y in yout}
    finally:
        for Y in yout:
            abi.dag_set_output(d.h, Y, None)
        d.close()
        for p, _ in list(xin.values()) + list(yout.values()):
            abi.dag_host_free(p)
    return runs, dev


def _check_whole(w, runs, dev):
    for ins, got in runs:
        ref = oracle.run(w, ins)
        for Y, g in got.items():
            dt = w.buffers[Y].dtype
            e = oracle.rel_err(storage_to_f64(g, dt), storage_to_f64(oracle.view(w, ref, Y), dt))
            assert e <= node_tolerance(w, Y), f"{w.name} sink {Y}: rel err {e:.3e}"
    for Y, g in runs[-1][1].items():
        assert np.array_equal(g.view(np.uint8), dev[Y].view(np.uint8)), f"sink {Y}: readback != dag_get_output"


@pytest.mark.parametrize("make", [
    lambda: fork_join(256),
    lambda: encoder_block(batch=2, seq=128, d_model=256, heads=4, d_head=64, ffn=512, seed=21),
], ids=["fork_join_256_f32", "encoder_small_bf16"])
def test_registered_readback_matches_oracle_and_device(make):
    w = make()
    runs, dev = _run_e2e(w, 3)
    # each submit saw its own activations: the sinks differ from submit to submit
    Y = w.output_ids()[0]
    assert not np.array_equal(runs[0][1][Y], runs[1][1][Y])
    _check_whole(w, runs, dev)


@pytest.mark.parametrize("dt", ["bf16", "f32"])
def test_registered_readback_full_size_mlp(dt):
    """The benchmark's e2e workload at its full size (batch 512, width 2048):
    three submits, every sink compared on sampled rows with the oracle and
    bit for bit with the device copy."""
    w = branchy_mlp(dt)
    runs, dev = _run_e2e(w, 3)
    rows = np.array([0, 129, 511])
    for ins, got in runs:
        ws, ref = oracle_rows(w, ins, rows)
        for Y, g in got.items():
            d = w.buffers[Y].dtype
            e = oracle.rel_err(storage_to_f64(g[rows], d), storage_to_f64(oracle.view(ws, ref, Y), d))
            assert e <= node_tolerance(w, Y), f"sink {Y}: rel err {e:.3e}"
    for Y, g in runs[-1][1].items():
        assert np.array_equal(g.view(np.uint8), dev[Y].view(np.uint8))


def test_back_to_back_batch_launches_read_back_their_own_sinks():
    """The end-to-end path's form for a batch: shares of the DAGs on separate
    handles, submitted back to back on one stream with streamed activations
    and registered readbacks, each launch's readback overlapping the next
    launch.  Every sink of every DAG equals the oracle on its inputs and, bit
    for bit, what dag_get_output reads from its handle afterwards."""
    import bench
    from synth.workloads import concat, random_batch
    wl = random_batch(12, base_seed=1300, max_nodes=24, sizes=(64, 128, 256, 512))
    parts = []
    try:
        for part, _ in bench.e2e_chunks(wl, 3):
            w = concat(part)
            X_ids = activation_ids(w)
            d = Dag.batch(part, options(use_graph=1), resident_inputs=False, streamed=set(X_ids))
            base = w.make_inputs()
            d.set_inputs({k: v for k, v in base.items() if k not in X_ids})
            d.run()
            pins = {}
            for i in X_ids:
                b = w.buffers[i]
                p = abi.dag_host_alloc(b.rows * b.cols * (4 if b.dtype == "f32" else 2))
                v = _pinned_view(p, b)
                v[:] = synth.fill("uniform", 90_000 + i, (b.rows, b.cols), b.dtype, -1.0, 1.0)
                base[i] = v.copy()
                abi.dag_set_input(d.h, i, p)
                pins[i] = p
            outs = {}
            for Y in w.output_ids():
                b = w.buffers[Y]
                p = abi.dag_host_alloc(b.rows * b.cols * (4 if b.dtype == "f32" else 2))
                outs[Y] = (p, _pinned_view(p, b))
                abi.dag_set_output(d.h, Y, p)
            parts.append((w, d, base, pins, outs))
        for _ in range(2):
            for _, d, _, _, _ in parts:
                d.submit()
            for _, d, _, _, _ in parts:
                abi.check(d.wait(), "dag_wait")
        for w, d, base, _, outs in parts:
            ref = oracle.run(w, base)
            for Y, (_, v) in outs.items():
                dt = w.buffers[Y].dtype
                e = oracle.rel_err(storage_to_f64(v.copy(), dt), storage_to_f64(oracle.view(w, ref, Y), dt))
                assert e <= node_tolerance(w, Y), f"{w.name} sink {Y}: rel err {e:.3e}"
                assert np.array_equal(v.view(np.uint8), d.output(Y).view(np.uint8)), f"sink {Y}: readback != device"
    finally:
        for w, d, _, pins, outs in parts:
            for Y in outs:
                abi.dag_set_output(d.h, Y, None)
            d.close()
            for p in list(pins.values()) + [p for p, _ in outs.values()]:
                abi.dag_host_free(p)
