"""The serving loop: requests admitted continuously into free slots and
device memory, overlapping on the GPU; each result equals the FP64 oracle's
on that request's inputs (within the per-buffer tolerance) and is the same,
bit for bit, alone and in the mix."""
import numpy as np
import pytest

import synth
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag, describe, options
from paper_2009_07482_gb300.serving import Server, activation_ids
from synth import storage_to_f64
from synth.workloads import branchy_mlp, encoder_block, fork_join
from tests.gpu_util import node_tolerance
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _models():
    return [branchy_mlp("bf16", batch=16, width=256, hidden=512, out=128, seed=7),
            branchy_mlp("bf16", batch=64, width=256, hidden=512, out=128, seed=7),
            encoder_block(batch=1, seq=64, d_model=128, heads=4, d_head=32, ffn=256, seed=4),
            fork_join(128, seed=3)]


def _request_inputs(w, seed):
    """Fresh activations for a request (same shapes, new draws)."""
    ins = {}
    for i in activation_ids(w):
        b = w.buffers[i]
        ins[i] = synth.fill("uniform", 90_000 + seed * 31 + i, (b.rows, b.cols), b.dtype, -1.0, 1.0)
    return ins


def test_each_result_is_the_same_alone_and_in_the_mix():
    ws = _models()
    weights = [w.make_inputs() for w in ws]
    reqs = [(k % len(ws), k) for k in range(24)]
    # alone: one DAG per request, run by itself; and the oracle on the same inputs
    alone, want = [], []
    for m, seed in reqs:
        w = ws[m]
        ins = dict(weights[m])
        ins.update(_request_inputs(w, seed))
        d = Dag(w, options(), resident_inputs=True)
        d.set_inputs(ins)
        d.run()
        alone.append({b: d.output(b) for b in w.output_ids()})
        d.close()
        ref = oracle.run(w, ins)
        want.append({b: oracle.view(w, ref, b) for b in w.output_ids()})
    # in the mix: all queued at once, three slots, admitted as slots free up
    srv = Server(ws, weights, max_slots=3)
    pend = [srv.submit(m, _request_inputs(ws[m], seed)) for m, seed in reqs]
    infos = [abi.dag_server_wait(srv.s, t) for t, _ in pend]
    assert abi.dag_server_slots(srv.s) <= 3
    for (m, seed), (t, outs), ref, exact, info in zip(reqs, pend, alone, want, infos):
        assert info.status == 0 and info.t_done_s >= info.t_launch_s >= info.t_arrive_s
        for b, got in outs.items():
            dt = ws[m].buffers[b].dtype
            e = oracle.rel_err(storage_to_f64(got, dt), storage_to_f64(exact[b], dt))
            tol = node_tolerance(ws[m], b)
            assert e <= tol, f"request {seed} (model {m}) buffer {b}: rel err {e:.3e} > {tol}"
            assert np.array_equal(got, ref[b])   # same plan, same tiles: the same bits
    srv.close()


def test_admission_is_bounded_by_free_device_memory():
    import torch
    w = branchy_mlp("bf16", batch=256, width=1024, hidden=1024, out=256, seed=5)
    weights = [w.make_inputs()]
    footprint = sum(b.rows * ((b.cols + 15) // 16 * 16) * (4 if b.dtype == "f32" else 2)
                    for b in w.buffers if b.view_of < 0)
    free, _ = torch.cuda.mem_get_info()
    # leave room for about two slots only
    srv = Server([w], weights, max_slots=16, hbm_reserve_bytes=int(free - 2.5 * footprint - (64 << 20)))
    pend = [srv.submit(0, _request_inputs(w, s)) for s in range(10)]
    for t, _ in pend:
        assert abi.dag_server_wait(srv.s, t).status == 0
    assert 1 <= abi.dag_server_slots(srv.s) <= 2
    srv.close()


def test_requests_overlap_on_the_device():
    ws = _models()
    weights = [w.make_inputs() for w in ws]
    srv = Server(ws, weights, max_slots=16)
    for m, w in enumerate(ws):
        ins = dict(weights[m])
        srv.set_default_io(m, _request_inputs(w, 1000 + m))
        abi.dag_server_warm(srv.s, m, 3)
    seq = [int(x) % len(ws) for x in synth.splitmix64(3, 300)]
    lat, wall, mif = abi.dag_server_simulate(srv.s, seq, 20000.0, 11)
    assert mif >= 2, "requests never overlapped"
    assert np.all(lat > 0)
    srv.close()
