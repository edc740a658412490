"""Sibling GEMMs merged by the planner (dag_options.merge): GEMMs that read one
A with resident weights of their own run as one GEMM over their summed width,
their weights, biases and outputs laid out as column slices of parent
buffers.  Every output element is the same dot product in the same K order,
so a merged plan gives the bits of the unmerged one; both match the FP64
oracle, the trace stays dependency-legal when each merged tile stands for
its siblings' shares (Def. 5), and Alg. 1's streams (§4) give the same bits."""
import numpy as np
import pytest

import oracle
import synth
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag, options
from synth import BF16, F32
from synth.workloads import Workload, encoder_block
from tests.gpu_util import bits_equal, check_trace, compare, written_buffers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _siblings(dt, bias, act, widths, M=640, K=320, seed=0):
    w = Workload(f"siblings_{dt}_{'b' if bias else 'nb'}_{act}")
    X = w.buf(M, K, dt, "input", ("uniform", seed + 1))
    for i, N in enumerate(widths):
        W = w.buf(K, N, dt, "input", ("normal", seed + 10 + i, 0.05))
        b = w.buf(1, N, F32, "input", ("normal", seed + 30 + i, 0.5)) if bias else -1
        O = w.buf(M, N, dt, "inter")
        w.node("gemm", X, O, b=W, bias=b, act=act)
        w.node("unary", O, w.buf(M, N, F32, "output"), act="relu")
    return w


def _run(w, ins, o):
    d = Dag(w, o, resident_inputs=True)
    try:
        d.set_inputs(ins)
        d.run()
        got = {b: d.output(b) for b in written_buffers(w, d.fusion())}
        check_trace(w, d)
        lead, off = d.merges()
        d.run(coarse=True)
        assert bits_equal(got, {b: d.output(b) for b in got}), "coarse and fine paths differ"
        cq = {}
        for comps in (abi.DAG_TC_WHOLE, abi.DAG_TC_PER_KERNEL):
            d.run_cq(n_queues=2, components=comps)
            cq[comps] = {b: d.output(b) for b in got}
    finally:
        d.close()
    for comps, g in cq.items():
        assert bits_equal(got, g), f"Alg. 1 (components {comps}) differs"
    return got, lead, off


@pytest.mark.parametrize("dt", [BF16, F32])
@pytest.mark.parametrize("bias,act", [(False, "none"), (True, "gelu")])
def test_merged_siblings_give_the_bits_of_their_own_gemms(dt, bias, act):
    w = _siblings(dt, bias, act, [64, 128, 32, 64, 96])
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    got, lead, off = _run(w, ins, options(trace=1))
    gemms = [v for v, n in enumerate(w.nodes) if n.op == "gemm"]
    assert [lead[v] for v in gemms] == [gemms[0]] * len(gemms), "siblings not merged"
    assert [off[v] for v in gemms] == [0, 64, 192, 224, 288]
    compare(w, got, ref)
    alone, lead1, _ = _run(w, ins, options(trace=1, merge=1))
    assert all(h < 0 for h in lead1)
    assert bits_equal(got, alone)


def test_encoder_projections_merged_across_heads():
    """The encoder block's 12 Q/K/V projections (4 heads of 64) read one X:
    one GEMM of 768 columns; the heads then read their Q, K and V as column
    slices of it."""
    w = encoder_block(batch=2, seq=128, d_model=256, heads=4, d_head=64, ffn=512, seed=21)
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    got, lead, off = _run(w, ins, options(trace=1))
    proj = [v for v, n in enumerate(w.nodes) if (n.name or "").startswith("proj_")]
    assert len(proj) == 12 and len({lead[v] for v in proj}) == 1 and lead[proj[0]] == proj[0]
    assert sorted(off[v] for v in proj) == list(range(0, 768, 64))
    compare(w, got, ref)
    alone, _, _ = _run(w, ins, options(trace=1, merge=1))
    assert bits_equal(got, alone)


@pytest.mark.parametrize("dt", [BF16, F32])
def test_merged_weights_read_back_and_update(dt):
    """A merged sibling's weight is a slice of its parent (kept K-major): it
    reads back as given, and a new upload of one weight changes exactly that
    sibling's output, as the oracle says."""
    w = _siblings(dt, True, "relu", [64, 64, 128], seed=5)
    ins = w.make_inputs()
    d = Dag(w, options(), resident_inputs=True)
    try:
        assert any(h >= 0 for h in d.merges()[0])
        d.set_inputs(ins)
        d.run()
        for b in w.input_ids():
            assert np.array_equal(d.output(b).view(np.uint8), ins[b].view(np.uint8)), f"input {b} reads back changed"
        W1 = [n.b for n in w.nodes if n.op == "gemm"][1]
        ins2 = dict(ins)
        b = w.buffers[W1]
        ins2[W1] = synth.fill("normal", 999, (b.rows, b.cols), b.dtype, 0.05)
        d.set_inputs({W1: ins2[W1]})
        d.run()
        got = {b: d.output(b) for b in written_buffers(w, d.fusion())}
    finally:
        d.close()
    compare(w, got, oracle.run(w, ins2))


@pytest.mark.parametrize("dt", [BF16, F32])
def test_merged_siblings_with_split_k(dt):
    """Siblings with a long K loop on a level of few tiles: the merged GEMM
    also splits K (bf16: 128 x 64 tiles in two partials; f32: the wide 3 x TF32
    form over the parent weight kept K-major, in four), within the oracle's
    tolerance and with the same bits on every submit path."""
    w = _siblings(dt, True, "relu", [64, 64, 128], M=256, K=2048, seed=3)
    ins = w.make_inputs()
    d = Dag(w, options(), resident_inputs=True)
    try:
        tiles = d.tiles()
    finally:
        d.close()
    gemm = [v for v, n in enumerate(w.nodes) if n.op == "gemm"]
    mine = tiles[tiles[:, 0] == gemm[0]]
    assert len(mine) == len(tiles[np.isin(tiles[:, 0], gemm)]) and ((mine[:, 5] >> 16) & 0xFF).max() >= 2
    got, lead, _ = _run(w, ins, options(trace=1))
    assert [lead[v] for v in gemm] == [gemm[0]] * 3
    compare(w, got, oracle.run(w, ins))


def test_merge_parents_are_not_caller_buffers():
    """The parent buffers the planner adds for a merged group are internal:
    every buffer call rejects their ids as it rejects any id the caller did
    not describe, while the siblings' own buffers stay addressable."""
    w = _siblings(BF16, True, "relu", [64, 64, 128], seed=7)
    d = Dag(w, options(), resident_inputs=True)
    host = np.zeros(1 << 20, np.uint8)
    try:
        assert any(h >= 0 for h in d.merges()[0])
        nb = len(w.buffers)
        for bad in (nb, nb + 1, nb + 2, -1):
            for call in (abi.dag_set_input, abi.dag_set_output, abi.dag_get_output):
                with pytest.raises(abi.DagError) as e:
                    call(d.h, bad, host.ctypes.data)
                assert e.value.status == abi.DAG_EINVAL
            assert not abi.dag_device_ptr(d.h, bad)[0]
        d.set_inputs(w.make_inputs())
        d.run()
        O = [n.out for n in w.nodes if n.op == "gemm"][1]
        assert abi.dag_device_ptr(d.h, O)[0]
    finally:
        d.close()
