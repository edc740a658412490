"""Resident GEMM weights kept transposed (K-major) on the device: the same
bits as with the caller's layout (keep_layout = 1), on every submit path,
with batched B blocks and shared weights; the weight reads back in the
caller's layout; buffers that are not pure B operands keep theirs."""
import numpy as np
import pytest

import oracle
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag, options
from synth import BF16, F32
from synth.workloads import Workload, branchy_mlp, transformer_heads
from tests.gpu_util import bits_equal, check_trace, compare, written_buffers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _run(w, ins, **opt):
    d = Dag(w, options(trace=1, **opt), resident_inputs=True)
    d.set_inputs(ins)
    d.run()
    keep = written_buffers(w)
    out = {b: d.output(b) for b in keep}
    check_trace(w, d)
    d.run(coarse=True)
    assert bits_equal(out, {b: d.output(b) for b in keep}), "kernel-by-kernel launches differ"
    d.run_cq(n_queues=2, components=abi.DAG_TC_WHOLE)
    assert bits_equal(out, {b: d.output(b) for b in keep}), "Alg. 1 on streams differs"
    return d, out


def _check(w, transposed):
    """Weights kept K-major: oracle parity; and the same bits as the caller's
    layout under one tile form.  f32 GEMMs with a K-major B take the wide
    128 x 128 / 256 tiles by default, whose partial sums are cut differently
    from the 128 x 64 tiles an MN-major B gets, so for the bit comparison
    both runs use the 128 x 64 form (DAG_F32_GEMM_TENSOR_NARROW)."""
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    d, got = _run(w, ins)
    compare(w, got, ref)
    for b, want in transposed.items():
        assert (abi.dag_device_ptr(d.h, b)[0] is None) == want, b
    # every input reads back in the caller's layout
    for b in w.input_ids():
        assert np.array_equal(d.output(b).view(np.uint8), np.ascontiguousarray(ins[b]).view(np.uint8)), b
    d.close()
    f32 = any(w.buffers[n.a].dtype == F32 for n in w.nodes if n.op == "gemm")
    form = {"f32_gemm": abi.DAG_F32_GEMM_TENSOR_NARROW} if f32 else {}
    if f32:
        n, got = _run(w, ins, **form)
        compare(w, got, ref)
        n.close()
    u, base = _run(w, ins, keep_layout=1, **form)
    for b in transposed:
        assert abi.dag_device_ptr(u.h, b)[0] is not None
    u.close()
    assert bits_equal(got, base), "K-major and caller-layout weights give different bits"


def test_branchy_mlp_bf16():
    w = branchy_mlp(BF16, batch=256, width=512, hidden=1024, out=256, seed=51)
    weights = {n.b: True for n in w.nodes if n.op == "gemm"}
    _check(w, weights)


def test_branchy_mlp_f32():
    w = branchy_mlp(F32, batch=256, width=512, hidden=1024, out=256, seed=52)
    _check(w, {n.b: True for n in w.nodes if n.op == "gemm"})


def test_transformer_heads_f32():
    w = transformer_heads(2, 64, seed=53)
    _check(w, {})


def test_batched_shared_and_mixed_use():
    w = Workload("layouts")
    # batched B blocks: 3 x (96 x 200), one per batch
    A = w.buf(3 * 100, 96, BF16, "input", ("uniform", 61))
    Bb = w.buf(3 * 96, 200, BF16, "input", ("normal", 62, 0.05))
    C = w.buf(3 * 100, 200, F32, "output")
    w.node("gemm", A, C, b=Bb, batch=3)
    # one weight shared by two GEMMs of one shape
    X1 = w.buf(130, 64, BF16, "input", ("uniform", 63))
    X2 = w.buf(130, 64, BF16, "input", ("uniform", 64))
    W = w.buf(64, 72, BF16, "input", ("normal", 65, 0.1))
    w.node("gemm", X1, w.buf(130, 72, F32, "output"), b=W)
    w.node("gemm", X2, w.buf(130, 72, F32, "output"), b=W)
    # a buffer read as B by one GEMM and as A by another keeps its layout
    Q = w.buf(64, 64, BF16, "input", ("normal", 66, 0.1))
    w.node("gemm", X1, w.buf(130, 64, BF16, "output"), b=Q)
    w.node("gemm", Q, w.buf(64, 64, F32, "output"), b=w.buf(64, 64, BF16, "input", ("uniform", 67)))
    _check(w, {Bb: True, W: True, Q: False})


def test_streamed_weights_keep_the_callers_layout():
    w = branchy_mlp(BF16, batch=128, width=256, hidden=512, out=128, seed=54)
    ins = w.make_inputs()
    d = Dag(w, options(), resident_inputs=False)
    assert all(abi.dag_device_ptr(d.h, n.b)[0] is not None for n in w.nodes if n.op == "gemm")
    d.set_inputs(ins)
    d.run()
    compare(w, {b: d.output(b) for b in written_buffers(w)}, oracle.run(w, ins))
    d.close()
