"""dag_run_noalloc: the entry point for callers that cannot allocate device
memory (their device memory is fully reserved by their own pool, or they run
inside an allocator or an error path).  On two calls in a row (the fixed
working area is reused and must be cleared between calls) it must give the
same bits as the dag_create / dag_submit path planned the same way (no split
K, the caller's weight layout), and values within the per-buffer tolerance
of the FP64 oracle; it must accept caller row pitches wider than the
library's own (with head outputs written as column slices of a wider
buffer); and it must turn away a DAG whose plan does not fit that fixed area.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import oracle
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import describe, options
from synth import BF16, F32, storage_to_f64
from synth.workloads import Workload, encoder_block, fork_join
from tests.gpu_util import node_tolerance, run_gpu, written_buffers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _caller_buffers(w, inputs, extra=0):
    """Device buffers owned by the caller (this test), one per root buffer,
    with a row pitch of round_up(cols, 16) + `extra` elements; inputs copied
    in."""
    import torch
    tensors, ptrs, pitch = {}, [], []
    for i, b in enumerate(w.buffers):
        if b.view_of >= 0:
            ptrs.append(0)
            pitch.append(0)
            continue
        ld = (b.cols + 15) // 16 * 16 + extra
        t = torch.zeros((b.rows, ld), dtype=torch.float32 if b.dtype == F32 else torch.int16, device="cuda")
        if i in inputs:
            arr = inputs[i] if b.dtype == F32 else inputs[i].view(np.int16)
            t[:, : b.cols].copy_(torch.from_numpy(np.ascontiguousarray(arr)))
        tensors[i] = t
        ptrs.append(t.data_ptr())
        pitch.append(ld)
    torch.cuda.synchronize()
    return tensors, ptrs, pitch


def _read(w, tensors, bid):
    b = w.buffers[bid]
    root = bid if b.view_of < 0 else b.view_of
    off = 0 if b.view_of < 0 else b.col_offset
    a = tensors[root][:, off: off + b.cols].cpu().numpy()
    return np.ascontiguousarray(a if b.dtype == F32 else a.view(np.uint16))


@pytest.mark.parametrize("extra", [0, 48], ids=["pitch_16", "pitch_wide"])
@pytest.mark.parametrize("make", [
    lambda: fork_join(256, seed=5),
    lambda: encoder_block(batch=2, seq=128, d_model=256, heads=4, d_head=64, ffn=512, seed=13),
], ids=["fork_join_f32", "encoder_bf16"])
def test_no_alloc_matches_the_allocating_path_twice(make, extra):
    import torch
    w = make()
    ins = w.make_inputs()
    # the dag_create / dag_submit path, planned as the no-alloc path plans:
    # no split K (it needs scratch memory), weights in the caller's layout
    ref = run_gpu(w, ins, resident=True, opts=options(split_k=1, keep_layout=1))
    exact = oracle.run(w, ins)
    nodes, _, bufs = describe(w, resident_inputs=True)
    written = written_buffers(w, abi.dag_fusion_host(nodes, [], bufs))
    assert set(written) <= set(ref)
    tensors, ptrs, pitch = _caller_buffers(w, ins, extra)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        for bid in written:               # outputs start from garbage each call
            root = bid if w.buffers[bid].view_of < 0 else w.buffers[bid].view_of
            tensors[root].fill_(-1)
        torch.cuda.synchronize()
        st = abi.dag_run_noalloc(nodes, bufs, ptrs, pitch, None, stream)
        assert st == abi.DAG_OK, abi.last_error()
        for bid in written:
            got = _read(w, tensors, bid)
            assert np.array_equal(got.view(np.uint8), ref[bid].view(np.uint8)), (call, bid)
            dt = w.buffers[bid].dtype
            err = oracle.rel_err(storage_to_f64(got, dt), storage_to_f64(oracle.view(w, exact, bid), dt))
            assert err <= node_tolerance(w, bid), (call, bid, err)
        # the pitch padding of every caller buffer is left as the caller wrote it
        for root, t in tensors.items():
            if extra and root in {b if w.buffers[b].view_of < 0 else w.buffers[b].view_of for b in written}:
                pad = t[:, w.buffers[root].cols + (-w.buffers[root].cols) % 16:]
                assert bool((pad == -1).all()), (call, root)


def test_no_alloc_rejects_a_plan_larger_than_its_fixed_area():
    import torch
    # 16384 x 32768 f32 GEMM: 32768 tiles of 128 x 128, far beyond the fixed area
    w = Workload("too_big")
    A = w.buf(16384, 64, F32, "input", ("uniform", 1))
    B = w.buf(64, 32768, F32, "input", ("uniform", 2))
    C = w.buf(16384, 32768, F32, "output")
    w.node("gemm", A, C, b=B)
    nodes, _, bufs = describe(w, resident_inputs=True)
    tensors, ptrs, pitch = _caller_buffers(w, {})
    st = abi.dag_run_noalloc(nodes, bufs, ptrs, pitch, None, torch.cuda.current_stream().cuda_stream)
    assert st == abi.DAG_ENOMEM
    assert "fixed scratch" in abi.last_error()
    del tensors
    torch.cuda.empty_cache()
