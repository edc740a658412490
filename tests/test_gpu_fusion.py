"""Epilogue fusion on the GPU: elementwise kernels computed inside the
epilogue of the tensor-core GEMM whose output they read.  Each step rounds to
the dtype of the buffer it stands for, so the fused plan must give the same
bits as the unfused one (DAG_FUSE_NONE), match the oracle within tolerance, keep
a legal trace, and give the same bits kernel by kernel and under the paper's
Alg. 1 on streams."""
import numpy as np
import pytest

import oracle
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag, options
from synth import BF16, F32
from synth.workloads import Workload, branchy_mlp, fork_join
from tests.gpu_util import bits_equal, check_trace, compare, written_buffers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _check(w, n_fused, resident=True, **opt):
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    d = Dag(w, options(trace=1, **opt), resident_inputs=resident)
    fused = d.fusion()
    assert sum(h >= 0 for h in fused) == n_fused
    d.set_inputs(ins)
    d.run()
    keep = written_buffers(w, fused)
    got = {b: d.output(b) for b in keep}
    compare(w, got, ref)
    check_trace(w, d)
    d.run(coarse=True)
    assert bits_equal(got, {b: d.output(b) for b in keep}), "kernel-by-kernel launches differ"
    d.run_cq(n_queues=3, components=abi.DAG_TC_PER_KERNEL)
    assert bits_equal(got, {b: d.output(b) for b in keep}), "Alg. 1 on streams differs"
    d.close()
    u = Dag(w, options(**{**opt, "fuse": abi.DAG_FUSE_NONE}), resident_inputs=resident)
    assert all(h < 0 for h in u.fusion())
    u.set_inputs(ins)
    u.run()
    assert bits_equal(got, {b: u.output(b) for b in keep}), "fused and unfused plans differ"
    u.close()


ALL = abi.DAG_FUSE_ALL


def test_branchy_mlp_bf16():
    _check(branchy_mlp(BF16, batch=256, width=512, hidden=1024, out=256, seed=21), 3, fuse=ALL)


def test_branchy_mlp_f32_tensor_cores():
    _check(branchy_mlp(F32, batch=256, width=512, hidden=1024, out=256, seed=22), 3, fuse=ALL)


def test_fork_join_streamed_inputs():
    _check(fork_join(200, seed=23), 1, resident=False, fuse=ALL)


def _chain(M, N, K, x_dt, out_dt, x_view_offset=None, batch=1, act="gelu", seed=0):
    """gemm (bf16, + bias) -> activation (bf16) -> + X -> out, X an input."""
    w = Workload(f"chain_{M}x{N}x{K}")
    A = w.buf(batch * M, K, BF16, "input", ("uniform", seed + 1))
    B = w.buf(batch * K, N, BF16, "input", ("normal", seed + 2, 0.05))
    bias = w.buf(1, N, F32, "input", ("normal", seed + 3, 0.1))
    C = w.buf(batch * M, N, BF16)
    w.node("gemm", A, C, b=B, bias=bias, batch=batch)
    S = w.buf(batch * M, N, BF16)
    w.node("unary", C, S, act=act)
    if x_view_offset is None:
        X = w.buf(batch * M, N, x_dt, "input", ("uniform", seed + 4))
    else:
        P = w.buf(batch * M, N + x_view_offset, x_dt, "input", ("uniform", seed + 4))
        X = w.buf(batch * M, N, x_dt, "inter", view_of=P, col_offset=x_view_offset)
    w.node("add", S, w.buf(batch * M, N, out_dt, "output"), b=X)
    return w


@pytest.mark.parametrize("case", [
    dict(M=256, N=256, K=128, x_dt=F32, out_dt=F32),
    dict(M=200, N=100, K=96, x_dt=BF16, out_dt=BF16, resident=False), # ragged; X uploaded each submit
    dict(M=130, N=72, K=64, x_dt=F32, out_dt=BF16, x_view_offset=3),  # X rows not 16-byte aligned
    dict(M=100, N=160, K=80, x_dt=BF16, out_dt=F32, batch=3, act="relu"),
], ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_activation_then_add_chain(case):
    case = dict(case)
    resident = case.pop("resident", True)
    _check(_chain(**case, seed=31), 1, resident=resident, fuse=abi.DAG_FUSE_ACT)
    _check(_chain(**case, seed=32), 2, resident=resident, fuse=ALL)


def test_split_k_gemm_with_a_fused_add():
    """A long-K GEMM on a level with few tiles is split; its finishing partials
    also run the fused add (waiting for the partials and for X)."""
    w = Workload("split_fused")
    A = w.buf(256, 4096, BF16, "input", ("uniform", 41))
    B = w.buf(4096, 512, BF16, "input", ("normal", 42, 0.02))
    C = w.buf(256, 512, BF16)
    w.node("gemm", A, C, b=B)
    A2 = w.buf(256, 256, BF16, "input", ("uniform", 43))
    B2 = w.buf(256, 512, BF16, "input", ("normal", 44, 0.05))
    X = w.buf(256, 512, F32)
    w.node("gemm", A2, X, b=B2)
    w.node("add", C, w.buf(256, 512, F32, "output"), b=X)
    d = Dag(w, options(fuse=ALL))
    splits = {int(t[0]): int(t[5]) >> 16 for t in d.tiles()}
    d.close()
    assert splits[0] & 0xFF >= 2, "the long-K GEMM should be split"
    _check(w, 1, fuse=ALL)
