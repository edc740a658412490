"""The per-buffer parity tolerance of the GPU tests (tests/gpu_util.py): the
bf16 tolerance (2e-2) only for buffers whose values depend on bf16
arithmetic -- a bf16-stored buffer, the output of a GEMM with bf16 operands,
and what is computed from either -- and the f32 tolerance (1e-5) for every
other buffer, also inside one batch that mixes bf16 and f32 DAGs."""
from synth import BF16, F32
from synth.workloads import Workload, concat, encoder_block, fork_join, random_layered
from tests.gpu_util import TOL, bf16_tainted, node_tolerance


def test_mixed_batch_keeps_f32_dags_at_the_f32_tolerance():
    parts = [random_layered(2000 + i, 6, 24, 4, sizes=(64, 128, 256)) for i in range(12)]
    parts += [fork_join(128, seed=3), encoder_block(batch=2, seq=64, d_model=128, heads=4, d_head=32, ffn=256, seed=4)]
    w = concat(parts)
    off = 0
    n_f32 = n_bf16 = 0
    for x in parts:
        bf = any(b.dtype == BF16 for b in x.buffers)
        for b in x.output_ids():
            assert node_tolerance(w, off + b) == (TOL[BF16] if bf else TOL[F32]), (x.name, b)
            n_bf16 += bf
            n_f32 += not bf
        off += len(x.buffers)
    assert n_f32 and n_bf16


def test_taint_follows_producers_not_the_dag():
    w = Workload("taint")
    a16 = w.buf(4, 8, BF16, "input", ("uniform", 1))
    a32 = w.buf(4, 8, F32, "input", ("uniform", 2))
    r32 = w.buf(4, 8, F32, "inter")     # relu of exact bf16 input values: exact in f32
    w.node("unary", a16, r32, act="relu")
    s32 = w.buf(4, 8, F32, "output")    # f32 arithmetic only
    w.node("add", r32, s32, b=a32)
    r16 = w.buf(4, 8, BF16, "inter")    # stored bf16: rounded once
    w.node("unary", a16, r16, act="relu")
    b16 = w.buf(8, 8, BF16, "input", ("uniform", 3))
    g32 = w.buf(4, 8, F32, "inter")     # bf16 GEMM, f32 output
    w.node("gemm", r16, g32, b=b16)
    y = w.buf(4, 8, F32, "output")      # downstream of the bf16 GEMM
    w.node("unary", g32, y, act="relu")
    par = w.buf(4, 16, F32, "output")   # written through two views, one tainted
    v0 = w.buf(4, 8, F32, "inter", view_of=par, col_offset=0)
    v1 = w.buf(4, 8, F32, "inter", view_of=par, col_offset=8)
    w.node("unary", a32, v0, act="relu")
    w.node("unary", g32, v1, act="relu")
    t = bf16_tainted(w)
    assert {r16, g32, y, v1, par} <= t
    assert not ({a16, a32, r32, s32, v0} & t)
    assert node_tolerance(w, s32) == TOL[F32] and node_tolerance(w, y) == TOL[BF16]
