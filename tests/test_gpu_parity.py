"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Sizes here span several tiles with ragged tails; the full workload sizes are
in test_gpu_full.py.  Tolerances (normwise per buffer): 1e-5 for f32 nodes,
2e-2 for bf16-input / f32-accumulate nodes.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.dag import Dag, options
from synth import BF16, F32
from synth.workloads import Workload, branchy_mlp, encoder_block, fork_join, from_arrays, random_layered
from tests.gpu_util import bits_equal, check_trace, compare, run_gpu, written_buffers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _roundtrip(w, opts=None, coarse_too=True):
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    d = Dag(w, opts or options(trace=1))
    d.set_inputs(ins)
    d.run()
    got = {b: d.output(b) for b in written_buffers(w, d.fusion())}
    errs = compare(w, got, ref)
    check_trace(w, d)
    if coarse_too:
        d.run(coarse=True)
        got_c = {b: d.output(b) for b in got}
        assert bits_equal(got, got_c), "coarse and fine paths differ"
    d.close()
    return errs


def test_gelu_elementwise_accuracy():
    """GELU (erf form) of every f32 on a dense grid over [-12, 12], element by
    element against the FP64 oracle rounded to f32: within 4e-7 |x| (the
    erf approximation's 1.5e-7 and a few ulp of f32 evaluation of the erfc
    term, scaled by 0.5 |x|) plus two f32 spacings of the result."""
    x = np.linspace(-12.0, 12.0, 512 * 1000).reshape(512, 1000)
    w, ids = from_arrays("gelu_grid", {"x": (x, F32)})
    y = w.buf(512, 1000, F32, "output")
    w.node("unary", ids["x"], y, act="gelu")
    ins = w.make_inputs()
    ref = oracle.run(w, ins)[y]
    got = run_gpu(w, ins)[y]
    xx = ins[ids["x"]].astype(np.float64)
    bound = 4e-7 * np.abs(xx) + 2 * np.spacing(np.abs(ref)).astype(np.float64)
    err = np.abs(got.astype(np.float64) - ref.astype(np.float64))
    assert np.all(err <= bound), float(np.max(err / bound))
    assert got[-1, -1] == np.float32(12.0)


@pytest.mark.parametrize("n", [256, 200, 64, 130])
def test_fork_join_f32(n):
    _roundtrip(fork_join(n, seed=n))


def test_fork_join_bf16():
    _roundtrip(fork_join(256, dtype=BF16))


def _gemm_case(M, N, K, dt, trans_b=0, batch=1, bias=True, act="none", out_dt=F32, scale=1.0, seed=0):
    w = Workload(f"gemm_{M}x{N}x{K}_{dt}_t{trans_b}_b{batch}")
    A = w.buf(batch * M, K, dt, "input", ("uniform", seed + 1))
    B = w.buf(batch * N if trans_b else batch * K, K if trans_b else N, dt, "input", ("uniform", seed + 2))
    bb = w.buf(1, N, F32, "input", ("normal", seed + 3, 0.5)) if bias else -1
    C = w.buf(batch * M, N, out_dt, "output")
    w.node("gemm", A, C, b=B, bias=bb, trans_b=trans_b, batch=batch, act=act, scale=scale)
    return w


GEMM_CASES = [
    dict(M=256, N=256, K=256, dt=BF16),
    dict(M=300, N=200, K=130, dt=BF16),                       # ragged M, N, K
    dict(M=128, N=64, K=64, dt=BF16, trans_b=1),
    dict(M=256, N=512, K=320, dt=BF16, trans_b=1, act="relu"),
    dict(M=100, N=96, K=72, dt=BF16, batch=3),                # batched, ragged per batch
    dict(M=64, N=128, K=200, dt=BF16, batch=4, trans_b=1, act="gelu", out_dt=BF16),
    dict(M=512, N=1024, K=512, dt=BF16, act="gelu", out_dt=BF16, scale=0.5),
    dict(M=256, N=256, K=256, dt=F32),
    dict(M=300, N=200, K=130, dt=F32, act="relu"),
    dict(M=100, N=96, K=72, dt=F32, batch=3, trans_b=1),
    dict(M=77, N=33, K=19, dt=F32, act="gelu", out_dt=BF16),
]


@pytest.mark.parametrize("case", GEMM_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_gemm(case):
    _roundtrip(_gemm_case(**case))


@pytest.mark.parametrize("case", [c for c in GEMM_CASES if c["dt"] == F32],
                         ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_gemm_f32_simt(case):
    """The same f32 cases on the SM cores (exact-f32 FFMA tiles)."""
    _roundtrip(_gemm_case(**case), options(trace=1, f32_gemm=abi.DAG_F32_GEMM_SIMT))


TF32_CASES = [
    dict(M=128, N=64, K=32, dt=F32),                          # one tile, one stage
    dict(M=384, N=640, K=4096, dt=F32, act="relu"),           # long K: the stage ring wraps many times
    dict(M=257, N=65, K=33, dt=F32, trans_b=1),               # ragged in every dimension
    dict(M=200, N=300, K=1000, dt=F32, out_dt=BF16, act="gelu", scale=0.25),
    dict(M=64, N=96, K=160, dt=F32, batch=5),                 # batched, M below one tile
    dict(M=96, N=128, K=96, dt=F32, batch=2, trans_b=1, bias=False),
]


@pytest.mark.parametrize("case", TF32_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_gemm_f32_tensor_cores(case):
    """3 x TF32 tiles within the f32 tolerance (a one-term tf32 product would
    miss it by about two orders of magnitude), in both B layouts."""
    w = _gemm_case(**case)
    d = Dag(w, options())
    assert ((d.tiles()[:, 5] & 0xFFFF) >= 64).all()  # planned as tensor-core f32 tiles
    d.close()
    _roundtrip(w)


def _resident_roundtrip(w, opts=None):
    """Inputs resident (weights read only as B are kept K-major on the
    device); oracle parity, trace legality, and the kernel-by-kernel launch
    giving the same bits.  Returns the planned tile table."""
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    d = Dag(w, opts or options(trace=1), resident_inputs=True)
    d.set_inputs(ins)
    d.run()
    got = {b: d.output(b) for b in written_buffers(w, d.fusion())}
    compare(w, got, ref)
    check_trace(w, d)
    tiles = d.tiles()
    d.run(coarse=True)
    assert bits_equal(got, {b: d.output(b) for b in got}), "coarse and fine paths differ"
    d.close()
    return tiles, got


WIDE_CASES = [
    dict(M=128, N=128, K=16, dt=F32),                         # one tile, one stage, one partial
    dict(M=384, N=640, K=4096, dt=F32, act="relu"),           # 256 stages: 32 partial sums; ragged last tile
    dict(M=257, N=200, K=33, dt=F32),                         # ragged M, N, K (K tail zero-filled)
    dict(M=200, N=300, K=1000, dt=F32, out_dt=BF16, act="gelu", scale=0.25),
    dict(M=64, N=96, K=160, dt=F32, batch=5),                 # batched, M below one tile
    dict(M=96, N=256, K=136, dt=F32, batch=2, trans_b=1, bias=False),
    dict(M=130, N=512, K=2048, dt=F32, trans_b=1, act="relu"),
]


@pytest.mark.parametrize("bn", [128, 256])
@pytest.mark.parametrize("case", WIDE_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_gemm_f32_wide_tiles(case, bn):
    """The wide 3 x TF32 form (128 x 128 / 128 x 256 tiles, B K-major, K in
    stages of 16, partial sums every 128 of K added up in f32) within the
    f32 tolerance of the oracle, in both launch forms, whole K per tile."""
    w = _gemm_case(**case)
    tiles, _ = _resident_roundtrip(w, options(trace=1, tile_override=bn, split_k=1))
    assert set((tiles[:, 5] & 0xFFFF).tolist()) == {bn}, "not planned as wide f32 tiles of that width"
    assert not ((tiles[:, 5] >> 16) > 0).any()


def test_gemm_f32_wide_and_narrow_agree_with_the_oracle():
    """The same f32 GEMM in the wide and the 128 x 64 form: both within the
    f32 tolerance (their bits differ: the partial sums are cut differently)."""
    w = _gemm_case(M=256, N=384, K=1536, dt=F32, act="relu")
    t_w, g_w = _resident_roundtrip(w, options(trace=1, f32_gemm=abi.DAG_F32_GEMM_TENSOR_WIDE))
    t_n, g_n = _resident_roundtrip(w, options(trace=1, f32_gemm=abi.DAG_F32_GEMM_TENSOR_NARROW))
    assert set((t_w[:, 5] & 0xFFFF).tolist()) <= {128, 256} and set((t_n[:, 5] & 0xFFFF).tolist()) == {64}


WIDE_SPLIT_CASES = [
    dict(M=128, N=256, K=2048, dt=F32),                       # one output tile: 4 partials
    dict(M=200, N=130, K=1000, dt=F32, act="gelu", out_dt=BF16),
    dict(M=64, N=192, K=1024, dt=F32, batch=2, trans_b=1, scale=0.5),
]


@pytest.mark.parametrize("case", WIDE_SPLIT_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_gemm_f32_wide_split_k(case):
    """A wide f32 GEMM with few output tiles runs as split-K partials summed
    in a fixed order by the finishing tile: within the f32 tolerance, and the
    same bits on every run, grid size and on Alg. 1's streams."""
    w = _gemm_case(**case)
    wide = abi.DAG_F32_GEMM_TENSOR_WIDE
    tiles, outs = _resident_roundtrip(w, options(trace=1, f32_gemm=wide))
    assert ((tiles[:, 5] >> 16) > 0).any(), "not split"
    assert set((tiles[:, 5] & 0xFFFF).tolist()) <= {128, 256}
    ins = w.make_inputs()
    for o in (options(max_ctas=3, f32_gemm=wide), options(max_ctas=1, f32_gemm=wide), options(f32_gemm=wide)):
        d = Dag(w, o, resident_inputs=True)
        d.set_inputs(ins)
        d.run()
        again = {b: d.output(b) for b in outs}
        d.run_cq(n_queues=2, components=abi.DAG_TC_PER_KERNEL)
        cq = {b: d.output(b) for b in outs}
        d.close()
        assert bits_equal(outs, again) and bits_equal(outs, cq)


def test_wide_f32_tiles_between_other_tensor_tiles_in_one_cta():
    """One CTA (and three) running bf16 tiles, wide f32 tiles of 256 columns
    (which hold both TMEM accumulator buffers), wide ones of 128 and 128 x 64
    f32 tiles in turn: the accumulator hand-over between them stays right."""
    w = Workload("mixed_wide")
    outs = []
    specs = [(BF16, 256, 0), (F32, 256, 1), (BF16, 128, 0), (F32, 128, 1), (F32, 64, 1), (F32, 512, 1),
             (BF16, 64, 1)]
    for i, (dt, N, tb) in enumerate(specs):
        K = 96 + 32 * i
        # 2048 rows: enough tiles per level that the planner keeps 256-column tiles
        A = w.buf(2048, K, dt, "input", ("uniform", 40 + i))
        B = w.buf(N if tb else K, K if tb else N, dt, "input", ("uniform", 60 + i))
        C = w.buf(2048, N, F32, "output")
        w.node("gemm", A, C, b=B, trans_b=tb, act="relu")
        outs.append(C)
    base = None
    for o in (options(trace=1, max_ctas=1), options(trace=1, max_ctas=1, scheduler=abi.DAG_SCHED_FIFO),
              options(trace=1, max_ctas=3), options(trace=1)):
        tiles, got = _resident_roundtrip(w, o)
        kinds = set((tiles[:, 5] & 0xFFFF).tolist())
        assert {64, 128, 256} <= kinds
        if base is None:
            base = got
        assert bits_equal(base, got)


def test_wide_f32_single_partial_tiles_after_long_epilogues():
    """256-column wide f32 tiles with one partial (K <= 128), each right
    after a tile whose epilogue is long (GELU, bf16 out) or whose partials
    are many, in one CTA and in three: the MMA issuer starts such a tile in
    the buffer the previous one freed early and takes the other buffer's
    release in turn, so the hand-over holds whichever side is first."""
    w = Workload("wide_single_partial")
    outs = []
    for i, K in enumerate([64, 2048, 16, 128, 1024, 48, 64]):
        A = w.buf(2048, K, F32, "input", ("uniform", 80 + i))
        B = w.buf(512, K, F32, "input", ("uniform", 90 + i))
        C = w.buf(2048, 512, BF16 if K >= 1024 else F32, "output")
        w.node("gemm", A, C, b=B, trans_b=1, act="gelu" if K >= 1024 else "relu")
        outs.append(C)
    wide = abi.DAG_F32_GEMM_TENSOR_WIDE
    base = None
    for o in (options(trace=1, max_ctas=1, f32_gemm=wide, tile_override=256, split_k=1),
              options(trace=1, max_ctas=3, f32_gemm=wide, tile_override=256, split_k=1)):
        tiles, got = _resident_roundtrip(w, o)
        assert set((tiles[:, 5] & 0xFFFF).tolist()) == {256}
        if base is None:
            base = got
        assert bits_equal(base, got)


@pytest.mark.parametrize("K,bn", [(16, 256), (200, 128), (2048, 256), (1000, 128)])
def test_wide_f32_weight_kept_k_major_matches_the_callers_k_major_copy(K, bn):
    """A resident f32 weight W (K x N, trans_b = 0) is kept K-major on the
    device, made at upload, so that wide f32 tiles can read it.  The same
    GEMM over the caller's own K-major copy W^T (trans_b = 1) gives the same
    bits; both match the oracle, and the transposed copy takes exactly the
    device memory of the caller's N x K form."""
    M, N = 640, 512
    outs = {}
    mem = {}
    for form in ("kn", "nk"):
        w = Workload("k_major_" + form)
        A = w.buf(M, K, F32, "input", ("uniform", 11))
        W = w.buf(K, N, F32, "input", ("uniform", 12)) if form == "kn" else w.buf(N, K, F32, "input")
        C = w.buf(M, N, F32, "output")
        w.node("gemm", A, C, b=W, trans_b=0 if form == "kn" else 1, act="relu")
        if form == "kn":
            ins = w.make_inputs()
        else:
            ins = {A: base_ins[A], W: np.ascontiguousarray(base_ins[W].T)}
        ref = oracle.run(w, ins)
        d = Dag(w, options(trace=1, f32_gemm=abi.DAG_F32_GEMM_TENSOR_WIDE, tile_override=bn, split_k=1),
                resident_inputs=True)
        try:
            assert set((d.tiles()[:, 5] & 0xFFFF).tolist()) == {bn}
            d.set_inputs(ins)
            d.run()
            got = {C: d.output(C)}
            compare(w, got, ref)
            check_trace(w, d)
            outs[form] = got[C]
            mem[form] = abi.dag_plan_get(d.h).buffer_bytes
        finally:
            d.close()
        if form == "kn":
            base_ins = ins
    assert np.array_equal(outs["kn"].view(np.uint32), outs["nk"].view(np.uint32))
    assert mem["kn"] == mem["nk"] > 0


def test_f32_unaligned_view_runs_on_simt_tiles():
    w = Workload("f32_view")
    P = w.buf(256, 100, F32, "input", ("uniform", 1))
    A = w.buf(256, 96, F32, "inter", view_of=P, col_offset=1)   # 4-byte offset: no TMA
    C = w.buf(256, 200, F32, "output")
    w.node("gemm", A, C, b=w.buf(96, 200, F32, "input", ("uniform", 2)))
    d = Dag(w, options())
    assert set(d.tiles()[:, 5].tolist()) <= {0, 1, 2}
    d.close()
    _roundtrip(w)


def test_bf16_and_f32_gemms_interleaved_in_one_cta():
    """One CTA runs bf16 and f32 tensor-core tiles alternately, so stages of
    the ring change hands between the MMA issuer and the splitter warps."""
    w = Workload("mixed")
    xs = []
    for i, dt in enumerate([BF16, F32, BF16, F32]):
        A = w.buf(256, 192 + 64 * i, dt, "input", ("uniform", 10 + i))
        B = w.buf(192 + 64 * i, 128, dt, "input", ("uniform", 20 + i))
        C = w.buf(256, 128, F32, "inter")
        w.node("gemm", A, C, b=B, act="relu")
        xs.append(C)
    S = w.buf(256, 128, F32, "inter")
    w.node("add", xs[0], S, b=xs[1])
    T = w.buf(256, 128, F32, "inter")
    w.node("add", xs[2], T, b=xs[3])
    U = w.buf(256, 128, F32, "output")
    w.node("add", S, U, b=T)
    for sched in (abi.DAG_SCHED_RANK_MODEL, abi.DAG_SCHED_FIFO):
        _roundtrip(w, options(trace=1, max_ctas=1, scheduler=sched), coarse_too=False)
    _roundtrip(w, options(trace=1))


@pytest.mark.parametrize("bn", [64, 128, 256])
@pytest.mark.parametrize("trans_b", [0, 1])
@pytest.mark.parametrize("out_dt", [F32, BF16])
def test_gemm_bf16_every_tile_width(bn, trans_b, out_dt):
    # N = 600: a ragged last n-tile for every width; every output chunk width
    w = _gemm_case(384, 600, 448, BF16, trans_b=trans_b, act="relu", out_dt=out_dt)
    _roundtrip(w, options(trace=1, tile_override=bn), coarse_too=False)


@pytest.mark.parametrize("N,dt_in,dt_out,scale", [(256, F32, BF16, 0.125), (1000, F32, F32, 1.0),
                                                  (2048, BF16, F32, 0.5), (33, BF16, BF16, 2.0),
                                                  # vector path (N a multiple of 4, at most 256): both
                                                  # halves of a lane's elements, one, and partial rows
                                                  (128, BF16, BF16, 1.0), (252, F32, F32, 1.0),
                                                  (4, F32, BF16, 1.0), (60, BF16, F32, 0.25), (132, F32, F32, 0.5),
                                                  # rows of 257..2048 held in registers (4 / 8 / 16 groups
                                                  # of 4 per lane), ragged last groups, and the fallbacks
                                                  # beyond (N > 2048, N not a multiple of 4)
                                                  (260, F32, F32, 1.0), (516, BF16, BF16, 0.5), (772, F32, BF16, 1.0),
                                                  (1500, BF16, F32, 0.125), (2044, F32, F32, 0.25),
                                                  (2052, F32, F32, 1.0), (1023, BF16, BF16, 1.0)])
def test_softmax(N, dt_in, dt_out, scale):
    w = Workload("softmax")
    x = w.buf(300, N, dt_in, "input", ("uniform", 5))
    s = w.buf(300, N, dt_in, name="xs")
    y = w.buf(300, N, dt_out, "output")
    w.node("unary", x, s)          # routes the input through a producer tile
    w.node("softmax", s, y, scale=scale * 8)
    _roundtrip(w)


@pytest.mark.parametrize("cols", [2048, 1001, 8, 3])
@pytest.mark.parametrize("dt", [F32, BF16])
def test_eltwise(cols, dt):
    w = Workload("elt")
    a = w.buf(70, cols, dt, "input", ("uniform", 1))
    b = w.buf(70, cols, F32, "input", ("uniform", 2))
    c = w.buf(70, cols, dt, name="c")
    y = w.buf(70, cols, F32, "output")
    w.node("add", a, c, b=b, act="relu")
    w.node("unary", c, y, act="gelu")
    _roundtrip(w)


@pytest.mark.parametrize("dt", [F32, BF16])
def test_branchy_mlp_small(dt):
    _roundtrip(branchy_mlp(dt, batch=200, width=256, hidden=512, out=128, seed=7))


def test_encoder_small():
    _roundtrip(encoder_block(batch=2, seq=128, d_model=256, heads=4, d_head=64, ffn=512, seed=9))


@pytest.mark.parametrize("seed", [1000, 1001, 1002, 1003])
def test_random_layered_small(seed):
    _roundtrip(random_layered(seed, 6, 16, 4, sizes=(64, 128, 256)))


def test_schedules_and_grid_sizes_give_identical_bits():
    """No reduction is split across tiles, so every legal schedule gives the same bits."""
    w = encoder_block(batch=2, seq=128, d_model=256, heads=4, d_head=64, ffn=512, seed=11)
    ins = w.make_inputs()
    base = run_gpu(w, ins)
    for o in (options(scheduler=abi.DAG_SCHED_FIFO), options(max_ctas=1), options(max_ctas=7),
              options(scheduler=abi.DAG_SCHED_FIFO, max_ctas=3)):
        assert bits_equal(base, run_gpu(w, ins, opts=o))


def test_streamed_inputs_and_repeated_submits():
    """Inputs uploaded on the copy streams each submit (ready flags) give the
    same bits as resident inputs, over several submits (epoch counters)."""
    w = branchy_mlp(BF16, batch=128, width=256, hidden=256, out=128, seed=3)
    ins = w.make_inputs()
    base = run_gpu(w, ins, resident=True)
    d = Dag(w)
    d.set_inputs(ins)
    for _ in range(3):
        d.run()
        assert bits_equal(base, {b: d.output(b) for b in base})
    # new data in the streamed input changes the result; the old data restores it
    X = w.input_ids()[0]
    ins2 = dict(ins)
    ins2[X] = synth.to_storage(synth.uniform(99, (128, 256)), BF16)
    d.set_inputs({X: ins2[X]})
    d.run()
    ref2 = oracle.run(w, ins2)
    compare(w, {b: d.output(b) for b in base}, ref2)
    d.set_inputs({X: ins[X]}, pinned=True)
    d.run()
    assert bits_equal(base, {b: d.output(b) for b in base})
    d.close()


def test_device_wait_timeout_reports_and_context_survives():
    """A tile waiting on a counter nothing releases gives up after the limit;
    dag_wait reports DAG_ETIMEOUT, the handle is poisoned, and the GPU context
    stays usable for a fresh DAG."""
    w = fork_join(64)
    ins = w.make_inputs()
    d = Dag(w, options(timeout_ns=50_000_000, debug_never_ready=1))
    d.set_inputs(ins)
    d.submit()
    st = d.wait(10_000_000_000)
    assert st == abi.DAG_ETIMEOUT
    with pytest.raises(abi.DagError):
        d.submit()
    d.close()
    got = run_gpu(w, ins)
    compare(w, got, oracle.run(w, ins))


def test_empty_and_degenerate_dags():
    w = Workload("one_elem")
    a = w.buf(1, 1, F32, "input", ("array", [[2.0]]))
    b = w.buf(1, 1, F32, "input", ("array", [[-3.0]]))
    y = w.buf(1, 1, F32, "output")
    w.node("gemm", a, y, b=b, act="relu")
    _roundtrip(w)
    w = Workload("single_row_softmax")
    x = w.buf(1, 1, F32, "input", ("array", [[5.0]]))
    y = w.buf(1, 1, F32, "output")
    w.node("softmax", x, y)
    _roundtrip(w)
    # a DAG with no kernels: submit and wait are no-ops
    w = Workload("empty")
    w.buf(4, 4, F32, "input", ("uniform", 1))
    d = Dag(w)
    d.run()
    d.close()


SPLIT_CASES = [
    dict(M=256, N=256, K=4096, dt=BF16),                                    # 8 tiles -> 4 partials each
    dict(M=200, N=100, K=3000, dt=BF16, act="gelu", out_dt=BF16),           # ragged, 2 partials
    dict(M=64, N=128, K=2048, dt=BF16, batch=2, trans_b=1, scale=0.5),     # batched, K-major B
]


@pytest.mark.parametrize("case", SPLIT_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_gemm_split_k(case):
    """A bf16 GEMM with few output tiles and a long K loop runs as split-K
    partials; the finishing partial adds them in a fixed order, so results
    are the same on every run, in both launch forms and on Alg. 1's streams."""
    w = _gemm_case(**case)
    d = Dag(w, options())
    split = d.tiles()[:, 5] >> 16
    assert (split > 0).any()
    d.close()
    _roundtrip(w)
    ins = w.make_inputs()
    d = Dag(w, options(max_ctas=3), resident_inputs=True)
    d.set_inputs(ins)
    d.run()
    outs = {b: d.output(b) for b in written_buffers(w, d.fusion())}
    d.run()
    again = {b: d.output(b) for b in outs}
    d.run_cq(n_queues=2, components=abi.DAG_TC_PER_KERNEL)
    cq = {b: d.output(b) for b in outs}
    d.close()
    assert bits_equal(outs, again) and bits_equal(outs, cq)
