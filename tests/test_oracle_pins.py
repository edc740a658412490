"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a hand-worked example, a
closed form, a published table, an independent library routine, or brute
force over every order.  CPU only.
"""
import itertools

import numpy as np
import pytest
from scipy import special, stats

import oracle
import synth
from synth import BF16, F32
from synth.workloads import Workload, encoder_block, fork_join, from_arrays, random_layered
from tests.conftest import load_golden


def f64(a, dt):
    return synth.storage_to_f64(a, dt)


# --------------------------------------------------------------------------
# input generator and storage rounding
# --------------------------------------------------------------------------
def test_splitmix64_published_vectors():
    g = load_golden("splitmix64.json")
    assert [int(x) for x in synth.splitmix64(0, 4)] == [int(h, 16) for h in g["seed0"]]
    assert [int(x) for x in synth.splitmix64(1234567, 3)] == g["seed1234567"]


def test_uniform_normal_moments():
    u = synth.uniform(7, (200000,))
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1 / 3) < 0.01
    z = synth.normal(8, (200000,), 0.02)
    assert abs(z.mean()) < 3e-4 and abs(z.std() - 0.02) < 3e-4
    # same seed, same draw
    assert np.array_equal(synth.uniform(7, (100,)), synth.uniform(7, (100,)))


def test_fast_fill_matches_the_numpy_definitions():
    for dt in (F32, BF16):
        assert np.array_equal(synth.fill("uniform", 77, (300, 333), dt, -1.0, 1.0),
                              synth.to_storage(synth.uniform(77, (300, 333)), dt))
        assert np.array_equal(synth.fill("normal", 78, (300, 333), dt, 0.02),
                              synth.to_storage(synth.normal(78, (300, 333), 0.02), dt))


def test_bf16_rounding_hand_cases():
    g = load_golden("bf16_rounding.json")
    for (label, hexbits), v in zip(g["cases"], g["values"]):
        assert oracle.f64_to_bf16(v) == int(hexbits, 16), label
    assert oracle.f64_to_bf16(float("nan")) & 0x7F80 == 0x7F80


def test_bf16_rounding_matches_independent_f32_routine():
    # f32 -> f64 is exact, so rounding f64 -> bf16 must agree with the integer
    # round-to-nearest-even on the f32 bit pattern used by the input generator.
    x = synth.uniform(11, (4000,)) * np.exp2(synth.uniform(12, (4000,)) * 60)
    x32 = x.astype(np.float32)
    ref = synth.f32_to_bf16_bits(x32)
    got = np.array([oracle.f64_to_bf16(float(v)) for v in x32.astype(np.float64)], np.uint16)
    assert np.array_equal(got, ref)


# --------------------------------------------------------------------------
# hand-worked DAG (paper Fig. 1 fork-join)
# --------------------------------------------------------------------------
def _fork_join_2x2(dt=F32):
    g = load_golden("fork_join_2x2.json")
    w, ids = from_arrays("fj2", {k: (g[k], dt) for k in ("A0", "B0", "B1", "B2")})
    C0 = w.buf(2, 2, dt, name="C0")
    C1 = w.buf(2, 2, dt, name="C1")
    C2 = w.buf(2, 2, dt, name="C2")
    C3 = w.buf(2, 2, F32, "output", name="C3")
    w.node("gemm", ids["A0"], C0, b=ids["B0"])
    w.node("gemm", C0, C1, b=ids["B1"])
    w.node("gemm", C0, C2, b=ids["B2"])
    w.node("add", C1, C3, b=C2)
    return w, g, dict(C0=C0, C1=C1, C2=C2, C3=C3)


@pytest.mark.parametrize("dt", [F32, BF16])
def test_fork_join_hand_computed(dt):
    w, g, out = _fork_join_2x2(dt)
    st = oracle.run(w, w.make_inputs())
    for k, bid in out.items():
        assert np.array_equal(f64(st[bid], w.buffers[bid].dtype), np.array(g[k], float)), k


# --------------------------------------------------------------------------
# closed forms and special cases
# --------------------------------------------------------------------------
def _single(op, a, out_shape, dt=F32, **kw):
    w, ids = from_arrays("one", {"a": (a, dt), **({"b": (kw.pop("b"), dt)} if "b" in kw else {}),
                                **({"bias": (kw.pop("bias"), F32)} if "bias" in kw else {})})
    o = w.buf(out_shape[0], out_shape[1], kw.pop("out_dt", F32), "output")
    w.node(op, ids["a"], o, b=ids.get("b", -1), bias=ids.get("bias", -1), **kw)
    st = oracle.run(w, w.make_inputs())
    return f64(st[o], w.buffers[o].dtype)


def test_gemm_identity_returns_a():
    A = synth.to_storage(synth.uniform(3, (5, 7)), F32).astype(np.float64)
    got = _single("gemm", A, (5, 7), b=np.eye(7))
    assert np.array_equal(got, A)


def test_gemm_zero_b_gives_activated_bias():
    g = load_golden("gelu_normal_cdf.json")
    x = np.array(g["x"])
    n = len(x)
    A = np.ones((3, 4))
    for act, ref in (("none", x), ("relu", np.maximum(x, 0)), ("gelu", np.array(g["gelu"]))):
        got = _single("gemm", A, (3, n), b=np.zeros((4, n)), bias=x[None, :], act=act)
        ref32 = np.broadcast_to(ref.astype(np.float32).astype(np.float64), (3, n))
        assert np.allclose(got, ref32, rtol=2e-7, atol=1e-30), act


def test_gelu_is_not_the_tanh_approximation():
    # tanh form 0.5x(1+tanh(sqrt(2/pi)(x+0.044715x^3))) differs at x=1 by ~1.5e-4
    got = _single("unary", np.array([[1.0]]), (1, 1), act="gelu")[0, 0]
    assert abs(got - 0.8413447460685429) < 1e-7
    tanh_form = 0.5 * (1 + np.tanh(np.sqrt(2 / np.pi) * (1 + 0.044715)))
    assert abs(got - tanh_form) > 1e-4


def test_gelu_matches_library_normal_cdf():
    x = synth.to_storage(synth.uniform(5, (4, 33)) * 6, F32).astype(np.float64)
    got = _single("unary", x, x.shape, act="gelu")
    ref = (x * stats.norm.cdf(x)).astype(np.float32).astype(np.float64)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-6)) < 2.5e-7


def test_softmax_closed_forms():
    # constant row -> 1/N; a row with one entry far above the rest -> one-hot
    got = _single("softmax", np.full((2, 4), 3.25), (2, 4))
    assert np.array_equal(got, np.full((2, 4), 0.25))
    got = _single("softmax", np.array([[0.0, 100.0, 0.0, -5.0]]), (1, 4))
    assert got[0, 1] == 1.0 and np.all(got[0, [0, 2, 3]] < 1e-40)
    # large inputs must not overflow (max subtraction)
    got = _single("softmax", np.array([[1000.0, 1000.0]]), (1, 2))
    assert np.array_equal(got, [[0.5, 0.5]])


def test_softmax_scale_and_shift():
    x = synth.to_storage(synth.uniform(9, (6, 50)) * 4, F32).astype(np.float64)
    a = _single("softmax", x, x.shape, scale=0.5)
    b = _single("softmax", x * 0.5, x.shape, scale=1.0)      # x*0.5 exact
    c = _single("softmax", x * 0.5 + 2.0, x.shape, scale=1.0)  # exact shift (|x| < 2)
    assert np.array_equal(a, b)
    assert np.max(np.abs(a - c)) <= 2 ** -24
    assert np.all(np.abs(a.sum(1) - 1) < 50 * 2 ** -24)


def test_softmax_matches_library():
    x = synth.to_storage(synth.uniform(10, (9, 257)) * 8, F32).astype(np.float64)
    got = _single("softmax", x, x.shape, scale=0.125)
    ref = special.softmax(0.125 * x, axis=1).astype(np.float32).astype(np.float64)
    assert np.max(np.abs(got - ref) / ref) <= 2 ** -23


@pytest.mark.parametrize("trans_b,batch", [(0, 1), (1, 1), (0, 3), (1, 3)])
def test_gemm_matches_numpy_float64(trans_b, batch):
    M, N, K = 13, 29, 53
    A = synth.to_storage(synth.uniform(1, (batch * M, K)), F32).astype(np.float64)
    Bs = (batch * N, K) if trans_b else (batch * K, N)
    B = synth.to_storage(synth.uniform(2, Bs), F32).astype(np.float64)
    bias = synth.to_storage(synth.uniform(3, (1, N)), F32).astype(np.float64)
    got = _single("gemm", A, (batch * M, N), b=B, bias=bias, trans_b=trans_b, batch=batch, act="relu", scale=0.75)
    ref = np.zeros((batch * M, N))
    for t in range(batch):
        Bt = B[t * N:(t + 1) * N].T if trans_b else B[t * K:(t + 1) * K]
        ref[t * M:(t + 1) * M] = np.maximum(0.75 * (A[t * M:(t + 1) * M] @ Bt) + bias, 0)
    ref32 = ref.astype(np.float32).astype(np.float64)
    # numpy sums in another order: the f64 results differ by ~1e-16 relative,
    # so the f32-rounded values agree to within one f32 ulp
    assert np.all(np.abs(got - ref32) <= np.spacing(np.abs(ref32).astype(np.float32)).astype(np.float64))


def test_add_and_relu_exact():
    a = synth.to_storage(synth.uniform(4, (7, 9)), F32).astype(np.float64)
    b = synth.to_storage(synth.uniform(5, (7, 9)), F32).astype(np.float64)
    got = _single("add", a, a.shape, b=b, act="relu")
    assert np.array_equal(got, np.maximum(a + b, 0).astype(np.float32).astype(np.float64))


def test_bf16_output_rounding_of_gemm():
    A = np.array([[1.0, 2.0 ** -8]])
    B = np.array([[1.0], [1.0]])
    got = _single("gemm", A, (1, 1), b=B, out_dt=BF16)
    assert got[0, 0] == 1.0                     # 1 + 2^-8 ties to even
    got = _single("gemm", A, (1, 1), b=np.array([[1.0], [3.0]]), out_dt=BF16)
    assert got[0, 0] == 1.0 + 2 ** -6           # 1 + 3*2^-8 ties to even (up)


def test_attention_with_zero_query_weights_averages_values():
    # Wq = 0 -> scores 0 -> uniform softmax (1/seq, exact in bf16) -> P.V is the
    # per-sequence column mean of V (closed form).
    w = encoder_block(batch=2, seq=16, d_model=32, heads=2, d_head=8, ffn=64, seed=21)
    ins = w.make_inputs()
    for i, b in enumerate(w.buffers):
        if b.name.startswith("Wq"):
            ins[i] = np.zeros_like(ins[i])
    st = oracle.run(w, ins)
    for h in range(2):
        P = next(i for i, b in enumerate(w.buffers) if b.name == f"P{h}")
        V = next(i for i, b in enumerate(w.buffers) if b.name == f"v{h}")
        Zh = next(i for i, b in enumerate(w.buffers) if b.name == f"Z{h}")
        assert np.all(f64(st[P], BF16) == 1.0 / 16)
        v = f64(st[V], BF16)
        z = f64(oracle.view(w, st, Zh), BF16)
        for s in range(2):
            mean = v[s * 16:(s + 1) * 16].mean(axis=0)
            ref = f64(np.array([oracle.f64_to_bf16(m) for m in mean], np.uint16), BF16)
            assert np.array_equal(z[s * 16:(s + 1) * 16], np.broadcast_to(ref, (16, 8)))


# --------------------------------------------------------------------------
# validation
# --------------------------------------------------------------------------
def test_validation_errors():
    w = Workload("bad")
    a = w.buf(4, 4, F32, "input", ("uniform", 1))
    b0 = w.buf(4, 4)
    b1 = w.buf(4, 4)
    w.node("gemm", a, b0, b=b1)
    w.node("gemm", a, b1, b=b0)
    assert oracle.validate(w) == 0
    with pytest.raises(oracle.OracleError) as e:
        oracle.topo_order(w)
    assert e.value.code == 2  # cycle
    w2 = Workload("mw")
    a = w2.buf(4, 4, F32, "input", ("uniform", 1))
    o = w2.buf(4, 4)
    w2.node("unary", a, o)
    w2.node("unary", a, o)
    assert oracle.validate(w2) == 5  # two writers
    w3 = Workload("inplace")
    a = w3.buf(4, 4, F32, "input", ("uniform", 1))
    w3.node("unary", a, a)
    assert oracle.validate(w3) == 5
    w4 = Workload("shape")
    a = w4.buf(4, 5, F32, "input", ("uniform", 1))
    b = w4.buf(4, 5, F32, "input", ("uniform", 2))
    o = w4.buf(4, 5)
    w4.node("gemm", a, o, b=b)
    assert oracle.validate(w4) == 3
    w5 = Workload("view")
    p = w5.buf(4, 8, F32)
    w5.buf(4, 4, BF16, view_of=p, col_offset=4)
    assert oracle.validate(w5) == 4
    for b_shape in [(4, 5), (5, 4)]:                  # an add's second operand of another shape
        w6 = Workload("add_shape")
        a = w6.buf(4, 4, F32, "input", ("uniform", 1))
        b = w6.buf(*b_shape, F32, "input", ("uniform", 2))
        w6.node("add", a, w6.buf(4, 4), b=b)
        assert oracle.validate(w6) == 3, b_shape
    for bias_shape in [(1, 3), (2, 4)]:               # a bias that is not one row of N
        w7 = Workload("bias_shape")
        a = w7.buf(4, 4, F32, "input", ("uniform", 1))
        b = w7.buf(4, 4, F32, "input", ("uniform", 2))
        bias = w7.buf(*bias_shape, F32, "input", ("uniform", 3))
        w7.node("gemm", a, w7.buf(4, 4), b=b, bias=bias)
        assert oracle.validate(w7) == 3, bias_shape


# --------------------------------------------------------------------------
# invariance over topological orders (brute force)
# --------------------------------------------------------------------------
def _linear_extensions(n, edges, limit=5000):
    preds = {v: set() for v in range(n)}
    for u, v in edges:
        preds[v].add(u)
    out = []

    def rec(prefix, placed):
        if len(out) >= limit:
            return
        if len(prefix) == n:
            out.append(list(prefix))
            return
        for v in range(n):
            if v not in placed and preds[v] <= placed:
                placed.add(v)
                prefix.append(v)
                rec(prefix, placed)
                prefix.pop()
                placed.remove(v)

    rec([], set())
    return out


def _node_edges(w):
    edges = []
    for v, n in enumerate(w.nodes):
        for bid in (n.a, n.b, n.bias):
            if bid < 0:
                continue
            for u, m in enumerate(w.nodes):
                if u == v:
                    continue
                wb, rb = w.buffers[m.out], w.buffers[bid]
                wroot = m.out if wb.view_of < 0 else wb.view_of
                rroot = bid if rb.view_of < 0 else rb.view_of
                if wroot != rroot:
                    continue
                wc = (0, wb.cols) if wb.view_of < 0 else (wb.col_offset, wb.col_offset + wb.cols)
                rc = (0, rb.cols) if rb.view_of < 0 else (rb.col_offset, rb.col_offset + rb.cols)
                if wc[0] < rc[1] and rc[0] < wc[1]:
                    edges.append((u, v))
    return edges


@pytest.mark.parametrize("make", [
    lambda: fork_join(16, seed=3),
    lambda: random_layered(5, 6, 8, 3, sizes=(8, 16, 32)),
    lambda: random_layered(6, 6, 8, 4, sizes=(8, 16)),
    lambda: encoder_block(batch=2, seq=8, d_model=16, heads=2, d_head=4, ffn=32, seed=4),
])
def test_every_topological_order_gives_identical_bits(make):
    w = make()
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    orders = _linear_extensions(len(w.nodes), _node_edges(w), limit=200)
    assert len(orders) >= 2
    for o in orders:
        assert oracle.is_topological(w, o)
        st = oracle.run(w, ins, order=o)
        for k in ref:
            assert np.array_equal(st[k].view(np.uint8), ref[k].view(np.uint8))


def test_bias_produced_by_a_later_kernel_is_waited_for():
    # kernel 0 reads as its bias the output of kernel 1 (an add): the order must
    # be [1, 0], and the value is A.B + (x + y), exact in small integers
    A = np.array([[1, 2], [3, -1]], float)
    B = np.array([[2, 0, 1], [-1, 1, 3]], float)
    x = np.array([[1, -2, 4]], float)
    y = np.array([[3, 5, -1]], float)
    w, ids = from_arrays("late_bias", {"A": (A, F32), "B": (B, F32), "x": (x, F32), "y": (y, F32)})
    bias = w.buf(1, 3)
    c = w.buf(2, 3, F32, "output")
    w.node("gemm", ids["A"], c, b=ids["B"], bias=bias)
    w.node("add", ids["x"], bias, b=ids["y"])
    assert oracle.topo_order(w) == [1, 0]
    st = oracle.run(w, w.make_inputs())
    assert np.array_equal(st[c], (A @ B + x + y).astype(np.float32))


def test_kahn_order_smallest_id_first():
    w = fork_join(8)
    assert oracle.topo_order(w) == [0, 1, 2, 3]
    assert not oracle.is_topological(w, [1, 0, 2, 3])


# --------------------------------------------------------------------------
# tile schedules: brute-force legality on tiny DAGs, and the trace checker
# --------------------------------------------------------------------------
def _tiny_dags():
    yield fork_join(8, seed=1), 4, 4
    w, ids = from_arrays("chain", {"x": (synth.uniform(3, (8, 6)), F32), "W": (synth.uniform(4, (6, 6)), F32)})
    h = w.buf(8, 6)
    s = w.buf(8, 6)
    y = w.buf(8, 6, F32, "output")
    w.node("gemm", ids["x"], h, b=ids["W"], act="relu")
    w.node("softmax", h, s)
    w.node("unary", s, y, act="gelu")
    yield w, 4, 6
    # a GEMM (kernel 0) whose B operand (8 x 8, two row blocks) and bias are
    # written tile by tile by later kernels
    w, ids = from_arrays("produced_operands", {"x": (synth.uniform(5, (4, 8)), F32),
                                               "Ws": (synth.uniform(6, (8, 8)), F32),
                                               "p": (synth.uniform(7, (1, 8)), F32),
                                               "q": (synth.uniform(8, (1, 8)), F32)})
    Wb = w.buf(8, 8)
    bias = w.buf(1, 8)
    y = w.buf(4, 8, F32, "output")
    w.node("gemm", ids["x"], y, b=Wb, bias=bias)
    w.node("unary", ids["Ws"], Wb, act="relu")
    w.node("add", ids["p"], bias, b=ids["q"])
    yield w, 4, 4


def _random_linear_extensions(n, edges, count, seed):
    """`count` linear extensions drawn by picking uniformly among the ready
    tiles at every step (seeded), to reach orders far from the lexicographic
    ones that _linear_extensions lists first."""
    rng = np.random.default_rng(seed)
    preds = {v: set() for v in range(n)}
    for u, v in edges:
        preds[v].add(u)
    out = []
    for _ in range(count):
        placed, order = set(), []
        while len(order) < n:
            ready = [v for v in range(n) if v not in placed and preds[v] <= placed]
            v = ready[int(rng.integers(len(ready)))]
            placed.add(v)
            order.append(v)
        out.append(order)
    return out


@pytest.mark.parametrize("case", list(range(3)))
def test_all_tile_orders_match_untiled(case):
    w, bm, bn = list(_tiny_dags())[case]
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    tiles = oracle.make_tiles(w, bm, bn)
    assert 6 <= len(tiles) <= 16
    deps = oracle.tile_deps(w, tiles)
    orders = _linear_extensions(len(tiles), deps, limit=3000)
    assert len(orders) > 10
    orders += _random_linear_extensions(len(tiles), deps, 300, seed=case)
    for o in orders:
        st = oracle.run_tiles(w, ins, tiles, o)
        for k in ref:
            assert np.array_equal(st[k].view(np.uint8), ref[k].view(np.uint8))
        # tickets drawn in this order are legal
        start = np.zeros(len(tiles), np.uint32)
        end = np.zeros(len(tiles), np.uint32)
        for pos, t in enumerate(o):
            start[t], end[t] = 2 * pos, 2 * pos + 1
        assert oracle.check_trace(w, tiles, start, end)[0] == 0
    # an order that breaks one edge reads poisoned data and is flagged
    u, v = deps[0]
    o = orders[0]
    bad = [t for t in o if t not in (u, v)]
    bad.insert(0, u)
    bad.insert(0, v)  # v before u
    st = oracle.run_tiles(w, ins, tiles, bad)
    assert any(not np.array_equal(st[k].view(np.uint8), ref[k].view(np.uint8)) for k in ref)
    start = np.zeros(len(tiles), np.uint32)
    end = np.zeros(len(tiles), np.uint32)
    for pos, t in enumerate(bad):
        start[t], end[t] = 2 * pos, 2 * pos + 1
    rc, bu, bv = oracle.check_trace(w, tiles, start, end)
    assert rc == 3 and (bu, bv) in deps


def test_softmax_tiles_split_by_columns():
    # A softmax tile may cover part of a row: its statistics still span the
    # whole row, and it depends on every producer tile of its rows.  Producer
    # (GELU) and softmax are both tiled 4 x 4 over 8 x 8, so a softmax tile
    # reads two producer tiles.
    w, ids = from_arrays("split_softmax", {"x": (synth.uniform(9, (8, 8)) * 4, F32)})
    h = w.buf(8, 8)
    y = w.buf(8, 8, F32, "output")
    w.node("unary", ids["x"], h, act="gelu")
    w.node("softmax", h, y, scale=0.5)
    ins = w.make_inputs()
    ref = oracle.run(w, ins)
    tiles = np.array([(k, r, r + 4, c, c + 4) for k in range(2) for r in (0, 4) for c in (0, 4)], np.int32)
    deps = set(oracle.tile_deps(w, tiles))
    for i, (k, r0, _, c0, _) in enumerate(tiles):
        if k == 1:
            assert {u for u, v in deps if v == i} == {j for j, t in enumerate(tiles) if t[0] == 0 and t[1] == r0}
    orders = _linear_extensions(len(tiles), deps, limit=500) + _random_linear_extensions(len(tiles), deps, 200, 7)
    for o in orders:
        st = oracle.run_tiles(w, ins, tiles, o)
        assert np.array_equal(st[y].view(np.uint8), ref[y].view(np.uint8))


def test_trace_checker_coverage_and_ticket_errors():
    w = fork_join(8)
    tiles = oracle.make_tiles(w, 4, 4)
    n = len(tiles)
    start = np.arange(n, dtype=np.uint32) * 2
    end = start + 1
    assert oracle.check_trace(w, tiles, start, end)[0] == 0
    assert oracle.check_trace(w, tiles[:-1], start[:-1], end[:-1])[0] == 1      # a hole
    dup = np.vstack([tiles, tiles[:1]])
    rc, bu, _ = oracle.check_trace(w, dup, np.append(start, 2 * n), np.append(end, 2 * n + 1))
    assert (rc, bu) == (1, n)                                                  # the second cover is named
    e2 = end.copy()
    e2[3] = start[3]
    assert oracle.check_trace(w, tiles, start, e2)[0] == 2
    # tickets come from one counter, so end(u) == start(v) never happens in a
    # legal run: the checker demands end(u) < start(v) strictly
    deps = oracle.tile_deps(w, tiles)
    v = deps[0][1]
    u = max((a for a, b in deps if b == v), key=lambda a: end[a])          # v's last predecessor
    s2 = start.copy()
    s2[v] = end[u]
    assert s2[v] < end[v]
    assert oracle.check_trace(w, tiles, s2, end)[:3] == (3, u, v)


def test_column_slice_views_depend_only_on_their_columns():
    w = encoder_block(batch=1, seq=8, d_model=16, heads=2, d_head=4, ffn=16, seed=5)
    tiles = oracle.make_tiles(w, 8, 4)
    deps = set(oracle.tile_deps(w, tiles))
    pv0 = [i for i, t in enumerate(tiles) if w.nodes[t[0]].name == "pv0"]
    pv1 = [i for i, t in enumerate(tiles) if w.nodes[t[0]].name == "pv1"]
    outp = [i for i, t in enumerate(tiles) if w.nodes[t[0]].name == "out_proj"]
    assert all((u, v) in deps for u in pv0 + pv1 for v in outp)
    assert not any((u, v) in deps or (v, u) in deps for u in pv0 for v in pv1)
