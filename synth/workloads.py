"""Workload descriptions: the application DAGs the library is exercised on.

A workload is the paper's DAG G = <(K,B),(E_I,E_O,E)> (§3 Problem Formulation)
written as plain data: a list of buffers and a list of kernel nodes, each node
naming the buffers it reads and the one buffer it writes, plus how to draw each
input buffer.  Nothing here computes a node; the oracle and the GPU library
each interpret the description on their own.

Buffer fields
    rows, cols   logical shape (row-major)
    dtype        "f32" | "bf16"
    role         "input" (uploaded / resident), "output" (read back),
                 "inter" (intermediate)
    view_of      -1, or the id of a parent buffer this one is a column slice of
    col_offset   first parent column of the slice
    init         for inputs: ("uniform", seed) | ("normal", seed, std)

Node fields
    op      "gemm" | "add" | "softmax" | "unary"
    a, b    input buffer ids (b = -1 for softmax/unary)
    bias    bias buffer id (1 x N) or -1 (gemm only)
    out     output buffer id
    trans_b gemm: B stored N x K per batch (K-major) instead of K x N
    act     "none" | "relu" | "gelu"
    scale   gemm: C = act(scale * A.B + bias); softmax: y = softmax(scale * x)
    batch   gemm: number of independent row-stacked problems
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import BF16, F32, fill, normal, to_storage, uniform


@dataclass
class Buffer:
    rows: int
    cols: int
    dtype: str = F32
    role: str = "inter"
    view_of: int = -1
    col_offset: int = 0
    init: Optional[Tuple] = None
    name: str = ""


@dataclass
class Node:
    op: str
    a: int
    out: int
    b: int = -1
    bias: int = -1
    trans_b: int = 0
    act: str = "none"
    scale: float = 1.0
    batch: int = 1
    name: str = ""
    component: int = 0  # task component id (the paper's partition T of the kernels)


@dataclass
class Workload:
    name: str
    buffers: List[Buffer] = field(default_factory=list)
    nodes: List[Node] = field(default_factory=list)
    meta: Dict = field(default_factory=dict)

    # -- construction helpers -------------------------------------------
    def buf(self, rows, cols, dtype=F32, role="inter", init=None, name="", view_of=-1, col_offset=0) -> int:
        self.buffers.append(Buffer(rows, cols, dtype, role, view_of, col_offset, init, name))
        return len(self.buffers) - 1

    def node(self, op, a, out, **kw) -> int:
        self.nodes.append(Node(op=op, a=a, out=out, **kw))
        return len(self.nodes) - 1

    # -- inputs ----------------------------------------------------------
    def input_ids(self) -> List[int]:
        return [i for i, b in enumerate(self.buffers) if b.role == "input"]

    def output_ids(self) -> List[int]:
        return [i for i, b in enumerate(self.buffers) if b.role == "output"]

    def make_inputs(self, cache: Optional[Dict] = None) -> Dict[int, np.ndarray]:
        """Draw every input buffer and round it to its storage dtype.  `cache`
        (a dict the caller keeps) reuses draws of equal recipe and shape."""
        out = {}
        for i in self.input_ids():
            b = self.buffers[i]
            key = (b.init[0], b.init[1], b.init[2] if len(b.init) > 2 else None, b.rows, b.cols, b.dtype) \
                if b.init[0] != "array" else None
            if cache is not None and key in cache:
                out[i] = cache[key]
                continue
            kind = b.init[0]
            if kind == "uniform":
                out[i] = fill("uniform", b.init[1], (b.rows, b.cols), b.dtype, -1.0, 1.0)
            elif kind == "normal":
                out[i] = fill("normal", b.init[1], (b.rows, b.cols), b.dtype, b.init[2])
            elif kind == "array":
                out[i] = to_storage(np.asarray(b.init[1], dtype=np.float64).reshape(b.rows, b.cols), b.dtype)
            else:
                raise ValueError(kind)
            if cache is not None and key is not None:
                cache[key] = out[i]
        return out

    def clone(self) -> "Workload":
        return dataclasses.replace(
            self,
            buffers=[dataclasses.replace(b) for b in self.buffers],
            nodes=[dataclasses.replace(n) for n in self.nodes],
            meta=dict(self.meta),
        )

    # -- algorithmic work ------------------------------------------------
    def node_flops(self, k: int) -> float:
        n = self.nodes[k]
        if n.op != "gemm":
            return float(self.buffers[n.out].rows * self.buffers[n.out].cols)
        M, N, K = gemm_mnk(self, n)
        return 2.0 * n.batch * M * N * K

    def node_bytes(self, k: int) -> float:
        """Each input read once plus the output written once, at stored dtype."""
        n = self.nodes[k]
        tot = 0
        for bid in (n.a, n.b, n.bias, n.out):
            if bid >= 0:
                b = self.buffers[bid]
                tot += b.rows * b.cols * (4 if b.dtype == F32 else 2)
        return float(tot)


def gemm_mnk(w: Workload, n: Node) -> Tuple[int, int, int]:
    """Per-batch (M, N, K) of a gemm node from its buffer shapes."""
    A, B = w.buffers[n.a], w.buffers[n.b]
    M = A.rows // n.batch
    K = A.cols
    N = B.rows // n.batch if n.trans_b else B.cols
    return M, N, K


def _seed(base: int, i: int) -> int:
    return base * 1_000_003 + i


# ---------------------------------------------------------------------------
# Fork-join DAG of the paper's Fig. 1: K0 -> {K1, K2} -> K3 (§1 Introduction)
# ---------------------------------------------------------------------------
def fork_join(n: int = 256, seed: int = 0, dtype: str = F32) -> Workload:
    """K0: C0=A0.B0, K1: C1=C0.B1, K2: C2=C0.B2, K3: C3=C1+C2; n x n, U[-1,1]."""
    w = Workload(f"fork_join_{n}_{dtype}")
    A0 = w.buf(n, n, dtype, "input", ("uniform", _seed(seed, 0)), "A0")
    B0 = w.buf(n, n, dtype, "input", ("uniform", _seed(seed, 1)), "B0")
    B1 = w.buf(n, n, dtype, "input", ("uniform", _seed(seed, 2)), "B1")
    B2 = w.buf(n, n, dtype, "input", ("uniform", _seed(seed, 3)), "B2")
    C0 = w.buf(n, n, dtype, "inter", name="C0")
    C1 = w.buf(n, n, dtype, "inter", name="C1")
    C2 = w.buf(n, n, dtype, "inter", name="C2")
    C3 = w.buf(n, n, F32, "output", name="C3")
    w.node("gemm", A0, C0, b=B0, name="K0")
    w.node("gemm", C0, C1, b=B1, name="K1")
    w.node("gemm", C0, C2, b=B2, name="K2")
    w.node("add", C1, C3, b=C2, name="K3")
    return w


# ---------------------------------------------------------------------------
# Branchy MLP inference DAG (ML-inference workload in the spirit of §5)
# ---------------------------------------------------------------------------
def branchy_mlp(dtype: str = BF16, batch: int = 512, width: int = 2048, branches: int = 4,
                depth: int = 3, hidden: int = 4096, out: int = 1024, seed: int = 1) -> Workload:
    """X -> `branches` x (`depth` x Linear+bias+ReLU) -> pairwise add tree -> Linear+ReLU -> Linear.

    Weights N(0, 0.02), biases N(0, 0.02), activations U[-1,1].  In the bf16
    variant every intermediate that feeds a GEMM is stored bf16 and the final
    output is f32; in the f32 variant everything is f32.
    """
    assert branches & (branches - 1) == 0, "add tree needs a power-of-two branch count"
    w = Workload(f"branchy_mlp_{dtype}_b{batch}_w{width}")
    s = 0

    def nxt():
        nonlocal s
        s += 1
        return _seed(seed, s)

    X = w.buf(batch, width, dtype, "input", ("uniform", nxt()), "X")
    heads = []
    for br in range(branches):
        h = X
        for l in range(depth):
            W = w.buf(width, width, dtype, "input", ("normal", nxt(), 0.02), f"W{br}_{l}")
            bvec = w.buf(1, width, F32, "input", ("normal", nxt(), 0.02), f"b{br}_{l}")
            o = w.buf(batch, width, dtype, "inter", name=f"h{br}_{l}")
            w.node("gemm", h, o, b=W, bias=bvec, act="relu", name=f"fc{br}_{l}")
            h = o
        heads.append(h)
    lvl = 0
    while len(heads) > 1:
        nh = []
        for i in range(0, len(heads), 2):
            o = w.buf(batch, width, dtype, "inter", name=f"sum{lvl}_{i // 2}")
            w.node("add", heads[i], o, b=heads[i + 1], name=f"add{lvl}_{i // 2}")
            nh.append(o)
        heads = nh
        lvl += 1
    W1 = w.buf(width, hidden, dtype, "input", ("normal", nxt(), 0.02), "WL1")
    b1 = w.buf(1, hidden, F32, "input", ("normal", nxt(), 0.02), "bL1")
    H1 = w.buf(batch, hidden, dtype, "inter", name="L1")
    w.node("gemm", heads[0], H1, b=W1, bias=b1, act="relu", name="L1")
    W2 = w.buf(hidden, out, dtype, "input", ("normal", nxt(), 0.02), "WL2")
    b2 = w.buf(1, out, F32, "input", ("normal", nxt(), 0.02), "bL2")
    Y = w.buf(batch, out, F32, "output", name="Y")
    w.node("gemm", H1, Y, b=W2, bias=b2, name="L2")
    return w


# ---------------------------------------------------------------------------
# Transformer encoder block (the paper's head DAG of §5, generalised)
# ---------------------------------------------------------------------------
def encoder_block(batch: int = 8, seq: int = 256, d_model: int = 1024, heads: int = 16,
                  d_head: int = 64, ffn: int = 4096, seed: int = 2, softmax_scale: Optional[float] = None) -> Workload:
    """Per head h: Q=X.Wq, K=X.Wk, V=X.Wv; S=Q.K^T (batched per sequence);
    P=softmax(scale*S); Z[:, h] = P.V; then Out = Z.Wo+bo, H = GELU(Out.W1+b1),
    Y = H.W2+b2.  bf16 storage, f32 scores and f32 final output.
    """
    if softmax_scale is None:
        softmax_scale = 1.0 / float(np.sqrt(d_head))
    T = batch * seq
    w = Workload(f"encoder_b{batch}_s{seq}_d{d_model}_h{heads}")
    s = 0

    def nxt():
        nonlocal s
        s += 1
        return _seed(seed, s)

    X = w.buf(T, d_model, BF16, "input", ("uniform", nxt()), "X")
    Z = w.buf(T, heads * d_head, BF16, "inter", name="Z")
    for h in range(heads):
        proj = []
        for nm in ("q", "k", "v"):
            Wt = w.buf(d_model, d_head, BF16, "input", ("normal", nxt(), 0.02), f"W{nm}{h}")
            o = w.buf(T, d_head, BF16, "inter", name=f"{nm}{h}")
            w.node("gemm", X, o, b=Wt, name=f"proj_{nm}{h}")
            proj.append(o)
        Q, Kb, V = proj
        S = w.buf(T, seq, F32, "inter", name=f"S{h}")
        w.node("gemm", Q, S, b=Kb, trans_b=1, batch=batch, name=f"qk{h}")
        P = w.buf(T, seq, BF16, "inter", name=f"P{h}")
        w.node("softmax", S, P, scale=softmax_scale, name=f"softmax{h}")
        Zh = w.buf(T, d_head, BF16, "inter", view_of=Z, col_offset=h * d_head, name=f"Z{h}")
        w.node("gemm", P, Zh, b=V, batch=batch, name=f"pv{h}")
    Wo = w.buf(heads * d_head, d_model, BF16, "input", ("normal", nxt(), 0.02), "Wo")
    bo = w.buf(1, d_model, F32, "input", ("normal", nxt(), 0.02), "bo")
    O = w.buf(T, d_model, BF16, "inter", name="O")
    w.node("gemm", Z, O, b=Wo, bias=bo, name="out_proj")
    W1 = w.buf(d_model, ffn, BF16, "input", ("normal", nxt(), 0.02), "W1")
    b1 = w.buf(1, ffn, F32, "input", ("normal", nxt(), 0.02), "b1")
    H = w.buf(T, ffn, BF16, "inter", name="H")
    w.node("gemm", O, H, b=W1, bias=b1, act="gelu", name="ffn1")
    W2 = w.buf(ffn, d_model, BF16, "input", ("normal", nxt(), 0.02), "W2")
    b2 = w.buf(1, d_model, F32, "input", ("normal", nxt(), 0.02), "b2")
    Y = w.buf(T, d_model, F32, "output", name="Y")
    w.node("gemm", H, Y, b=W2, bias=b2, name="ffn2")
    return w


def transformer_heads(heads: int = 16, beta: int = 256, dtype: str = F32, seed: int = 4,
                      softmax_scale: float = 1.0) -> Workload:
    """The paper's transformer-layer DAG of §5 (its Experiments 1-3): every
    matrix beta x beta; per head h: Q=X.Wq, K=X.Wk, V=X.Wv, A=Q.K^T (K read
    as a K-major operand: the transpose kernel is fused away), B=softmax(A),
    C=B.V, Z[:, h] = C.Wh (heads concatenated in place).  Each head is one
    task component (the paper's clustering partition).  X ~ U[-1,1), weights
    N(0, 0.02); the softmax scale defaults to the paper's literal form (1).
    """
    w = Workload(f"transformer_heads_h{heads}_b{beta}_{dtype}")
    s = 0

    def nxt():
        nonlocal s
        s += 1
        return _seed(seed, s)

    X = w.buf(beta, beta, dtype, "input", ("uniform", nxt()), "X")
    Z = w.buf(beta, heads * beta, dtype, "output", name="Z")
    for h in range(heads):
        proj = []
        for nm in ("q", "k", "v"):
            Wt = w.buf(beta, beta, dtype, "input", ("normal", nxt(), 0.02), f"W{nm}{h}")
            o = w.buf(beta, beta, dtype, "inter", name=f"{nm}{h}")
            w.node("gemm", X, o, b=Wt, name=f"proj_{nm}{h}", component=h)
            proj.append(o)
        Q, Kb, V = proj
        A = w.buf(beta, beta, F32, "inter", name=f"A{h}")
        w.node("gemm", Q, A, b=Kb, trans_b=1, name=f"qk{h}", component=h)
        B = w.buf(beta, beta, dtype, "inter", name=f"B{h}")
        w.node("softmax", A, B, scale=softmax_scale, name=f"softmax{h}", component=h)
        C = w.buf(beta, beta, dtype, "inter", name=f"C{h}")
        w.node("gemm", B, C, b=V, name=f"bv{h}", component=h)
        Wh = w.buf(beta, beta, dtype, "input", ("normal", nxt(), 0.02), f"Wh{h}")
        Zh = w.buf(beta, beta, dtype, "inter", view_of=Z, col_offset=h * beta, name=f"Z{h}")
        w.node("gemm", C, Zh, b=Wh, name=f"cw{h}", component=h)
    return w


# ---------------------------------------------------------------------------
# Seeded random layered DAGs (batched workload)
# ---------------------------------------------------------------------------
_POW2 = [64, 128, 256, 512, 1024, 2048]


class _Draw:
    """Sequential integer draws from one SplitMix64 stream."""

    def __init__(self, seed: int):
        from . import splitmix64
        self._seed = seed
        self._i = 0
        self._sm = splitmix64

    def u64(self) -> int:
        v = int(self._sm(self._seed, 1, self._i)[0])
        self._i += 1
        return v

    def randint(self, lo: int, hi: int) -> int:  # inclusive
        return lo + self.u64() % (hi - lo + 1)

    def unit(self) -> float:
        return (self.u64() >> 11) * 2.0 ** -53

    def choice(self, seq):
        return seq[self.u64() % len(seq)]


def random_layered(seed: int, min_nodes: int = 8, max_nodes: int = 64, max_width: int = 8,
                   sizes=tuple(_POW2), dtype: Optional[str] = None) -> Workload:
    """Random layered DAG: layers of width U{1..max_width} until the node budget.

    Each node: gemm 70% / eltwise 20% (add if it has two predecessors of equal
    shape, else relu) / softmax 10%.  Root gemms draw M, N, K from `sizes`; a
    non-root gemm takes A = its first predecessor's output (so M, K inherit)
    and draws N.  dtype is drawn per DAG (50/50) unless given.
    """
    d = _Draw(seed)
    if dtype is None:
        dtype = BF16 if d.u64() & 1 else F32
    n_nodes = d.randint(min_nodes, max_nodes)
    w = Workload(f"random_{seed}_{dtype}")
    layers: List[List[int]] = []   # node ids per layer
    out_of: Dict[int, int] = {}    # node -> output buffer
    s = 0

    def nxt():
        nonlocal s
        s += 1
        return _seed(seed, s)

    count = 0
    while count < n_nodes:
        width = min(d.randint(1, max_width), n_nodes - count)
        layer = []
        for _ in range(width):
            r = d.unit()
            prev = [k for L in layers[-2:] for k in L]
            if not prev:
                op = "gemm"
            else:
                op = "gemm" if r < 0.7 else ("eltwise" if r < 0.9 else "softmax")
            if op == "gemm":
                if not prev:
                    M, K = d.choice(sizes), d.choice(sizes)
                    a = w.buf(M, K, dtype, "input", ("uniform", nxt()))
                else:
                    p = d.choice(prev)
                    a = out_of[p]
                    M, K = w.buffers[a].rows, w.buffers[a].cols
                N = d.choice(sizes)
                B = w.buf(K, N, dtype, "input", ("normal", nxt(), float(1.0 / np.sqrt(K))))
                o = w.buf(M, N, dtype, "inter")
                act = "relu" if d.u64() % 2 else "none"
                k = w.node("gemm", a, o, b=B, act=act)
            elif op == "eltwise":
                p = d.choice(prev)
                a = out_of[p]
                shape = (w.buffers[a].rows, w.buffers[a].cols)
                same = [q for q in prev if q != p and (w.buffers[out_of[q]].rows, w.buffers[out_of[q]].cols) == shape]
                o = w.buf(shape[0], shape[1], dtype, "inter")
                if same:
                    k = w.node("add", a, o, b=out_of[d.choice(same)])
                else:
                    k = w.node("unary", a, o, act="relu")
            else:
                p = d.choice(prev)
                a = out_of[p]
                o = w.buf(w.buffers[a].rows, w.buffers[a].cols, dtype, "inter")
                k = w.node("softmax", a, o, scale=1.0)
            out_of[k] = o
            layer.append(k)
            count += 1
        layers.append(layer)
    # every buffer nobody reads is a DAG output (sink, END in the paper's terms)
    read = {b for n in w.nodes for b in (n.a, n.b, n.bias) if b >= 0}
    for k, o in out_of.items():
        if o not in read:
            w.buffers[o].role = "output"
            w.buffers[o].dtype = F32
    return w


# ---------------------------------------------------------------------------
# Tiny hand-checkable DAGs
# ---------------------------------------------------------------------------
def from_arrays(name: str, inputs: Dict[str, Tuple[np.ndarray, str]]) -> Tuple[Workload, Dict[str, int]]:
    """Start a workload whose inputs are given literally (for hand-computed tests)."""
    w = Workload(name)
    ids = {}
    for nm, (arr, dt) in inputs.items():
        arr = np.atleast_2d(np.asarray(arr, dtype=np.float64))
        ids[nm] = w.buf(arr.shape[0], arr.shape[1], dt, "input", ("array", arr), nm)
    return w, ids


def concat(workloads: List[Workload], name: str = "batch") -> Workload:
    """One workload holding several DAGs side by side (ids offset in order),
    matching the buffer and node numbering of a batched plan."""
    w = Workload(name)
    for x in workloads:
        boff = len(w.buffers)
        for b in x.buffers:
            nb = dataclasses.replace(b)
            if nb.view_of >= 0:
                nb.view_of += boff
            w.buffers.append(nb)
        for n in x.nodes:
            nn = dataclasses.replace(n)
            nn.a += boff
            nn.out += boff
            if nn.b >= 0:
                nn.b += boff
            if nn.bias >= 0:
                nn.bias += boff
            w.nodes.append(nn)
    return w


def random_batch(n_dags: int = 256, base_seed: int = 1000, **kw) -> List[Workload]:
    """The batched workload: seeded random layered DAGs, seed base_seed + i."""
    return [random_layered(base_seed + i, **kw) for i in range(n_dags)]


def chain_and_fill(chain: int = 48, fill: int = 4, fill_dim: int = 4096, dtype: str = BF16, seed: int = 9) -> Workload:
    """A latency-bound chain beside wide filler work: `chain` GEMMs
    128 x 256 x 256 (+ReLU) in sequence -- one tile each, whose time is set by
    per-tile latency rather than by their few flops -- and `fill` independent
    fill_dim^3 GEMMs.  The chain is the critical path, but a roofline time
    model prices each of its GEMMs at a fraction of its measured time, so
    ranks from that model put the filler first.  Inputs U[-1,1), weights
    N(0, 0.06) (chain) / N(0, 0.02) (filler)."""
    w = Workload(f"chain{chain}_fill{fill}x{fill_dim}_{dtype}")
    s = 0

    def nxt():
        nonlocal s
        s += 1
        return _seed(seed, s)

    x = w.buf(128, 256, dtype, "input", ("uniform", nxt()), "x")
    for i in range(chain):
        W = w.buf(256, 256, dtype, "input", ("normal", nxt(), 0.06), f"Wc{i}")
        last = i == chain - 1
        y = w.buf(128, 256, F32 if last else dtype, "output" if last else "inter", name=f"c{i}")
        w.node("gemm", x, y, b=W, act="relu", name=f"chain{i}")
        x = y
    for j in range(fill):
        A = w.buf(fill_dim, fill_dim, dtype, "input", ("uniform", nxt()), f"F{j}")
        B = w.buf(fill_dim, fill_dim, dtype, "input", ("normal", nxt(), 0.02), f"G{j}")
        w.node("gemm", A, w.buf(fill_dim, fill_dim, F32, "output", name=f"H{j}"), b=B, name=f"fill{j}")
    return w
