"""JSON specification frontend (paper §4.A, "Design Frontend").

A specification file describes an application DAG the way the paper's
PySchedCL frontend does, and this module turns it into the C ABI's structs:

  {
    "name": "...",
    "symbols": {"M": 256, "N": 256, "K": 256},      default symbol values
    "cq": {"gpu": 3},                                 command queues per device
    "tc": [[0, 2], [1]],                              the task component partition
    "kernels": [
      {"id": 0, "name": "matmul", "dev": "gpu",
       "workDimension": 2, "globalWorkSize": ["M", "N", 1],
       "inputBuffers":  [{"type": "float", "size": "M*K", "pos": 0},
                         {"type": "float", "size": "K*N", "pos": 1}],
       "outputBuffers": [{"type": "float", "size": "M*N", "pos": 2}],
       "varArguments":  [{"type": "int", "pos": 3, "value": "M"}, ...],
       "attrs": {"act": "relu", "scale": 1.0}},       this library's extension
      ...
    ],
    "edges": ["0,2 -> 2,0", ...]                      k_i,b_r -> k_j,b_s
  }

A kernel is one of this library's operations, chosen by its name: matmul /
gemm (arguments A, B, C[, bias]; C = act(scale * A.B + bias); M, N, K from
the variable arguments or globalWorkSize [M, N]), matmul_t (the same with B
given as N x K), add / vadd (A, B, C), softmax (A, B, row-wise over
globalWorkSize [rows, cols]), relu / gelu (A, B), and transpose (A, B),
which is fused into the GEMM that reads its output as the B operand (that
GEMM reads B K-major instead).  Buffer sizes, work sizes and variable
arguments may be symbolic expressions over the symbols (+ - * / // % ** and
parentheses), resolved with the defaults in "symbols" overridden by the
caller (the paper's command-line values).  A buffer's size is checked
against the shape its role implies.  An edge says that argument b_r (an
output) of kernel k_i is argument b_s (an input) of kernel k_j: on one GPU
both are one buffer.  Inputs that no edge feeds are the DAG's inputs (the
paper's isolated writes); outputs that no edge consumes are its outputs.

Not supported, with an error: ioBuffers (in-place kernels: every buffer has
one writer), devices other than "gpu" (one GPU, no CPU device), kernel names
outside the list above.
"""
from __future__ import annotations

import ast
import json
import operator
import re
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

__all__ = ["SpecError", "SpecDag", "load", "loads", "evaluate"]


class SpecError(ValueError):
    pass


# ---------------------------------------------------------------------------
# symbolic sizes
# ---------------------------------------------------------------------------
_BINOPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul, ast.Div: operator.truediv,
           ast.FloorDiv: operator.floordiv, ast.Mod: operator.mod, ast.Pow: operator.pow}


def evaluate(expr, symbols: Dict[str, float]) -> int:
    """An integer from a constant or an arithmetic expression over symbols."""
    if isinstance(expr, bool):
        raise SpecError(f"not a size: {expr!r}")
    if isinstance(expr, (int, float)):
        v = expr
    elif isinstance(expr, str):
        try:
            tree = ast.parse(expr.strip(), mode="eval")
        except SyntaxError as e:
            raise SpecError(f"cannot parse {expr!r}: {e.msg}") from None

        def ev(n):
            if isinstance(n, ast.Expression):
                return ev(n.body)
            if isinstance(n, ast.Constant) and isinstance(n.value, (int, float)) and not isinstance(n.value, bool):
                return n.value
            if isinstance(n, ast.Name):
                if n.id not in symbols:
                    raise SpecError(f"unknown symbol {n.id!r} in {expr!r}")
                return symbols[n.id]
            if isinstance(n, ast.BinOp) and type(n.op) in _BINOPS:
                return _BINOPS[type(n.op)](ev(n.left), ev(n.right))
            if isinstance(n, ast.UnaryOp) and isinstance(n.op, (ast.UAdd, ast.USub)):
                x = ev(n.operand)
                return x if isinstance(n.op, ast.UAdd) else -x
            raise SpecError(f"only arithmetic over symbols is allowed: {expr!r}")

        v = ev(tree)
    else:
        raise SpecError(f"not a size: {expr!r}")
    if float(v) != int(v):
        raise SpecError(f"{expr!r} = {v} is not an integer")
    return int(v)


# ---------------------------------------------------------------------------
# the DAG a specification describes (the shape dag.describe expects)
# ---------------------------------------------------------------------------
@dataclass
class SpecBuffer:
    rows: int
    cols: int
    dtype: str          # "f32" | "bf16"
    role: str           # "input" | "inter" | "output"
    view_of: int = -1
    col_offset: int = 0
    name: str = ""


@dataclass
class SpecNode:
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
    component: int = 0


@dataclass
class SpecDag:
    name: str
    buffers: List[SpecBuffer] = field(default_factory=list)
    nodes: List[SpecNode] = field(default_factory=list)
    edges: List[Tuple[int, int, int, int]] = field(default_factory=list)  # node, buf -> node, buf
    queues: int = 1                       # command queues of the GPU ("cq")
    kernel_of_node: List[int] = field(default_factory=list)  # spec kernel id per node
    symbols: Dict[str, int] = field(default_factory=dict)

    def input_ids(self):
        return [i for i, b in enumerate(self.buffers) if b.role == "input"]

    def output_ids(self):
        return [i for i, b in enumerate(self.buffers) if b.role == "output"]

    def to_workload(self, seed: int = 7):
        """The same DAG as a seeded synthetic workload, for running it with
        generated data: matmul B operands and biases (the weights) ~ N(0, 0.02),
        every other input ~ U[-1, 1), as in the paper's transformer workload."""
        from synth.workloads import Workload
        w = Workload(self.name)
        weights = {n.b for n in self.nodes if n.op == "gemm"} | {n.bias for n in self.nodes if n.bias >= 0}
        for i, b in enumerate(self.buffers):
            init = None
            if b.role == "input":
                init = ("normal", seed * 1000 + i, 0.02) if i in weights else ("uniform", seed * 1000 + i)
            w.buf(b.rows, b.cols, b.dtype, b.role, init, b.name, view_of=b.view_of, col_offset=b.col_offset)
        for n in self.nodes:
            w.node(n.op, n.a, n.out, b=n.b, bias=n.bias, trans_b=n.trans_b, act=n.act, scale=n.scale,
                   batch=n.batch, name=n.name, component=n.component)
        w.edges = list(self.edges)
        return w


# ---------------------------------------------------------------------------
# kernel signatures: argument roles by position order
# ---------------------------------------------------------------------------
_DTYPES = {"float": "f32", "float32": "f32", "f32": "f32", "bfloat16": "bf16", "bf16": "bf16"}
_OPS = {"matmul": "gemm", "gemm": "gemm", "matmul_t": "gemm_t", "add": "add", "vadd": "add",
        "softmax": "softmax", "relu": "relu", "gelu": "gelu", "transpose": "transpose"}
_EDGE = re.compile(r"^\s*(\d+)\s*,\s*(\d+)\s*->\s*(\d+)\s*,\s*(\d+)\s*$")


def loads(text: str, symbols: Optional[Dict[str, int]] = None) -> SpecDag:
    return _build(json.loads(text), symbols or {})


def load(path: str, symbols: Optional[Dict[str, int]] = None) -> SpecDag:
    with open(path) as f:
        return _build(json.load(f), symbols or {})


def _build(spec: dict, overrides: Dict[str, int]) -> SpecDag:
    sym = {k: evaluate(v, {}) for k, v in spec.get("symbols", {}).items()}
    sym.update({k: int(v) for k, v in overrides.items()})
    kernels = spec.get("kernels")
    if not kernels:
        raise SpecError("no kernels")
    by_id = {}
    for k in kernels:
        if "id" not in k or "name" not in k:
            raise SpecError(f"kernel without id or name: {k}")
        if k["id"] in by_id:
            raise SpecError(f"duplicate kernel id {k['id']}")
        by_id[k["id"]] = k
        dev = k.get("dev", "gpu")
        if dev != "gpu":
            raise SpecError(f"kernel {k['id']}: device {dev!r}: this library runs on one GPU")
        if k.get("ioBuffers"):
            raise SpecError(f"kernel {k['id']}: ioBuffers (in-place) are not supported: one writer per buffer")
        if k["name"] not in _OPS:
            raise SpecError(f"kernel {k['id']}: unknown kernel {k['name']!r} (known: {sorted(_OPS)})")

    # edges: (k_i, pos_r) -> (k_j, pos_s)
    edges = []
    for e in spec.get("edges", []):
        m = _EDGE.match(e) if isinstance(e, str) else None
        if m is None:
            raise SpecError(f"edge {e!r} is not of the form 'k_i,b_r -> k_j,b_s'")
        ki, br, kj, bs = map(int, m.groups())
        if ki not in by_id or kj not in by_id:
            raise SpecError(f"edge {e!r}: unknown kernel")
        outs = {b["pos"] for b in by_id[ki].get("outputBuffers", [])}
        ins = {b["pos"] for b in by_id[kj].get("inputBuffers", [])}
        if br not in outs:
            raise SpecError(f"edge {e!r}: argument {br} is not an output of kernel {ki}")
        if bs not in ins:
            raise SpecError(f"edge {e!r}: argument {bs} is not an input of kernel {kj}")
        edges.append((ki, br, kj, bs))
    feeds = {}  # (k_j, pos_s) -> (k_i, pos_r)
    for ki, br, kj, bs in edges:
        if (kj, bs) in feeds:
            raise SpecError(f"input {bs} of kernel {kj} has two producers")
        feeds[(kj, bs)] = (ki, br)
    consumed = {(ki, br) for ki, br, _, _ in edges}

    # task components
    comp = {kid: 0 for kid in by_id}
    tc = spec.get("tc")
    if tc:
        seen = set()
        for ci, part in enumerate(tc):
            for kid in part:
                if kid not in by_id:
                    raise SpecError(f"tc: unknown kernel {kid}")
                if kid in seen:
                    raise SpecError(f"tc: kernel {kid} in two task components")
                seen.add(kid)
                comp[kid] = ci
        if seen != set(by_id):
            raise SpecError(f"tc: kernels {sorted(set(by_id) - seen)} in no task component")

    dag = SpecDag(spec.get("name", "spec"), symbols=sym)
    cq = spec.get("cq", {})
    dag.queues = evaluate(cq.get("gpu", 1), sym) if isinstance(cq, dict) else 1
    if dag.queues < 1:
        raise SpecError("cq: the GPU needs at least one command queue")

    # topological order of the spec kernels (so producers' buffers exist first)
    order, indeg = [], {kid: 0 for kid in by_id}
    succ = {kid: [] for kid in by_id}
    for ki, _, kj, _ in edges:
        indeg[kj] += 1
        succ[ki].append(kj)
    ready = sorted(k for k, d in indeg.items() if d == 0)
    while ready:
        k = ready.pop(0)
        order.append(k)
        for j in succ[k]:
            indeg[j] -= 1
            if indeg[j] == 0:
                ready.append(j)
                ready.sort()
    if len(order) != len(by_id):
        raise SpecError("the edges form a cycle")

    buf_of = {}           # (kernel id, pos) -> buffer id
    transposed = {}       # transpose kernel's output (kid, pos) -> the buffer it transposes

    def dt_of(b):
        t = b.get("type", "float")
        if t not in _DTYPES:
            raise SpecError(f"unknown buffer type {t!r}")
        return _DTYPES[t]

    def check_size(kid, b, rows, cols):
        size = evaluate(b["size"], sym) if "size" in b else rows * cols
        if size != rows * cols:
            raise SpecError(f"kernel {kid}, argument {b['pos']}: size {size} but its role needs {rows} x {cols}")

    def input_buffer(kid, b, rows, cols):
        pos = b["pos"]
        if (kid, pos) in feeds:
            src = feeds[(kid, pos)]
            if src in transposed:
                raise SpecError(f"kernel {kid}: a transposed matrix can only be the B operand of a matmul")
            bid = buf_of[src]
            sb = dag.buffers[bid]
            if (sb.rows, sb.cols) != (rows, cols):
                raise SpecError(f"kernel {kid}, argument {pos}: producer's buffer is {sb.rows} x {sb.cols}, "
                                f"needs {rows} x {cols}")
            if sb.dtype != dt_of(b):
                raise SpecError(f"kernel {kid}, argument {pos}: dtype differs from its producer's")
            return bid
        check_size(kid, b, rows, cols)
        dag.buffers.append(SpecBuffer(rows, cols, dt_of(b), "input", name=f"k{kid}.arg{pos}"))
        return len(dag.buffers) - 1

    def output_buffer(kid, b, rows, cols):
        check_size(kid, b, rows, cols)
        role = "inter" if (kid, b["pos"]) in consumed else "output"
        dag.buffers.append(SpecBuffer(rows, cols, dt_of(b), role, name=f"k{kid}.arg{b['pos']}"))
        buf_of[(kid, b["pos"])] = len(dag.buffers) - 1
        return len(dag.buffers) - 1

    for kid in order:
        k = by_id[kid]
        op = _OPS[k["name"]]
        ins = sorted(k.get("inputBuffers", []), key=lambda b: b["pos"])
        outs = sorted(k.get("outputBuffers", []), key=lambda b: b["pos"])
        var = [evaluate(v["value"], sym) for v in sorted(k.get("varArguments", []), key=lambda v: v["pos"])]
        gws = [evaluate(x, sym) for x in k.get("globalWorkSize", [])]
        attrs = k.get("attrs", {})
        if len(outs) != 1:
            raise SpecError(f"kernel {kid}: needs exactly one output buffer")

        def dims2():
            g = [x for x in gws if x != 1] or [1]
            if len(gws) >= 2:
                return gws[0], gws[1]
            return 1, g[0]

        if op in ("gemm", "gemm_t"):
            # variable arguments in position order are M, N, K; globalWorkSize [M, N] may stand for the first two
            if len(var) >= 3:
                M, N, K = var[:3]
            elif len(var) == 1 and len(gws) >= 2:
                M, N, K = gws[0], gws[1], var[0]
            else:
                raise SpecError(f"kernel {kid}: matmul needs M, N, K (varArguments, or globalWorkSize [M, N] and K)")
            if len(ins) not in (2, 3):
                raise SpecError(f"kernel {kid}: matmul takes A, B[, bias]")
            a = input_buffer(kid, ins[0], M, K)
            bsrc = feeds.get((kid, ins[1]["pos"]))
            trans_b = 1 if op == "gemm_t" else 0
            if bsrc in transposed:  # transpose fused: read the untransposed matrix K-major
                if trans_b:
                    raise SpecError(f"kernel {kid}: matmul_t of a transposed matrix")
                bb = transposed[bsrc]
                if (dag.buffers[bb].rows, dag.buffers[bb].cols) != (N, K):
                    raise SpecError(f"kernel {kid}: transposed operand has the wrong shape")
                trans_b = 1
            else:
                bb = input_buffer(kid, ins[1], N if trans_b else K, K if trans_b else N)
            bias = input_buffer(kid, ins[2], 1, N) if len(ins) == 3 else -1
            out = output_buffer(kid, outs[0], M, N)
            dag.nodes.append(SpecNode("gemm", a, out, b=bb, bias=bias, trans_b=trans_b,
                                      act=attrs.get("act", "none"), scale=float(attrs.get("scale", 1.0)),
                                      name=f"{k['name']}{kid}", component=comp[kid]))
        elif op == "transpose":
            rows, cols = dims2()
            if len(ins) != 1:
                raise SpecError(f"kernel {kid}: transpose takes one input")
            src = input_buffer(kid, ins[0], rows, cols)
            check_size(kid, outs[0], cols, rows)
            users = [(kj, bs) for ki, br, kj, bs in edges if ki == kid]
            for kj, bs in users:
                kb = by_id[kj]
                b_pos = sorted(kb.get("inputBuffers", []), key=lambda b: b["pos"])
                if _OPS[kb["name"]] != "gemm" or len(b_pos) < 2 or b_pos[1]["pos"] != bs:
                    raise SpecError(f"kernel {kid}: a transpose must feed only the B operand of matmuls")
            transposed[(kid, outs[0]["pos"])] = src
            continue
        else:
            rows, cols = dims2()
            if op == "add":
                if len(ins) != 2:
                    raise SpecError(f"kernel {kid}: add takes two inputs")
                a = input_buffer(kid, ins[0], rows, cols)
                bb = input_buffer(kid, ins[1], rows, cols)
                out = output_buffer(kid, outs[0], rows, cols)
                dag.nodes.append(SpecNode("add", a, out, b=bb, act=attrs.get("act", "none"),
                                          name=f"{k['name']}{kid}", component=comp[kid]))
            else:
                if len(ins) != 1:
                    raise SpecError(f"kernel {kid}: {k['name']} takes one input")
                a = input_buffer(kid, ins[0], rows, cols)
                out = output_buffer(kid, outs[0], rows, cols)
                if op == "softmax":
                    dag.nodes.append(SpecNode("softmax", a, out, scale=float(attrs.get("scale", 1.0)),
                                              name=f"{k['name']}{kid}", component=comp[kid]))
                else:
                    dag.nodes.append(SpecNode("unary", a, out, act=op, name=f"{k['name']}{kid}",
                                              component=comp[kid]))
        dag.kernel_of_node.append(kid)

    # the paper's edges, as ABI edges between the nodes that remain; an edge
    # into a fused transpose continues to the matmuls that read its output
    node_of_kernel = {kid: i for i, kid in enumerate(dag.kernel_of_node)}
    for ki, br, kj, bs in edges:
        if ki not in node_of_kernel:
            continue
        b = buf_of[(ki, br)]
        targets = [kj] if kj in node_of_kernel else [kl for kt, _, kl, _ in edges if kt == kj]
        for kl in targets:
            e = (node_of_kernel[ki], b, node_of_kernel[kl], b)
            if e not in dag.edges:
                dag.edges.append(e)
    return dag


def main(argv=None) -> int:
    """python -m paper_2009_07482_gb300.spec dag.json [-D M=512 ...] [--run]
    Prints the DAG; with --run, executes it on the GPU with seeded inputs,
    persistent and with the paper's Alg. 1 on the spec's queues."""
    import argparse
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("spec")
    ap.add_argument("-D", action="append", default=[], metavar="SYM=VALUE")
    ap.add_argument("--run", action="store_true")
    a = ap.parse_args(argv)
    over = {}
    for d in a.D:
        k, _, v = d.partition("=")
        over[k.strip()] = evaluate(v, {})
    dag = load(a.spec, over)
    print(f"{dag.name}: {len(dag.nodes)} kernels, {len(dag.buffers)} buffers, "
          f"{len(set(n.component for n in dag.nodes))} task components, {dag.queues} queue(s); symbols {dag.symbols}")
    for i, n in enumerate(dag.nodes):
        print(f"  node {i} (kernel {dag.kernel_of_node[i]}): {n.op} {n.name} a={n.a} b={n.b} -> {n.out} "
              f"trans_b={n.trans_b} act={n.act} component={n.component}")
    if a.run:
        from . import _binding as abi
        from .dag import Dag, options
        w = dag.to_workload()
        with Dag(w, options(), resident_inputs=True) as d:
            d.set_inputs(w.make_inputs())
            d.run()
            r = d.run_cq(n_queues=dag.queues, components=abi.DAG_TC_GIVEN)
            print(f"ran: Alg. 1 on {dag.queues} stream(s): device {r.device_us:.1f} us, host {r.host_us:.1f} us, "
                  f"{r.n_callbacks} callbacks")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
