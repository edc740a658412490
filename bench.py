#!/usr/bin/env python3
"""Benchmark: DAG makespan and DAGs/s of the fine-grained persistent executor.

Default workload: the batched configuration, 256 seeded random layered DAGs
(8-64 nodes, layer widths 1-8; GEMM 70% / elementwise 20% / softmax 10%;
M, N, K in {64..2048}; bf16 or f32 per DAG) in one persistent launch replayed
from a captured CUDA graph.  One step = one submission of the whole batch,
weights and activations resident in HBM; L2 is flushed (a 256 MiB write)
between timed steps, outside the timed events.

Also measured and reported on the same JSON line:
  coarse     every kernel as given (no sibling GEMMs merged), its tiles
             launched kernel by kernel on one stream
  epilogue_fusion  the persistent executor with the opt-in epilogue fusion
             modes, when the DAG has kernels they would fuse (single DAGs)
  e2e        the same metric through the C ABI with host buffers: upload of
             the activations from pinned memory, execution, readback of every
             sink, every step
  roofline   the executor kernel's achieved TFLOP/s against the measured peak
  cp_roofline  makespan against the DAG's critical-path / total-work bounds
  learned    (batched) makespan under the learned, profiled and roofline
             ranks and FIFO order
  configs    (batched, one GPU) the single-DAG configurations measured the
             same way: fork-join 256^3 f32 (the paper's Fig. 1), branchy MLP
             bf16 and f32, encoder block bf16 -- makespan, kernel-by-kernel,
             the paper's Alg. 1 on streams at its best queue count, and the
             fractions of the critical-path and work bounds
  cpu_baseline the FP64 oracle on a bounded sample, on one host core
  cpu_baseline_all_cores  the same on every host core at once

--impl reference times the FP64 oracle (the only reference implementation of
this method) on the host cores instead: each step runs whole units of the
workload (a block of batch rows, a sequence, a head, rows of several DAGs of
the batch) and the rate is the units done over the time spent.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DAGs/s (fine-grained persistent executor, device makespan)"
UNIT = "DAGs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["mlp_bf16", "mlp_f32", "fork_join", "encoder", "heads", "softmax", "add", "batched",
                             "serving", "exp1"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="batched: skip the cost-model comparison")
    ap.add_argument("--no-configs", action="store_true", help="batched: skip the single-DAG configurations")
    ap.add_argument("--dags", type=int, default=256,
                    help="batched: number of DAGs (256 = the configuration; fewer only for profiling captures)")
    ap.add_argument("--profile", action="store_true", help="few steps, no side measurements (for ncu)")
    ap.add_argument("--f32-simt", action="store_true", help="f32 GEMMs on the SM cores (FFMA) instead of 3 x TF32")
    ap.add_argument("--tile-override", type=int, default=0, choices=[0, 64, 128, 256],
                    help="diagnostic: force the tensor-core GEMM tile width (dag_options.tile_override; "
                         "0 = the planner's choice)")
    ap.add_argument("--timeline", action="store_true",
                    help="diagnostic: per-kernel phases of traced launches (claim, dependencies, K loop, epilogue, "
                         "release) instead of the measured line")
    ap.add_argument("--chrome-trace", metavar="PATH", default=None,
                    help="with --timeline: also write the last traced launch as a Chrome trace-event file")
    return ap.parse_args()


# phases of one tile, in the order the executor stamps them (dag_trace_stamps)
STAMPS = ["claim", "ready", "loaded", "mma0", "mma1", "work", "acc", "body", "sync", "end"]


def run_timeline(args, w, d, abi, stream, flush, reps=8):
    """Per-kernel timeline of `reps` traced launches of the handle `d`
    (created with trace = 1): each kernel's window in the launch (first claim,
    first dependency release, last release; medians over launches, in us from
    the launch's first claim) and the median time of each phase of its tiles
    (between consecutive stamps the tile kind records)."""
    import numpy as np
    windows, phases, spans, lw = {}, {}, [], []
    for _ in range(reps):
        flush.zero_()
        d.submit(stream.cuda_stream)
        abi.check(d.wait(), "wait")
        recs = d.trace()
        st = abi.dag_trace_stamps(d.h).astype(np.int64)
        enter, leave = abi.dag_trace_launch(d.h)
        node = np.array([r.node for r in recs])
        t0 = st[:, 0].min()
        spans.append((st[:, 9].max() - t0) / 1e3)
        lw.append(((t0 - enter) / 1e3, (leave - st[:, 9].max()) / 1e3, (leave - enter) / 1e3))
        for v in range(len(w.nodes)):
            S = st[node == v]
            if not len(S):
                continue
            windows.setdefault(v, []).append(((S[:, 0].min() - t0) / 1e3, (S[:, 1].min() - t0) / 1e3,
                                              (S[:, 9].max() - t0) / 1e3, len(S)))
            used = [i for i in range(10) if (S[:, i] > 0).all()]
            for a, b in zip(used[:-1], used[1:]):
                phases.setdefault(v, {}).setdefault(f"{STAMPS[a]}->{STAMPS[b]}", []).extend(
                    list((S[:, b] - S[:, a]) / 1e3))
    out = []
    for v in sorted(windows):
        win = np.median(np.array(windows[v]), axis=0)
        n = w.nodes[v]
        out.append({"kernel": v, "name": getattr(n, "name", "") or f"{n.op}{v}", "op": n.op,
                    "tiles": int(win[3]), "first_claim_us": round(float(win[0]), 2),
                    "first_ready_us": round(float(win[1]), 2), "last_release_us": round(float(win[2]), 2),
                    "phase_median_us": {k: round(float(np.median(x)), 2) for k, x in phases[v].items()}})
    lw = np.array(lw)
    return {"traced_launch_us_median": round(float(np.median(spans)), 2),
            "launch_window_us_median": {"entry_to_first_claim": round(float(np.median(lw[:, 0])), 2),
                                        "last_release_to_exit": round(float(np.median(lw[:, 1])), 2),
                                        "entry_to_exit": round(float(np.median(lw[:, 2])), 2)},
            "kernels": out}


def e2e_chunks(wl, n):
    """The batch in n consecutive shares of DAGs, for the end-to-end path's
    back-to-back launches: [(DAGs, {buffer id in concat(wl): id in concat(DAGs)})]."""
    per = -(-len(wl) // n)
    out, goff = [], 0
    for c in range(0, len(wl), per):
        part = wl[c:c + per]
        nbuf = sum(len(x.buffers) for x in part)
        out.append((part, {g: g - goff for g in range(goff, goff + nbuf)}))
        goff += nbuf
    return out


def make_workload(name, n_dags=256):
    """(workload, description); for "batched" the workload is the list of DAGs."""
    from synth.workloads import branchy_mlp, encoder_block, fork_join, random_batch
    if name == "batched":
        rank = int(os.environ.get("RANK", 0))
        return random_batch(n_dags, base_seed=1000 + 256 * rank), (
            f"{n_dags} seeded random layered DAGs (8-64 nodes, widths 1-8; GEMM 70% / eltwise 20% / "
            "softmax 10%; M,N,K in {64..2048}; bf16 or f32 per DAG) in one persistent launch "
            "replayed from a CUDA graph")
    if name == "mlp_bf16":
        return branchy_mlp("bf16"), ("branchy MLP inference DAG, bf16 in / f32 accumulate: batch 512, 4 branches x 3 "
                                     "Linear(2048,2048)+bias+ReLU, add tree, Linear(2048,4096)+ReLU, Linear(4096,1024)")
    if name == "mlp_f32":
        return branchy_mlp("f32"), "branchy MLP inference DAG, f32: batch 512, widths as mlp_bf16"
    if name == "fork_join":
        return fork_join(256), "fork-join DAG (paper Fig. 1): 3 GEMMs 256^3 f32 + add"
    if name == "softmax":
        from synth.workloads import Workload
        w = Workload("attention_softmax_level")
        for h in range(16):
            a = w.buf(2048, 256, "f32", "input", ("uniform", 100 + h), f"S{h}")
            w.node("softmax", a, w.buf(2048, 256, "bf16", "output", name=f"P{h}"), scale=0.125, name=f"softmax{h}")
        return w, ("the encoder's attention softmax level alone: 16 heads x (8 x 256) rows x 256, f32 scores in, "
                   "bf16 out, scale 1/8 (memory-bound)")
    if name == "add":
        from synth.workloads import Workload
        w = Workload("add_tree_4096")
        xs = [w.buf(4096, 4096, "bf16", "input", ("uniform", 200 + i), f"X{i}") for i in range(4)]
        s0 = w.buf(4096, 4096, "bf16", name="S0")
        s1 = w.buf(4096, 4096, "bf16", name="S1")
        w.node("add", xs[0], s0, b=xs[1], name="add0")
        w.node("add", xs[2], s1, b=xs[3], name="add1")
        w.node("add", s0, w.buf(4096, 4096, "bf16", "output", name="Y"), b=s1, name="add2")
        return w, ("a two-level add tree ((X0+X1)+(X2+X3)) of 4096 x 4096 bf16 matrices, 32 MiB each, "
                   "larger than L2 together (memory-bound)")
    if name == "heads":
        from synth.workloads import transformer_heads
        return transformer_heads(16, 256), ("the paper's transformer-layer DAG (§5): 16 heads, beta = 256, f32; "
                                            "per head 3 projections, Q.K^T, softmax, B.V, C.W_h")
    return encoder_block(), ("transformer encoder block DAG: 8 x 256 tokens, d_model 1024, 16 heads as fork "
                             "branches, out proj, FFN 4096 GELU; bf16 in / f32 accumulate")


def paper_alg1(d, abi, reps=8):
    """The paper's own form (Alg. 1 on CUDA streams, dag_submit_cq) on the
    same DAG: the task components as given (the whole DAG when none are) with
    q = 1..5 command queues, and eager (every kernel a component, one queue,
    a host callback per kernel).  Median device makespans in us."""
    import statistics
    out = {"components_given": {}, "eager_us": None, "eager_gap_us": None}
    for q in range(1, 6):
        rs = [d.run_cq(n_queues=q, components=abi.DAG_TC_GIVEN) for _ in range(reps)]
        out["components_given"][q] = statistics.median(r.device_us for r in rs)
        out["n_components"] = rs[0].n_components
    rs = [d.run_cq(n_queues=1, components=abi.DAG_TC_PER_KERNEL) for _ in range(reps)]
    out["eager_us"] = statistics.median(r.device_us for r in rs)
    out["eager_gap_us"] = statistics.median(r.gap_us for r in rs)
    best_q = min(out["components_given"], key=out["components_given"].get)
    out["best_q"] = best_q
    out["best_us"] = out["components_given"][best_q]
    out["speedup_best_q_over_q1"] = out["components_given"][1] / out["best_us"]
    return out


def run_exp1(args):
    """The paper's Experiment 1 on this GPU: transformer DAGs with H heads at
    beta = 256 (f32); per H the persistent executor, the kernel-by-kernel
    path, and Alg. 1 on streams (clustering: one component per head,
    q = 1..5; eager).  One JSON line."""
    import statistics
    import torch
    from paper_2009_07482_gb300 import _binding as abi
    from paper_2009_07482_gb300 import build as libbuild
    from paper_2009_07482_gb300.dag import Dag, options
    from synth.workloads import transformer_heads
    libbuild.build()
    stream = torch.cuda.current_stream()
    rows = []
    with ClockSampler(0) as clk:
        for H in (1, 2, 4, 8, 16):
            w = transformer_heads(H, 256)
            d = Dag(w, options(), resident_inputs=True)
            d.set_inputs(w.make_inputs(_INPUTS))

            def timed(submit, n):
                out = []
                for i in range(n + 3):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    submit(stream.cuda_stream)
                    b.record(stream)
                    abi.check(d.wait(), "wait")
                    if i >= 3:
                        out.append(a.elapsed_time(b) * 1e3)
                return statistics.median(out)

            row = {"heads": H, "persistent_us": timed(d.submit, 30)}
            d.close()
            # the paper's forms run every kernel as given: no sibling GEMMs merged
            d = Dag(w, options(merge=1), resident_inputs=True)
            d.set_inputs(w.make_inputs(_INPUTS))
            row["coarse_us"] = timed(d.submit_coarse, 10)
            row.update(paper_alg1(d, abi, reps=6))
            row["speedup_persistent_over_best"] = row["best_us"] / row["persistent_us"]
            rows.append(row)
            d.close()
        # Experiments 2-3: H = 16, beta 64..512; clustering (best q) against the
        # dynamic coarse policies with a host callback per kernel: eager (F by
        # rank) and FIFO order.  HEFT on a single device places every kernel on
        # it, so it reduces to the rank-ordered list (eager) here.
        rows23 = []
        for beta in (64, 128, 256, 512):
            w = transformer_heads(16, beta)
            d = Dag(w, options(), resident_inputs=True)
            d.set_inputs(w.make_inputs(_INPUTS))
            pers = []
            for i in range(23):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                d.submit(stream.cuda_stream)
                b.record(stream)
                abi.check(d.wait(), "wait")
                if i >= 3:
                    pers.append(a.elapsed_time(b) * 1e3)
            row = {"beta": beta, "persistent_us": statistics.median(pers)}
            d.close()
            d = Dag(w, options(merge=1), resident_inputs=True)  # Alg. 1 runs every kernel as given
            d.set_inputs(w.make_inputs(_INPUTS))
            clus = {q: statistics.median(d.run_cq(n_queues=q, components=abi.DAG_TC_GIVEN).device_us
                                         for _ in range(4)) for q in (1, 2, 3, 4, 5)}
            row["clustering_best_q"] = min(clus, key=clus.get)
            row["clustering_us"] = clus[row["clustering_best_q"]]
            for name, fifo in (("eager_rank_us", 0), ("eager_fifo_us", 1)):
                rs = [d.run_cq(n_queues=1, components=abi.DAG_TC_PER_KERNEL, fifo=fifo) for _ in range(4)]
                row[name] = statistics.median(r.device_us for r in rs)
                if not fifo:
                    row["eager_gap_us"] = statistics.median(r.gap_us for r in rs)
            row["speedup_clustering_over_eager"] = row["eager_rank_us"] / row["clustering_us"]
            row["speedup_persistent_over_clustering"] = row["clustering_us"] / row["persistent_us"]
            rows23.append(row)
            d.close()
    last = rows[-1]
    line = {"metric": "DAG makespan (us), paper §5 Experiment 1 transformer DAGs (beta 256, f32)",
            "value": last["persistent_us"], "unit": "us", "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32", "data": "synthetic (seeded SplitMix64)",
            "config": {"workload": "transformer_heads H in {1,2,4,8,16}, beta 256; value = persistent executor at H=16",
                       "f32_gemm": "tensor cores (3 x TF32 split)"},
            "sweep": rows, "exp2_3": rows23, "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (rows of the batch are independent in the MLP
# and fork-join DAGs; a sequence is independent in the encoder)
# ---------------------------------------------------------------------------
_INPUTS = {}


def _oracle_seconds(w, ins, repeat=1, min_s=0.5):
    """Mean seconds of one oracle run of w.  A run shorter than min_s counts as
    a warm-up, and the timed runs are repeated until they add up to min_s."""
    import oracle
    t0 = time.perf_counter()
    oracle.run(w, ins)
    t = time.perf_counter() - t0
    if t >= min_s and repeat == 1:
        return t
    n = max(repeat, -(-min_s // max(t, 1e-6)))
    t0 = time.perf_counter()
    for _ in range(int(n)):
        oracle.run(w, ins)
    return (time.perf_counter() - t0) / n


# workloads whose oracle sample is one of `units` independent parts of the DAG
UNIT_SAMPLES = ("encoder", "heads", "softmax", "add")
E2E_CHUNKS = 8  # persistent launches per batch step on the end-to-end path


def unit_sample(workload):
    """(sample workload, units per DAG, description) for UNIT_SAMPLES."""
    from synth.workloads import Workload, encoder_block, transformer_heads
    if workload == "encoder":
        return encoder_block(batch=1), 8, "encoder block: 1 of 8 independent sequences (all 99 kernels)"
    if workload == "heads":
        return transformer_heads(1, 256), 16, "transformer heads: 1 of 16 independent heads (7 kernels)"
    if workload == "softmax":
        w = Workload("one_head_softmax")
        a = w.buf(2048, 256, "f32", "input", ("uniform", 100), "S0")
        w.node("softmax", a, w.buf(2048, 256, "bf16", "output"), scale=0.125)
        return w, 16, "softmax level: 1 of 16 heads"
    if workload == "add":
        w = Workload("add_tree_rows")
        xs = [w.buf(256, 4096, "bf16", "input", ("uniform", 200 + i)) for i in range(4)]
        s0, s1 = w.buf(256, 4096, "bf16"), w.buf(256, 4096, "bf16")
        w.node("add", xs[0], s0, b=xs[1])
        w.node("add", xs[2], s1, b=xs[3])
        w.node("add", s0, w.buf(256, 4096, "bf16", "output"), b=s1)
        return w, 16, "add tree: 256 of 4096 rows"
    raise ValueError(workload)


def _row_subset(w, ins, rows):
    """The DAG w restricted to batch rows `rows` of every row-space buffer
    (the random layered DAGs and the MLPs are row-wise: row i of every kernel
    output depends on row i of its row-space inputs and on whole weights),
    with its inputs: the oracle on it computes exactly those rows."""
    import dataclasses
    weights = {n.b for n in w.nodes if n.op == "gemm"} | {n.bias for n in w.nodes if n.op == "gemm" and n.bias >= 0}
    rs = {i for i, b in enumerate(w.buffers) if b.role != "input" or i not in weights}
    ws = w.clone()
    for i in rs:
        ws.buffers[i] = dataclasses.replace(ws.buffers[i], rows=len(rows))
    return ws, {i: (a[rows] if i in rs else a) for i, a in ins.items()}


def _gemm_flops(w):
    return sum(w.node_flops(k) for k, n in enumerate(w.nodes) if n.op == "gemm")


BATCH_ROWS = 4


def batch_sample(stride=8, first=0):
    """The 256-DAG batch and a bounded sample of it: the first BATCH_ROWS rows
    of every `stride`-th DAG (from `first`), each run whole over those rows.
    Returns (DAGs, picked ids, GEMM flops of the sample, GEMM flops of the
    batch); all work of these DAGs is row-wise, so the sample's share of the
    batch's work is the ratio of GEMM flops."""
    from synth.workloads import random_batch
    ws = random_batch(256)
    pick = list(range(first, len(ws), stride))
    rows = BATCH_ROWS
    f_sample = sum(sum(w.node_flops(k) * rows / w.buffers[n.a].rows for k, n in enumerate(w.nodes) if n.op == "gemm")
                   for w in (ws[i] for i in pick))
    return ws, pick, f_sample, sum(_gemm_flops(x) for x in ws)


def _batch_sample_seconds(ws, pick, inputs=None):
    """Seconds of the oracle on the batch sample (inputs drawn beforehand)."""
    import numpy as np
    import oracle
    rows = np.arange(BATCH_ROWS)
    subs = []
    for i in pick:
        ins = inputs[i] if inputs else ws[i].make_inputs()
        subs.append(_row_subset(ws[i], ins, rows))
    t0 = time.perf_counter()
    for w, ins in subs:
        oracle.run(w, ins)
    return time.perf_counter() - t0


def oracle_model(workload, ra=4, rb=12):
    """Seconds per full DAG of the FP64 oracle on one host core, from a bounded
    sample.  MLP / fork-join rows are independent, so the time is
    fixed + rows * slope (the fixed part widens each weight once); two row
    counts give both terms.  The encoder's sequences are independent: one
    sequence, times 8."""
    import oracle
    from synth.workloads import branchy_mlp, encoder_block, fork_join
    oracle.build()
    if workload.startswith("mlp"):
        dt = "bf16" if workload == "mlp_bf16" else "f32"
        wa, wb = branchy_mlp(dt, batch=ra), branchy_mlp(dt, batch=rb)
        ta = _oracle_seconds(wa, wa.make_inputs(_INPUTS))
        tb = _oracle_seconds(wb, wb.make_inputs(_INPUTS))
        slope = max(tb - ta, 0.0) / (rb - ra)
        full = ta + (512 - ra) * slope
        desc = (f"branchy MLP {dt} on {ra} and {rb} of 512 batch rows (all 17 kernels; {ta:.2f} s, {tb:.2f} s), "
                f"extrapolated linearly in rows to 512")
        return full, desc, (wa, ra, ta, slope)
    if workload == "fork_join":
        w = fork_join(256)
        t = _oracle_seconds(w, w.make_inputs(), repeat=3)
        return t, "fork-join 256^3 f32: the whole DAG, mean of 3 runs", (w, 256, t, 0.0)
    if workload in UNIT_SAMPLES:
        w, units, what = unit_sample(workload)
        t = _oracle_seconds(w, w.make_inputs(_INPUTS))
        return units * t, f"{what} ({t:.2f} s), times {units}", (w, 1, t, 0.0)
    if workload == "batched":
        ws, pick, f_s, f_b = batch_sample()
        t = _batch_sample_seconds(ws, pick)
        return (t * f_b / f_s,
                f"random batch: the first {BATCH_ROWS} rows of each of {len(pick)} DAGs (every 8th) in {t:.2f} s; "
                f"extrapolated to the 256-DAG batch by GEMM flops (x{f_b / f_s:.0f})",
                (None, 0, t, 0.0))
    raise ValueError(f"no oracle sample for workload {workload}")


def oracle_sample(workload):
    full, desc, _ = oracle_model(workload)
    n_dags = 256 if workload == "batched" else 1
    return {"value": n_dags / full, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}


def _oracle_rows_proc(dt, ra, rb, barrier, out):
    """One process of oracle_all_cores (MLP): build the samples, then time the
    oracle on ra and on rb batch rows, each start aligned with the others."""
    import oracle
    from synth.workloads import branchy_mlp
    oracle.build()
    wa, wb = branchy_mlp(dt, batch=ra), branchy_mlp(dt, batch=rb)
    cache = {}                              # both samples share one draw of the weights
    ia, ib = wa.make_inputs(cache), wb.make_inputs(cache)
    barrier.wait(timeout=300)
    ta = _oracle_seconds(wa, ia)
    barrier.wait(timeout=300)
    tb = _oracle_seconds(wb, ib)
    out.put((ta, tb))


def _oracle_unit_proc(workload, barrier, out):
    """One process of oracle_all_cores (UNIT_SAMPLES): time the oracle on one
    independent part of the DAG, the start aligned with the others."""
    import oracle
    oracle.build()
    w, _, _ = unit_sample(workload)
    ins = w.make_inputs()
    barrier.wait(timeout=300)
    out.put(_oracle_seconds(w, ins))


def _oracle_batch_proc(barrier, out):
    """One process of oracle_all_cores (batched): time the batch's sample."""
    import oracle
    oracle.build()
    ws, pick, _, _ = batch_sample()
    ins = {i: ws[i].make_inputs() for i in pick}
    barrier.wait(timeout=300)
    out.put(_batch_sample_seconds(ws, pick, ins))


def _spawn_timed(target, args, P):
    """Run target(*args, barrier, queue) in P spawned processes (none inherits
    the parent's CUDA context) and return what each put on the queue; a process
    that fails or stalls raises instead of hanging the caller."""
    import multiprocessing as mp
    import queue
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(P), ctx.Queue()
    ps = [ctx.Process(target=target, args=(*args, barrier, out)) for _ in range(P)]
    for p in ps:
        p.start()
    res, deadline = [], time.time() + 420
    try:
        while len(res) < P:
            try:
                res.append(out.get(timeout=2))
            except queue.Empty:
                if any(p.exitcode not in (None, 0) for p in ps) or time.time() > deadline:
                    raise RuntimeError("a worker process of the all-cores oracle timing failed or ran too long")
    finally:
        for p in ps:
            p.join(timeout=5)
            if p.is_alive():
                p.terminate()
    return res


def oracle_all_cores(workload, ra=4, rb=20, procs=None):
    """The FP64 oracle on every host core at once (at most 64 processes, about
    0.3 GB each), from the same bounded samples as oracle_model, all started
    together so that they share the machine as a parallel run would.

    MLP: the batch rows are independent, so a DAG splits into one share of rows
    per core; each process times ra and rb rows and extrapolates its share,
    fixed + ceil(512 / procs) * slope (each share widens the weights once).
    UNIT_SAMPLES: the sample is one of `units` independent parts (a sequence, a
    head, a row block); min(procs, units) processes each time one, and a DAG
    takes ceil(units / processes) of them.  Batched: every process times the
    batch's three-DAG sample, and the batch, scaled by GEMM flops, spreads over
    the processes.  The processes are alike, so the median time stands for them
    (the slowest would mostly measure noise)."""
    P = procs or min(len(os.sched_getaffinity(0)), 64)
    if workload.startswith("mlp"):
        dt = "bf16" if workload == "mlp_bf16" else "f32"
        res = _spawn_timed(_oracle_rows_proc, (dt, ra, rb), P)
        rows = -(-512 // P)

        def share(ta, tb):  # one process's share of a DAG, from its own two samples
            slope = max(tb - ta, 0.0) / (rb - ra)
            return max(ta - ra * slope, 0.0) + rows * slope

        shares = sorted(share(ta, tb) for ta, tb in res)
        full = shares[len(shares) // 2]
        sample = (f"branchy MLP {dt}: {P} processes at once, each timing {ra} and {rb} batch rows and "
                  f"extrapolating its share of {rows} rows ({shares[0]:.1f} to {shares[-1]:.1f} s); "
                  f"one DAG = the median share")
    elif workload in UNIT_SAMPLES:
        _, units, what = unit_sample(workload)
        P = min(P, units)
        ts = sorted(_spawn_timed(_oracle_unit_proc, (workload,), P))
        waves = -(-units // P)
        full = ts[len(ts) // 2] * waves
        sample = (f"{what}: {P} processes at once, each timing one part ({ts[0]:.2f} to {ts[-1]:.2f} s); "
                  f"one DAG = {waves} x the median")
    elif workload == "batched":
        _, pick, f_s, f_b = batch_sample()
        ts = sorted(_spawn_timed(_oracle_batch_proc, (), P))
        full = ts[len(ts) // 2] * (f_b / f_s) / P / 256    # per DAG, the batch's DAGs spread over P cores
        sample = (f"random batch: {P} processes at once, each timing the first {BATCH_ROWS} rows of each of "
                  f"{len(pick)} DAGs ({ts[0]:.2f} to {ts[-1]:.2f} s); the batch = the median x {f_b / f_s:.0f} "
                  f"(GEMM flops) / {P} processes")
    else:
        raise ValueError(f"no all-cores oracle sample for workload {workload}")
    return {"value": 1.0 / full, "unit": UNIT, "cores": P, "kind": "oracle", "sample": sample}


def reference_units(workload, step):
    """Whole units of work for the reference arm's step `step`: a list of
    (oracle workload, its inputs) plus the fraction of one DAG of the
    benchmark's workload they make up, and a description.  Inputs are drawn
    here, before the step's timer starts."""
    from synth.workloads import branchy_mlp, fork_join
    if workload.startswith("mlp"):
        rows = 64
        w = branchy_mlp("bf16" if workload == "mlp_bf16" else "f32", batch=rows)
        return [(w, w.make_inputs(_INPUTS))], rows / 512, f"a block of {rows} of the 512 batch rows (all 17 kernels)"
    if workload == "fork_join":
        w = fork_join(256)
        return [(w, w.make_inputs(_INPUTS))], 1.0, "the whole DAG"
    if workload in UNIT_SAMPLES:
        w, units, what = unit_sample(workload)
        return [(w, w.make_inputs(_INPUTS))], 1.0 / units, what
    if workload == "batched":
        import numpy as np
        ws, _, _, f_b = _REF_BATCH or _ref_batch()
        k0 = (8 * step) % 256
        units, f = [], 0.0
        for k in range(k0, k0 + 8):
            w = ws[k]
            units.append(_row_subset(w, w.make_inputs(), np.arange(BATCH_ROWS)))
            f += sum(w.node_flops(j) * BATCH_ROWS / w.buffers[n.a].rows for j, n in enumerate(w.nodes) if n.op == "gemm")
        return units, f / (f_b / 256), (f"the first {BATCH_ROWS} rows of 8 DAGs of the batch (DAGs 8s..8s+7 at "
                                        f"step s), counted in DAGs of the batch's mean GEMM work")
    raise ValueError(workload)


_REF_BATCH = None


def _ref_batch():
    global _REF_BATCH
    _REF_BATCH = batch_sample()
    return _REF_BATCH


def run_reference(args):
    """The FP64 oracle as the reference arm, on one host core: every step
    runs whole units of the workload (see reference_units) and is timed as
    it ran; the rate is the DAG fraction those units make up, summed over the
    timed steps, over the time they took.  Nothing is extrapolated into the
    timed figures; the full-DAG time the rate implies is reported beside them
    under its own name."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload in ("serving", "exp1"):
        print(json.dumps({"impl": "reference", "unavailable": f"--workload {args.workload} has no oracle arm; "
                          "its DAGs are timed in the other workloads"}))
        return 0
    import oracle
    oracle.build()
    _, desc = make_workload(args.workload)
    per, frac = [], []
    what = ""
    for i in range(args.warmup + args.steps):
        units, f, what = reference_units(args.workload, i)
        t0 = time.perf_counter()
        for w, ins in units:
            oracle.run(w, ins)
        t = time.perf_counter() - t0
        if i >= args.warmup:
            per.append(t)
            frac.append(f)
    rate = sum(frac) / sum(per)
    ms = statistics.mean(per) * 1e3
    sample = f"each step: the oracle on {what}; rate = DAG fraction done / time spent over the timed steps"
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": desc, "parallelism": "host oracle, rank 0 only"},
            "dag_fraction_per_step": statistics.mean(frac),
            "implied_seconds_per_full_dag": 1.0 / rate,
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.15)
        self.t0 = time.time()
        return self

    def __exit__(self, *a):
        self.t1 = time.time()
        time.sleep(0.1)
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if not (self.t0 - 0.06 <= ts <= self.t1 + 0.06):
                    continue
                sm.append(float(f[2]))
                mx = max(mx, float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def traffic_for(workload):
    """DRAM bytes per executor launch from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2009_07482_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    sha = h.hexdigest()[:16]
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if os.path.exists(p):
        for line in open(p):
            f = line.split()
            if len(f) >= 3 and f[0] == workload and f[1] == sha:
                return float(f[2]), sha
    return None, sha


def learned_eval_batched(wl, ins, abi, Dag, options, timed_fn):
    """Ranks for the 256-DAG batch from three cost sources -- the planner's
    roofline model (default), a measured profile (tile times traced on a run
    of this batch) and the learned MLP (trained on traces of other random
    DAGs) -- plus FIFO order; reports the median makespan of each and the
    prediction error of the model-based sources against the profile."""
    import numpy as np
    from paper_2009_07482_gb300.costmodel import (CostModel, features, measure, mape,
                                                  node_costs_from_tile_times)
    from synth.workloads import concat
    # profile of the batch itself
    d = Dag.batch(wl, options(trace=1, use_graph=1), resident_inputs=True)
    d.set_inputs(ins)
    for _ in range(2):
        d.run()
    st = abi.dag_trace_stamps(d.h).astype(np.int64)
    tiles = d.tiles()
    grid = d.plan().grid
    model_costs = abi.dag_node_costs_get(d.h).astype(np.float64)
    d.close()
    nn = sum(len(x.nodes) for x in wl)
    dur = (st[:, 9] - st[:, 1]) / 1e3
    per = [[] for _ in range(nn)]
    for t, v in enumerate(tiles[:, 0]):
        per[v].append(dur[t])
    prof_tile = np.array([np.median(x) if x else 0.0 for x in per])
    counts = np.bincount(tiles[:, 0], minlength=nn)
    prof_costs = node_costs_from_tile_times(prof_tile, counts, grid)
    model_tile = model_costs / np.ceil(np.maximum(counts, 1) / grid)
    # learned model trained on traces of other random DAGs, alone and in
    # batches of 2..64 (so its concurrency feature covers batched plans)
    from synth.workloads import random_batch, random_layered
    trF, trT = [], []
    seed = 5000
    for k in (1, 1, 1, 1, 2, 4, 8, 16, 32, 64):
        rw = concat(random_batch(k, base_seed=seed))
        seed += k
        F, t, *_ = measure(rw, rw.make_inputs(_INPUTS))
        trF.append(F)
        trT.append(t)
    for i in range(8):  # single DAGs with sizes up to 4096 (beyond the batch's 2048)
        rw = random_layered(5200 + i, 8, 24, 4, sizes=(64, 128, 256, 512, 1024, 2048, 4096))
        F, t, *_ = measure(rw, rw.make_inputs(_INPUTS))
        trF.append(F)
        trT.append(t)
    cm = CostModel().fit(np.concatenate(trF), np.concatenate(trT))
    # features of each DAG inside the batch plan (level concurrency of the batch)
    wcat = concat(wl)
    Fb = features(wcat, tiles, grid)
    learn_tile = cm.predict_tile_us(Fb)
    learn_costs = node_costs_from_tile_times(learn_tile, counts, grid)
    chain = chain_and_fill_eval(cm, abi, Dag, options, timed_fn)
    cm.close()
    res = {"mape_learned_vs_profile": mape(learn_tile, prof_tile),
           "mape_roofline_vs_profile": mape(model_tile, prof_tile), "makespan_us": {}}
    for name, o in (("rank_roofline_model", options(use_graph=1)),
                    ("rank_profile", options(use_graph=1, scheduler=abi.DAG_SCHED_RANK_GIVEN, node_cost_us=prof_costs)),
                    ("rank_learned", options(use_graph=1, scheduler=abi.DAG_SCHED_RANK_GIVEN, node_cost_us=learn_costs)),
                    ("fifo", options(use_graph=1, scheduler=abi.DAG_SCHED_FIFO))):
        dd = Dag.batch(wl, o, resident_inputs=True)
        dd.set_inputs(ins)
        dd.run()
        res["makespan_us"][name] = statistics.median(timed_fn(dd, 5))
        dd.close()
    ms = res["makespan_us"]
    res["regret_learned_vs_profile"] = ms["rank_learned"] / ms["rank_profile"] - 1.0
    res["gain_learned_vs_roofline_model"] = ms["rank_roofline_model"] / ms["rank_learned"] - 1.0
    res["chain_and_fill"] = chain
    return res


def chain_and_fill_eval(cm, abi, Dag, options, timed_fn, reps=9):
    """The DAG where the cost source decides the order: a chain of 48 small,
    latency-bound bf16 GEMMs (the critical path; the roofline model prices each
    at a fraction of its measured time) beside four 4096^3 GEMMs.  Makespan
    with the critical-path priority under roofline, measured-profile and
    learned costs, and FIFO."""
    from paper_2009_07482_gb300.costmodel import profile_costs
    from synth.workloads import chain_and_fill
    w = chain_and_fill()
    ins = w.make_inputs(_INPUTS)
    learned = cm.node_costs(w)
    prof = profile_costs(w, ins)
    cp = abi.DAG_RANK_CRITICAL_PATH
    out = {"workload": w.name, "priority": "critical path (upward + downward rank)", "makespan_us": {}}
    for name, o in (("roofline_model", options(rank_form=cp)),
                    ("profile", options(rank_form=cp, scheduler=abi.DAG_SCHED_RANK_GIVEN, node_cost_us=prof)),
                    ("learned", options(rank_form=cp, scheduler=abi.DAG_SCHED_RANK_GIVEN, node_cost_us=learned)),
                    ("fifo", options(scheduler=abi.DAG_SCHED_FIFO))):
        d = Dag(w, o, resident_inputs=True)
        d.set_inputs(ins)
        d.run()
        out["makespan_us"][name] = statistics.median(timed_fn(d, reps))
        d.close()
    ms = out["makespan_us"]
    out["gain_learned_vs_roofline_model"] = ms["roofline_model"] / ms["learned"] - 1.0
    out["regret_learned_vs_profile"] = ms["learned"] / ms["profile"] - 1.0
    return out


def serving_models():
    """The serving mix: fork-join 256^3 f32; branchy MLP bf16 at batch 1, 16,
    256; encoder block at 1 and 2 sequences of 256 tokens."""
    from synth.workloads import branchy_mlp, encoder_block, fork_join
    return [fork_join(256), branchy_mlp("bf16", batch=1), branchy_mlp("bf16", batch=16),
            branchy_mlp("bf16", batch=256), encoder_block(batch=1), encoder_block(batch=2)]


def run_serving(args):
    """Open-loop serving: Poisson arrivals of requests drawn from the model
    mix, continuous admission into slots by free device memory; latency =
    completion (outputs in host memory) minus scheduled arrival."""
    import numpy as np
    import torch
    import synth
    from paper_2009_07482_gb300 import _binding as abi
    from paper_2009_07482_gb300 import build as libbuild
    from paper_2009_07482_gb300.costmodel import CostModel, measure, node_costs_from_tile_times
    from paper_2009_07482_gb300.serving import Server, activation_ids
    from synth.workloads import random_layered
    libbuild.build()
    torch.cuda.set_device(0)
    ws = serving_models()
    weights = [w.make_inputs(_INPUTS) for w in ws]
    n_req = 2000
    seq = [int(x) % len(ws) for x in synth.splitmix64(3, n_req)]

    # kernel costs for the slots' ranks: measured profile, and the learned model
    prof, feats = [], []
    for w, ins in zip(ws, weights):
        F, med, counts, grid, _ = measure(w, ins)
        prof.append(node_costs_from_tile_times(med, counts, grid))
        feats.append((F, counts, grid))
    trF, trT = [], []
    for i in range(24):
        rw = random_layered(5000 + i, 8, 24, 4, sizes=(64, 128, 256, 512, 1024))
        F, t, *_ = measure(rw, rw.make_inputs(_INPUTS))
        trF.append(F)
        trT.append(t)
    cm = CostModel().fit(np.concatenate(trF), np.concatenate(trT))
    learned = [node_costs_from_tile_times(cm.predict_tile_us(F), c, g) for F, c, g in feats]
    cm.close()

    def server(costs):
        srv = Server(ws, weights, max_slots=64, hbm_reserve_bytes=8 << 30, node_costs=costs)
        for m, w in enumerate(ws):
            srv.set_default_io(m, {i: weights[m][i] for i in activation_ids(w)})
            abi.dag_server_warm(srv.s, m, 4)
        abi.dag_server_simulate(srv.s, seq[:200], 1e7, 1)  # warm-up
        return srv

    srv = server(prof)
    abi.dag_server_simulate(srv.s, seq, 1e9, 5)                 # untimed: creates the slots the mix needs
    _, wall, _ = abi.dag_server_simulate(srv.s, seq, 1e9, 7)   # all at once: saturation throughput
    sat = n_req / wall
    sweep = []
    for f in (0.25, 0.5, 0.75, 1.0, 1.25):
        lat, wall, mif = abi.dag_server_simulate(srv.s, seq, f * sat, 11)
        sweep.append({"rate_frac": f, "rate_dags_per_s": f * sat, "dags_per_s": n_req / wall,
                      "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                      "max_in_flight": mif})
    slots = abi.dag_server_slots(srv.s)
    srv.close()
    compare = {}
    for name, costs in (("profile", prof), ("learned", learned)):
        srv = server(costs)
        lat, wall, _ = abi.dag_server_simulate(srv.s, seq, 0.75 * sat, 13)
        compare[name] = {"p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                         "dags_per_s": n_req / wall}
        srv.close()
    compare["learned_p99_regret"] = compare["learned"]["p99_us"] / compare["profile"]["p99_us"] - 1.0
    line = {"metric": "DAGs/s (serving, open-loop Poisson arrivals)", "value": sat, "unit": UNIT, "n_gpus": 1,
            "steps": n_req, "warmup": 200, "ms_per_step": 1e3 / sat, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic (seeded SplitMix64)",
            "config": {"workload": "serving mix: " + ", ".join(w.name for w in ws), "requests": n_req,
                       "slots_created": slots, "admission": "by free HBM (8 GiB reserve), 64 slots max"},
            "serving": sweep, "scheduler_compare_at_0.75": compare, "gpu_launches": n_req}
    print(json.dumps(line))
    return 0


def roofline_of(w, info, mean_us, peaks, peaks_src, f32_simt):
    """Roofline of one executor launch of workload w taking mean_us: achieved
    TFLOP/s (GB/s for a DAG without GEMMs) against the measured peak of the
    arithmetic the GEMMs run in.  f32 GEMMs: the larger of the FP32 ALU peak
    (152 SMs x 128 FFMA/clk x 2 flop x max SM clock) and the 3 x TF32 tensor
    peak (measured bf16 x the nominal tf32/bf16 ratio 1.1/2.25, / 3
    products); the executor runs them on the tensor cores unless f32_simt.
    A DAG with both takes the flop-weighted peak.  Returns (roof, flops by
    dtype)."""
    simt_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    tc_peak = peaks["bf16_tflops"] * (1.1 / 2.25) / 3.0
    f32_peak = simt_peak if f32_simt else max(simt_peak, tc_peak)
    fl = {"bf16": 0.0, "f32": 0.0}
    for k, n in enumerate(w.nodes):
        if n.op == "gemm":
            fl[w.buffers[n.a].dtype] += w.node_flops(k)
    t_bound_us = (fl["bf16"] / peaks["bf16_tflops"] + fl["f32"] / f32_peak) / 1e6
    achieved = info.flops / (mean_us * 1e-6) / 1e12
    src_bf16 = f"{peaks_src} bf16 burst (MEASURED_PEAKS.json)" if peaks_src == "measured" else "fallback 1.9 PF/s"
    src_f32 = ("3 x TF32 on the tensor cores: measured bf16 burst x 1.1/2.25 (nominal tf32/bf16) / 3"
               if f32_peak == tc_peak else "derived: 152 SMs x 128 f32 FMA/clk x 2 flop x max SM clock")
    if fl["f32"] == 0 and fl["bf16"] == 0:  # no GEMM: the DAG is bound by HBM bandwidth
        roof = {"bound": "hbm", "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "peak_source": f"{peaks_src} HBM copy bandwidth (MEASURED_PEAKS.json)"}
    elif fl["f32"] == 0:
        roof = {"bound": "tensor", "peak": peaks["bf16_tflops"], "peak_source": src_bf16}
    elif fl["bf16"] == 0:
        roof = {"bound": "alu" if f32_simt else "tensor", "peak": f32_peak, "peak_source": src_f32}
    else:
        roof = {"bound": "tensor", "peak": info.flops / t_bound_us / 1e6,
                "peak_source": f"flop-weighted: bf16 at {src_bf16}, f32 at {src_f32}"}
    if roof["bound"] == "hbm":
        achieved = info.bytes / (mean_us * 1e-6) / 1e9
        roof.update({"achieved": achieved, "frac": achieved / roof["peak"]})
    else:
        roof.update({"achieved": achieved, "unit": "TFLOP/s", "frac": achieved / roof["peak"]})
    return roof, fl


CONFIGS = ("fork_join", "mlp_bf16", "mlp_f32", "encoder")


def config_extras(args, abi, Dag, options, stream, flush, peaks, peaks_src, reps=20):
    """The single-DAG configurations, each measured as the main line measures
    its workload (inputs resident, L2 flushed between steps, CUDA events on
    the launching stream): device makespan of the persistent executor, the
    kernel-by-kernel path, the paper's Alg. 1 on streams (given components,
    q = 1..5, best), and the fractions of the critical-path and work bounds
    and of the measured peak."""
    import torch
    sp = stream.cuda_stream
    out = {}

    def timed(submit, dd, n):
        for _ in range(3):
            submit(sp)
            abi.check(dd.wait(), "wait")
        ts = []
        for _ in range(n):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            submit(sp)
            b.record(stream)
            abi.check(dd.wait(), "wait")
            ts.append(a.elapsed_time(b) * 1e3)
        return ts

    for name in CONFIGS:
        w, desc = make_workload(name)
        d = Dag(w, options(), resident_inputs=True)
        d.set_inputs(w.make_inputs(_INPUTS))
        d.run()
        fine = timed(d.submit, d, max(reps, args.steps))
        info = d.plan()
        # the kernel-by-kernel path and Alg. 1 launch every kernel as given (no
        # sibling GEMMs merged), as the paper's forms do
        dk = Dag(w, options(merge=1), resident_inputs=True)
        dk.set_inputs(w.make_inputs(_INPUTS))
        dk.run()
        coarse = timed(dk.submit_coarse, dk, max(5, reps // 2))
        alg1 = paper_alg1(dk, abi, reps=5)
        dk.close()
        med = statistics.median(fine)
        roof, _ = roofline_of(w, info, statistics.mean(fine), peaks, peaks_src, False)
        out[name] = {"workload": desc, "tiles": info.n_tiles,
                     "makespan_us": {"median": med, "mean": statistics.mean(fine), "min": min(fine)},
                     "dags_per_s": 1e6 / statistics.mean(fine),
                     "coarse_us": statistics.median(coarse),
                     "speedup_fine_over_coarse": statistics.median(coarse) / med,
                     "paper_alg1": {"best_q": alg1["best_q"], "best_us": alg1["best_us"],
                                    "eager_us": alg1["eager_us"],
                                    "speedup_persistent_over_best": alg1["best_us"] / med},
                     "cp_roofline": {"critical_path_us": info.critical_path_us, "work_bound_us": info.work_bound_us,
                                     "frac_of_cp": info.critical_path_us / med,
                                     "frac_of_work_bound": info.work_bound_us / med},
                     "roofline": {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "frac")}}
        d.close()
        _INPUTS.clear()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "exp1":
        return run_exp1(args)
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2009_07482_gb300 import _binding as abi
    from paper_2009_07482_gb300 import build as libbuild
    from paper_2009_07482_gb300.dag import Dag, describe, options
    libbuild.build()
    abi.dag_set_device(local)
    peaks, peaks_src = load_peaks()
    abi.dag_set_peaks(peaks["bf16_tflops"], 0.0, peaks["hbm_gbs"])

    wl, desc = make_workload(args.workload, args.dags)
    batched = isinstance(wl, list)
    from synth.workloads import concat
    w = concat(wl) if batched else wl
    n_dags = len(wl) if batched else 1
    if batched:
        ins, off = {}, 0
        for x in wl:
            ins.update({off + i: a for i, a in x.make_inputs(_INPUTS).items()})
            off += len(x.buffers)
    else:
        ins = w.make_inputs(_INPUTS)
    # per-step inputs: the activations (inputs not used as GEMM weights or biases)
    weights = {n.b for n in w.nodes if n.op == "gemm"} | {n.bias for n in w.nodes if n.op == "gemm" and n.bias >= 0}
    X_ids = [i for i in w.input_ids() if i not in weights]
    Y_ids = w.output_ids()

    def make_dag(streamed, fuse=0, trace=0, merge=0):
        o = options(use_graph=1 if batched else 0, f32_gemm=abi.DAG_F32_GEMM_SIMT if args.f32_simt else 0,
                    fuse=fuse, trace=trace, merge=merge, tile_override=args.tile_override)
        if batched:
            return Dag.batch(wl, o, resident_inputs=not streamed, streamed=set(X_ids) if streamed else None)
        return Dag(w, o, streamed=set(X_ids)) if streamed else Dag(w, o, resident_inputs=True)

    # device-resident run: every input resident
    d = make_dag(False)
    d.set_inputs(ins)
    d.run()
    info = d.plan()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(submit, steps, warmup, dd=None):
        dd = dd or d
        for _ in range(warmup):
            submit(sp)
            abi.check(dd.wait(), "wait")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        t0 = time.perf_counter()
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            submit(sp)
            b.record(stream)
            abi.check(dd.wait(), "wait")
        barrier()
        wall = time.perf_counter() - t0
        return [a.elapsed_time(b) * 1e3 for a, b in evs], wall  # us

    launches_per_step = 1
    with ClockSampler(local) as clk:
        fine_us, wall = timed(d.submit, args.steps, max(3, args.warmup))
    if args.profile:
        print(json.dumps({"profile_run": True, "median_us": statistics.median(fine_us)}))
        d.close()
        return 0
    if args.timeline:
        dt = make_dag(False, trace=1)
        dt.set_inputs(ins)
        for _ in range(max(3, args.warmup)):
            dt.run()
        tl = run_timeline(args, w, dt, abi, stream, flush)
        if args.chrome_trace:
            dt.write_chrome_trace(args.chrome_trace)
        dt.close()
        d.close()
        print(json.dumps({"timeline": args.workload, "config": {"workload": desc},
                          "untraced_makespan_us_median": round(statistics.median(fine_us), 2), **tl}))
        return 0
    # kernel by kernel: every kernel as given (no sibling GEMMs merged), one
    # launch per kernel not fused into a GEMM, two for a split GEMM
    dk = make_dag(False, merge=1)
    dk.set_inputs(ins)
    dk.run()
    coarse_us, _ = timed(dk.submit_coarse, min(10, max(3, args.steps // 4)) if batched else max(10, args.steps // 4), 3,
                         dd=dk)
    fused = dk.fusion()
    tl = dk.tiles()
    dk.close()
    split_nodes = {int(t[0]) for t in tl if (int(t[5]) >> 16) & 0xFF}
    n_coarse_launches = sum(1 + (v in split_nodes) for v in range(len(w.nodes)) if fused[v] < 0)
    # the opt-in epilogue-fusion modes (the measured line runs without fusion)
    unfused = None
    for name, mode in (() if batched else (("activations", abi.DAG_FUSE_ACT), ("activations_and_adds", abi.DAG_FUSE_ALL))):
        fo = options(fuse=mode, f32_gemm=abi.DAG_F32_GEMM_SIMT if args.f32_simt else 0)
        n_f = sum(h >= 0 for h in abi.dag_fusion_host(*describe(w, resident_inputs=True), fo))
        if not n_f:
            continue
        u = make_dag(False, fuse=mode)
        u.set_inputs(ins)
        u.run()
        u_us, _ = timed(u.submit, max(5, args.steps // 2), 3, u)
        unfused = unfused or {"mode": "none"}
        unfused[name] = {"fused_kernels": int(n_f), "median_us": statistics.median(u_us)}
        u.close()
    alg1 = None if batched else paper_alg1(d, abi, reps=8)

    # max over ranks of the mean step time
    mean_us = statistics.mean(fine_us)
    if world > 1:
        t = torch.tensor([mean_us], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        mean_us = float(t.item())
    value = world * n_dags * 1e6 / mean_us
    med = statistics.median(fine_us)
    q = np.percentile(fine_us, [10, 90])
    cmed = statistics.median(coarse_us)

    # e2e: host buffers through the C ABI (activations streamed from pinned
    # memory every step, every sink read back into pinned memory).  The batch
    # goes as E2E_CHUNKS persistent launches of an equal share of its DAGs, one
    # handle each, submitted back to back on one stream: a launch's readback
    # (after its own end) and the next launches' uploads run on the copy
    # engines while the following launch computes.
    d.close()
    e2e_parts = []  # (handle, {global buffer id: local id})
    if batched:
        for part, loc in e2e_chunks(wl, E2E_CHUNKS):
            o = options(use_graph=1, f32_gemm=abi.DAG_F32_GEMM_SIMT if args.f32_simt else 0)
            eh = Dag.batch(part, o, resident_inputs=False, streamed={loc[i] for i in X_ids if i in loc})
            e2e_parts.append((eh, loc))
    else:
        e2e_parts.append((make_dag(True), {i: i for i in range(len(w.buffers))}))
    pins = []
    ybytes = 0
    for eh, loc in e2e_parts:
        eh.set_inputs({loc[k]: v for k, v in ins.items() if k in loc and k not in X_ids})
        eh.run()
        eh.set_inputs({loc[k]: ins[k] for k in X_ids if k in loc}, pinned=True)
        for Y in Y_ids:
            if Y not in loc:
                continue
            nb = w.buffers[Y].rows * w.buffers[Y].cols * (4 if w.buffers[Y].dtype == "f32" else 2)
            pins.append(abi.dag_host_alloc(nb))
            abi.dag_set_output(eh.h, loc[Y], pins[-1])
            ybytes += nb

    def e2e_step():
        for eh, _ in e2e_parts:
            eh.submit(sp)
        for eh, _ in e2e_parts:
            abi.check(eh.wait(), "wait")

    for _ in range(max(3, args.warmup)):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = args.steps if not batched else min(10, max(3, args.steps // 4))
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    xbytes = sum(ins[k].nbytes for k in X_ids)
    for eh, loc in e2e_parts:
        for Y in Y_ids:
            if Y in loc:
                abi.dag_set_output(eh.h, loc[Y], None)
        eh.close()
    for pnt in pins:
        abi.dag_host_free(pnt)

    # roofline of the executor kernel (the only kernel of a step)
    roof, fl = roofline_of(w, info, mean_us, peaks, peaks_src, args.f32_simt)
    bf16 = fl["bf16"] > 0 and fl["f32"] == 0
    traffic, sha = traffic_for(args.workload)
    roof["traffic"] = traffic
    roof["algorithmic"] = {"flops_per_launch": info.flops, "bytes_per_launch": info.bytes}
    roof["kernel"] = "dagx::dag_exec_kernel"
    roof["kernel_src_sha"] = sha

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_us / 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32+bf16 (no GEMM)" if roof["bound"] == "hbm" else "bf16" if bf16
                  else ("f32" if fl["bf16"] == 0 else "bf16+f32")),
        "data": "synthetic (seeded SplitMix64)",
        "config": {"workload": desc, "dags_per_step": n_dags, "nodes": len(w.nodes), "tiles": info.n_tiles,
                   "grid": info.grid,
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "f32_gemm": "SM cores (FFMA)" if args.f32_simt else "tensor cores (3 x TF32 split)",
                   **({"tile_override": args.tile_override} if args.tile_override else {}),
                   "parallelism": f"replicas x{world} (independent DAGs per GPU)" if world > 1 else "1 GPU"},
        "makespan_us": {"median": med, "p10": float(q[0]), "p90": float(q[1]), "mean": statistics.mean(fine_us)},
        "coarse": {"median_us": cmed, "launches_per_step": n_coarse_launches,
                   "speedup_fine_over_coarse": cmed / med},
        "cp_roofline": {"critical_path_us": info.critical_path_us, "work_bound_us": info.work_bound_us,
                        "frac_of_cp": info.critical_path_us / med, "frac_of_work_bound": info.work_bound_us / med},
        "roofline": roof,
        "e2e": {"value": world * n_dags / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(xbytes),
                "d2h_bytes_per_step": int(ybytes), "ms_per_step": e2e_s * 1e3,
                "launches_per_step": len(e2e_parts)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if alg1:
        alg1["speedup_persistent_over_best"] = alg1["best_us"] / med
        line["paper_alg1"] = alg1
    if unfused:
        line["epilogue_fusion"] = unfused
    if batched and not args.no_learned:
        def timed_fn(dd, n):
            out = []
            for _ in range(n):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                dd.submit(sp)
                b.record(stream)
                abi.check(dd.wait(), "wait")
                out.append(a.elapsed_time(b) * 1e3)
            return out
        line["learned"] = learned_eval_batched(wl, ins, abi, Dag, options, timed_fn)
    if batched and world == 1 and not args.no_configs:
        line["configs"] = config_extras(args, abi, Dag, options, stream, flush, peaks, peaks_src)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(args.workload)
        if args.workload.startswith("mlp") or args.workload in UNIT_SAMPLES or batched:
            try:
                line["cpu_baseline_all_cores"] = oracle_all_cores(args.workload)
            except Exception as e:  # a host-side extra: never costs the measured line
                line["cpu_baseline_all_cores"] = {"unavailable": str(e)[:200]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
