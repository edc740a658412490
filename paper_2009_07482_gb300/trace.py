"""Chrome trace-event export of an executor launch (a Gantt chart per SM).

The paper reads its schedules off Gantt charts of OpenCL command timings
(write / ndrange / read per queue, §2 and §5).  Here the unit of work is a
tile, and the executor's trace (dag_trace_get, with dag_options.trace = 1)
records for each tile the SM it ran on and four %globaltimer times: the claim
of its queue position, the end of its dependency waits, the moment the worker
warps picked it up, and its release.  This module turns those records into
the trace-event JSON that chrome://tracing and Perfetto open: one process per
SM with two rows,

  dispatch   claim -> dependencies met (the scheduler warp waiting on counters)
  tile       workers start -> release (epilogue / body, release included)

Events of one row never overlap: a tile's bar is cut where the next tile of
the same row begins (the uncut times stay in the event's args).

kernel_windows_trace does the same for whole-kernel windows, such as those
of the paper's own Alg. 1 on CUDA streams.
"""
from __future__ import annotations

import json
from typing import Dict, List, Optional, Sequence


def chrome_trace(records: Sequence, names: Optional[Sequence[str]] = None) -> Dict:
    """Trace-event JSON (a dict) from dag_trace_record-like objects (fields
    node, r0, r1, c0, c1, smid, split, start_ticket, end_ticket, t_claim_ns,
    t_start_ns, t_work_ns, t_end_ns).  `names[node]` labels the events
    (default "kernel <node>").  Times are microseconds from the earliest claim."""
    recs = [r for r in records if r.t_claim_ns]
    if not recs:
        return {"traceEvents": [], "displayTimeUnit": "ns"}
    t0 = min(r.t_claim_ns for r in recs)

    def us(t):
        return (t - t0) / 1e3

    def label(r):
        return names[r.node] if names is not None and r.node < len(names) else f"kernel {r.node}"

    rows: Dict[tuple, List[dict]] = {}
    for r in recs:
        args = {"node": int(r.node), "rows": [int(r.r0), int(r.r1)], "cols": [int(r.c0), int(r.c1)],
                "tickets": [int(r.start_ticket), int(r.end_ticket)], "split": int(r.split)}
        if r.t_start_ns >= r.t_claim_ns:
            rows.setdefault((int(r.smid), 0), []).append(
                {"name": f"wait {label(r)}", "ts": us(r.t_claim_ns), "end": us(r.t_start_ns), "args": args})
        work = r.t_work_ns if r.t_work_ns else r.t_start_ns
        if r.t_end_ns >= work:
            rows.setdefault((int(r.smid), 1), []).append(
                {"name": label(r), "ts": us(work), "end": us(r.t_end_ns),
                 "args": dict(args, work_us=us(work), release_us=us(r.t_end_ns))})
    events = []
    for (sm, row), evs in sorted(rows.items()):
        evs.sort(key=lambda e: e["ts"])
        for i, e in enumerate(evs):
            end = e["end"] if i + 1 == len(evs) else min(e["end"], evs[i + 1]["ts"])
            events.append({"name": e["name"], "ph": "X", "pid": sm, "tid": row, "ts": e["ts"],
                           "dur": max(end - e["ts"], 0.0), "args": e["args"]})
    for sm in sorted({sm for sm, _ in rows}):
        events.append({"name": "process_name", "ph": "M", "pid": sm, "args": {"name": f"SM {sm}"}})
        events.append({"name": "thread_name", "ph": "M", "pid": sm, "tid": 0, "args": {"name": "dispatch"}})
        events.append({"name": "thread_name", "ph": "M", "pid": sm, "tid": 1, "args": {"name": "tile"}})
    return {"traceEvents": events, "displayTimeUnit": "ns"}


def write_chrome_trace(path: str, records: Sequence, names: Optional[Sequence[str]] = None) -> None:
    with open(path, "w") as f:
        json.dump(chrome_trace(records, names), f)


def kernel_windows_trace(start_us: Sequence[float], end_us: Sequence[float], names: Sequence[str],
                         groups: Optional[Sequence[int]] = None, group_label: str = "component") -> Dict:
    """Trace-event JSON of whole-kernel windows, as the paper's Gantt charts of
    its schedules (§5): e.g. the [start, end) of each kernel under the paper's
    Alg. 1 on streams (dag_submit_cq with per-kernel times).  One process per
    group (task component); inside it, kernels are packed in start order onto
    the first lane free at their start, so a lane never holds two kernels at
    once and the lanes show the concurrency the queues achieved.  Kernels
    without a window (end <= start, e.g. fused into another) are skipped."""
    n = len(names)
    groups = list(groups) if groups is not None else [0] * n
    lanes: Dict[int, List[float]] = {}            # group -> end time of each lane
    events = []
    for v in sorted(range(n), key=lambda v: (float(start_us[v]), v)):
        s, e = float(start_us[v]), float(end_us[v])
        if not e > s:
            continue
        g = int(groups[v])
        ends = lanes.setdefault(g, [])
        lane = next((i for i, t in enumerate(ends) if t <= s), len(ends))
        if lane == len(ends):
            ends.append(e)
        else:
            ends[lane] = e
        events.append({"name": names[v], "ph": "X", "pid": g, "tid": lane, "ts": s, "dur": e - s,
                       "args": {"kernel": v}})
    for g in sorted(lanes):
        events.append({"name": "process_name", "ph": "M", "pid": g, "args": {"name": f"{group_label} {g}"}})
        for i in range(len(lanes[g])):
            events.append({"name": "thread_name", "ph": "M", "pid": g, "tid": i, "args": {"name": f"lane {i}"}})
    return {"traceEvents": events, "displayTimeUnit": "ns"}
