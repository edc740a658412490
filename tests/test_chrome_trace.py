"""Chrome trace-event export of an executor trace (host only, fake records)."""
import json
import types

from paper_2009_07482_gb300.trace import chrome_trace, write_chrome_trace


def _rec(node, sm, claim, start, work, end, r=(0, 128), c=(0, 256), tickets=(0, 1)):
    return types.SimpleNamespace(node=node, r0=r[0], r1=r[1], c0=c[0], c1=c[1], smid=sm, split=0,
                                 start_ticket=tickets[0], end_ticket=tickets[1], t_claim_ns=claim,
                                 t_start_ns=start, t_work_ns=work, t_end_ns=end)


def test_rows_per_sm_times_and_no_overlap(tmp_path):
    base = 5_000_000_000
    recs = [
        _rec(0, 3, base + 0, base + 500, base + 600, base + 10_000),
        # SM 3's next tile: claimed while the first still runs; its work starts
        # before the first one's release (the releaser warp runs alongside)
        _rec(1, 3, base + 2_000, base + 9_000, base + 9_500, base + 15_000, tickets=(2, 3)),
        _rec(1, 7, base + 100, base + 9_100, base + 9_200, base + 14_000, tickets=(4, 5)),
        _rec(2, 7, 0, 0, 0, 0),          # a record that never ran (no claim): skipped
    ]
    tr = chrome_trace(recs, names=["fc0", "fc1", "add"])
    ev = [e for e in tr["traceEvents"] if e["ph"] == "X"]
    meta = [e for e in tr["traceEvents"] if e["ph"] == "M"]
    assert {(e["pid"], e["args"]["name"]) for e in meta if e["name"] == "process_name"} == {(3, "SM 3"), (7, "SM 7")}
    assert len(ev) == 6
    sm3_tile = sorted((e for e in ev if e["pid"] == 3 and e["tid"] == 1), key=lambda e: e["ts"])
    assert [e["name"] for e in sm3_tile] == ["fc0", "fc1"]
    assert sm3_tile[0]["ts"] == 0.6 and sm3_tile[0]["dur"] == 8.9        # cut at the next tile's start (9.5 us)
    assert sm3_tile[0]["args"]["release_us"] == 10.0                     # the uncut release time is kept
    assert sm3_tile[1]["ts"] == 9.5 and sm3_tile[1]["dur"] == 5.5
    waits = sorted((e for e in ev if e["tid"] == 0), key=lambda e: (e["pid"], e["ts"]))
    assert [(e["pid"], e["name"], e["ts"], e["dur"]) for e in waits] == [
        (3, "wait fc0", 0.0, 0.5), (3, "wait fc1", 2.0, 7.0), (7, "wait fc1", 0.1, 9.0)]
    for row in {(e["pid"], e["tid"]) for e in ev}:          # no two events of a row overlap
        es = sorted((e for e in ev if (e["pid"], e["tid"]) == row), key=lambda e: e["ts"])
        assert all(a["ts"] + a["dur"] <= b["ts"] + 1e-9 for a, b in zip(es, es[1:]))
    p = tmp_path / "t.json"
    write_chrome_trace(str(p), recs, ["fc0", "fc1", "add"])
    assert json.loads(p.read_text()) == json.loads(json.dumps(tr))


def test_empty_trace():
    assert chrome_trace([])["traceEvents"] == []


def test_kernel_windows_pack_into_non_overlapping_lanes():
    from paper_2009_07482_gb300.trace import kernel_windows_trace
    # component 0: k0 [0,10) and k1 [2,6) overlap -> two lanes; k2 [6,9) reuses lane 1;
    # component 1: k3 [10,20); k4 has no window (fused into another kernel) and is skipped
    start = [0.0, 2.0, 6.0, 10.0, 5.0]
    end = [10.0, 6.0, 9.0, 20.0, 5.0]
    tr = kernel_windows_trace(start, end, ["k0", "k1", "k2", "k3", "k4"], groups=[0, 0, 0, 1, 1])
    ev = {e["name"]: e for e in tr["traceEvents"] if e["ph"] == "X"}
    assert set(ev) == {"k0", "k1", "k2", "k3"}
    assert [(ev[k]["pid"], ev[k]["tid"], ev[k]["ts"], ev[k]["dur"]) for k in ("k0", "k1", "k2", "k3")] == [
        (0, 0, 0.0, 10.0), (0, 1, 2.0, 4.0), (0, 1, 6.0, 3.0), (1, 0, 10.0, 10.0)]
    lanes = [e for e in tr["traceEvents"] if e["ph"] == "M" and e["name"] == "thread_name"]
    assert sorted((e["pid"], e["tid"]) for e in lanes) == [(0, 0), (0, 1), (1, 0)]
