"""bench.py --timeline: the per-kernel windows and phase medians computed from
trace stamps (host arithmetic only; the records are fakes with known times)."""
import types

import numpy as np

import bench
from synth.workloads import fork_join


class _FakeDag:
    def __init__(self, stamps, nodes):
        self.h = None
        self._stamps = stamps
        self._nodes = nodes

    def submit(self, stream):
        pass

    def wait(self):
        return 0

    def trace(self):
        return [types.SimpleNamespace(node=v) for v in self._nodes]


def test_timeline_windows_and_phases():
    w = fork_join(8)                       # kernels 0..3
    # kernel 0: two GEMM-like tiles stamped at every phase; kernel 3: one
    # elementwise tile (no load / MMA / accumulator stamps)
    base = 1_000_000
    g0 = [0, 500, 900, 1000, 3000, 1200, 3500, 4500, 4700, 6000]
    g1 = [100, 700, 1100, 1200, 3300, 1300, 3600, 4800, 5000, 6500]
    e3 = [6600, 7000, 0, 0, 0, 7100, 0, 8100, 8200, 9000]
    stamps = np.array([g0, g1, e3], dtype=np.int64) + base
    stamps[2, [2, 3, 4, 6]] = 0            # phases an elementwise tile does not stamp
    # the launch: entered 2 us before the first claim, left 1.5 us after the last release
    fake_abi = types.SimpleNamespace(check=lambda st, what: None,
                                     dag_trace_stamps=lambda h: stamps.astype(np.uint64),
                                     dag_trace_launch=lambda h: (base - 2000, base + 9000 + 1500))
    flush = types.SimpleNamespace(zero_=lambda: None)
    stream = types.SimpleNamespace(cuda_stream=0)
    d = _FakeDag(stamps, [0, 0, 3])
    out = bench.run_timeline(None, w, d, fake_abi, stream, flush, reps=3)
    assert out["traced_launch_us_median"] == 9.0
    assert out["launch_window_us_median"] == {"entry_to_first_claim": 2.0, "last_release_to_exit": 1.5,
                                              "entry_to_exit": 12.5}
    k = {x["kernel"]: x for x in out["kernels"]}
    assert set(k) == {0, 3}
    assert (k[0]["tiles"], k[0]["first_claim_us"], k[0]["first_ready_us"], k[0]["last_release_us"]) == (2, 0.0, 0.5, 6.5)
    ph = k[0]["phase_median_us"]
    assert ph["claim->ready"] == 0.55 and ph["mma0->mma1"] == 2.05 and ph["sync->end"] == 1.4
    assert list(ph) == ["claim->ready", "ready->loaded", "loaded->mma0", "mma0->mma1", "mma1->work", "work->acc",
                        "acc->body", "body->sync", "sync->end"]
    ph3 = k[3]["phase_median_us"]
    assert list(ph3) == ["claim->ready", "ready->work", "work->body", "body->sync", "sync->end"]
    assert ph3["work->body"] == 1.0 and k[3]["first_claim_us"] == 6.6
