"""bench.py's all-cores oracle baseline: spawned processes, each timing the
oracle on its own batch rows at the same moment (CPU only, two processes);
and the end-to-end path's split of the batch into back-to-back launches."""
import pytest

import bench


def test_all_cores_baseline_runs_and_reports_its_processes():
    r = bench.oracle_all_cores("mlp_bf16", ra=1, rb=2, procs=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["unit"] == bench.UNIT
    assert 0 < r["value"] < 100          # DAGs/s of a float64 CPU executor on 512 rows
    assert "2 processes" in r["sample"] and "share of 256 rows" in r["sample"]


def test_a_failing_worker_is_reported_not_waited_for():
    import time

    import pytest

    t0 = time.time()
    with pytest.raises(RuntimeError, match="failed or ran too long"):
        bench.oracle_all_cores("mlp_bf16", ra=0, rb=1, procs=2)    # a 0-row DAG: the oracle rejects it
    assert time.time() - t0 < 120


def test_all_cores_baseline_of_independent_parts():
    # the softmax level: one head of 16 per process; two processes take 8 heads each
    r = bench.oracle_all_cores("softmax", procs=2)
    assert r["cores"] == 2 and r["value"] > 0
    assert "2 processes" in r["sample"] and "one DAG = 8 x the median" in r["sample"]
    # never more processes than parts: the encoder's 8 sequences
    assert bench.unit_sample("encoder")[1] == 8


def test_all_cores_baseline_of_the_batch():
    r = bench.oracle_all_cores("batched", procs=2)
    assert r["cores"] == 2 and r["value"] > 0
    assert "/ 2 processes" in r["sample"] and "rows of each of 32 DAGs" in r["sample"]


def test_reference_arm_times_whole_units():
    """The reference arm's rate is the DAG fraction of the units it ran over
    the time it spent: a step is whole units (here: rows of 8 DAGs of the
    batch), and the batch's sample covers every DAG over 32 steps."""
    units, f, what = bench.reference_units("batched", 0)
    assert len(units) == 8 and 0 < f < 1 and "8 DAGs" in what
    u2, f2, _ = bench.reference_units("batched", 32)
    assert f2 == f                       # step 32 wraps to DAGs 0..7
    units, f, _ = bench.reference_units("encoder", 0)
    assert f == 1 / 8 and len(units) == 1


@pytest.mark.parametrize("n_dags,n", [(256, 8), (13, 4), (3, 8)])
def test_end_to_end_chunks_cover_the_batch_once(n_dags, n):
    """The end-to-end path's shares of the batch: consecutive, every DAG in
    one share, and each share's buffer ids those of concat(share) shifted
    from concat(batch) -- so inputs, streamed activations and sinks land on
    the handle that owns them."""
    from synth.workloads import concat, random_batch
    wl = random_batch(n_dags)
    chunks = bench.e2e_chunks(wl, n)
    assert len(chunks) <= n and [x for part, _ in chunks for x in part] == wl
    whole = concat(wl)
    seen = set()
    for part, loc in chunks:
        local = concat(part)
        assert sorted(loc.values()) == list(range(len(local.buffers)))
        for g, l in loc.items():
            assert whole.buffers[g] == local.buffers[l]
        seen |= set(loc)
    assert seen == set(range(len(whole.buffers)))
