"""bench.py's all-cores oracle baseline: spawned processes, each timing the
oracle on its own batch rows at the same moment (CPU only, two processes)."""
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
