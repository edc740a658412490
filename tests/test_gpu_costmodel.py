"""The learned cost model on the GPU: its forward/backward kernels against the
FP64 oracle (oracle/mlp.py), Adam steps against the oracle's, and what the
trained network buys the scheduler over the untrained network and the
planner's roofline estimates."""
import numpy as np
import pytest

import synth
from oracle import mlp as omlp
from paper_2009_07482_gb300 import _binding as abi
from paper_2009_07482_gb300.costmodel import CostModel, N_FEATURES, mape, measure, model_tile_us
from paper_2009_07482_gb300.dag import Dag, options
from synth.workloads import random_layered
from tests.gpu_util import bits_equal, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2009_07482_gb300 import build
    build.build()
    abi.lib()


def _params(in_dim, seed, scale=0.3):
    return (synth.uniform(seed, (omlp.n_params(in_dim),)) * scale).astype(np.float32)


@pytest.mark.parametrize("n", [1, 63, 64, 200, 1000])
def test_loss_and_gradient_match_the_oracle(n):
    in_dim = N_FEATURES
    p = _params(in_dim, 7)
    X = synth.uniform(8, (n, in_dim)).astype(np.float32)
    y = synth.uniform(9, (n,)).astype(np.float32)
    m = abi.dag_mlp_create(in_dim)
    abi.dag_mlp_set_params(m, p)
    loss, g = abi.dag_mlp_loss_grad(m, X, y)
    pred = abi.dag_mlp_predict(m, X)
    abi.dag_mlp_destroy(m)
    ref_loss, ref_g = omlp.loss_grad(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64), in_dim)
    ref_out, _ = omlp.forward(p.astype(np.float64), X.astype(np.float64), in_dim)
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, ref_loss)
    assert np.max(np.abs(g - ref_g)) <= 1e-5 * max(1.0, np.max(np.abs(ref_g)))
    assert np.max(np.abs(pred - ref_out)) <= 1e-5 * max(1.0, np.max(np.abs(ref_out)))


def test_adam_steps_match_the_oracle():
    in_dim, n = 9, 300
    p = _params(in_dim, 17)
    X = synth.uniform(18, (n, in_dim)).astype(np.float32)
    y = (np.sin(X.sum(1)) * 0.5).astype(np.float32)
    m = abi.dag_mlp_create(in_dim)
    abi.dag_mlp_set_params(m, p)
    abi.dag_mlp_train(m, X, y, steps=20, batch=64, lr=1e-3)
    got = abi.dag_mlp_get_params(m)
    abi.dag_mlp_destroy(m)
    ref = omlp.adam_train(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64), in_dim, 20, 64, 1e-3)
    # 20 steps of at most lr each: f32 rounding stays far below one step
    assert np.max(np.abs(got - ref)) <= 2e-5


def test_learned_costs_beat_untrained_and_roofline_estimates():
    """Trained on tile times the executor recorded for one set of random DAGs,
    the network predicts the tile times of other DAGs better than its untrained
    self and than the planner's roofline time model; scheduling with its ranks
    changes no output bit."""
    train, test = [], []
    for i in range(24):
        w = random_layered(5000 + i, 8, 24, 4, sizes=(64, 128, 256, 512, 1024))
        F, t, *_ = measure(w, w.make_inputs())
        train.append((F, t))
    for i in range(6):
        w = random_layered(6000 + i, 8, 24, 4, sizes=(64, 128, 256, 512, 1024))
        ins = w.make_inputs()
        F, t, counts, grid, _ = measure(w, ins)
        test.append((w, ins, F, t, counts, grid))
    F = np.concatenate([f for f, _ in train])
    T = np.concatenate([t for _, t in train])
    Ft = np.concatenate([x[2] for x in test])
    Tt = np.concatenate([x[3] for x in test])
    cm = CostModel()
    err_untrained = mape(cm.predict_tile_us(Ft), Tt)
    cm.fit(F, T)
    err_trained = mape(cm.predict_tile_us(Ft), Tt)
    err_roof = mape(np.concatenate([model_tile_us(x[0]) for x in test]), Tt)
    assert err_trained < 0.5 * err_untrained, (err_trained, err_untrained)
    assert err_trained < err_roof, (err_trained, err_roof)
    # ranks from the model reorder the queue, never the results
    w, ins = test[0][0], test[0][1]
    base = run_gpu(w, ins)
    costs = cm.node_costs(w)
    assert bits_equal(base, run_gpu(w, ins, opts=options(scheduler=abi.DAG_SCHED_RANK_GIVEN, node_cost_us=costs)))
    cm.close()


def _training_traces():
    """Tile times the executor recorded on random DAGs alone (sizes 64..4096)
    and in batches of 2..32 (so the concurrency feature covers batched plans)."""
    from synth.workloads import concat, random_batch
    F, T = [], []
    for i in range(16):
        w = random_layered(5000 + i, 8, 24, 4, sizes=(64, 128, 256, 512, 1024, 2048, 4096))
        f, t, *_ = measure(w, w.make_inputs())
        F.append(f)
        T.append(t)
    seed = 7000
    for k in (2, 8, 32):
        w = concat(random_batch(k, base_seed=seed))
        seed += k
        f, t, *_ = measure(w, w.make_inputs())
        F.append(f)
        T.append(t)
    return np.concatenate(F), np.concatenate(T)


def test_learned_costs_put_a_latency_bound_chain_first_and_shorten_the_makespan():
    """What the trained network gains over the planner's roofline model: on a
    DAG whose critical path is a chain of 48 small GEMMs (latency-bound: the
    roofline model prices each at a fraction of its measured time) beside four
    4096^3 GEMMs, the learned costs -- like the measured profile, and unlike
    the roofline model -- make the chain the most expensive path, and with the
    critical-path priority the executor then runs the chain alongside the
    filler instead of after it.  Medians of 9 runs; the gain must exceed the
    runs' spread several times over."""
    import statistics

    import torch
    from paper_2009_07482_gb300.costmodel import profile_costs
    from synth.workloads import chain_and_fill
    F, T = _training_traces()
    cm = CostModel().fit(F, T)
    w = chain_and_fill()
    ins = w.make_inputs()
    chain = [k for k, n in enumerate(w.nodes) if n.name.startswith("chain")]
    fill = [k for k, n in enumerate(w.nodes) if n.name.startswith("fill")]
    learned = cm.node_costs(w)
    cm.close()
    prof = profile_costs(w, ins)
    d = Dag(w, options(), resident_inputs=True)
    roof = abi.dag_node_costs_get(d.h).astype(float).tolist()
    d.close()
    path = lambda c: sum(c[k] for k in chain)
    assert path(prof) > max(prof[k] for k in fill)        # measured: the chain is the longest path
    assert path(learned) > max(learned[k] for k in fill)  # learned: the same
    assert path(roof) < max(roof[k] for k in fill)        # roofline: the filler looks longer

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def makespans(costs):
        o = options(rank_form=abi.DAG_RANK_CRITICAL_PATH)
        if costs is not None:
            o = options(rank_form=abi.DAG_RANK_CRITICAL_PATH, scheduler=abi.DAG_SCHED_RANK_GIVEN, node_cost_us=costs)
        dd = Dag(w, o, resident_inputs=True)
        dd.set_inputs(ins)
        out = []
        for i in range(12):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dd.submit(stream.cuda_stream)
            b.record(stream)
            abi.check(dd.wait(), "wait")
            if i >= 3:
                out.append(a.elapsed_time(b) * 1e3)
        dd.close()
        return out

    t_roof, t_learn, t_prof = makespans(None), makespans(learned), makespans(prof)
    spread = max(max(x) - min(x) for x in (t_roof, t_learn, t_prof))
    gain = statistics.median(t_roof) - statistics.median(t_learn)
    assert gain > 4 * spread, (statistics.median(t_roof), statistics.median(t_learn), spread)
    assert statistics.median(t_learn) < 0.85 * statistics.median(t_roof)
    # the learned ranks come within 10 % of the measured profile's
    assert statistics.median(t_learn) < 1.1 * statistics.median(t_prof)
