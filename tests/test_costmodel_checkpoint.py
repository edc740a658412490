"""Checkpoints of the learned cost model and the measured-profile store
(host logic; the MLP's GPU kernels are replaced by an in-memory fake)."""
import numpy as np
import pytest

from paper_2009_07482_gb300 import costmodel as cm
from synth.workloads import branchy_mlp, fork_join

GB300 = {"gpu": "NVIDIA GB300", "sms": 152, "sm_max_mhz": 2070.0}
OTHER = {"gpu": "NVIDIA B200", "sms": 148, "sm_max_mhz": 1965.0}


@pytest.fixture
def fake_mlp(monkeypatch):
    n = cm.N_FEATURES * 64 + 64 + 64 * 64 + 64 + 64 + 1
    a = cm.abi
    monkeypatch.setattr(a, "dag_mlp_create", lambda in_dim: {"p": np.zeros(n, np.float32)})
    monkeypatch.setattr(a, "dag_mlp_param_count", lambda h: n)
    monkeypatch.setattr(a, "dag_mlp_set_params", lambda h, p: h.__setitem__("p", np.array(p, np.float32)))
    monkeypatch.setattr(a, "dag_mlp_get_params", lambda h: h["p"].copy())
    monkeypatch.setattr(a, "dag_mlp_predict", lambda h, X: (np.asarray(X, np.float32) @ h["p"][:cm.N_FEATURES]))
    monkeypatch.setattr(a, "dag_mlp_destroy", lambda h: None)
    return n


def test_cost_model_round_trip(fake_mlp, tmp_path):
    m = cm.CostModel()
    p = np.arange(fake_mlp, dtype=np.float32) / fake_mlp
    cm.abi.dag_mlp_set_params(m.h, p)
    m.mu = np.linspace(0, 1, cm.N_FEATURES).astype(np.float32)
    m.sd = np.linspace(1, 2, cm.N_FEATURES).astype(np.float32)
    F = np.random.default_rng(0).random((5, cm.N_FEATURES))
    path = str(tmp_path / "cost.npz")
    m.save(path, device=GB300)
    m2 = cm.CostModel.load(path, device=GB300)
    assert np.array_equal(cm.abi.dag_mlp_get_params(m2.h), p)
    assert np.array_equal(m2.mu, m.mu) and np.array_equal(m2.sd, m.sd)
    assert np.array_equal(m2.predict_tile_us(F), m.predict_tile_us(F))


def test_cost_model_refuses_another_device(fake_mlp, tmp_path):
    m = cm.CostModel()
    path = str(tmp_path / "cost.npz")
    m.save(path, device=GB300)
    with pytest.raises(ValueError, match="B200"):
        cm.CostModel.load(path, device=OTHER)
    cm.CostModel.load(path, device=OTHER, any_device=True)
    # the clock is recorded, not compared
    cm.CostModel.load(path, device=dict(GB300, sm_max_mhz=1500.0))


def test_profile_db_round_trip_and_signatures(tmp_path):
    a, b = fork_join(64), fork_join(128)
    mlp = branchy_mlp("bf16", batch=8, width=64, hidden=128, out=32)
    assert len({cm.dag_signature(x) for x in (a, b, mlp)}) == 3
    assert cm.dag_signature(fork_join(64, seed=9)) == cm.dag_signature(a)   # inputs' values do not matter
    db = cm.ProfileDB(device=GB300)
    db.record(a, [1.0, 2.0, 3.0, 4.0])
    db.record(mlp, list(range(len(mlp.nodes))))
    with pytest.raises(ValueError):
        db.record(b, [1.0])
    path = str(tmp_path / "profile.json")
    db.save(path)
    db2 = cm.ProfileDB.load(path, device=GB300)
    assert db2.get(a) == [1.0, 2.0, 3.0, 4.0] and db2.get(mlp) == [float(i) for i in range(len(mlp.nodes))]
    assert db2.get(b) is None
    with pytest.raises(ValueError):
        cm.ProfileDB.load(path, device=OTHER)
