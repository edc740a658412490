"""Learned and measured per-kernel costs for the ready-queue ranks.

The executor orders its queue by bottom-level rank (paper §5, clustering: the
priority queue F ordered by the bottom-level rank of each component's FRONT
kernels; HEFT takes the kernel times from profiling).  A rank needs a time
per kernel.  Three sources:

  * the planner's roofline model (DAG_SCHED_RANK_MODEL, the default);
  * a measured profile: per-kernel tile times recorded by the executor's own
    trace on an earlier run of the same DAG (profile_costs);
  * the learned model: a 3-layer MLP (64 hidden; dag_mlp_* kernels) that
    predicts a kernel's tile time from its features and so generalises to
    DAGs never run before (CostModel.node_costs).

Per-kernel cost = tile time x waves (tiles / grid, rounded up).  Argument
marshalling and bookkeeping only; forward, backward and Adam run on the GPU.
"""
from __future__ import annotations

import hashlib
import json
import math
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import _binding as abi
from .dag import Dag, describe, options

N_FEATURES = 12
# per-SM rates of the roofline feature (measured GB300 peaks / 152 SMs): bf16
# tensor, f32 on the tensor cores as 3 x TF32, and HBM bandwidth
_SM_BF16, _SM_F32, _SM_BW = 1.9e12 / 152, 0.31e12 / 152, 6.7e12 / 152
STAMP_READY, STAMP_END = 1, 9


def _depths(w) -> List[int]:
    writer = {}
    for v, n in enumerate(w.nodes):
        b = w.buffers[n.out]
        writer.setdefault(n.out if b.view_of < 0 else b.view_of, []).append(v)
    d = [0] * len(w.nodes)
    for v, n in enumerate(w.nodes):  # nodes of these workloads are listed in topological order
        for bid in (n.a, n.b, n.bias):
            if bid < 0:
                continue
            b = w.buffers[bid]
            for u in writer.get(bid if b.view_of < 0 else b.view_of, []):
                if u < v:
                    d[v] = max(d[v], d[u] + 1)
    return d


def features(w, tiles: np.ndarray, grid: int) -> np.ndarray:
    """(n_nodes, 12) features: op kind one-hot (bf16 GEMM, f32 GEMM, add,
    activation, softmax), log2 of M, N, K+1, tile area, tile count, of
    1 + (tiles at the kernel's depth level) / grid, and of a tile's roofline
    time on one SM (max of its flops over the SM's share of the tensor peak
    and its bytes over its share of HBM bandwidth, in us): the network then
    learns a correction to the roofline, which carries over to sizes it was
    not trained on."""
    nn = len(w.nodes)
    count = np.bincount(tiles[:, 0], minlength=nn)
    area = np.zeros(nn)
    trows = np.zeros(nn)
    tcols = np.zeros(nn)
    for r in tiles:
        if area[r[0]] == 0:
            area[r[0]] = (r[2] - r[1]) * (r[4] - r[3])
            trows[r[0]], tcols[r[0]] = r[2] - r[1], r[4] - r[3]
    dep = _depths(w)
    level = {}
    for v in range(nn):
        level[dep[v]] = level.get(dep[v], 0) + count[v]
    F = np.zeros((nn, N_FEATURES), np.float32)
    for v, n in enumerate(w.nodes):
        out = w.buffers[n.out]
        if n.op == "gemm":
            kind = 0 if w.buffers[n.a].dtype == "bf16" else 1
            A = w.buffers[n.a]
            M, K = A.rows // n.batch, A.cols
            N = out.cols
        else:
            kind = {"add": 2, "unary": 3, "softmax": 4}[n.op]
            M, N, K = out.rows, out.cols, 0
        F[v, kind] = 1.0
        F[v, 5] = math.log2(M)
        F[v, 6] = math.log2(N)
        F[v, 7] = math.log2(K + 1)
        F[v, 8] = math.log2(max(1.0, area[v]))
        F[v, 9] = math.log2(max(1, count[v]))
        F[v, 10] = math.log2(1.0 + level[dep[v]] / grid)
        a = max(1.0, area[v])
        if n.op == "gemm":
            es = 2 if w.buffers[n.a].dtype == "bf16" else 4
            t_flop = 2.0 * a * K / (_SM_BF16 if es == 2 else _SM_F32)
            t_byte = ((trows[v] + tcols[v]) * K * es + a * 4) / _SM_BW
        else:
            t_flop, t_byte = 0.0, a * 3 * 4 / _SM_BW
        F[v, 11] = math.log2(max(t_flop, t_byte) * 1e6 + 1e-3)
    return F


def measure(w, inputs, runs: int = 2, opts=None):
    """Run w with tracing; returns (features, median tile time per kernel in
    microseconds, tile counts, grid, makespan of the last run in
    microseconds)."""
    o = opts or options()
    o.trace = 1
    d = Dag(w, o, resident_inputs=True)
    try:
        d.set_inputs(inputs)
        for _ in range(runs):
            d.run()
        st = abi.dag_trace_stamps(d.h).astype(np.int64)
        tiles = d.tiles()
        grid = d.plan().grid
    finally:
        d.close()
    nn = len(w.nodes)
    dur = (st[:, STAMP_END] - st[:, STAMP_READY]) / 1e3
    per = [[] for _ in range(nn)]
    for t, v in enumerate(tiles[:, 0]):
        per[v].append(dur[t])
    med = np.array([np.median(x) if x else 0.0 for x in per])
    span = (st[:, STAMP_END].max() - st[st[:, 0] > 0, 0].min()) / 1e3
    return features(w, tiles, grid), med, np.bincount(tiles[:, 0], minlength=nn), grid, span


def model_tile_us(w) -> np.ndarray:
    """The planner's roofline time model, per kernel, as a tile time (its
    kernel cost divided by the kernel's waves)."""
    d = Dag(w, options(), resident_inputs=True)
    try:
        costs = abi.dag_node_costs_get(d.h).astype(np.float64)
        tiles = d.tiles()
        grid = d.plan().grid
    finally:
        d.close()
    counts = np.bincount(tiles[:, 0], minlength=len(w.nodes))
    return costs / np.ceil(np.maximum(counts, 1) / grid)


def node_costs_from_tile_times(tile_us: Sequence[float], counts: Sequence[int], grid: int) -> List[float]:
    """Tile time x waves; 0 for a kernel with no tiles of its own (computed in
    the epilogue of the GEMM it is fused into)."""
    return [float(t) * math.ceil(c / grid) if c else 0.0 for t, c in zip(tile_us, counts)]


def profile_costs(w, inputs, opts=None) -> List[float]:
    """Measured-profile costs: tile times recorded on a run of this DAG."""
    _, med, counts, grid, _ = measure(w, inputs, runs=2, opts=opts)
    return node_costs_from_tile_times(med, counts, grid)


class CostModel:
    """The learned cost model (dag_mlp_*): log tile time from features."""

    def __init__(self, seed: int = 11):
        import synth
        self.h = abi.dag_mlp_create(N_FEATURES)
        n = abi.dag_mlp_param_count(self.h)
        # fan-in-scaled uniform initialisation from the seeded generator
        p = np.zeros(n, np.float32)
        o = 0
        for fan_in, size in ((N_FEATURES, N_FEATURES * 64), (0, 64), (64, 64 * 64), (0, 64), (64, 64), (0, 1)):
            if fan_in:
                p[o:o + size] = synth.uniform(seed + o, (size,)) / math.sqrt(fan_in)
            o += size
        self.init_params = p
        abi.dag_mlp_set_params(self.h, p)
        self.mu = np.zeros(N_FEATURES, np.float32)
        self.sd = np.ones(N_FEATURES, np.float32)

    def _norm(self, F):
        return (np.asarray(F, np.float32) - self.mu) / self.sd

    def fit(self, F: np.ndarray, tile_us: np.ndarray, steps: int = 3000, batch: int = 256, lr: float = 2e-3,
            seed: int = 5):
        import synth
        keep = tile_us > 0
        F, y = np.asarray(F, np.float32)[keep], np.log(tile_us[keep]).astype(np.float32)
        self.mu = F.mean(0)
        self.sd = np.maximum(F.std(0), 1e-3).astype(np.float32)
        order = np.argsort(synth.splitmix64(seed, len(y)))  # a seeded shuffle of the samples
        abi.dag_mlp_train(self.h, self._norm(F[order]), y[order], steps, batch, lr)
        return self

    def predict_tile_us(self, F: np.ndarray) -> np.ndarray:
        return np.exp(abi.dag_mlp_predict(self.h, self._norm(F)).astype(np.float64))

    def node_costs(self, w, n_sm: int = 152) -> List[float]:
        """Predicted per-kernel costs for a DAG, from its host plan."""
        nodes, edges, bufs = describe(w, resident_inputs=True)
        tiles, info = abi.dag_plan_host(nodes, edges, bufs, None, n_sm)
        F = features(w, tiles, info.grid)
        counts = np.bincount(tiles[:, 0], minlength=len(w.nodes))
        return node_costs_from_tile_times(self.predict_tile_us(F), counts, info.grid)

    # -- checkpoints -------------------------------------------------------
    def save(self, path: str, device: Optional[Dict] = None) -> None:
        """Weights, feature normalisation and the device they were trained on
        (tile times are only meaningful on the GPU and clocks they came from)."""
        meta = {"format": CHECKPOINT_FORMAT, "n_features": N_FEATURES, "hidden": 64,
                "device": device if device is not None else device_info()}
        with open(path, "wb") as f:
            np.savez(f, params=abi.dag_mlp_get_params(self.h), mu=self.mu, sd=self.sd,
                     meta=np.frombuffer(json.dumps(meta).encode(), np.uint8))

    @classmethod
    def load(cls, path: str, device: Optional[Dict] = None, any_device: bool = False) -> "CostModel":
        """A model saved by save(); refuses one trained on another GPU model or
        SM count unless any_device (clocks are recorded, not compared: they
        vary from run to run)."""
        with np.load(path) as z:
            meta = json.loads(z["meta"].tobytes().decode())
            params, mu, sd = z["params"], z["mu"], z["sd"]
        if meta.get("format") != CHECKPOINT_FORMAT or meta.get("n_features") != N_FEATURES:
            raise ValueError(f"{path}: not a cost-model checkpoint of this version")
        if not any_device:
            check_same_device(meta.get("device", {}), device if device is not None else device_info(), path)
        m = cls()
        if params.size != abi.dag_mlp_param_count(m.h):
            m.close()
            raise ValueError(f"{path}: {params.size} parameters, the network has {abi.dag_mlp_param_count(m.h)}")
        abi.dag_mlp_set_params(m.h, params)
        m.mu, m.sd = mu.astype(np.float32), sd.astype(np.float32)
        return m

    def close(self):
        if self.h:
            abi.dag_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CHECKPOINT_FORMAT = 1


def device_info(ordinal: int = 0) -> Dict:
    """What a recorded time depends on: the GPU model, its SM count and its
    maximum SM clock (from nvidia-smi, if it answers)."""
    info = {"gpu": "none", "sms": 0, "sm_max_mhz": None}
    try:
        import torch
        if torch.cuda.is_available():
            pr = torch.cuda.get_device_properties(ordinal)
            info["gpu"], info["sms"] = pr.name, int(pr.multi_processor_count)
    except Exception:
        pass
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(ordinal), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
        if out.returncode == 0 and out.stdout.strip():
            info["sm_max_mhz"] = float(out.stdout.strip().splitlines()[0])
    except Exception:
        pass
    return info


def check_same_device(saved: Dict, current: Dict, what: str) -> None:
    if saved.get("gpu") != current.get("gpu") or saved.get("sms") != current.get("sms"):
        raise ValueError(f"{what}: recorded on {saved.get('gpu')} ({saved.get('sms')} SMs), "
                         f"this is {current.get('gpu')} ({current.get('sms')} SMs)")


def dag_signature(w) -> str:
    """A DAG's identity for a profile: every buffer's shape, dtype, role and
    view, and every kernel's operation, operands and attributes."""
    h = hashlib.sha256()
    for b in w.buffers:
        h.update(repr((b.rows, b.cols, b.dtype, b.role, b.view_of, b.col_offset)).encode())
    for n in w.nodes:
        h.update(repr((n.op, n.a, n.b, n.bias, n.out, n.trans_b, n.act, float(n.scale), n.batch)).encode())
    return h.hexdigest()[:32]


class ProfileDB:
    """Measured per-kernel costs (profile_costs) of DAGs, by signature, saved
    to and loaded from a JSON file that records the device they came from."""

    def __init__(self, device: Optional[Dict] = None):
        self.device = device if device is not None else device_info()
        self.costs: Dict[str, List[float]] = {}

    def record(self, w, costs: Sequence[float]) -> None:
        if len(costs) != len(w.nodes):
            raise ValueError(f"{len(costs)} costs for {len(w.nodes)} kernels")
        self.costs[dag_signature(w)] = [float(c) for c in costs]

    def get(self, w) -> Optional[List[float]]:
        return self.costs.get(dag_signature(w))

    def save(self, path: str) -> None:
        with open(path, "w") as f:
            json.dump({"format": CHECKPOINT_FORMAT, "device": self.device, "costs": self.costs}, f)

    @classmethod
    def load(cls, path: str, device: Optional[Dict] = None, any_device: bool = False) -> "ProfileDB":
        with open(path) as f:
            d = json.load(f)
        if d.get("format") != CHECKPOINT_FORMAT:
            raise ValueError(f"{path}: not a profile database of this version")
        cur = device if device is not None else device_info()
        if not any_device:
            check_same_device(d.get("device", {}), cur, path)
        db = cls(d.get("device", cur))
        db.costs = {k: [float(c) for c in v] for k, v in d.get("costs", {}).items()}
        return db


def mape(pred: np.ndarray, true: np.ndarray) -> float:
    m = true > 0
    return float(np.mean(np.abs(pred[m] - true[m]) / true[m]))
