"""Learned format selector.

The paper picks each intermediate's format with a gray-box cost model (Sec. 5.2,
"Determining a good format combination"), driven by cheap data characteristics:
the number of elements, the bit-width histogram and the sort order.  This module
learns such a model from traces the engine itself produces.

* features (16 fp32) come from the GPU statistics pass ``ms_column_stats``:
  log2 n, the 8-bucket histogram of per-block bit widths, the global, FOR and
  DELTA widths, sortedness, run density, the producing operator and whether a
  consumer reads the column at random;
* labels are, for each of the five formats, log2 bytes per value and log2
  nanoseconds per value of writing the column in that format and reading it
  once.  They are measured by compressing the intermediate into every format:
  the exhaustive try-all-formats choice, which is also the reference the
  selector's regret is measured against;
* the network (16 -> 64 -> 64 -> 10, ReLU, fp32) is trained with the library's
  own forward/backward and Adam kernels (``ms_mlp_*``);
* a plan asks for formats before its intermediates exist: the plan runs once on a
  prefix sample with uncompressed intermediates, and their statistics, scaled to
  the full length, feed the network.

All choices change formats only; every result stays bit-exact.
"""
from __future__ import annotations

import json
import math

import numpy as np
import torch

from . import morphstore as ms

N_FEATURES = 16
N_OUT = 10
OPS = {"base": 0, "select": 1, "project": 2, "calc": 3, "semijoin": 4, "group": 5}
OBJECTIVES = ("size", "time")


# ------------------------------------------------------------------ features

def features_from_stats(stats, op: str = "base", random_reads: bool = False, n_scale: float = 1.0) -> np.ndarray:
    """16 features from the MS_STATS_WORDS statistics of one column."""
    st = np.asarray(stats, dtype=np.uint64).astype(np.float64)
    n = st[0] * n_scale
    chunks = max(st[2], 1.0)
    hist = st[8:8 + 65]
    f = np.zeros(N_FEATURES, dtype=np.float32)
    f[0] = math.log2(n + 1.0) / 32.0
    for b in range(65):  # 8 buckets of 8 bits; width 0 counts with the first
        f[1 + min(max(b - 1, 0) // 8, 7)] += hist[b] / chunks
    f[9] = (int(st[1]).bit_length()) / 64.0
    f[10] = st[3] / chunks / 64.0
    f[11] = st[4] / chunks / 64.0
    pairs = max(st[0] - st[2], 1.0)
    f[12] = st[5] / pairs
    f[13] = math.log2(st[6] + 1.0) / math.log2(st[0] + 2.0)
    f[14] = OPS.get(op, 0) / 8.0
    f[15] = 1.0 if random_reads else 0.0
    return f


def column_features(ctx, col, op="base", random_reads=False, n_scale=1.0) -> np.ndarray:
    stats = ctx.column_stats(col).cpu().numpy().view(np.uint64)
    return features_from_stats(stats, op, random_reads, n_scale)


def static_width(stats) -> int:
    return max(1, int(np.uint64(stats[1])).bit_length())


# -------------------------------------------------------------------- labels

def measure_formats(ctx, d_values: torch.Tensor, stats, reps: int = 2):
    """Exhaustive try-all-formats measurement of one intermediate: its size in
    bytes and its write+read time (compress into the format, then one agg_sum
    pass over it) in nanoseconds, for each of the five formats."""
    n = d_values.numel()
    bw = static_width(stats)
    sizes = np.zeros(5)
    times = np.zeros(5)
    res = torch.empty(1, dtype=torch.int64, device=d_values.device)
    for f in range(5):
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            col = ctx.compress(d_values, f, bw if f == ms.STATIC_BP else 0)
            ctx.agg_sum(col, out=res)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e6)
            sizes[f] = ctx.info(col)["size_bytes"]
            ctx.free(col)
        times[f] = best
    return sizes, times


def labels_from(sizes, times, n) -> np.ndarray:
    n = max(n, 1)
    return np.concatenate([np.log2(np.maximum(sizes, 1.0) / n), np.log2(np.maximum(times, 1.0) / n)]).astype(np.float32)


# ------------------------------------------------------------------- network

class Selector:
    """The MLP with its target standardisation; parameters live on the device."""

    def __init__(self, device, seed: int = 0):
        self.device = device
        rng = np.random.default_rng(seed)
        p = [rng.normal(0, math.sqrt(2.0 / 16), (16, 64)), np.zeros(64), rng.normal(0, math.sqrt(2.0 / 64), (64, 64)),
             np.zeros(64), rng.normal(0, math.sqrt(1.0 / 64), (64, 10)), np.zeros(10)]
        theta = np.concatenate([a.ravel() for a in p]).astype(np.float32)
        self.params = torch.from_numpy(theta).to(device)
        self.mu = np.zeros(N_OUT, dtype=np.float32)
        self.sd = np.ones(N_OUT, dtype=np.float32)
        self.loss_history = []

    def train(self, X: np.ndarray, Y: np.ndarray, M: np.ndarray | None = None, epochs: int = 400,
              lr: float = 3e-3) -> list:
        """Full-batch Adam on the device with the library's kernels."""
        dev = self.device
        if M is None:
            M = np.ones_like(Y)
        self.mu = (Y * M).sum(0) / np.maximum(M.sum(0), 1)
        self.sd = np.sqrt(((Y - self.mu) ** 2 * M).sum(0) / np.maximum(M.sum(0), 1)) + 1e-3
        x = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
        y = torch.from_numpy(np.ascontiguousarray((Y - self.mu) / self.sd, np.float32)).to(dev)
        m = torch.from_numpy(np.ascontiguousarray(M, np.float32)).to(dev)
        inv = 1.0 / max(float(M.sum()), 1.0)
        grad = torch.zeros(ms.MLP_PARAMS, dtype=torch.float32, device=dev)
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        parts = torch.zeros(600 * (ms.MLP_PARAMS + 1), dtype=torch.float32, device=dev)
        mo = torch.zeros_like(self.params)
        ve = torch.zeros_like(self.params)
        hist = []
        for step in range(1, epochs + 1):
            ms.mlp_loss_grad(self.params, x, y, m, inv, grad, loss, parts)
            ms.mlp_adam(self.params, grad, mo, ve, step, lr=lr)
            if step % 20 == 0 or step == 1:
                hist.append((step, float(loss.item())))
        self.loss_history = hist
        return hist

    # --------------------------------------------------------- checkpoint
    def save(self, prefix: str) -> None:
        """Writes the network as <prefix>.bin (MS_MLP_PARAMS little-endian fp32 in the
        packed layout of include/morphstore.h) and <prefix>.json (target scaling,
        loss history)."""
        theta = self.params.detach().to("cpu", torch.float32).numpy().astype("<f4")
        theta.tofile(prefix + ".bin")
        meta = {"params": int(theta.size), "layout": "W1[16][64] b1[64] W2[64][64] b2[64] W3[64][10] b3[10]",
                "mu": [float(v) for v in self.mu], "sd": [float(v) for v in self.sd],
                "loss_history": [[int(a), float(b)] for a, b in self.loss_history]}
        with open(prefix + ".json", "w") as f:
            json.dump(meta, f, indent=1)

    @classmethod
    def load(cls, prefix: str, device) -> "Selector":
        with open(prefix + ".json") as f:
            meta = json.load(f)
        theta = np.fromfile(prefix + ".bin", dtype="<f4")
        if theta.size != ms.MLP_PARAMS or meta.get("params") != ms.MLP_PARAMS:
            raise ValueError("not a selector checkpoint: wrong parameter count")
        sel = cls(device)
        sel.params = torch.from_numpy(theta.astype(np.float32)).to(device)
        sel.mu = np.asarray(meta["mu"], dtype=np.float32)
        sel.sd = np.asarray(meta["sd"], dtype=np.float32)
        sel.loss_history = [tuple(v) for v in meta.get("loss_history", [])]
        return sel

    def predict(self, X: np.ndarray) -> np.ndarray:
        x = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(self.device)
        y = ms.mlp_forward(self.params, x).cpu().numpy()
        return y * self.sd + self.mu

    def choose(self, X: np.ndarray, objective: str = "size", allowed=None) -> np.ndarray:
        """Format with the smallest predicted cost; `allowed` restricts the candidates
        (a plan cannot pick static BP before the intermediate's width is known)."""
        y = self.predict(np.atleast_2d(X))
        cost = (y[:, :5] if objective == "size" else y[:, 5:]).copy()
        if allowed is not None:
            mask = np.ones(5, dtype=bool)
            mask[list(allowed)] = False
            cost[:, mask] = np.inf
        return np.argmin(cost, axis=1)


def regret(chosen: np.ndarray, costs: np.ndarray) -> float:
    """sum cost(chosen) / sum cost(exhaustive best) - 1 over a set of intermediates."""
    costs = np.asarray(costs, dtype=np.float64)
    picked = costs[np.arange(len(chosen)), chosen].sum()
    return float(picked / costs.min(axis=1).sum() - 1.0)


# ------------------------------------------------------------- trace harvest

def synthetic_intermediates(seed: int, count: int, lo_log2: int = 16, hi_log2: int = 22):
    """Columns with the shapes the engine's plans produce: skewed per-block widths,
    sorted keys and position lists at several selectivities, products of the two,
    Table 1 shapes, run-length-heavy columns and narrow ranges of huge values.
    Yields (name, op, random_reads, numpy uint64 array)."""
    from . import synth
    rng = np.random.default_rng(seed)
    kinds = ("skewed", "sorted", "positions", "product", "C1", "C2", "C3", "C4", "runs", "narrow_huge", "uniform")
    for i in range(count):
        n = int(2 ** rng.uniform(lo_log2, hi_log2))
        kind = kinds[i % len(kinds)]
        s = int(rng.integers(1 << 30))
        if kind == "skewed":
            x, op = synth.skewed_widths(s, n), "base"
        elif kind == "sorted":
            x, op = synth.sorted_gaps(s, n), "base"
        elif kind == "positions":
            # the positions a select keeps at selectivity sel: gaps between kept rows
            # are geometric with mean 1/sel (generated in O(n), not by scanning n/sel rows)
            sel = float(rng.choice([0.001, 0.01, 0.1, 0.5, 0.9]))
            u = (synth.splitmix64(s, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
            gaps = 1 + np.floor(np.log1p(-u) / np.log1p(-sel)) if sel < 1.0 else np.ones(n)
            x, op = (np.cumsum(gaps.astype(np.uint64)) - np.uint64(1)), "select"
        elif kind == "product":
            with np.errstate(over="ignore"):
                x = synth.skewed_widths(s, n, widths=(3, 8, 16)) * synth.sorted_gaps(s + 1, n)
            op = "calc"
        elif kind in ("C1", "C2", "C3", "C4"):
            x, op = synth.table1_column(kind, n, seed=s), "project"
        elif kind == "runs":
            vals = synth.uniform(s, n // 8 + 1, 0, 1 << int(rng.integers(4, 40)))
            lens = 1 + (synth.splitmix64(s + 1, vals.size) % np.uint64(int(rng.integers(2, 1000))))
            x, op = np.repeat(vals, lens.astype(np.int64))[:n], "project"
        elif kind == "narrow_huge":
            b = int(rng.integers(1, 20))
            x, op = synth.uniform(s, n, 2**62, 2**62 + (1 << b)), "project"
        else:
            x, op = synth.uniform(s, n, 0, 1 << int(rng.integers(1, 64))), "project"
        yield kind, op, bool(rng.random() < 0.3), x


def harvest(ctx, items, reps: int = 2):
    """Features and exhaustive labels for every item (name, op, random, array)."""
    X, Y, S, T, names = [], [], [], [], []
    for name, op, rand, x in items:
        d = ms.as_device_u64(x, ctx.device)
        col = ctx.compress(d, ms.UNCOMPR)
        stats = ctx.column_stats(col).cpu().numpy().view(np.uint64)
        ctx.free(col)
        f = features_from_stats(stats, op, rand)
        sizes, times = measure_formats(ctx, d, stats, reps=reps)
        X.append(f)
        Y.append(labels_from(sizes, times, x.size))
        S.append(sizes)
        T.append(times)
        names.append(name)
    return np.array(X), np.array(Y), np.array(S), np.array(T), names
