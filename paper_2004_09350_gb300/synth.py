"""Seeded synthetic inputs (SplitMix64), shared by the tests, the bench and the oracle runs.

This module holds data generation only -- none of the method's arithmetic.  Every
array is a numpy ``uint64`` array produced from a counter-based SplitMix64 stream
(value i of stream ``seed`` is ``mix(seed + (i + 1) * GAMMA)``), so the same seed
gives the same column on any machine.

Shapes and distributions follow the paper's synthetic columns (Sec. 5.1, Table 1)
and the workloads this project measures:
  * ``table1_column``   -- C1..C4 of Table 1 (C1 uniform in [0,63]; C2 with 0.01%
    outliers 2^63-1; C3 uniform in [2^62, 2^62+63]; C4 sorted in [2^47, 2^47+100K]),
  * ``tiny_fragment``   -- two 2^20-row columns: A ~ U[0,2^12), B ~ U[0,2^20),
  * ``skewed_widths``   -- per-512-block bit width drawn from {3,8,16,27,40},
  * ``sorted_gaps``     -- sorted keys with geometric gaps of mean 4,
  * ``star_fact`` / ``star_dims`` -- a star-schema-shaped fact table and dimensions,
  * ``batch_fragments`` -- thousands of select -> project -> agg_sum fragments with
    log-uniform lengths and per-fragment widths and shapes.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BLOCK = 512


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Values offset .. offset+n-1 of the counter-based SplitMix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers in [lo, hi) (hi - lo >= 1).  Power-of-two spans take the top bits;
    other spans (< 2^32) scale the top 32 bits: ((z >> 32) * span) >> 32."""
    span = hi - lo
    if span <= 0:
        raise ValueError("empty range")
    z = splitmix64(seed, n)
    if span & (span - 1) == 0:
        k = span.bit_length() - 1
        r = (z >> np.uint64(64 - k)) if k > 0 else np.zeros(n, dtype=np.uint64)
    else:
        if span >= 1 << 32:
            raise ValueError("non-power-of-two spans must be < 2^32")
        r = ((z >> np.uint64(32)) * np.uint64(span)) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return r + np.uint64(lo)


# ------------------------------------------------ the same streams on the GPU

def _torch_mix(z):
    import torch
    m30 = (1 << 34) - 1
    m27 = (1 << 37) - 1
    m31 = (1 << 33) - 1
    z = z ^ ((z >> 30) & m30)
    z = z * torch.tensor(int(np.int64(np.uint64(0xBF58476D1CE4E5B9).view(np.int64))), dtype=torch.int64,
                         device=z.device)
    z = z ^ ((z >> 27) & m27)
    z = z * torch.tensor(int(np.int64(np.uint64(0x94D049BB133111EB).view(np.int64))), dtype=torch.int64,
                         device=z.device)
    return z ^ ((z >> 31) & m31)


def splitmix64_torch(seed: int, n: int, device, offset: int = 0):
    """splitmix64() computed with int64 tensor arithmetic on `device` (same bits)."""
    import torch
    gamma = int(np.uint64(GAMMA).view(np.int64))
    s = int(np.uint64(seed & 0xFFFFFFFFFFFFFFFF).view(np.int64))
    i = torch.arange(offset + 1, offset + n + 1, dtype=torch.int64, device=device)
    return _torch_mix(i * gamma + s)


def uniform_torch(seed: int, n: int, lo: int, hi: int, device):
    """uniform() on `device`, as an int64 tensor holding the same uint64 bits."""
    span = hi - lo
    z = splitmix64_torch(seed, n, device)
    if span & (span - 1) == 0:
        k = span.bit_length() - 1
        r = ((z >> (64 - k)) & ((1 << k) - 1)) if k > 0 else z * 0
    else:
        r = (((z >> 32) & 0xFFFFFFFF) * span) >> 32
    return r + lo


def geometric_gaps(seed: int, n: int) -> np.ndarray:
    """Gaps in {1, 2, ...} with P(g = k) = (3/4)^(k-1) / 4 (mean 4), capped at 33.

    Trial t succeeds when bits 2t, 2t+1 of the draw are both zero (probability 1/4);
    the gap is one plus the index of the first success.  The index comes from the
    lowest set bit of the "pair is 00" mask, located exactly with frexp.
    """
    z = splitmix64(seed, n)
    with np.errstate(over="ignore"):
        m = ~(z | (z >> np.uint64(1))) & np.uint64(0x5555555555555555)
        low = m & (~m + np.uint64(1))
    _, e = np.frexp(low.astype(np.float64))
    gap = (e.astype(np.int64) - 1) // 2 + 1
    gap[m == 0] = 33
    return gap.astype(np.uint64)


def runs(seed: int, n: int, mean_run: int, distinct: int = 6) -> np.ndarray:
    """A column of runs: run lengths uniform in [1, 2*mean_run - 1] (mean `mean_run`),
    run values uniform in [0, distinct), so that neighbouring runs of equal value merge
    into longer ones as in real low-cardinality columns."""
    if n == 0:
        return np.zeros(0, dtype=np.uint64)
    k = n // max(mean_run, 1) + 2
    while True:
        lens = uniform(seed, k, 1, 2 * mean_run)
        if int(lens.sum()) >= n:
            break
        k *= 2
    vals = uniform(seed + 1, k, 0, distinct)
    return np.repeat(vals, lens.astype(np.int64))[:n].copy()


# --------------------------------------------------------------- Table 1 columns

def table1_column(which: str, n: int, seed: int = 1) -> np.ndarray:
    """Synthetic columns C1-C4 (Sec. 5.1, Table 1), length n."""
    if which == "C1":
        return uniform(seed, n, 0, 64)
    if which == "C2":
        x = uniform(seed, n, 0, 64)
        out = splitmix64(seed + 7, n) % np.uint64(10000) == 0  # 0.01 % outliers
        x[out] = np.uint64(2**63 - 1)
        return x
    if which == "C3":
        return uniform(seed, n, 2**62, 2**62 + 64)
    if which == "C4":
        return np.sort(uniform(seed, n, 2**47, 2**47 + 100_000 + 1))
    raise ValueError(which)


def table1_point_select_variant(which: str, n: int, seed: int = 1) -> np.ndarray:
    """Sec. 5.1 single-operator input: 90% of values equal the column's lowest value."""
    x = table1_column(which, n, seed)
    lowest = {"C1": 0, "C2": 0, "C3": 2**62, "C4": 2**47}[which]
    pick = splitmix64(seed + 11, n) % np.uint64(10) != 0
    x = x.copy()
    x[pick] = np.uint64(lowest)
    if which == "C4":
        x = np.sort(x)
    return x


# ------------------------------------------------------------ measured workloads

def tiny_fragment(seed: int = 42, n: int = 1 << 20):
    """Two columns: A ~ U[0, 2^12) (static BP at 12 bits), B ~ U[0, 2^20)."""
    return uniform(seed, n, 0, 1 << 12), uniform(seed + 1, n, 0, 1 << 20)


WIDTH_CHOICES = (3, 8, 16, 27, 40)


def skewed_widths(seed: int, n: int, widths=WIDTH_CHOICES) -> np.ndarray:
    """Per 512-block width b drawn uniformly from ``widths``; values U[0, 2^b) with
    one value per block forced to have bit b-1 set, so the block's width is exactly b."""
    nblk = (n + BLOCK - 1) // BLOCK
    choice = np.asarray(widths, dtype=np.uint64)[splitmix64(seed, nblk) % np.uint64(len(widths))]
    b = np.repeat(choice, BLOCK)[:n]
    z = splitmix64(seed + 1, n)
    x = z >> (np.uint64(64) - b)
    first = np.arange(0, n, BLOCK)
    forced_at = first + (splitmix64(seed + 2, nblk) % np.uint64(BLOCK)).astype(np.int64)
    forced_at = np.minimum(forced_at, n - 1)
    x[forced_at] |= np.uint64(1) << (b[forced_at] - np.uint64(1))
    return x


def sorted_gaps(seed: int, n: int) -> np.ndarray:
    """Sorted keys: K_0 = 0 and K_i - K_{i-1} ~ Geometric(1/4) (mean 4)."""
    if n == 0:
        return np.zeros(0, dtype=np.uint64)
    g = geometric_gaps(seed, n)
    g[0] = 0
    return np.cumsum(g, dtype=np.uint64)


def value_at_rank(x: np.ndarray, s: float) -> int:
    """Value at rank floor(s*n) of x sorted ascending (threshold for `x < c` at selectivity ~s)."""
    k = min(int(s * x.size), x.size - 1)
    return int(np.partition(x, k)[k])


# ---------------------------------------------------------------- star schema

DIM_SIZES = (2_500_000, 200_000, 30_000, 2556)


def star_dims(seed: int = 7) -> dict:
    """Dimension attributes: D1.c5 ~ U[0,5) over 2.5e6 keys, D2.c25 ~ U[0,25) over
    2e5 keys, and the date dimension's year = (7 * key) // 2556 over 2556 keys
    (seven equal years)."""
    return {"d1_c5": uniform(seed, DIM_SIZES[0], 0, 5),
            "d2_c25": uniform(seed + 1, DIM_SIZES[1], 0, 25),
            "date_year": (np.arange(DIM_SIZES[3], dtype=np.uint64) * np.uint64(7)) // np.uint64(DIM_SIZES[3])}


def star_fact_torch(seed: int, n: int, device) -> dict:
    """star_fact() generated on `device` (int64 tensors with the same bits)."""
    import torch
    day = (torch.arange(n, dtype=torch.int64, device=device) * DIM_SIZES[3]) // max(n, 1)
    return {
        "fk1": uniform_torch(seed + 10, n, 0, DIM_SIZES[0], device),
        "fk2": uniform_torch(seed + 11, n, 0, DIM_SIZES[1], device),
        "fk3": uniform_torch(seed + 12, n, 0, DIM_SIZES[2], device),
        "fk_date": day,
        "quantity": uniform_torch(seed + 13, n, 1, 51, device),
        "discount": uniform_torch(seed + 14, n, 0, 11, device),
        "revenue": uniform_torch(seed + 15, n, 0, 1 << 23, device),
    }


def star_fact(seed: int, n: int) -> dict:
    """Fact columns: fk1..fk3 uniform over the dimension sizes, fk_date sorted over
    [0, 2556) with equal counts per day, quantity U[1,50], discount U[0,10],
    revenue U[0, 2^23)."""
    day = (np.arange(n, dtype=np.uint64) * np.uint64(DIM_SIZES[3])) // np.uint64(max(n, 1))
    return {
        "fk1": uniform(seed + 10, n, 0, DIM_SIZES[0]),
        "fk2": uniform(seed + 11, n, 0, DIM_SIZES[1]),
        "fk3": uniform(seed + 12, n, 0, DIM_SIZES[2]),
        "fk_date": day,
        "quantity": uniform(seed + 13, n, 1, 51),
        "discount": uniform(seed + 14, n, 0, 11),
        "revenue": uniform(seed + 15, n, 0, 1 << 23),
    }


# ----------------------------------------------------------- batched fragments

# ms_cmp ids: LT three times as often as the others
BATCH_CMPS = (2, 2, 2, 6, 5, 0, 1, 3, 4)
BATCH_Y_SHAPES = ("uniform", "offset", "sorted", "skewed")
BATCH_SELECTIVITIES = (0.001, 0.1, 0.9)


def _unit(z) -> float:
    return float(int(z) >> 11) / float(1 << 53)


def batch_fragments(seed: int, count: int, lo_log2: float = 10, hi_log2: float = 24, max_bits: int = 40) -> list:
    """Parameters of `count` fragments sum(y[i] for x[i] <cmp> c1 (c2)):
    n = floor(2^(lo + u (hi - lo))) (log-uniform), x ~ U[0, 2^bx), y of one of
    BATCH_Y_SHAPES at width by, with bx, by uniform in [1, max_bits], and a
    predicate whose constant sits at the quantile s of x's range, s drawn from
    BATCH_SELECTIVITIES (BETWEEN spans s/2 of the range above it)."""
    z = splitmix64(seed, 8 * count).reshape(count, 8)
    out = []
    for f in range(count):
        n = int(2.0 ** (lo_log2 + _unit(z[f, 0]) * (hi_log2 - lo_log2)))
        bx = 1 + int(z[f, 1] % np.uint64(max_bits))
        by = 1 + int(z[f, 2] % np.uint64(max_bits))
        shape = BATCH_Y_SHAPES[int(z[f, 3] % np.uint64(len(BATCH_Y_SHAPES)))]
        cmp = BATCH_CMPS[int(z[f, 4] % np.uint64(len(BATCH_CMPS)))]
        sel = BATCH_SELECTIVITIES[int(z[f, 5] % np.uint64(len(BATCH_SELECTIVITIES)))]
        c1 = int(sel * (1 << bx))
        c2 = c1 + int(sel * (1 << bx) / 2)
        sx = int(z[f, 7] & np.uint64(0xFFFFFFFF))
        out.append({"n": n, "bx": bx, "by": by, "shape": shape, "cmp": cmp, "c1": c1, "c2": c2,
                    "seed_x": sx, "seed_y": sx + 0x1000})
    return out


def _skew_widths(by: int):
    return (max(1, by // 4), max(1, by // 2), by)


def _sorted_gap_bits(by: int) -> int:
    return 1 + (by - 1) % 8


def batch_x(spec: dict) -> np.ndarray:
    return uniform(spec["seed_x"], spec["n"], 0, 1 << spec["bx"])


def batch_y(spec: dict) -> np.ndarray:
    """y of the fragment's shape: uniform U[0, 2^by); offset 2^(by-1) + U[0, 2^max(by-8,0))
    (narrow range, FOR-friendly); sorted prefix sums of U[0, 2^g) gaps, g = 1 + (by-1) % 8
    (DELTA-friendly); skewed per-block widths from {by/4, by/2, by} (dynamic-BP-friendly)."""
    n, by, sy, shape = spec["n"], spec["by"], spec["seed_y"], spec["shape"]
    if shape == "uniform":
        return uniform(sy, n, 0, 1 << by)
    if shape == "offset":
        with np.errstate(over="ignore"):
            return uniform(sy, n, 0, 1 << max(by - 8, 0)) + np.uint64(1 << (by - 1))
    if shape == "sorted":
        return np.cumsum(uniform(sy, n, 0, 1 << _sorted_gap_bits(by)), dtype=np.uint64)
    return skewed_widths(sy, n, _skew_widths(by))


def _umod_torch(z, m: int):
    """(z as uint64) mod m for an int64 tensor z and 0 < m < 2^31."""
    hi = (z >> 32) & 0xFFFFFFFF
    lo = z & 0xFFFFFFFF
    return ((hi % m) * ((1 << 32) % m) + lo % m) % m


def skewed_widths_torch(seed: int, n: int, widths, device):
    """skewed_widths() on `device` (int64 tensor, same bits)."""
    import torch
    nblk = (n + BLOCK - 1) // BLOCK
    w = torch.tensor(list(widths), dtype=torch.int64, device=device)
    choice = w[_umod_torch(splitmix64_torch(seed, nblk, device), len(widths))]
    b = choice.repeat_interleave(BLOCK)[:n]
    z = splitmix64_torch(seed + 1, n, device)
    x = (z >> (64 - b)) & ((torch.ones_like(b) << b) - 1)
    first = torch.arange(0, n, BLOCK, dtype=torch.int64, device=device)
    forced_at = torch.clamp(first + _umod_torch(splitmix64_torch(seed + 2, nblk, device), BLOCK), max=n - 1)
    x[forced_at] |= torch.ones_like(forced_at) << (b[forced_at] - 1)
    return x


def batch_x_torch(spec: dict, device):
    return uniform_torch(spec["seed_x"], spec["n"], 0, 1 << spec["bx"], device)


def batch_y_torch(spec: dict, device):
    """batch_y() on `device` (int64 tensor, same bits)."""
    import torch
    n, by, sy, shape = spec["n"], spec["by"], spec["seed_y"], spec["shape"]
    if shape == "uniform":
        return uniform_torch(sy, n, 0, 1 << by, device)
    if shape == "offset":
        return uniform_torch(sy, n, 0, 1 << max(by - 8, 0), device) + (1 << (by - 1))
    if shape == "sorted":
        return torch.cumsum(uniform_torch(sy, n, 0, 1 << _sorted_gap_bits(by), device), 0)
    return skewed_widths_torch(sy, n, _skew_widths(by), device)
