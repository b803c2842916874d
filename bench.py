#!/usr/bin/env python
"""Throughput of the on-the-fly morphing pipeline on one GB300 (or N replicas).

Default workload (star): a star-schema plan over a 6e8-row fact table of uint64
columns (foreign keys uniform over dimensions of 2.5e6, 2e5, 3e4 and 2556 rows,
a date-sorted key, quantity, discount, revenue) and three dimension attributes.
One step selects on two dimension attributes, semi-joins both into the fact
table, selects discount and quantity ranges, projects, computes group ids and
group-sums revenue into 105 groups.  Compressed pipeline: base columns dynamic
BP (the sorted date key DELTA+BP), positions DELTA+BP, values dynamic BP.  The
same plan with every column uncompressed is timed beside it.

value = fact rows per second of the compressed pipeline (whole job).
roofline = the dominant kernel's algorithmic bytes per launch / its mean launch
time, against the measured HBM copy peak.  e2e = the same plan through the C
ABI with the base columns imported from pinned host memory every step in their
format and the group sums read back (uncompressed.e2e: the uncompressed plan the
same way).  cpu_baseline = the CPU oracle on a bounded prefix sample of the same
workload.  Footprint: the sum of column sizes (base plus intermediates), and the
device peak (base columns, the arena's high-water mark of intermediates and the
context's work area).

Other workloads (--workload): sweep-plan (select(X<c) -> project X, K -> calc ->
agg_sum on 2^28-row columns), selector, batch, kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "logical rows/s and achieved HBM GB/s (% of peak), compressed vs uncompressed"
FALLBACK_HBM = 6800.0
BLOCK = 512


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--render-sweep-table", default="",
                    help="print the markdown table of a saved sweep-table JSON line and exit")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rows", type=int, default=0,
                    help="fact rows (star, default 6e8) or column rows (other workloads, default 2^28)")
    ap.add_argument("--selectivity", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=2020)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["star", "sweep-plan", "sweep-table", "selector", "batch", "kernel"],
                    default="star",
                    help="star: the star-schema plan on a 6e8-row fact table (default); "
                         "sweep-plan: the 2^28-row select/project/calc/sum plan; "
                         "sweep-table: every operator of that plan for every input/output format pair; "
                         "selector: train the learned format selector on engine traces and measure its regret; "
                         "batch: 4096 select->project->agg_sum fragments in one persistent launch; "
                         "kernel: one operator of the plan alone (--kernel), the case the ncu summaries use")
    ap.add_argument("--kernel", choices=["agg_sum", "select", "select_packed", "project", "project_uniform",
                                         "compress", "decompress"],
                    default="agg_sum",
                    help="project_uniform: project X at positions spread uniformly over the column "
                         "(--selectivity of the rows), the access pattern of the star plan's projects")
    ap.add_argument("--width", type=int, default=0,
                    help="kernel workload: every 512-block of X at this bit width (0: the plan's width mix)")
    ap.add_argument("--x-format", choices=["uncompr", "static_bp", "dyn_bp", "delta_bp", "for_bp"], default="dyn_bp",
                    help="kernel workload: the format X is stored in (static BP at X's largest width)")
    ap.add_argument("--selector-items", type=int, default=20000,
                    help="selector workload: engine traces to train and hold out (80/20), 2^16 rows up to "
                         "2^--selector-max-log2")
    ap.add_argument("--selector-max-log2", type=float, default=20.0)
    ap.add_argument("--selector-mid-items", type=int, default=2000,
                    help="selector workload: extra training traces of 2^20 .. 2^24 rows")
    ap.add_argument("--selector-large-items", type=int, default=200,
                    help="selector workload: extra held-out traces of 2^22 .. 2^26 rows")
    ap.add_argument("--fragments", type=int, default=4096)
    ap.add_argument("--batch-max-log2", type=float, default=24.0)
    ap.add_argument("--batch-train-items", type=int, default=400)
    a = ap.parse_args()
    a.warmup = max(a.warmup, 3)
    if not a.rows and a.workload != "star":
        a.rows = 1 << 28
    return a


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


# ----------------------------------------------------------------- workload

def make_inputs(rows, seed, sel):
    from paper_2004_09350_gb300 import synth
    x = synth.skewed_widths(seed, rows)
    k = synth.sorted_gaps(seed + 1, rows)
    c = synth.value_at_rank(x, sel)
    return x, k, c


PLAN_WORKLOAD = ("select(X<c)->project(X,K)->calc(X'*K')->agg_sum on 2^28-row columns, "
                 "X widths {3,8,16,27,40} per 512-block, K sorted gaps mean 4")
COMPRESSED = {"X": "dyn_bp", "K": "delta_bp", "P": "delta_bp", "X'": "dyn_bp", "K'": "delta_bp", "Y": "dyn_bp"}
UNCOMPRESSED = {k: "uncompr" for k in COMPRESSED}


def fmt_id(name):
    from paper_2004_09350_gb300 import morphstore as ms
    return ms.FORMAT_NAMES.index(name)


def run_plan(ctx, cx, ck, c, fm, res):
    """One step of the plan; frees its intermediates (LIFO) before returning."""
    from paper_2004_09350_gb300 import morphstore as ms
    pos = ctx.select(cx, ms.LT, c, fmt=fmt_id(fm["P"]))
    xp = ctx.project(cx, pos, fmt=fmt_id(fm["X'"]))
    kp = ctx.project(ck, pos, fmt=fmt_id(fm["K'"]))
    y = ctx.calc(ms.MUL, xp, kp, fmt=fmt_id(fm["Y"]))
    ctx.agg_sum(y, out=res)
    return [y, kp, xp, pos]


def free_all(ctx, cols):
    for col in cols:
        ctx.free(col)


# ------------------------------------------------------ algorithmic bytes

def block_widths(x, delta=False):
    nb = x.size // BLOCK
    blk = x[: nb * BLOCK].reshape(nb, BLOCK)
    if delta:
        d = np.diff(blk, axis=1)
        m = d.max(axis=1) if nb else np.zeros(0, np.uint64)
    else:
        m = blk.max(axis=1)
    w = np.zeros(nb, dtype=np.int64)
    v = m.copy()
    while np.any(v):
        nz = v != 0
        w[nz] += 1
        v >>= np.uint64(1)
    return w


def touched_bytes_dyn(x_widths, n, pos):
    """Bytes of the 512-value blocks of a dynamic-BP column that positions `pos`
    touch (header + payload of each touched block; the remainder's touched
    32-byte sectors): the unit of data movement of a block-format gather."""
    nb = x_widths.size
    p = pos.astype(np.int64)
    g = np.unique(p[p < nb * BLOCK] >> 9)
    rem = p[p >= nb * BLOCK]
    sectors = np.unique((8 * (rem - nb * BLOCK)) >> 5).size if rem.size else 0
    return int(16 * g.size + 64 * int(x_widths[g].sum()) + 32 * sectors)


def touched_bytes_delta(k_widths, pos):
    g = np.unique(pos.astype(np.int64) >> 9)
    g = g[g < k_widths.size]
    return int((64 * k_widths[g] + 16).sum())


# ------------------------------------------------------------------ clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "period_ms": 50}


# ------------------------------------------------------------- CPU oracle

def oracle_plan(x, k, c):
    """The same plan on the CPU oracle: every column passes through the oracle's
    codec in the pipeline's formats (decode inputs, encode each intermediate)."""
    import oracle
    f = {n: oracle.FORMAT_NAMES.index(v) for n, v in COMPRESSED.items()}
    bx, bk = oracle.compress(f["X"], x), oracle.compress(f["K"], k)
    t0 = time.perf_counter()
    xd = oracle.decompress(f["X"], x.size, bx)
    kd = oracle.decompress(f["K"], k.size, bk)
    pos = oracle.select(xd, oracle.LT, c)
    pd = oracle.decompress(f["P"], pos.size, oracle.compress(f["P"], pos))
    xp = oracle.project(xd, pd)
    kp = oracle.project(kd, pd)
    xpd = oracle.decompress(f["X'"], xp.size, oracle.compress(f["X'"], xp))
    kpd = oracle.decompress(f["K'"], kp.size, oracle.compress(f["K'"], kp))
    y = oracle.calc(oracle.MUL, xpd, kpd)
    yd = oracle.decompress(f["Y"], y.size, oracle.compress(f["Y"], y))
    s = oracle.agg_sum(yd)
    return time.perf_counter() - t0, s


def host_info():
    """The host the CPU baseline ran on: CPU model (lscpu, else the platform) and core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return {"cpu": model or platform.processor() or platform.machine(), "cores": os.cpu_count()}


def cpu_baseline(x, k, c, target_s=15.0):
    """Oracle on a bounded prefix sample sized for ~target_s seconds of CPU work."""
    probe = min(x.size, 1 << 15)
    t, _ = oracle_plan(x[:probe], k[:probe], c)
    rows = int(min(x.size, max(probe, probe * target_s / max(t, 1e-6))))
    rows -= rows % BLOCK
    t, _ = oracle_plan(x[:rows], k[:rows], c)
    return {"value": rows / t, "unit": "rows/s", "cores": 1, "host": host_info(), "kind": "oracle",
            "sample": f"first {rows} rows of X and K, same plan and formats, single thread ({t:.1f} s)"}


# ---------------------------------------------------------------- helpers

def source_digest():
    """Digest of the kernel sources' code: comments, blank lines and layout are left
    out, so that a comment edit keeps a committed traffic figure valid and any code
    edit invalidates it."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2004_09350_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(" ".join(line.split()) for line in text.splitlines() if line.strip())
        h.update(f.encode() + b"\0" + code.encode() + b"\0")
    return h.hexdigest()[:16]


def measured_traffic(kernel, key="dram_bytes_per_launch"):
    """A DRAM traffic figure (bytes per launch, or bytes per algorithmic byte) from the
    committed ncu summary, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    e = t.get(kernel)
    if not e or e.get("source_digest") != source_digest():
        return None
    return e.get(key)


def max_over_ranks(x, world, device=None):
    """The largest x over all ranks (the slowest replica sets the job's step time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rows_per_s(world, rows, ms_step):
    """Whole-job throughput: every replica processes `rows` per step."""
    return world * rows / (ms_step * 1e-3)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# -------------------------------------------------------------- our arm

def bench_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2004_09350_gb300 import morphstore as ms

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    n = args.rows
    x, k, c = make_inputs(n, args.seed, args.selectivity)
    dev = torch.device("cuda", local)
    ctx = ms.Ctx(local, arena_bytes=int(2.5 * 8 * n) + (1 << 30), max_rows=n)
    res = torch.zeros(1, dtype=torch.int64, device=dev)
    dx, dk = ms.as_device_u64(x, dev), ms.as_device_u64(k, dev)
    out = {}
    for label, fm in (("compressed", COMPRESSED), ("uncompressed", UNCOMPRESSED)):
        cx = ctx.compress(dx, fmt_id(fm["X"]))
        ck = ctx.compress(dk, fmt_id(fm["K"]))
        ctx.check(what="base columns")
        # warm-up, sizes of every column of the plan and the peak footprint
        for _ in range(args.warmup):
            free_all(ctx, run_plan(ctx, cx, ck, c, fm, res))
        ctx.reset_high_water()
        cols = run_plan(ctx, cx, ck, c, fm, res)
        sizes = {"X": ctx.info(cx)["size_bytes"], "K": ctx.info(ck)["size_bytes"]}
        for name, col in zip(("Y", "K'", "X'", "P"), cols):
            sizes[name] = ctx.info(col)["size_bytes"]
        m = ctx.info(cols[3])["n"]
        free_all(ctx, cols)
        base_use, high = ctx.arena_usage()
        ctx.check(what=f"{label} warm-up")
        want = None
        barrier()
        # the clock sampler (50 ms period) also runs over untimed steps just before and
        # after the timed ones, so that a short timed region still gets samples
        w0 = time.perf_counter()
        free_all(ctx, run_plan(ctx, cx, ck, c, fm, res))
        torch.cuda.synchronize()
        pad = max(1, int(0.4 / max(time.perf_counter() - w0, 1e-4)))
        clocks = Clocks(local) if label == "compressed" else None
        if clocks:
            for _ in range(pad):
                free_all(ctx, run_plan(ctx, cx, ck, c, fm, res))
        barrier()
        ctx.profile(True)
        # one event between consecutive steps: the mean over the whole region and the best step
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record()
        for i in range(args.steps):
            free_all(ctx, run_plan(ctx, cx, ck, c, fm, res))
            evs[i + 1].record()
        t0, t1 = evs[0], evs[-1]
        barrier()
        best_ms = min(evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps))
        prof = ctx.profile_collect()
        ctx.profile(False)
        if clocks:
            for _ in range(pad):
                free_all(ctx, run_plan(ctx, cx, ck, c, fm, res))
            torch.cuda.synchronize()
        ck_info = clocks.stop() if clocks else None
        ctx.check(what=f"{label} timed steps")
        ms_step = max_over_ranks(t0.elapsed_time(t1) / args.steps, world, dev)
        got = int(ms.to_numpy_u64(res)[0])
        out[label] = dict(ms_step=ms_step, best_ms=best_ms, sizes=sizes, m=m, prof=prof, clocks=ck_info, sum=got,
                          footprint=int(sum(sizes.values())), arena_peak=int(high - (base_use - 0)))
        ctx.free(ck)
        ctx.free(cx)
    assert out["compressed"]["sum"] == out["uncompressed"]["sum"], "pipelines disagree"

    # ---- algorithmic bytes of each kernel of the compressed plan (per launch)
    comp = out["compressed"]
    s, m = comp["sizes"], comp["m"]
    pos = np.flatnonzero(x < np.uint64(c))
    xw, kw = block_widths(x), block_widths(k, delta=True)
    nch = -(-n // BLOCK)
    alg = {
        "mark": s["X"] + n // 8 + 8 * nch,
        "emit": n // 8 + 8 * nch + s["P"],
        "project": (s["P"] + touched_bytes_dyn(xw, n, pos) + s["X'"]
                    + s["P"] + touched_bytes_delta(kw, pos) + s["K'"]) / 2,
        "calc": s["X'"] + s["K'"] + s["Y"],
        "agg_sum": s["Y"] + 8,
    }
    per_kernel = {}
    for kname, (launches, total) in comp["prof"].items():
        avg = total / max(launches, 1)
        gbs = alg.get(kname, 0) / (avg * 1e-3) / 1e9 if kname in alg else None
        per_kernel[kname] = {"launches": launches, "avg_ms": round(avg, 4),
                             "alg_bytes": int(alg.get(kname, 0)), "alg_GBps": None if gbs is None else round(gbs, 1)}
    dom = max(per_kernel, key=lambda kk: per_kernel[kk]["avg_ms"] * per_kernel[kk]["launches"])
    peak, peak_kind = peaks()
    ach = per_kernel[dom]["alg_GBps"]
    plan_bytes = sum(v * per_kernel.get(kk, {"launches": 0})["launches"] / args.steps for kk, v in alg.items())

    # ---- end to end through the C ABI from pinned host buffers: every step copies the
    # plan's base columns in, in their format, runs the plan and reads the sum back
    def e2e_run(fm):
        cx = ctx.compress(dx, fmt_id(fm["X"]))
        ck = ctx.compress(dk, fmt_id(fm["K"]))
        hx = torch.from_numpy(ctx.export_bytes(cx)).pin_memory()
        hk = torch.from_numpy(ctx.export_bytes(ck)).pin_memory()
        ctx.free(ck)
        ctx.free(cx)
        hres = torch.zeros(1, dtype=torch.int64).pin_memory()

        def e2e_step():
            ix = ctx.import_bytes(fmt_id(fm["X"]), n, hx)
            ik = ctx.import_bytes(fmt_id(fm["K"]), n, hk)
            free_all(ctx, run_plan(ctx, ix, ik, c, fm, res))
            hres.copy_(res, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            ctx.free(ik)
            ctx.free(ix)

        for _ in range(args.warmup):
            e2e_step()
        barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        ms_e = max_over_ranks((time.perf_counter() - t) * 1e3 / args.steps, world, dev)
        assert int(hres.numpy().view(np.uint64)[0]) == comp["sum"]
        return {"value": job_rows_per_s(world, n, ms_e), "unit": "rows/s",
                "h2d_bytes_per_step": int(hx.numel() + hk.numel()), "d2h_bytes_per_step": 8,
                "ms_per_step": round(ms_e, 3)}

    e2e = e2e_unc = None
    if not args.no_e2e:
        e2e = e2e_run(COMPRESSED)
        e2e_unc = e2e_run(UNCOMPRESSED)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(x, k, c)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None

    unc = out["uncompressed"]
    line = {
        "metric": METRIC,
        "value": job_rows_per_s(world, n, comp["ms_step"]),
        "unit": "rows/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(comp["ms_step"], 4),
        "ms_per_step_best": round(comp["best_ms"], 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic (seeded SplitMix64)",
        "config": {
            "workload": PLAN_WORKLOAD,
            "rows": n, "selectivity": round(comp["m"] / n, 5), "formats": COMPRESSED,
            "l2": "inputs larger than L2 (compressed X %.2f GB, K %.2f GB; uncompressed 2.1 GB each)"
                  % (comp["sizes"]["X"] / 1e9, comp["sizes"]["K"] / 1e9),
            "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": None if ach is None else round(ach / peak, 4), "peak_kind": peak_kind,
                     "traffic": measured_traffic(dom),
                     "alg_bytes_per_launch": per_kernel[dom]["alg_bytes"]},
        "per_kernel": per_kernel,
        "plan_GBps": round(plan_bytes / (comp["ms_step"] * 1e-3) / 1e9, 1),
        "uncompressed": {"value": job_rows_per_s(world, n, unc["ms_step"]), "ms_per_step": round(unc["ms_step"], 4),
                         "ms_per_step_best": round(unc["best_ms"], 4), "e2e": e2e_unc,
                         "footprint_bytes": unc["footprint"], "arena_peak_bytes": unc["arena_peak"]},
        "compressed": {"footprint_bytes": comp["footprint"], "arena_peak_bytes": comp["arena_peak"],
                       "sizes": comp["sizes"]},
        "speedup_vs_uncompressed": round(unc["ms_step"] / comp["ms_step"], 3),
        "gpu_launches": int(sum(v[0] for v in comp["prof"].values())),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": comp["clocks"],
    }
    return line


# ------------------------------------------------------------ reference arm

def bench_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return None
    if args.workload == "star":
        return bench_reference_star(args, world)
    x, k, c = make_inputs(args.rows, args.seed, args.selectivity)
    # each step runs the oracle on a bounded prefix so the whole run stays within minutes
    per_step_s = max(2.0, min(20.0, 150.0 / max(args.steps + args.warmup, 1)))
    probe = min(x.size, 1 << 15)
    t, _ = oracle_plan(x[:probe], k[:probe], c)
    rows = int(min(x.size, max(probe, probe * per_step_s / max(t, 1e-6))))
    rows -= rows % BLOCK
    for _ in range(args.warmup):
        oracle_plan(x[: min(rows, 1 << 15)], k[: min(rows, 1 << 15)], c)
    times = [oracle_plan(x[:rows], k[:rows], c)[0] for _ in range(args.steps)]
    tot = sum(times)
    value = rows * args.steps / tot
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded SplitMix64)",
            "config": {"workload": PLAN_WORKLOAD, "rows": int(x.size),
                       "selectivity": round(float(np.count_nonzero(x < np.uint64(c))) / max(x.size, 1), 5),
                       "formats": COMPRESSED, "parallelism": "1 host core"},
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "host": host_info(), "kind": "oracle",
                             "sample": f"first {rows} rows of the {x.size}-row workload per step "
                                       f"(the same plan and formats, single thread)"},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------- star plan

STAR_WORKLOAD = ("star-schema plan on a 6e8-row fact table: select D1.c5 = 0 and D2.c25 < 15, semi-join fk1 "
                 "and fk2, select 1 <= discount <= 3 and quantity < 25, project, calc, group_sum on 105 groups")


def oracle_star_plan(fact, dims, codec=True):
    """The star plan on the CPU oracle.  With codec=True every column passes through
    the oracle's codec in the compressed pipeline's formats: the base columns are
    decoded from their compressed bytes and every intermediate is encoded and
    decoded again, as an engine with compressed intermediates does."""
    import oracle
    from paper_2004_09350_gb300 import plans, synth
    fm = {k: int(v) for k, v in plans.STAR_COMPRESSED.items()}
    fb = {k: int(v) for k, v in plans.STAR_BASE_COMPRESSED.items()}
    packed = ({k: oracle.compress(fb[k], v, bw=plans.base_width(k, fb[k])) for k, v in {**fact, **dims}.items()}
              if codec else None)
    t0 = time.perf_counter()
    if codec:
        src = {**fact, **dims}
        b = {k: oracle.decompress(fb[k], src[k].size, packed[k], bw=plans.base_width(k, fb[k])) for k in src}
    else:
        b = {**fact, **dims}

    def inter(name, x):
        bw = plans.star_width(name, fm[name])
        return oracle.decompress(fm[name], x.size, oracle.compress(fm[name], x, bw=bw), bw=bw) if codec else x

    s1 = inter("S1", oracle.select(b["d1_c5"], oracle.EQ, 0))
    s2 = inter("S2", oracle.select(b["d2_c25"], oracle.LT, 15))
    p1 = inter("P1", oracle.semijoin(b["fk1"], s1, synth.DIM_SIZES[0]))
    f2 = inter("F2", oracle.project(b["fk2"], p1))
    q2 = inter("Q2", oracle.semijoin(f2, s2, synth.DIM_SIZES[1]))
    p2 = inter("P2", oracle.project(p1, q2))
    disc = inter("DISC", oracle.project(b["discount"], p2))
    q3 = inter("Q3", oracle.select(disc, oracle.BETWEEN, 1, 3))
    p3 = inter("P3", oracle.project(p2, q3))
    qty = inter("QTY", oracle.project(b["quantity"], p3))
    q4 = inter("Q4", oracle.select(qty, oracle.LT, 25))
    p4 = inter("P4", oracle.project(p3, q4))
    date = inter("DATE", oracle.project(b["fk_date"], p4))
    year = inter("YEAR", oracle.project(b["date_year"], date))
    f2b = inter("F2B", oracle.project(b["fk2"], p4))
    c25 = inter("C25", oracle.project(b["d2_c25"], f2b))
    g0 = inter("G0", oracle.calc(oracle.MUL, year, c=15))
    gid = inter("GID", oracle.calc(oracle.ADD, g0, c25))
    rev = inter("REV", oracle.project(b["revenue"], p4))
    sums = oracle.group_sum(gid, rev, plans.STAR_GROUPS)
    return time.perf_counter() - t0, sums


def star_host_sample(seed, rows):
    """The first `rows` fact rows and the dimensions, generated on the host (the
    same bits as the device generators)."""
    from paper_2004_09350_gb300 import synth
    return synth.star_fact(seed, rows), synth.star_dims(seed + 1)


def star_cpu_sample_rows(seed, target_s):
    """Fact rows of a prefix sample whose oracle star plan takes about target_s."""
    probe = 1 << 18
    f, d = star_host_sample(seed, probe)
    t, _ = oracle_star_plan(f, d)
    rows = int(probe * target_s / max(t, 1e-6))
    return max(probe, rows - rows % BLOCK)


def star_cpu_baseline(seed, n, target_s=15.0):
    rows = min(n, star_cpu_sample_rows(seed, target_s))
    f, d = star_host_sample(seed, rows)
    t, _ = oracle_star_plan(f, d)
    return {"value": rows / t, "unit": "rows/s", "cores": 1, "host": host_info(), "kind": "oracle",
            "build": "gcc -O2, single thread, not pinned to a core",
            "sample": f"first {rows} of the {n} fact rows, the same plan with every column passed through the "
                      f"oracle's codec in the compressed pipeline's formats ({t:.1f} s)"}


def _device_col_bytes(ctx, col):
    return ctx.export_bytes(col, device=True)


def project_touched_bytes(ctx, data, pos_t):
    """Bytes of the data column's units that sorted positions pos_t (int64 device
    tensor) touch: each touched 512-value block whole (header and payload) for the
    block formats and static BP, each touched 32-byte sector of an uncompressed
    column or of a block format's raw remainder."""
    import torch
    from paper_2004_09350_gb300 import morphstore as ms
    if pos_t.numel() == 0:
        return 0
    meta = ctx.info(data)
    n = meta["n"]
    if data.fmt == ms.UNCOMPR:
        return 32 * int(torch.unique_consecutive(pos_t >> 2).numel())
    if data.fmt == ms.STATIC_BP:
        full = n // BLOCK
        g = torch.unique_consecutive(pos_t >> 9)
        blk = int((g < full).sum())
        tail = pos_t[pos_t >= full * BLOCK]
        tail_sect = int(torch.unique_consecutive((tail - full * BLOCK) * meta["static_bw"] // 256).numel())
        return 64 * meta["static_bw"] * blk + 32 * tail_sect
    nb = meta["n_blocks"]
    raw = _device_col_bytes(ctx, data)
    hdr = raw[: 16 * nb].view(torch.int64).view(-1, 2)[:, 0] if nb else torch.zeros(0, dtype=torch.int64,
                                                                                      device=pos_t.device)
    g = torch.unique_consecutive(pos_t >> 9)
    gm = g[g < nb]
    b = (hdr[gm] & 255) if nb else gm
    rem = pos_t[pos_t >= nb * BLOCK]
    rem_sect = int(torch.unique_consecutive((rem - nb * BLOCK) >> 2).numel()) if rem.numel() else 0
    return int(16 * gm.numel() + 64 * int(b.sum())) + 32 * rem_sect


def star_kernel_bytes(ctx, trace):
    """Algorithmic bytes of one step of the star plan, per kernel (the operator
    definitions of the measurement plan; bytes(c) = physical column size):
      select    mark: bytes(in) + n/8 (match bitmap) + 4 per 512-row chunk (counts)
                emit: n/8 + 8 per chunk (offsets) + bytes(out)
      semijoin  build_keys: bytes(keys) + D/8;  mark: bytes(probe) + D/8 (key bitmap
                read) + n/8 + 4 per chunk;  emit as for select
      project   bytes(pos) + the data units the positions touch + bytes(out)
      calc      bytes(a) + bytes(b) + bytes(out);  group_sum  bytes(gid) + bytes(val) + 8G
    Scan and placement kernels move only bookkeeping and have no algorithmic bytes."""
    size = {}

    def sz(c):
        k = id(c)
        if k not in size:
            size[k] = ctx.info(c)
        return size[k]

    kb = {}

    def add(k, v):
        kb[k] = kb.get(k, 0) + int(v)

    for op, name, ins, out, extra, _, _ in trace:
        if op in ("select", "semijoin"):
            n = sz(ins[0])["n"]
            nch = -(-n // BLOCK)
            bitmap = n // 8
            add("mark", sz(ins[0])["size_bytes"] + bitmap + 4 * nch)
            add("emit", bitmap + 8 * nch + sz(out)["size_bytes"])
            if op == "semijoin":
                add("build_keys", sz(ins[1])["size_bytes"] + -(-extra // 8))
                add("mark", -(-extra // 8))
        elif op == "project":
            pos_t = ctx.decompress(ins[1])
            add("project", sz(ins[1])["size_bytes"] + project_touched_bytes(ctx, ins[0], pos_t)
                + sz(out)["size_bytes"])
            del pos_t
        elif op == "calc":
            add("calc", sum(sz(c)["size_bytes"] for c in ins) + sz(out)["size_bytes"])
        elif op == "group_sum":
            add("group_sum", sum(sz(c)["size_bytes"] for c in ins) + 8 * extra)
    return kb


def bench_star(args):
    """The star-schema plan at 6e8 fact rows (the default workload)."""
    import torch
    from paper_2004_09350_gb300 import morphstore as ms
    from paper_2004_09350_gb300 import plans, synth

    world, rank, local = dist_setup(args)
    n = args.rows or 600_000_000
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    fact = synth.star_fact_torch(args.seed, n, dev)
    dims = {k: ms.as_device_u64(v, dev) for k, v in synth.star_dims(args.seed + 1).items()}
    raw = {**fact, **dims}
    # arena: the base columns (uncompressed: 7 fact columns of 8 bytes) plus every
    # intermediate of one step (at most 8 bytes a fact row in the uncompressed plan), and
    # the compressed base columns, which stay for the end-to-end runs (12 bytes a row)
    ctx = ms.Ctx(local, arena_bytes=8 * 8 * n + 8 * n + 12 * n + (256 << 20), max_rows=n)
    out = {}

    def run_variant(label, base, fm):
        """Warm-up, one traced sizing step (sizes, footprint, per-operator times,
        algorithmic bytes) and the timed steps of the star plan in formats fm."""
        base_bytes = sum(ctx.info(c)["size_bytes"] for c in base.values())
        res = torch.zeros(plans.STAR_GROUPS, dtype=torch.int64, device=dev)
        for _ in range(args.warmup):
            _, cols = plans.star_plan(ctx, base, fm, out=res)
            plans.free_lifo(ctx, cols)
        use0, _ = ctx.arena_usage()
        ctx.reset_high_water()
        trace = []
        _, cols = plans.star_plan(ctx, base, fm, out=res, trace=trace)
        inter_bytes = plans.footprint(ctx, cols)
        _, high = ctx.arena_usage()
        torch.cuda.synchronize()
        op_ms = {rec[1]: round(rec[5].elapsed_time(rec[6]), 4) for rec in trace}
        kb = star_kernel_bytes(ctx, trace) if label == "compressed" else None
        plans.free_lifo(ctx, cols)
        del trace
        ctx.check(what=f"star {label} sizing step")
        barrier()
        clocks = Clocks(local) if label == "compressed" else None
        if clocks:  # let the sampler see load before the timed region
            w0 = time.perf_counter()
            while time.perf_counter() - w0 < 0.3:
                _, cols = plans.star_plan(ctx, base, fm, out=res)
                plans.free_lifo(ctx, cols)
                torch.cuda.synchronize()
        barrier()
        ctx.profile(True)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record()
        for i in range(args.steps):
            _, cols = plans.star_plan(ctx, base, fm, out=res)
            plans.free_lifo(ctx, cols)
            evs[i + 1].record()
        barrier()
        prof = ctx.profile_collect()
        ctx.profile(False)
        if clocks:
            w0 = time.perf_counter()
            while time.perf_counter() - w0 < 0.3:
                _, cols = plans.star_plan(ctx, base, fm, out=res)
                plans.free_lifo(ctx, cols)
                torch.cuda.synchronize()
        ck_info = clocks.stop() if clocks else None
        ctx.check(what=f"star {label} timed steps")
        ms_step = max_over_ranks(evs[0].elapsed_time(evs[-1]) / args.steps, world, dev)
        best = min(evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps))
        return {"ms_per_step": round(ms_step, 4), "ms_per_step_best": round(best, 4),
                "rows_per_s": job_rows_per_s(world, n, ms_step),
                "base_bytes": int(base_bytes), "intermediate_bytes": int(inter_bytes),
                "footprint_bytes": int(base_bytes + inter_bytes),
                "arena_peak_intermediates": int(high - use0),
                "device_peak_bytes": int(base_bytes + (high - use0) + ctx.work_bytes()),
                "sums": ms.to_numpy_u64(res).tolist(), "prof": prof, "kernel_bytes": kb,
                "clocks": ck_info, "op_ms_sizing_step": op_ms,
                "per_kernel_ms": {k: round(v[1] / args.steps, 4) for k, v in prof.items()}}

    base_c = plans.compress_base(ctx, raw, plans.STAR_BASE_COMPRESSED)
    ctx.check(what="star base")
    out["compressed"] = run_variant("compressed", base_c, plans.STAR_COMPRESSED)
    out["compressed"]["_base"] = base_c
    # the plan-level format search (Sec. 5.2): greedy per-intermediate runtime choice
    # over the compressed base columns
    t_g = time.perf_counter()
    fm_g, _, evals = plans.greedy_formats(ctx, lambda fm: plans.star_plan(ctx, base_c, fm), plans.STAR_NAMES,
                                          plans.STAR_COMPRESSED, "time", candidates=plans.STAR_CANDIDATES, reps=2)
    search_s = time.perf_counter() - t_g
    out["greedy"] = run_variant("greedy", base_c, fm_g)
    out["greedy"]["formats"] = {k: ms.FORMAT_NAMES[v] for k, v in fm_g.items()}
    out["greedy"]["search"] = {"evaluations": evals, "seconds": round(search_s, 1)}
    base_u = plans.compress_base(ctx, raw, plans.STAR_BASE_UNCOMPRESSED)
    ctx.check(what="star base")
    out["uncompressed"] = run_variant("uncompressed", base_u, plans.STAR_UNCOMPRESSED)
    out["uncompressed"]["_base"] = base_u
    assert out["greedy"]["sums"] == out["compressed"]["sums"], "greedy formats change the result"
    assert out["compressed"]["sums"] == out["uncompressed"]["sums"], "star pipelines disagree"
    comp, unc = out["compressed"], out["uncompressed"]

    # ---- roofline of the dominant kernel of the compressed plan
    per_kernel = {}
    for kname, (launches, total) in comp["prof"].items():
        alg = comp["kernel_bytes"].get(kname)
        per_step_ms = total / args.steps
        per_kernel[kname] = {"launches_per_step": launches // args.steps, "ms_per_step": round(per_step_ms, 4),
                             "alg_bytes_per_step": alg,
                             "alg_GBps": None if not alg else round(alg / (per_step_ms * 1e-3) / 1e9, 1)}
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms_per_step"])
    peak, peak_kind = peaks()
    ach = per_kernel[dom]["alg_GBps"]
    lps = max(per_kernel[dom]["launches_per_step"], 1)
    plan_bytes = sum(v for v in comp["kernel_bytes"].values())

    # ---- end to end through the C ABI: every step imports the base columns from
    # pinned host memory in their format, runs the plan and reads the sums back
    def e2e_run(label, base_fm, fm):
        base = out[label]["_base"]
        host = {k: ctx.export_bytes(c, pinned=True) for k, c in base.items()}
        rows = {k: ctx.info(c)["n"] for k, c in base.items()}
        hres = torch.zeros(plans.STAR_GROUPS, dtype=torch.int64).pin_memory()
        res = torch.zeros(plans.STAR_GROUPS, dtype=torch.int64, device=dev)

        def step():
            imp = {k: ctx.import_bytes(base_fm[k], rows[k], host[k], bw=plans.base_width(k, base_fm[k])) for k in base}
            _, cols = plans.star_plan(ctx, imp, fm, out=res)
            plans.free_lifo(ctx, cols)
            hres.copy_(res, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            for c in reversed(list(imp.values())):
                ctx.free(c)

        for _ in range(args.warmup):
            step()
        barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            step()
        barrier()
        ms_e = max_over_ranks((time.perf_counter() - t) * 1e3 / args.steps, world, dev)
        assert hres.numpy().view(np.uint64).tolist() == comp["sums"], "end-to-end sums differ"
        h2d = int(sum(h.numel() for h in host.values()))
        del host
        return {"value": job_rows_per_s(world, n, ms_e), "unit": "rows/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 8 * plans.STAR_GROUPS, "ms_per_step": round(ms_e, 3)}

    e2e = e2e_unc = None
    if not args.no_e2e:
        e2e = e2e_run("compressed", plans.STAR_BASE_COMPRESSED, plans.STAR_COMPRESSED)
        e2e_unc = e2e_run("uncompressed", plans.STAR_BASE_UNCOMPRESSED, plans.STAR_UNCOMPRESSED)
    for label in ("uncompressed", "compressed"):
        for c in reversed(list(out[label].pop("_base").values())):
            ctx.free(c)
    ctx.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = star_cpu_baseline(args.seed, n)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return None
    clocks = comp.get("clocks")
    launches = int(sum(p["launches_per_step"] for p in per_kernel.values()) * args.steps)
    greedy = out["greedy"]
    for v in (comp, unc, greedy):
        for k in ("sums", "prof", "kernel_bytes", "clocks"):
            v.pop(k, None)
    greedy["speedup_vs_uncompressed"] = round(unc["ms_per_step"] / greedy["ms_per_step"], 3)
    greedy["footprint_ratio"] = round(greedy["footprint_bytes"] / unc["footprint_bytes"], 4)
    return {
        "metric": METRIC, "value": comp["rows_per_s"], "unit": "rows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": comp["ms_per_step"],
        "ms_per_step_best": comp["ms_per_step_best"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded SplitMix64, generated on the GPU)",
        "config": {"workload": STAR_WORKLOAD, "fact_rows": n, "dimension_rows": list(synth.DIM_SIZES),
                   "formats": "base: columns read at positions static BP, fk_date DELTA+BP, scanned columns "
                              "dynamic BP; intermediates: positions DELTA+BP, values static BP at their "
                              "domain's width",
                   "l2": "inputs larger than L2 (compressed fact columns %.2f GB)" % (comp["base_bytes"] / 1e9),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": None if ach is None else round(ach / peak, 4), "peak_kind": peak_kind,
                     "traffic": measured_traffic("star_" + dom),
                     "alg_bytes_per_launch": None if not per_kernel[dom]["alg_bytes_per_step"]
                     else int(per_kernel[dom]["alg_bytes_per_step"] / lps),
                     "launches_per_step": lps},
        "per_kernel": per_kernel,
        "plan_alg_GBps": round(plan_bytes / (comp["ms_per_step"] * 1e-3) / 1e9, 1),
        "compressed": comp, "uncompressed": dict(unc, e2e=e2e_unc), "compressed_greedy_formats": greedy,
        "speedup_vs_uncompressed": round(unc["ms_per_step"] / comp["ms_per_step"], 3),
        "footprint_ratio": round(comp["footprint_bytes"] / unc["footprint_bytes"], 4),
        "device_peak_ratio": round(comp["device_peak_bytes"] / unc["device_peak_bytes"], 4),
        "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
    }


def bench_reference_star(args, world):
    """Reference arm of the star workload: the oracle as it stands, on one host core,
    each step a bounded prefix sample of the same fact table."""
    n = args.rows or 600_000_000
    per_step_s = max(2.0, min(20.0, 150.0 / max(args.steps + args.warmup, 1)))
    rows = min(n, star_cpu_sample_rows(args.seed, per_step_s))
    f, d = star_host_sample(args.seed, rows)
    fw, dw = star_host_sample(args.seed, 1 << 16)
    for _ in range(args.warmup):
        oracle_star_plan(fw, dw)
    times = [oracle_star_plan(f, d)[0] for _ in range(args.steps)]
    tot = sum(times)
    value = rows * args.steps / tot
    from paper_2004_09350_gb300 import synth
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded SplitMix64)",
            "config": {"workload": STAR_WORKLOAD, "fact_rows": n, "dimension_rows": list(synth.DIM_SIZES),
                       "parallelism": "1 host core"},
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "host": host_info(), "kind": "oracle",
                             "build": "gcc -O2, single thread, not pinned to a core",
                             "sample": f"first {rows} of the {n} fact rows per step, the same plan with every "
                                       f"column passed through the oracle's codec in the compressed formats"},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------- learned selector

PLAN_INTERMEDIATES = ("P", "X'", "K'", "Y")


def plan_time(ctx, cx, ck, c, fm, res, reps=3):
    import torch
    for _ in range(2):
        free_all(ctx, run_plan(ctx, cx, ck, c, fm, res))
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        free_all(ctx, run_plan(ctx, cx, ck, c, fm, res))
    t1.record()
    t1.synchronize()
    return t0.elapsed_time(t1) / reps


def bench_selector(args):
    import torch
    from paper_2004_09350_gb300 import morphstore as ms
    from paper_2004_09350_gb300 import plans, selector, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = ms.Ctx(0, arena_bytes=4 << 30, max_rows=1 << 26)
    # ---- 1. traces: every intermediate compressed into every format (items are
    # generated and labelled one at a time)
    t_h = time.perf_counter()
    items = selector.synthetic_intermediates(args.seed, args.selector_items, lo_log2=16,
                                             hi_log2=args.selector_max_log2)
    X, Y, S, T, names = selector.harvest(ctx, items, reps=2)
    harvest_s = time.perf_counter() - t_h
    # longer traces (2^20 .. 2^24 rows), all trained on: run times grow with the length
    # in ways the short traces alone do not show
    t_m = time.perf_counter()
    mid = selector.synthetic_intermediates(args.seed + 55, args.selector_mid_items, lo_log2=20, hi_log2=24)
    XM, YM, _, _, _ = selector.harvest(ctx, mid, reps=1)
    mid_s = time.perf_counter() - t_m
    # a held-out set of long intermediates (2^22 .. 2^26 rows), never trained on
    t_l = time.perf_counter()
    big = selector.synthetic_intermediates(args.seed + 99, args.selector_large_items, lo_log2=22, hi_log2=26)
    XL, _, SL, TL, _ = selector.harvest(ctx, big, reps=1)
    large_s = time.perf_counter() - t_l
    ctx.close()
    idx = np.random.default_rng(args.seed).permutation(len(X))
    cut = int(0.8 * len(X))
    tr, te = idx[:cut], idx[cut:]
    # ---- 2. training with the library's kernels
    sel = selector.Selector(dev, seed=args.seed)
    t_t = time.perf_counter()
    Xtr, Ytr = (np.concatenate([X[tr], XM]), np.concatenate([Y[tr], YM])) if len(XM) else (X[tr], Y[tr])
    hist = sel.train(Xtr, Ytr, epochs=800, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t_t
    held = {}
    for obj, feats_, costs in (("size", X[te], S[te]), ("time", X[te], T[te]), ("size_long", XL, SL),
                               ("time_long", XL, TL)):
        chosen = sel.choose(feats_, obj.split("_")[0])
        held[obj] = {"regret": round(selector.regret(chosen, costs), 4),
                     "static_bp_for_all_regret": round(selector.regret(np.full(len(costs), 1), costs), 4),
                     "best_fixed_format_regret": round(min(selector.regret(np.full(len(costs), f), costs)
                                                           for f in range(5)), 4)}
    # ---- 3. the 2^28-row plan with formats picked from a prefix sample
    n = args.rows
    x, k, c = make_inputs(n, args.seed, args.selectivity)
    ctx = ms.Ctx(0, arena_bytes=int(2.5 * 8 * n) + (1 << 30), max_rows=n)
    res = torch.zeros(1, dtype=torch.int64, device=dev)
    cx = ctx.compress(ms.as_device_u64(x, dev), ms.DYN_BP)
    ck = ctx.compress(ms.as_device_u64(k, dev), ms.DELTA_BP)
    sample = 1 << 16
    sx = ctx.compress(ms.as_device_u64(x[:sample], dev), ms.UNCOMPR)
    sk = ctx.compress(ms.as_device_u64(k[:sample], dev), ms.UNCOMPR)
    cols = run_plan(ctx, sx, sk, c, UNCOMPRESSED, res)  # [Y, K', X', P]
    ops = {"P": ("select", False), "X'": ("project", False), "K'": ("project", False), "Y": ("calc", False)}
    feats = {name: selector.column_features(ctx, col, *ops[name], n_scale=n / sample)
             for name, col in zip(("Y", "K'", "X'", "P"), cols)}
    free_all(ctx, cols)
    for col in (sk, sx):
        ctx.free(col)
    picks = {name: int(sel.choose(feats[name], "time", allowed=plans.PLAN_CANDIDATES)[0])
             for name in PLAN_INTERMEDIATES}
    fm_sel = {name: ms.FORMAT_NAMES[picks[name]] for name in PLAN_INTERMEDIATES}
    # greedy per-intermediate runtime search (Sec. 5.2) over the plan's intermediates
    # (plans.greedy_formats; static BP is not a candidate: its width must be known
    # before the intermediate exists)
    run = lambda fm: plans.select_project_calc_sum(ctx, cx, ck, c, fm, out=res)  # noqa: E731  (format ids)
    names_fm = {k2: v for k2, v in COMPRESSED.items() if k2 in PLAN_INTERMEDIATES}
    g_fm, _, _ = plans.greedy_formats(ctx, run, PLAN_INTERMEDIATES,
                                      {k2: fmt_id(v) for k2, v in names_fm.items()}, "time", reps=3)
    fm_g = dict(COMPRESSED, **{k2: ms.FORMAT_NAMES[v] for k2, v in g_fm.items()})
    t_sel = plan_time(ctx, cx, ck, c, dict(COMPRESSED, **fm_sel), res, reps=10)
    t_greedy = plan_time(ctx, cx, ck, c, fm_g, res, reps=10)
    t_fixed = plan_time(ctx, cx, ck, c, COMPRESSED, res, reps=10)
    ctx.check(what="selector plans")
    ctx.close()
    return {"workload": "selector", "metric": "learned format selector: regret vs exhaustive choice",
            "items": len(X), "train_items": len(tr), "heldout_items": len(te), "long_heldout_items": len(XL),
            "mid_train_items": len(XM), "rows_log2": [16, args.selector_max_log2], "mid_rows_log2": [20, 24],
            "long_rows_log2": [22, 26],
            "harvest_s": round(harvest_s, 1), "mid_harvest_s": round(mid_s, 1), "long_harvest_s": round(large_s, 1),
            "train_s": round(train_s, 2),
            "loss_first_last": [hist[0][1], hist[-1][1]], "heldout": held,
            "plan_2e28": {"rows": n, "selector_formats": fm_sel, "greedy_formats": {k2: fm_g[k2] for k2 in PLAN_INTERMEDIATES},
                          "ms_selector": round(t_sel, 4), "ms_greedy_search": round(t_greedy, 4),
                          "ms_fixed_formats": round(t_fixed, 4),
                          "regret_vs_greedy": round(t_sel / t_greedy - 1.0, 4)},
            "note": "time labels: write + one read of the intermediate; static BP excluded from the plan search "
                    "because its width must be known before the intermediate exists"}


# ------------------------------------------------------- batched fragments

def _events_ms(fn, steps, stream):
    """Per-step device milliseconds of fn() (CUDA events on `stream`)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in ev]


def oracle_fragment(sp):
    import oracle
    from paper_2004_09350_gb300 import synth
    x, y = synth.batch_x(sp), synth.batch_y(sp)
    t = time.perf_counter()
    pos = oracle.select(x, sp["cmp"], sp["c1"], sp["c2"])
    s = oracle.agg_sum(oracle.project(y, pos))
    return s, time.perf_counter() - t


def column_bound(n, fmt, bits):
    """Upper bound of a column's bytes in `fmt` for values of at most `bits` bits."""
    nb = n // BLOCK
    if fmt == 0:
        return 8 * n
    if fmt == 1:
        return (n * bits + 63) // 64 * 8
    w = 64 if fmt == 3 else bits
    return 16 * nb + nb * 64 * w + 8 * (n % BLOCK) + 256


def bench_batch(args):
    import torch
    from paper_2004_09350_gb300 import autotune, selector, synth
    from paper_2004_09350_gb300 import morphstore as ms

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    F = args.fragments
    specs = synth.batch_fragments(args.seed, F, lo_log2=10, hi_log2=args.batch_max_log2)
    rows = sum(sp["n"] for sp in specs)
    max_n = max(sp["n"] for sp in specs)
    # ---- 1. the format selector, trained on engine traces with the library's kernels
    t_s = time.perf_counter()
    hctx = ms.Ctx(0, arena_bytes=1 << 30, max_rows=1 << 18)
    items = list(selector.synthetic_intermediates(args.seed + 1, args.batch_train_items, lo_log2=12, hi_log2=18))
    X, Y, _, _, _ = selector.harvest(hctx, items, reps=1)
    hctx.close()
    sel = selector.Selector(dev, seed=args.seed)
    sel.train(X, Y, epochs=800, lr=3e-3)
    # ---- 2. statistics of every base column, then one batched prediction
    gens = (synth.batch_x_torch, synth.batch_y_torch)
    sctx = ms.Ctx(0, arena_bytes=8 * max_n + (64 << 20), max_rows=max_n)
    stats = torch.zeros((2 * F, ms.STATS_WORDS), dtype=torch.int64, device=dev)
    for f, sp in enumerate(specs):
        for j in range(2):
            col = sctx.compress(gens[j](sp, dev), ms.UNCOMPR)
            sctx.column_stats(col, out=stats[2 * f + j])
            sctx.free(col)
    sctx.check(what="batch statistics")
    sctx.close()
    st = stats.cpu().numpy().view(np.uint64)
    feats = np.stack([selector.features_from_stats(st[i], "base") for i in range(2 * F)])
    fmts = sel.choose(feats, "size", allowed=(ms.STATIC_BP, ms.DYN_BP, ms.DELTA_BP, ms.FOR_BP))
    bits = [max(1, int(st[i][1]).bit_length()) for i in range(2 * F)]
    setup_sel_s = time.perf_counter() - t_s
    # ---- 3. the base columns in the chosen formats
    arena = sum(column_bound(specs[i // 2]["n"], int(fmts[i]), bits[i]) for i in range(2 * F)) + (1 << 30)
    ctx = ms.Ctx(0, arena_bytes=arena, max_rows=max_n)
    cols = []
    for f, sp in enumerate(specs):
        for j in range(2):
            i = 2 * f + j
            cols.append(ctx.compress(gens[j](sp, dev), int(fmts[i]), bits[i] if fmts[i] == ms.STATIC_BP else 0))
    ctx.check(what="batch base columns")
    batch = ms.Batch(ctx, cols[0::2], cols[1::2], [sp["cmp"] for sp in specs], [sp["c1"] for sp in specs],
                     [sp["c2"] for sp in specs])
    info = batch.info()
    sums = torch.zeros(F, dtype=torch.int64, device=dev)
    # ---- 4. autotuning (every candidate gives the same bits)
    best, table = autotune.tune(batch, sums, reps=3, use_cache=False)
    default_ms = table.get(ms.DEFAULT_BATCH_CONFIG) or autotune.time_config(batch, sums, ms.DEFAULT_BATCH_CONFIG)
    # ---- 5. timing: one persistent launch (graph) vs one launch per fragment
    g_one = batch.graph(sums, cfg=best)
    for _ in range(args.warmup):
        g_one.launch(stream)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    t_wall = time.perf_counter()
    one = _events_ms(lambda: g_one.launch(stream), args.steps, stream)
    while time.perf_counter() - t_wall < 1.0:  # let the clock sampler see the load
        one += _events_ms(lambda: g_one.launch(stream), args.steps, stream)
    clk = clocks.stop()
    got = ms.to_numpy_u64(sums).copy()
    ctx.profile(True)
    for _ in range(args.steps):
        batch.run(sums, cfg=best, stream=stream)
    prof = ctx.profile_collect()
    ctx.profile(False)
    k_ms = prof["batch"][1] / prof["batch"][0]
    each = _events_ms(lambda: batch.run(sums, cfg=best, per_fragment=True, stream=stream), args.warmup, stream)
    each = _events_ms(lambda: batch.run(sums, cfg=best, per_fragment=True, stream=stream), args.steps, stream)
    got_each = ms.to_numpy_u64(sums).copy()
    g_each = batch.graph(sums, cfg=best, per_fragment=True)
    _events_ms(lambda: g_each.launch(stream), args.warmup, stream)
    each_g = _events_ms(lambda: g_each.launch(stream), args.steps, stream)
    g_each.close()
    ctx.check(what="batch runs")
    # operator-at-a-time per fragment: ms_select -> ms_project -> ms_agg_sum
    res = torch.zeros(F, dtype=torch.int64, device=dev)

    def op_at_a_time():
        for f in range(F):
            pos = ctx.select(cols[2 * f], specs[f]["cmp"], specs[f]["c1"], specs[f]["c2"], fmt=ms.DELTA_BP)
            yv = ctx.project(cols[2 * f + 1], pos, fmt=ms.DYN_BP)
            ctx.agg_sum(yv, out=res[f:f + 1])
            ctx.free(yv)
            ctx.free(pos)
    op_at_a_time()
    ops_ms = _events_ms(op_at_a_time, 1, stream)[0]
    ctx.check(what="operator-at-a-time fragments")
    got_ops = ms.to_numpy_u64(res).copy()
    assert (got == got_each).all() and (got == got_ops).all(), "batched runs disagree"
    # ---- 6. parity against the oracle on sampled fragments, and the CPU baseline
    order = np.argsort([sp["n"] for sp in specs])
    rng = np.random.default_rng(args.seed)
    sample = sorted(set(order[-4:].tolist()) | set(order[:4].tolist()) | set(rng.choice(F, 4, replace=False).tolist()))
    mism, cpu_rows, cpu_t = 0, 0, 0.0
    for f in sample:
        want, t = oracle_fragment(specs[f])
        mism += int(want != int(got[f]))
        cpu_rows += specs[f]["n"]
        cpu_t += t
    med = statistics.median(one)
    peak, peak_kind = peaks()
    achieved = info["bytes"] / (k_ms * 1e-3) / 1e9
    batch.close()
    g_one.close()
    counts = {ms.FORMAT_NAMES[k]: int((fmts == k).sum()) for k in range(5)}
    ctx.close()
    return {
        "metric": "aggregate rows/s of batched select->project->agg_sum fragments", "workload": "batch",
        "value": rows / (med * 1e-3), "unit": "rows/s", "n_gpus": 1, "steps": len(one), "warmup": args.warmup,
        "ms_per_step": round(med, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic (seeded SplitMix64, generated on the GPU)",
        "config": {"workload": f"{F} fragments sum(y[i] for x[i] <cmp> c), lengths log-uniform in "
                               f"[2^10, 2^{args.batch_max_log2:g}], x ~ U[0,2^bx), y uniform/offset/sorted/skewed "
                               f"at width by, bx, by ~ U[1,40]; base formats chosen by the learned selector",
                   "fragments": F, "rows": info["rows"], "chunks": info["chunks"], "bytes": info["bytes"],
                   "l2": "inputs larger than L2 (no flush)", "launch": "one persistent launch in a CUDA graph"},
        "gb_per_s": info["bytes"] / (med * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": (None if measured_traffic("batch", "dram_per_algorithmic_byte") is None
                                 else int(measured_traffic("batch", "dram_per_algorithmic_byte") * info["bytes"])),
                     "kernel": "k_batch", "kernel_ms": round(k_ms, 4)},
        "per_fragment_launches": {"ms_per_step": round(statistics.median(each), 3),
                                  "rows_per_s": rows / (statistics.median(each) * 1e-3),
                                  "speedup_of_one_launch": round(statistics.median(each) / med, 2)},
        "per_fragment_graph": {"ms_per_step": round(statistics.median(each_g), 3),
                               "speedup_of_one_launch": round(statistics.median(each_g) / med, 2)},
        "operator_at_a_time": {"ms_per_step": round(ops_ms, 2), "speedup_of_one_launch": round(ops_ms / med, 1)},
        "autotune": {"best": list(best), "best_ms": round(table[best], 4), "default_ms": round(default_ms, 4),
                     "worst_ms": round(max(table.values()), 4), "candidates": len(table)},
        "selector": {"train_items": len(X), "setup_s": round(setup_sel_s, 1), "base_formats": counts},
        "parity": {"sampled_fragments": len(sample), "mismatches": mism, "all_launch_modes_agree": True},
        "cpu_baseline": {"value": cpu_rows / cpu_t, "unit": "rows/s", "cores": 1, "host": host_info(), "kind": "oracle",
                         "sample": f"{len(sample)} fragments ({cpu_rows} rows) through the oracle's "
                                   f"select, project and agg_sum ({cpu_t:.1f} s)"},
        "clocks": clk, "gpu_launches": len(one),
    }


# ------------------------------------------------------------ format sweep table

def bench_sweep_table(args):
    """The format sweep at --rows (default 2^28): every operator of the plain plan for
    every input/output format pair, timed on its own (CUDA events, mean of --steps
    after 3 warm-ups): select X < c for X in 5 formats x positions in 5 formats at
    selectivities 0.1%, 10%, 90%; the specialized select on packed X; project X at
    the 10% positions (DELTA) for 5 data x 5 output formats, and uncompressed X at
    positions in 5 formats; calc X' * K' with both inputs in one of 5 formats x 5
    output formats; agg_sum of X in 5 formats.  Reports ms and logical rows/s
    (select, agg_sum: X's rows; project, calc: output rows)."""
    import torch
    from paper_2004_09350_gb300 import morphstore as ms

    n = args.rows
    x, k, _ = make_inputs(n, args.seed, 0.1)
    from paper_2004_09350_gb300 import synth
    dev = torch.device("cuda", 0)
    ctx = ms.Ctx(0, arena_bytes=int(14 * 8 * n) + (1 << 30), max_rows=n)
    bx = max(1, int(x.max()).bit_length())
    bk = max(1, int(k.max()).bit_length())
    F = list(range(5))
    dx, dk = ms.as_device_u64(x, dev), ms.as_device_u64(k, dev)
    X = {f: ctx.compress(dx, f, bx if f == ms.STATIC_BP else 0) for f in F}
    K = {f: ctx.compress(dk, f, bk if f == ms.STATIC_BP else 0) for f in F}
    del dx, dk
    ctx.check(what="sweep base columns")
    res = torch.zeros(1, dtype=torch.int64, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / args.steps

    name = ms.FORMAT_NAMES
    out = {"rows": n, "x_bytes": {name[f]: ctx.info(X[f])["size_bytes"] for f in F},
           "k_bytes": {name[f]: ctx.info(K[f])["size_bytes"] for f in F},
           "select": {}, "select_packed": {}, "project": {}, "project_positions": {}, "calc": {}, "agg_sum": {}}
    for sel in (0.001, 0.1, 0.9):
        c = synth.value_at_rank(x, sel)
        for fi in F:
            for fo in F:
                bwo = 0
                if fo == ms.STATIC_BP:
                    bwo = max(1, (n - 1).bit_length())
                t = timed(lambda: ctx.free(ctx.select(X[fi], ms.LT, c, fmt=fo, bw=bwo)))
                out["select"][f"{sel}|{name[fi]}|{name[fo]}"] = {"ms": round(t, 4), "rows_per_s": n / (t * 1e-3)}
            if fi != ms.UNCOMPR:
                t = timed(lambda: ctx.free(ctx.select_packed(X[fi], ms.LT, c, fmt=ms.DELTA_BP)))
                out["select_packed"][f"{sel}|{name[fi]}|delta_bp"] = {"ms": round(t, 4), "rows_per_s": n / (t * 1e-3)}
        ctx.check(what=f"select sweep {sel}")
    c = synth.value_at_rank(x, 0.1)
    P = ctx.select(X[ms.DYN_BP], ms.LT, c, fmt=ms.DELTA_BP)
    m = ctx.info(P)["n"]
    bxo = bx
    for fi in F:
        for fo in F:
            t = timed(lambda: ctx.free(ctx.project(X[fi], P, fmt=fo, bw=bxo if fo == ms.STATIC_BP else 0)))
            out["project"][f"{name[fi]}|{name[fo]}"] = {"ms": round(t, 4), "rows_per_s": m / (t * 1e-3)}
    ctx.check(what="project sweep")
    Pf = {f: ctx.morph(P, f, max(1, (n - 1).bit_length()) if f == ms.STATIC_BP else 0) for f in F}
    for fp in F:
        t = timed(lambda: ctx.free(ctx.project(X[ms.UNCOMPR], Pf[fp], fmt=ms.UNCOMPR)))
        out["project_positions"][f"{name[fp]}|uncompr"] = {"ms": round(t, 4), "rows_per_s": m / (t * 1e-3)}
    ctx.check(what="position-format sweep")
    for fi in F:
        xp = ctx.project(X[ms.UNCOMPR], P, fmt=fi, bw=bx if fi == ms.STATIC_BP else 0)
        kp = ctx.project(K[ms.UNCOMPR], P, fmt=fi, bw=bk if fi == ms.STATIC_BP else 0)
        for fo in F:
            # static BP output: the products need up to bx + bk bits
            bwo = min(64, bx + bk) if fo == ms.STATIC_BP else 0
            t = timed(lambda: ctx.free(ctx.calc(ms.MUL, xp, kp, fmt=fo, bw=bwo)))
            out["calc"][f"{name[fi]}|{name[fo]}"] = {"ms": round(t, 4), "rows_per_s": m / (t * 1e-3)}
        ctx.free(kp)
        ctx.free(xp)
    ctx.check(what="calc sweep")
    for fi in F:
        t = timed(lambda: ctx.agg_sum(X[fi], out=res))
        out["agg_sum"][name[fi]] = {"ms": round(t, 4), "rows_per_s": n / (t * 1e-3)}
    ctx.check(what="agg_sum sweep")
    out["positions"] = m

    # direct morphs (Sec. 3.2, on-the-fly morphing) of X for every ordered format pair,
    # against the round trip through uint64 (decompress into a buffer, compress again);
    # algorithmic bytes: bytes(input) + bytes(output)
    xb = out["x_bytes"]
    buf = torch.empty(n, dtype=torch.int64, device=dev)
    out["morph"], out["morph_staged"] = {}, {}
    for fi in F:
        for fo in F:
            bwo = bx if fo == ms.STATIC_BP else 0
            t = timed(lambda: ctx.free(ctx.morph(X[fi], fo, bwo)))
            gbps = (xb[name[fi]] + xb[name[fo]]) / (t * 1e6)
            out["morph"][f"{name[fi]}|{name[fo]}"] = {"ms": round(t, 4), "rows_per_s": n / (t * 1e-3),
                                                      "alg_GBps": round(gbps, 1)}
            t = timed(lambda: (ctx.decompress(X[fi], out=buf), ctx.free(ctx.compress(buf, fo, bwo))))
            out["morph_staged"][f"{name[fi]}|{name[fo]}"] = {"ms": round(t, 4), "rows_per_s": n / (t * 1e-3)}
    ctx.check(what="morph sweep")

    # RLE (Sec. 2.1) against uncompressed, dynamic BP and DELTA+BP on a column of long
    # runs (run lengths uniform in [1, 7999], 6 distinct values: a sorted low-cardinality
    # column's shape), every operator that reads it, and the encoders
    r = synth.runs(args.seed + 5, n, 4000)
    dr = ms.as_device_u64(r, dev)
    RF = [ms.UNCOMPR, ms.DYN_BP, ms.DELTA_BP, ms.RLE]
    Rc = {f: ctx.compress(dr, f) for f in RF}
    rb = {name[f]: ctx.info(Rc[f])["size_bytes"] for f in RF}
    rle = {"runs": ctx.info(Rc[ms.RLE])["n_blocks"], "bytes": rb, "compress": {}, "decompress": {},
           "morph_from_dyn_bp": {}, "select": {}, "agg_sum": {}, "project": {}}
    for f in RF:
        fn = name[f]
        t = timed(lambda: ctx.free(ctx.compress(dr, f)))
        rle["compress"][fn] = {"ms": round(t, 4), "alg_GBps": round((8 * n + rb[fn]) / (t * 1e6), 1)}
        t = timed(lambda: ctx.decompress(Rc[f], out=buf))
        rle["decompress"][fn] = {"ms": round(t, 4), "alg_GBps": round((8 * n + rb[fn]) / (t * 1e6), 1)}
        t = timed(lambda: ctx.free(ctx.morph(Rc[ms.DYN_BP], f)))
        rle["morph_from_dyn_bp"][fn] = {"ms": round(t, 4),
                                       "alg_GBps": round((rb["dyn_bp"] + rb[fn]) / (t * 1e6), 1)}
        t = timed(lambda: ctx.free(ctx.select(Rc[f], ms.LT, 1, fmt=ms.DELTA_BP)))
        rle["select"][fn] = {"ms": round(t, 4), "rows_per_s": n / (t * 1e-3)}
        t = timed(lambda: ctx.agg_sum(Rc[f], out=res))
        rle["agg_sum"][fn] = {"ms": round(t, 4), "rows_per_s": n / (t * 1e-3),
                             "alg_GBps": round(rb[fn] / (t * 1e6), 1)}
        t = timed(lambda: ctx.free(ctx.project(Rc[f], P, fmt=ms.UNCOMPR)))
        rle["project"][fn] = {"ms": round(t, 4), "rows_per_s": m / (t * 1e-3)}
    ctx.check(what="rle sweep")
    rle["select_selectivity"] = float(np.count_nonzero(r < 1)) / n
    out["rle"] = rle
    for f in reversed(RF):
        ctx.free(Rc[f])
    del dr

    # FOR / DELTA cascaded with static BP against the dynamic cascades: K (sorted) as
    # DELTA, X as FOR, the static width the column's widest block needs
    cas = {}
    for col, dyn, stat in (("K", K[ms.DELTA_BP], ms.DELTA_STATIC_BP), ("X", X[ms.FOR_BP], ms.FOR_STATIC_BP)):
        src = k if col == "K" else x
        bws = max(1, int(oracle_free_block_width(src, stat == ms.DELTA_STATIC_BP)))
        dsrc = ms.as_device_u64(src, dev)
        sc = ctx.compress(dsrc, stat, bws)
        e = {"static_bw": bws, "bytes": {name[ctx.info(dyn)["fmt"]]: ctx.info(dyn)["size_bytes"],
                                          name[stat]: ctx.info(sc)["size_bytes"]}}
        for key, cc, fm, bw_ in (("dyn", dyn, ctx.info(dyn)["fmt"], 0), ("static", sc, stat, bws)):
            e[key] = {
                "compress_ms": round(timed(lambda: ctx.free(ctx.compress(dsrc, fm, bw_))), 4),
                "decompress_ms": round(timed(lambda: ctx.decompress(cc, out=buf)), 4),
                "agg_sum_ms": round(timed(lambda: ctx.agg_sum(cc, out=res)), 4),
                "project_ms": round(timed(lambda: ctx.free(ctx.project(cc, P, fmt=ms.UNCOMPR))), 4)}
        cas[col] = e
        ctx.free(sc)
        del dsrc
    ctx.check(what="cascade sweep")
    out["static_cascades"] = cas
    ctx.close()
    return {"workload": "sweep-table", "metric": METRIC, **out}


def oracle_free_block_width(x: np.ndarray, delta: bool) -> int:
    """The widest 512-value block's residual width (DELTA: differences to the
    predecessor within the block; FOR: distance to the block minimum), from numpy."""
    nb = x.size // BLOCK
    if nb == 0:
        return 1
    b = x[: nb * BLOCK].reshape(nb, BLOCK)
    if delta:
        r = np.diff(b, axis=1)  # sorted input: no wrap-around
    else:
        r = b - b.min(axis=1, keepdims=True)
    return int(r.max()).bit_length()


def render_sweep_table(t: dict) -> str:
    """Markdown of a sweep-table line (--render-sweep-table FILE)."""
    F = ["uncompr", "static_bp", "dyn_bp", "delta_bp", "for_bp"]
    L = ["# Format sweep at 2^28 rows: every operator for every input/output format pair\n",
         "Columns: X with per-512-block widths in {3, 8, 16, 27, 40} (values below 2^b), K sorted with gaps",
         "Geometric(1/4); select X < c at three selectivities; project X and K at the positions of the 10%",
         f"select ({t['positions']:,} positions, DELTA+BP); calc X' * K'; agg_sum; morph X between every pair",
         "of formats; RLE on a column of long runs.  Milliseconds per call (CUDA events, mean of the timed",
         "calls after 3 warm-ups, every kernel of the call included: mark, scan, emit and placement for",
         "select).  One GB300.\n",
         "Command (committed files only): `python bench.py --workload sweep-table --steps 5`, rendered by",
         "`python bench.py --render-sweep-table <its JSON line>`.\n",
         "Column sizes (bytes): " + ", ".join(f"X {k} {v / 1e6:.0f} MB" for k, v in t["x_bytes"].items()) + "; "
         + ", ".join(f"K {k} {v / 1e6:.0f} MB" for k, v in t["k_bytes"].items()) + ".\n"]

    def grid(title, key, fmt_key, rows=F, cols=F, head="in \\ out"):
        L.append(title + "\n")
        L.append(f"| {head} | " + " | ".join(cols) + " |")
        L.append("|---|" + "---|" * len(cols))
        for a in rows:
            L.append(f"| {a} | " + " | ".join(f"{t[key][fmt_key(a, b)]['ms']:.3f}" for b in cols) + " |")
        L.append("")

    for sel in ("0.001", "0.1", "0.9"):
        grid(f"## select X < c, selectivity {float(sel) * 100:g}% (rows: X format; columns: positions format)",
             "select", lambda a, b, s=sel: f"{s}|{a}|{b}", head="X \\ out")
        sp = t["select_packed"]
        L.append("Specialized select on the packed codes (`ms_select_packed`, DELTA+BP positions): "
                 + ", ".join(f"{a} {sp[f'{sel}|{a}|delta_bp']['ms']:.3f}" for a in F if f"{sel}|{a}|delta_bp" in sp)
                 + " (general select with the same output: "
                 + ", ".join(f"{a} {t['select'][f'{sel}|{a}|delta_bp']['ms']:.3f}" for a in F if a != "uncompr")
                 + ").\n")
    grid("## project (rows: data format; columns: output format), 10% positions", "project",
         lambda a, b: f"{a}|{b}", head="data \\ out")
    L.append("Positions column format (X uncompressed, uncompressed output): "
             + ", ".join(f"{k.split('|')[0]} {v['ms']:.3f}" for k, v in t["project_positions"].items()) + ".\n")
    grid("## calc X' * K' (rows: X' format; columns: output format)", "calc", lambda a, b: f"{a}|{b}",
         head="X' \\ out")
    L.append("## agg_sum of X\n")
    L.append(" | ".join(f"{k} {v['ms']:.3f} ms ({v['rows_per_s'] / 1e9:.0f} G rows/s)"
                        for k, v in t["agg_sum"].items()) + "\n")
    if "morph" in t:
        grid("## morph X (Sec. 3.2 direct morphing; rows: from; columns: to)", "morph", lambda a, b: f"{a}|{b}",
             head="from \\ to")
        grid("The same through uint64 (ms_decompress into a buffer, then ms_compress):", "morph_staged",
             lambda a, b: f"{a}|{b}", head="from \\ to")
        L.append("Algorithmic GB/s of the direct morphs (bytes in + bytes out): "
                 + ", ".join(f"{k} {v['alg_GBps']:.0f}" for k, v in t["morph"].items()) + ".\n")
    if "rle" in t:
        r = t["rle"]
        RF = list(r["bytes"])
        L.append(f"## RLE on a column of long runs ({r['runs']:,} runs; run lengths uniform in [1, 7999], 6 values)\n")
        L.append("| operation | " + " | ".join(RF) + " |")
        L.append("|---|" + "---|" * len(RF))
        L.append("| bytes | " + " | ".join(f"{r['bytes'][f] / 1e6:.1f} MB" for f in RF) + " |")
        for op, what in (("compress", "compress from uint64"), ("decompress", "decompress to uint64"),
                         ("morph_from_dyn_bp", "morph from dynamic BP"),
                         ("select", f"select x < 1 ({100 * r['select_selectivity']:.1f}%), DELTA+BP positions"),
                         ("agg_sum", "agg_sum"), ("project", "project at the 10% positions of X")):
            L.append(f"| {what} | " + " | ".join(f"{r[op][f]['ms']:.3f}" for f in RF) + " |")
        L.append("")
    if "static_cascades" in t:
        L.append("## FOR / DELTA cascaded with static BP against the dynamic cascades (ms)\n")
        L.append("| column | format | bytes | compress | decompress | agg_sum | project at the 10% positions |")
        L.append("|---|---|---|---|---|---|---|")
        for col, e in t["static_cascades"].items():
            names = list(e["bytes"])
            for key, nm in (("dyn", names[0]), ("static", names[1])):
                d = e[key]
                label = nm + (f" (b = {e['static_bw']})" if key == "static" else "")
                L.append(f"| {col} | {label} | {e['bytes'][nm] / 1e6:.0f} MB | {d['compress_ms']:.3f} | "
                         f"{d['decompress_ms']:.3f} | {d['agg_sum_ms']:.3f} | {d['project_ms']:.3f} |")
        L.append("")
    return "\n".join(L)


# ------------------------------------------------------------ one kernel

def bench_kernel(args):
    """One operator of the plan on the plan's columns (X dynamic BP, K DELTA, positions
    of X < c at 10% as DELTA), built with bench.py's own generators at --rows: 3 warm-up
    and --steps timed calls, per-kernel CUDA-event times.  This is the case the
    profiles' ncu captures run (a few launches on a column larger than L2)."""
    import torch
    from paper_2004_09350_gb300 import morphstore as ms

    from paper_2004_09350_gb300 import synth

    n = args.rows
    x, k, c = make_inputs(n, args.seed, args.selectivity)
    if args.width:
        x = synth.skewed_widths(args.seed, n, widths=(args.width,))
        c = synth.value_at_rank(x, args.selectivity)
    dev = torch.device("cuda", 0)
    ctx = ms.Ctx(0, arena_bytes=int(2.5 * 8 * n) + (1 << 30), max_rows=n)
    fx = fmt_id(args.x_format)
    bw = max(1, int(x.max()).bit_length()) if fx == ms.STATIC_BP and x.size else 0
    cx = ctx.compress(ms.as_device_u64(x, dev), fx, bw)
    ck = ctx.compress(ms.as_device_u64(k, dev), ms.DELTA_BP)
    res = torch.zeros(1, dtype=torch.int64, device=dev)
    pos = ctx.select(cx, ms.LT, c, fmt=ms.DELTA_BP) if args.kernel == "project" else None
    if args.kernel == "project_uniform":
        u = ctx.compress(synth.uniform_torch(args.seed + 7, n, 0, 1 << 20, dev), ms.UNCOMPR)
        pos = ctx.select(u, ms.LT, int(args.selectivity * (1 << 20)), fmt=ms.DELTA_BP)

    raw = ms.as_device_u64(x, dev) if args.kernel in ("compress", "decompress") else None

    def once():
        if args.kernel == "agg_sum":
            ctx.agg_sum(cx, out=res)
        elif args.kernel == "select":
            ctx.free(ctx.select(cx, ms.LT, c, fmt=ms.DELTA_BP))
        elif args.kernel == "select_packed":
            ctx.free(ctx.select_packed(cx, ms.LT, c, fmt=ms.DELTA_BP))
        elif args.kernel == "project_uniform":
            ctx.free(ctx.project(cx, pos, fmt=ms.DYN_BP))
        elif args.kernel == "compress":  # X again, into a fresh arena column
            ctx.free(ctx.compress(raw, fx, bw))
        elif args.kernel == "decompress":  # X into a caller buffer
            ctx.decompress(cx, out=raw)
        else:
            ctx.free(ctx.project(cx, pos, fmt=ms.DYN_BP))
            ctx.free(ctx.project(ck, pos, fmt=ms.DELTA_BP))
    for _ in range(3):
        once()
    torch.cuda.synchronize()
    ctx.profile(True)
    for _ in range(args.steps):
        once()
    prof = ctx.profile_collect()
    ctx.check(what="kernel workload")
    out = {"workload": "kernel", "kernel": args.kernel, "rows": n, "x_format": args.x_format,
           "x_width": args.width or "plan mix",
           "bytes": {"X": ctx.info(cx)["size_bytes"], "K": ctx.info(ck)["size_bytes"]},
           "ms_per_launch": {kk: round(v[1] / v[0], 4) for kk, v in prof.items()}}
    if pos is not None:
        out["positions"] = ctx.info(pos)["n"]
    if args.kernel in ("compress", "decompress"):  # algorithmic bytes: 8n + bytes(col)
        key = "compress" if args.kernel == "compress" else "decompress"
        alg = 8 * n + out["bytes"]["X"]
        ms_k = sum(v for kk, v in out["ms_per_launch"].items() if kk in (key, "place"))
        out["alg_bytes"] = alg
        out["alg_GBps_with_placement"] = round(alg / (ms_k * 1e-3) / 1e9, 1) if ms_k else None
    ctx.close()
    return out


def main():
    args = parse()
    if args.render_sweep_table:
        with open(args.render_sweep_table) as f:
            print(render_sweep_table(json.loads(f.read().strip().splitlines()[-1])))
        return
    if args.workload == "kernel" and args.impl == "ours":
        print(json.dumps(bench_kernel(args)))
        return
    if args.workload == "sweep-table" and args.impl == "ours":
        print(json.dumps(bench_sweep_table(args)))
        return
    if args.workload == "batch" and args.impl == "ours":
        print(json.dumps(bench_batch(args)))
        return
    if args.workload == "selector" and args.impl == "ours":
        print(json.dumps(bench_selector(args)))
        return
    if args.impl == "reference":
        line = bench_reference(args)
    elif args.workload == "star":
        line = bench_star(args)
    else:
        line = bench_ours(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
