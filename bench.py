#!/usr/bin/env python3
"""Benchmark of the fast zeta and Moebius transforms on one GB300 (or N replicas).

One step = one pass of the whole hot path over one synthetic poset function:
the zeta transform (chain scan + niv gather) of f, then the Moebius transform
(forward substitution + V^-1) of the result. The value is node-values/s:
2 * n * B output values per step (n * B from each transform) over the
device time of the step, summed over K steps (CUDA events on the launching
stream; the L2 is flushed between steps, outside the timed events).

Default workload: planted-chain poset n = 2^20, k = 64 chains of 16384, cross
out-degree 3, f fp64 uniform in [-1, 1], B = 1 (plain FP64 GPU form). Extra
lines ("variants") time the same poset with int64 and FP32-compensated values
and the antichain-level Moebius schedule.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mz|reference]

For N > 1, launch under torch.distributed.run: every rank runs an independent
replica (its own poset, seed + rank) with no collective on the data path, and
the value is the sum over ranks divided by the slowest rank's time.
--impl reference times the CPU oracle (exact per-row definition) instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import posetgen as pg  # noqa: E402

METRIC = "zeta & Möbius node-values/s, % HBM peak; FP32-compensated vs FP64 plain"
FP64_ADDS_PER_S = 0.625e12   # GB300 nominal FP64 1.25 TFLOP/s (an FMA counts 2), one add per FMA slot
HOP_FLOOR_US = 0.45          # SM-to-SM store -> poll latency, measured unloaded on GB300
UNIT = "node-values/s"

WORKLOADS = {
    "c1": dict(n=4096, k=16, cross_p=4 / 4096, desc="planted poset n=4096, k=16 chains of 256, cross edges w.p. 4/n"),
    "c2": dict(n=1 << 20, k=64, cross_deg=3,
               desc="planted poset n=2^20, k=64 chains of 16384, cross-chain out-degree 3"),
    "c3": dict(n=1 << 22, k=128, cross_deg=2,
               desc="planted poset n=2^22, k=128 chains of 32768, cross-chain out-degree 2"),
    # the paper's own random DAGs (Sec. 5): Erdos-Renyi, average degree 4 or 6, chains by
    # Alg. 1's path cover (k ~ 0.3 n, so the niv map is kept sparse)
    "er1m4": dict(n=1 << 20, er_degree=4, desc="Erdos-Renyi DAG n=2^20, average degree 4, path-cover chains"),
    "er1m6": dict(n=1 << 20, er_degree=6, desc="Erdos-Renyi DAG n=2^20, average degree 6, path-cover chains"),
    "er9m4": dict(n=9_000_000, er_degree=4, desc="Erdos-Renyi DAG n=9e6, average degree 4, path-cover chains"),
    "er9m6": dict(n=9_000_000, er_degree=6, desc="Erdos-Renyi DAG n=9e6, average degree 6, path-cover chains"),
}
BATCH_WORKLOADS = {
    "c4": dict(count=4096, batch=32, cross_deg=2,
               desc="4096 planted posets, n log-uniform [1k,64k], k log-uniform [4,256], cross out-degree 2, "
                    "B=32 functions per poset"),
    "c4s": dict(count=256, batch=32, cross_deg=2,
                desc="256 planted posets drawn like the 4096-poset batch (n log-uniform [1k,64k], "
                     "k log-uniform [4,256], cross out-degree 2), B=32 functions per poset"),
}
DTYPES = {"f64": ("f64u", "fp64 uniform [-1,1]"), "i64": ("i64:1048576", "int64 uniform [-2^20,2^20]"),
          "f32c": ("f32u", "fp32 uniform [-1,1] as F32C pairs")}


def make_poset(wl: str, seed: int):
    w = WORKLOADS[wl]
    if "er_degree" in w:
        return pg.er_dag(w["n"], w["er_degree"], seed)
    kw = {"cross_p": w["cross_p"]} if "cross_p" in w else {"cross_deg": w["cross_deg"]}
    return pg.planted_chain_poset(w["n"], w["k"], seed, **kw)


def time_single(mz, torch, wl: str, dtype_key: str, steps: int = 10, seed: int = 1):
    """zeta + Moebius of one function on one poset (a variant line): build time, per-transform
    times and node-values/s, and the shape of the plan."""
    p = make_poset(wl, seed)
    t0 = time.perf_counter()
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    build_s = time.perf_counter() - t0
    kind = DTYPES[dtype_key][0]
    x = to_dev(pg.function_values(p.n, 1, kind, 2)[:, 0], dtype_key, torch)
    g = plan.zeta(x)
    y = plan.mobius(g)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    for _ in range(steps):
        plan.zeta(x, out=g)
    e[1].record()
    for _ in range(steps):
        plan.mobius(g, out=y)
    e[2].record()
    e[2].synchronize()
    plan.check()
    tz, tm = e[0].elapsed_time(e[1]) / steps, e[1].elapsed_time(e[2]) / steps
    info = plan.info
    plan.close()
    out = {"workload": WORKLOADS[wl]["desc"], "dtype": dtype_key, "n": p.n, "k": info["k"],
           "nnz": info["nnz"], "ulevels": info["ulevels"], "sparse_map": bool(info["sparse"]),
           "host_build_s": round(build_s, 2), "zeta_ms": round(tz, 4), "mobius_ms": round(tm, 4),
           "value": round(2 * p.n / ((tz + tm) / 1e3), 1), "unit": UNIT}
    if p.chain_id is None:
        # the same poset built on the device, Alg. 1's matching included (another maximum
        # matching: the same number of chains)
        try:
            t0 = time.perf_counter()
            pd = mz.Plan(p.n, p.src, p.dst, None, device_build=2)
            out["device_build_s"] = round(time.perf_counter() - t0, 2)
            out["device_build_same_k"] = pd.info["k"] == info["k"]
            pd.close()
        except Exception as exc:      # keep the measured line; say what failed
            out["device_build_error"] = f"{type(exc).__name__}: {exc}"
    return out


def time_plan_file(mz, plan, info):
    """The plan's precomputation written to a file and loaded back into a device plan
    (mz_plan_save / mz_plan_load): sizes and wall times; outside every timed region."""
    import tempfile
    try:
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "plan.mzplan")
            t0 = time.perf_counter()
            plan.save(path)
            save_s = time.perf_counter() - t0
            size = os.path.getsize(path)
            t0 = time.perf_counter()
            loaded = mz.Plan.load(path)
            load_s = time.perf_counter() - t0
            same = loaded.info == info
            loaded.close()
        return {"bytes": size, "save_s": round(save_s, 3), "load_s": round(load_s, 3), "same_plan_info": bool(same)}
    except Exception as exc:          # keep the measured line; say what failed
        return {"error": f"{type(exc).__name__}: {exc}"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("mz_kernels.cu", "mz_arith.cuh"):
        with open(os.path.join(ROOT, "paper_2211_13706_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str, workload: str, dtype: str):
    """DRAM bytes per launch from the committed ncu summary, or None if absent/stale."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src_hash = None
    vals = {}
    for line in open(path):
        line = line.strip()
        if line.startswith("source_hash:"):
            src_hash = line.split(":", 1)[1].strip()
        elif line and not line.startswith("#") and "=" in line:
            key, v = line.split("=", 1)
            vals[key.strip()] = v.split()[0]
    if src_hash != kernel_source_hash():
        return None
    v = vals.get(f"{kernel}/{workload}/{dtype}")
    return float(v) if v else None


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:   # sampling has begun before the timed steps
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- device arm
def algorithmic_bytes(kernel: str, n: int, k: int, B: int, nnz: int, wave=None) -> int:
    """Bytes a launch must move: the finite entries of the niv map it needs (nnz(N), or
    nnz(N) - n without the own-chain entries), its inputs and its outputs; the prefix
    array y' counts only where a kernel writes it or reads it as its own input.
    wave = (rows, entries): the rows of the Moebius forward substitution and their finite
    entries on other chains (U-level schedule: the rows another chain reads; None: all
    rows, as in the antichain schedule)."""
    wr, we = wave if wave is not None else (n, nnz - n)
    if kernel == "chain_scan":
        return 8 * n * B + 4 * (n + k) + 8 * (n + k) * B
    if kernel == "niv_gather":
        return 4 * nnz + 4 * n + 8 * n * B
    if kernel == "mob_init":
        return (n + k) + 4 * (n + k) + 8 * (n + k) * B
    if kernel == "mob_wave":
        return 4 * we + 12 * wr + 8 * wr * B + 8 * wr * B
    if kernel == "mob_leaf":
        leaves = n - wr
        return 4 * nnz + 8 * n + 8 * leaves * B + 8 * leaves * B
    if kernel == "mob_diff":
        return 4 * (n + k) + 8 * (n + k) * B + 8 * n * B
    raise KeyError(kernel)


ZETA_KERNELS = ["chain_scan", "niv_gather"]
MOB_KERNELS = ["mob_init", "mob_wave", "mob_leaf", "mob_diff"]
MOB_KERNELS_ANTI = ["mob_init", "mob_wave"]


def to_dev(x, dtype_key, torch):
    if dtype_key == "f32c":
        hi = np.asarray(x, dtype=np.float32)
        return torch.from_numpy(np.stack([hi, np.zeros_like(hi)])).cuda()
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def time_transforms(mz, plan, x, steps, warmup, torch, flush, anti=False, sampler=None):
    """Runs `warmup` + `steps` steps (zeta then Moebius); returns per-kernel mean ms,
    total device ms of the timed steps, and the launch count."""
    stream = torch.cuda.current_stream()
    nz, nm = len(ZETA_KERNELS), len(MOB_KERNELS_ANTI if anti else MOB_KERNELS)
    ev_z = [torch.cuda.Event(enable_timing=True) for _ in range(nz + 1)]
    ev_m = [torch.cuda.Event(enable_timing=True) for _ in range(nm + 1)]
    for e in ev_z + ev_m:            # create the underlying cudaEvent_t
        e.record(stream)
    torch.cuda.synchronize()
    g = torch.empty_like(x)
    y = torch.empty_like(x)
    sums = np.zeros(nz + nm)
    total = 0.0
    launches = 0
    for it in range(warmup + steps):
        if it == warmup:
            torch.cuda.synchronize()
            if sampler:
                sampler.start()
        flush.zero_()                 # L2 flush, outside the timed events
        mz.mz_set_launch_events([e.cuda_event for e in ev_z])
        plan.zeta(x, out=g)
        lz = mz.mz_last_launch_count()
        mz.mz_set_launch_events([e.cuda_event for e in ev_m])
        plan.mobius(g, out=y)
        lm = mz.mz_last_launch_count()
        mz.mz_set_launch_events(None)
        ev_m[-1].synchronize()
        if it >= warmup:
            tz = [ev_z[i].elapsed_time(ev_z[i + 1]) for i in range(nz)]
            tm = [ev_m[i].elapsed_time(ev_m[i + 1]) for i in range(nm)]
            sums += np.array(tz + tm)
            total += ev_z[0].elapsed_time(ev_z[-1]) + ev_m[0].elapsed_time(ev_m[-1])
            launches += lz + lm
    clocks = sampler.stop() if sampler else None
    plan.check()
    names = ZETA_KERNELS + (MOB_KERNELS_ANTI if anti else MOB_KERNELS)
    return {n_: s / steps for n_, s in zip(names, sums)}, total, launches, clocks, g, y


def time_e2e(mz, plan, f_np, dtype_key, steps, torch):
    """The step through the public API from pinned host memory: H2D of f, zeta, Moebius,
    D2H of both results, every step inside the timed region. Double-buffered on three
    streams: step i+1's input goes up and step i's results come down while the GPU
    computes, as a user streaming many functions through one plan would run it."""
    x = to_dev(f_np, dtype_key, torch)
    h_in = x.cpu().pin_memory()
    main = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    d_in = [torch.empty_like(x) for _ in range(2)]
    d_g = [torch.empty_like(x) for _ in range(2)]
    d_f = [torch.empty_like(x) for _ in range(2)]
    h_g = [torch.empty_like(h_in).pin_memory() for _ in range(2)]
    h_f = [torch.empty_like(h_in).pin_memory() for _ in range(2)]
    ev = lambda: [torch.cuda.Event() for _ in range(2)]
    uploaded, g_ready, f_ready, downloaded = ev(), ev(), ev(), ev()

    def run(nsteps):
        for i in range(nsteps):
            s = i % 2
            if i >= 2:
                up.wait_event(g_ready[s])          # step i-2 has read d_in[s]
            with torch.cuda.stream(up):
                d_in[s].copy_(h_in, non_blocking=True)
            uploaded[s].record(up)
            main.wait_event(uploaded[s])
            if i >= 2:
                main.wait_event(downloaded[s])     # step i-2's results are on the host
            plan.zeta(d_in[s], out=d_g[s])
            g_ready[s].record(main)
            plan.mobius(d_g[s], out=d_f[s])
            f_ready[s].record(main)
            down.wait_event(g_ready[s])
            with torch.cuda.stream(down):
                h_g[s].copy_(d_g[s], non_blocking=True)
            down.wait_event(f_ready[s])
            with torch.cuda.stream(down):
                h_f[s].copy_(d_f[s], non_blocking=True)
            downloaded[s].record(down)
        main.wait_stream(down)

    run(2)                                          # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    up.wait_stream(main)
    run(steps)
    e1.record(main)
    e1.synchronize()
    total = e0.elapsed_time(e1)
    plan.check()
    nbytes = x.numel() * x.element_size()
    return total, nbytes, 2 * nbytes


def cpu_baseline(p, f_np, budget_s: float, max_rows: int):
    """The CPU oracle as it stands: exact zeta rows (BFS reachability + exact sum)."""
    import oracle
    rng = np.random.default_rng(123)
    rows = rng.choice(p.n, max_rows, replace=False).tolist()
    t0 = time.perf_counter()
    done = 0
    for r in rows:
        oracle.zeta_rows(p.n, p.src, p.dst, f_np, [r])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} zeta rows of this poset (exact: BFS reachability + exact sum), single thread; "
                      "the oracle's Moebius has no per-row form cheaper than O(|out(x)|^2)"}


def _as_f64(v):
    return v[0].astype(np.float64) + v[1].astype(np.float64) if isinstance(v, tuple) else np.asarray(v, np.float64)


def oracle_row_errors(p, outs, rows):
    """Per-result error of GPU results against the oracle (exact sums, correctly rounded)
    on the listed rows. outs: {dtype: (f, g, m)}: the input f, the GPU's zeta g = Z f and
    the GPU's Moebius m = M g of that g, each fp64 or an F32C (hi, lo) pair. Returns per
    dtype the largest componentwise error of zeta, |g(x) - (Z f)(x)| / (Z|f|)(x), and of
    the Moebius residual, |(Z m)(x) - g(x)| / ((Z|m|)(x) + |g(x)|) (its backward error)."""
    import oracle
    tiny = np.finfo(np.float64).tiny
    res = {}
    for dk, (f, g, m) in outs.items():
        ref = oracle.zeta_rows(p.n, p.src, p.dst, f, rows)
        fa = (np.abs(f[0]), np.abs(f[1])) if isinstance(f, tuple) else np.abs(f)
        mag = oracle.zeta_rows(p.n, p.src, p.dst, fa, rows)
        ez = np.abs(_as_f64(g)[rows] - np.asarray(ref, np.float64)) / np.maximum(np.asarray(mag, np.float64), tiny)
        res[dk] = {"zeta_max_rel": float(ez.max())}
        # The Moebius transform of rounded data grows like 10^(0.23 U-levels) on these posets
        # for any algorithm; where that overflows the output type there is no residual to take.
        if np.all(np.isfinite(_as_f64(m))):
            r, rm = oracle.mobius_residual_rows(p.n, p.src, p.dst, m, g, rows)
            em = np.abs(np.asarray(r, np.float64)) / np.maximum(np.asarray(rm, np.float64), tiny)
            res[dk]["mobius_residual_max_rel"] = float(em.max())
            res[dk]["mobius_max_abs"] = float(np.max(np.abs(_as_f64(m))))
        else:
            res[dk]["mobius_residual_max_rel"] = None
            res[dk]["mobius_overflow"] = True
    return res


def accuracy_leg(cases, budget_s: float):
    """The CPU-baseline leg's second product: the GPU results of each case checked against
    the oracle on sampled rows, case after case until the time budget is spent (every
    case gets at least one row). cases: list of (name, poset, outs, n_rows)."""
    t0 = time.perf_counter()
    out = {}
    for name, p, outs, n_rows in cases:
        rows = np.random.default_rng(7).choice(p.n, min(n_rows, p.n), replace=False).tolist()
        worst = out.setdefault(name, {"rows": 0})    # cases of one name (several posets) merge
        done = worst.pop("rows")
        for r in rows:
            for dk, e in oracle_row_errors(p, outs, [r]).items():
                w = worst.setdefault(dk, {})
                for key, v in e.items():
                    if isinstance(v, bool):
                        w[key] = w.get(key, False) or v
                    elif v is None or (key in w and w[key] is None):
                        w[key] = None
                    else:
                        w[key] = max(w.get(key, 0.0), v)
            done += 1
            if time.perf_counter() - t0 > budget_s:
                break
        worst["rows"] = done
        out[name] = worst
    out["note"] = ("largest componentwise error on sampled rows against the oracle (exact sums, correctly "
                   "rounded): zeta |g - Zf| / Z|f|, Moebius residual (backward error) |Z m - g| / (Z|m| + |g|) "
                   "of m = Moebius(g) for the GPU's own zeta output g; F32C values are (hi, lo) pairs taken "
                   "exactly; inputs of the F32C and fp64 lines are the same fp32 values (C2, C3), or each "
                   "dtype's own random values (C4). mobius_overflow: |M g| of rounded data exceeds the output "
                   "type (it grows like 10^(0.23 U-levels) for any algorithm), so no residual exists")
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def _gen_one(spec_and_deg):
    (n, k, seed), deg = spec_and_deg
    p = pg.planted_chain_poset(n, k, seed, cross_deg=deg)
    return p.n, p.src, p.dst, p.chain_id


def gen_batch_posets(wl: str, seed: int):
    """The posets of a batch workload, generated in a spawned process pool (started
    before this process touches the GPU)."""
    import multiprocessing as mp
    w = BATCH_WORKLOADS[wl]
    specs = pg.planted_batch_specs(w["count"], seed)
    work = [(sp, w["cross_deg"]) for sp in specs]
    if w["count"] <= 64:
        return [_gen_one(x) for x in work]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_one, work, chunksize=16)


def time_batch(mz, plan, x, steps, warmup, torch, use_graph):
    """zeta then Moebius of x per step, replayed from a captured CUDA graph when
    use_graph (else launched directly); returns (total device ms of `steps` steps, graph used)."""
    g = torch.empty_like(x)
    y = torch.empty_like(x)
    step = lambda: (plan.zeta(x, out=g), plan.mobius(g, out=y))
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    graph = None
    if use_graph:
        try:
            cg = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                step()                       # warm the workspace on the capture stream
            torch.cuda.current_stream().wait_stream(side)
            with torch.cuda.graph(cg):
                step()
            graph = cg
        except Exception as exc:            # capture unsupported: launch directly
            print(f"graph capture failed ({exc}); timing direct launches", file=sys.stderr)
            torch.cuda.synchronize()
            graph = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for _ in range(steps):
        e0.record()
        if graph is not None:
            graph.replay()
        else:
            step()
        e1.record()
        e1.synchronize()
        total += e0.elapsed_time(e1)
    plan.check()
    return total, graph is not None


def batch_values(n, B, dtype_key, seed, torch):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    if dtype_key == "f32c":
        hi = torch.rand((n, B), generator=gen, device="cuda", dtype=torch.float32) * 2 - 1
        return torch.stack([hi, torch.zeros_like(hi)])
    if dtype_key == "f64":
        return torch.rand((n, B), generator=gen, device="cuda", dtype=torch.float64) * 2 - 1
    return torch.randint(-1000, 1001, (n, B), generator=gen, device="cuda", dtype=torch.int64)


def time_batch_e2e(plan, x, steps, torch):
    """The batched step through the public API from pinned host memory: H2D of the
    inputs, zeta, Moebius of the result, D2H of both results, every step inside the
    timed region (one buffer set, copies and compute in stream order)."""
    h_in = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
    h_in.copy_(x)
    h_g = torch.empty_like(h_in, pin_memory=True)
    h_f = torch.empty_like(h_in, pin_memory=True)
    d_in = torch.empty_like(x)
    g = torch.empty_like(x)
    y = torch.empty_like(x)

    def step():
        d_in.copy_(h_in, non_blocking=True)
        plan.zeta(d_in, out=g)
        plan.mobius(g, out=y)
        h_g.copy_(g, non_blocking=True)
        h_f.copy_(y, non_blocking=True)

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    e1.synchronize()
    plan.check()
    nbytes = x.numel() * x.element_size()
    return e0.elapsed_time(e1), nbytes, 2 * nbytes


def run_batch_workload(mz, wl, posets, steps, warmup, torch, dtypes=("f32c", "f64"), graph=True, e2e_steps=0,
                       samples=None, compare_builds=False):
    """Builds one plan for all posets on the device, autotunes it and times each dtype (CUDA
    graph replay); with e2e_steps also the end-to-end step from pinned host memory.
    compare_builds: first builds the same plan on the host (timed, compared, freed).
    samples: a list of (poset index, column) whose inputs and outputs are copied to the
    host (key "_samples", for the accuracy check of the CPU-baseline leg)."""
    from paper_2211_13706_gb300 import autotune
    w = BATCH_WORKLOADS[wl]
    spec = [(n, s_, d_, c) for n, s_, d_, c in posets]
    host_s = host_info = None
    if compare_builds:
        t0 = time.perf_counter()
        hp = mz.Plan.batch(spec)
        host_s = time.perf_counter() - t0
        host_info = hp.info
        hp.close()
        torch.cuda.empty_cache()
    t0 = time.perf_counter()
    plan = mz.Plan.batch(spec, device_build=True)
    build_s = time.perf_counter() - t0
    info = plan.info
    out = {"workload": w["desc"], "posets": info["components"], "n_total": info["n"], "k_total": info["k"],
           "nnz": info["nnz"], "max_ulevels": info["ulevels"], "wave_rows": info["wave_rows"], "batch": w["batch"],
           "device_build_s": round(build_s, 2)}
    if compare_builds:
        out["host_build_s"] = round(host_s, 2)
        out["same_plan_info"] = all(host_info[key] == info[key] for key in host_info)
    peak, peak_kind = load_peaks()
    n, k, B, nnz = info["n"], info["k"], w["batch"], info["nnz"]
    wave = (info["wave_rows"], info["wave_entries"])
    offs = np.cumsum([0] + [int(q[0]) for q in posets])
    kept = {}
    for dk in dtypes:
        x = batch_values(n, B, dk, 11, torch)
        tuned = autotune.tune(plan, x, reps=1)
        tot, used_graph = time_batch(mz, plan, x, steps, warmup, torch, graph)
        units = 2 * n * B * steps
        out[dk] = {"value": round(units / (tot / 1e3), 1), "unit": UNIT, "ms_per_step": round(tot / steps, 3),
                   "steps": steps, "cuda_graph": used_graph, "tuning": tuned}
        # per-kernel times of the same step, launched directly (inputs exceed L2: no flush)
        kt, _, _, _, g, y = time_transforms(mz, plan, x, 3, 1, torch, torch.empty(1, device="cuda"))
        out[dk]["kernels"] = {name: {"mean_ms": round(v, 4), "share": round(v / sum(kt.values()), 4),
                                     "alg_GBps": round(algorithmic_bytes(name, n, k, B, nnz, wave) / (v / 1e3) / 1e9, 1)}
                              for name, v in kt.items()}
        dom = max(kt, key=kt.get)
        alg = algorithmic_bytes(dom, n, k, B, nnz, wave)
        achieved = alg / (kt[dom] / 1e3) / 1e9
        out[dk]["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                               "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                               "traffic": None, "algorithmic_bytes": alg, "mean_launch_ms": round(kt[dom], 4)}
        # the gathers' arithmetic roof: one add per gathered term and function (zeta gather:
        # nnz(N) terms; leaf gather: the same tiles)
        terms = nnz * B
        alu = {}
        for kname in ("niv_gather", "mob_leaf"):
            t_g = kt[kname] / 1e3
            if dk == "f32c":     # Sum2 step: TwoSum (6 fp32 adds) + 2 adds per term
                ops, peak_ops = 8 * terms, torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2.07e9
                alu[kname] = {"fp32_ops": ops, "achieved_Tops": round(ops / t_g / 1e12, 2),
                              "peak_Tops": round(peak_ops / 1e12, 2), "frac": round(ops / t_g / peak_ops, 4),
                              "note": "peak = SMs x 128 fp32 lanes x 2.07 GHz (one add per lane per clock)"}
            elif dk == "f64":
                alu[kname] = {"fp64_adds": terms, "achieved_Tadds": round(terms / t_g / 1e12, 3),
                              "peak_Tadds": FP64_ADDS_PER_S / 1e12, "frac": round(terms / t_g / FP64_ADDS_PER_S, 4)}
        out[dk]["gather_alu"] = alu.get("niv_gather")
        out[dk]["leaf_alu"] = alu.get("mob_leaf")
        if samples:
            for (pi, b) in samples:
                sl = slice(int(offs[pi]), int(offs[pi + 1]))
                if dk == "f32c":
                    pick = lambda t: (t[0, sl, b].cpu().numpy(), t[1, sl, b].cpu().numpy())
                else:
                    pick = lambda t: t[sl, b].cpu().numpy()
                kept.setdefault((pi, b), {})[dk] = (pick(x), pick(g), pick(y))
        del g, y
        if e2e_steps:
            torch.cuda.empty_cache()
            ms, h2d, d2h = time_batch_e2e(plan, x, e2e_steps, torch)
            out[dk]["e2e"] = {"value": round(2 * n * B * e2e_steps / (ms / 1e3), 1), "unit": UNIT,
                              "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                              "ms_per_step": round(ms / e2e_steps, 3),
                              "copies": "pinned host memory, H2D of f, D2H of zeta(f) and Moebius(zeta(f)), "
                                        "in stream order"}
        del x
        torch.cuda.empty_cache()
    plan.close()
    if samples:
        out["_samples"] = kept
    return out


def time_c3(mz, torch, flush, steps: int = 10):
    """The precision workload: n = 2^22, k = 128 chains, cross out-degree 2, B = 1, f fp32
    uniform [-1, 1] and log-normal (sigma = 3, random signs); compensated F32C and plain
    fp64 on the same values, plan built on the device and its launch shapes autotuned.
    Returns the timings and the poset with host copies of inputs and outputs (for the
    accuracy check of the CPU-baseline leg)."""
    from paper_2211_13706_gb300 import autotune
    p = make_poset("c3", 1)
    t0 = time.perf_counter()
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, device_build=True)
    build_s = time.perf_counter() - t0
    info = plan.info
    res = {"workload": WORKLOADS["c3"]["desc"] + "; B=1", "n": p.n, "k": info["k"], "nnz": info["nnz"],
           "ulevels": info["ulevels"], "wave_rows": info["wave_rows"], "device_build_s": round(build_s, 2)}
    kept = {}
    for kind in ("u", "ln"):
        f32 = pg.function_values(p.n, 1, "f32" + kind, 13)[:, 0]
        res[kind] = {}
        for dk in ("f32c", "f64"):
            x = to_dev(f32 if dk == "f32c" else f32.astype(np.float64), dk, torch)
            tuned = autotune.tune(plan, x, reps=2)
            kt, total, _, _, g, y = time_transforms(mz, plan, x, steps, 3, torch, flush)
            zms = kt["chain_scan"] + kt["niv_gather"]
            res[kind][dk] = {"value": round(2 * p.n * steps / (total / 1e3), 1), "unit": UNIT,
                             "zeta_ms": round(zms, 4), "mobius_ms": round(total / steps - zms, 4),
                             "kernels_ms": {a: round(b, 4) for a, b in kt.items()}, "tuning": tuned}
            if dk == "f32c":
                host = lambda t: (t[0].cpu().numpy(), t[1].cpu().numpy())
                kept.setdefault(kind, {})[dk] = ((f32, np.zeros_like(f32)), host(g), host(y))
            else:
                kept.setdefault(kind, {})[dk] = (f32.astype(np.float64), g.cpu().numpy(), y.cpu().numpy())
            del x, g, y
    plan.close()
    torch.cuda.empty_cache()
    return res, p, kept


def time_seeds(mz, torch, wl: str, dtype_key: str, flush, seeds=(1, 2, 3, 4, 5), steps: int = 20):
    """The headline step (zeta + Moebius, B = 1) on the workload drawn with each seed; plans
    built on the device. Returns per-seed node-values/s and their median."""
    vals = []
    for sd in seeds:
        p = make_poset(wl, sd)
        plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, device_build=True)
        x = to_dev(pg.function_values(p.n, 1, DTYPES[dtype_key][0], 2)[:, 0], dtype_key, torch)
        g, y = plan.zeta(x), None
        y = plan.mobius(g)
        ts = []
        for it in range(steps + 3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.zeta(x, out=g)
            plan.mobius(g, out=y)
            e1.record()
            e1.synchronize()
            if it >= 3:
                ts.append(e0.elapsed_time(e1))
        plan.check()
        vals.append(round(2 * p.n / (statistics.median(ts) / 1e3), 1))
        plan.close()
    return {"seeds": list(seeds), "values": vals, "median": statistics.median(vals), "unit": UNIT,
            "note": "median step time of 20 per seed, L2 flushed between steps"}


def cpu_paper_method(mz, plan, f_np, dtype_key, gpu_g=None):
    """The paper's fast transforms on the host cores (cpubase/: Alg. 3, Alg. 4 in Alg. 5's
    antichain order, OpenMP), timed on this plan's structures: all threads and one."""
    import cpubase
    if plan.info["sparse"]:
        return None
    cp = cpubase.CpuPlan(plan, mz.MZ_EXPORT_NIV, mz.MZ_EXPORT_CHAIN_ID, mz.MZ_EXPORT_CHAIN_POS, mz.MZ_EXPORT_LEVEL,
                         mz.MZ_EXPORT_ULEVEL)
    x = np.asarray(f_np, np.int64 if dtype_key == "i64" else np.float64)
    out = {"kind": "paper_method_cpu", "dtype": "int64" if dtype_key == "i64" else "f64"}
    all_threads = cpubase.threads()
    for label, t, reps in (("all_cores", all_threads, 3), ("one_core", 1, 1)):
        cpubase.set_threads(t)
        tz, tm, tu = [], [], []
        for _ in range(reps):
            t0 = time.perf_counter()
            g = cp.zeta(x)
            t1 = time.perf_counter()
            y = cp.mobius(g)
            t2 = time.perf_counter()
            yu = cp.mobius_u(g)
            t3 = time.perf_counter()
            tz.append(t1 - t0)
            tm.append(t2 - t1)
            tu.append(t3 - t2)
        z, m, u = statistics.median(tz), statistics.median(tm), statistics.median(tu)
        out[label] = {"threads": t, "zeta_ms": round(z * 1e3, 2), "mobius_ms": round(m * 1e3, 2),
                      "value": round(2 * plan.info["n"] / (z + m), 1), "unit": UNIT,
                      "mobius_ulevel_schedule_ms": round(u * 1e3, 2),
                      "value_ulevel_schedule": round(2 * plan.info["n"] / (z + u), 1)}
    cpubase.set_threads(all_threads)
    if dtype_key == "i64":   # exact: Moebius(zeta(f)) = f, under both schedules
        out["check"] = {"moebius_of_zeta_is_f": bool(np.array_equal(y, x) and np.array_equal(yu, x))}
    elif gpu_g is not None:  # fp64 Moebius at this size is too ill-conditioned for a round trip
        err = float(np.max(np.abs(g - gpu_g)) / max(1e-300, float(np.max(np.abs(gpu_g)))))
        out["check"] = {"zeta_vs_gpu_max_rel": err}
    out["note"] = ("transforms only, on the plan's chains and dense niv map; Moebius in the antichain order "
                   "of Alg. 5 (value) and in the order of U's dependency levels (value_ulevel_schedule); "
                   "the fair CPU reference point for the GPU numbers")
    return out


def rank_seed(rank: int) -> int:
    """Seed of the poset a rank runs: ranks hold independent problems (replicas)."""
    return 1 + rank


def reduce_over_ranks(local_ms: float, units_per_rank: int, dist=None, device=None):
    """(slowest rank's time in ms, whole-job node-values/s): every rank's units over the
    slowest rank's time. `dist` is torch.distributed or None for one process."""
    world = 1
    t = local_ms
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        x = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, units_per_rank * world / (t / 1e3)


def time_differentiation(mz, torch, steps=5, warmup=2):
    """C5: loss = sum(w * Moebius(zeta(f) * h)) on n = 2^20, k = 64 (cross out-degree 3),
    B = 16, forward and backward (zeta, Moebius, Moebius^T, zeta^T); fp32 (compensated
    transforms) and fp64. Units: 4 transforms * n * B node-values per step."""
    p = pg.planted_chain_poset(1 << 20, 64, 5, cross_deg=3)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, build_transpose=True)
    out = {"workload": "planted poset n=2^20, k=64, cross out-degree 3, B=16, loss=sum(w*Moebius(zeta(f)*h))"}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        gen = torch.Generator(device="cuda").manual_seed(5)
        f, w, h = ((torch.rand((p.n, 16), generator=gen, device="cuda", dtype=dt) * 2 - 1) for _ in range(3))
        f.requires_grad_()

        def step():
            f.grad = None
            loss = (w * mz.MobiusFn.apply(mz.ZetaFn.apply(f, plan) * h, plan)).sum()
            loss.backward()

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_fwd_bwd": round(ms, 3), "value": round(4 * p.n * 16 / (ms / 1e3), 1), "unit": UNIT}
    plan.check()
    plan.close()
    return out


def device_arm(args):
    import torch
    import paper_2211_13706_gb300 as mz

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # batch-workload posets: generated before this process touches the GPU
    batch_posets = None
    if args.workload in BATCH_WORKLOADS:
        return batch_arm(args, gen_batch_posets(args.workload, rank_seed(rank)))
    if not args.no_variants:
        batch_posets = gen_batch_posets("c4", rank_seed(rank))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = WORKLOADS[args.workload]
    p = make_poset(args.workload, rank_seed(rank))
    t0 = time.perf_counter()
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    build_s = time.perf_counter() - t0
    info = plan.info
    kind, fdesc = DTYPES[args.dtype]
    f_np = pg.function_values(p.n, 1, kind, 2 + rank)[:, 0]
    x = to_dev(f_np, args.dtype, torch)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    # launch shapes picked by the autotuner for this plan and input (results do not depend on them)
    from paper_2211_13706_gb300 import autotune
    tuned = autotune.tune(plan, x)

    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    kt, total_ms, launches, clocks, g, y = time_transforms(mz, plan, x, args.steps, args.warmup, torch, flush,
                                                           sampler=sampler)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    n, k, B = p.n, info["k"], 1
    total_ms, value = reduce_over_ranks(total_ms, 2 * n * B * args.steps, dist, "cuda")

    # round-trip sanity on the timed data (Moebius(zeta(f)) = f)
    if args.dtype == "i64":
        assert torch.equal(y, x), "Moebius(zeta(f)) != f"

    # the accuracy inputs: one fp32-valued function through the F32C and the fp64 path (the
    # same values), outputs kept on the host for the CPU-baseline leg's oracle rows
    f32 = pg.function_values(p.n, 1, "f32u", 20 + rank)[:, 0]
    acc_c2 = {}
    for dk in ("f32c", "f64"):
        xa = to_dev(f32 if dk == "f32c" else f32.astype(np.float64), dk, torch)
        mz.mz_plan_tune(plan.handle, **tuned)
        ga = plan.zeta(xa)
        ma = plan.mobius(ga)
        plan.check()
        if dk == "f32c":
            host = lambda t: (t[0].cpu().numpy(), t[1].cpu().numpy())
            acc_c2[dk] = ((f32, np.zeros_like(f32)), host(ga), host(ma))
        else:
            acc_c2[dk] = (f32.astype(np.float64), ga.cpu().numpy(), ma.cpu().numpy())
        del xa, ga, ma

    e2e_ms, h2d, d2h = time_e2e(mz, plan, f_np, args.dtype, max(5, min(args.steps, 50)), torch)
    e2e_steps = max(5, min(args.steps, 50))
    e2e_val = 2 * n * B * e2e_steps * world / (e2e_ms / 1e3)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_kind = load_peaks()
    dom = max(kt, key=kt.get)
    wave = (info["wave_rows"], info["wave_entries"])
    alg = algorithmic_bytes(dom, n, k, B, info["nnz"], wave)
    achieved = alg / (kt[dom] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_kind,
            "traffic": load_traffic(dom, args.workload, args.dtype), "algorithmic_bytes": alg,
            "mean_launch_ms": round(kt[dom], 5)}
    kernels = {name: {"mean_ms": round(v, 5), "share": round(v / sum(kt.values()), 4),
                      "alg_GBps": round(algorithmic_bytes(name, n, k, B, info["nnz"], wave) / (v / 1e3) / 1e9, 1)}
               for name, v in kt.items()}
    # The gather's other roof: one add per gathered term (nnz(N) per launch). In fp64 it is
    # bound by the FP64 pipe: nominal 1.25 TFLOP/s = 0.625e12 adds/s on GB300.
    adds = info["nnz"] * B
    kernels["niv_gather"]["adds_per_s"] = round(adds / (kt["niv_gather"] / 1e3), 1)
    if args.dtype == "f64":
        kernels["niv_gather"]["fp64_add_frac_of_nominal"] = round(adds / (kt["niv_gather"] / 1e3) / FP64_ADDS_PER_S, 4)
    # The forward substitution's roof is latency: U's dependency graph has `ulevels`
    # levels, and each level costs at least one store-to-poll hop between SMs
    # (measured unloaded on GB300: about 0.45 us one way).
    lat_ms = info["ulevels"] * HOP_FLOOR_US / 1e3
    latency = {"kernel": "mob_wave", "levels": info["ulevels"], "hop_floor_us": HOP_FLOOR_US,
               "bound_ms": round(lat_ms, 4), "achieved_ms": round(kt["mob_wave"], 4),
               "frac": round(lat_ms / kt["mob_wave"], 4)}

    variants = {}
    c3 = p3 = acc_c3 = None
    if not args.no_variants:
        for vd in ("i64", "f32c"):
            if vd == args.dtype:
                continue
            fv = pg.function_values(p.n, 1, DTYPES[vd][0], 3)[:, 0]
            xv = to_dev(fv, vd, torch)
            ktv, tot, _, _, _, _ = time_transforms(mz, plan, xv, args.variant_steps, 3, torch, flush)
            variants[vd] = {"value": 2 * n * args.variant_steps / (tot / 1e3),
                            "ms_per_step": tot / args.variant_steps,
                            "kernels_ms": {a: round(b, 5) for a, b in ktv.items()}}
        if not info["sparse"]:
            # the same plan built by the device build (Thm. 4's recurrence, U levels and
            # layouts in kernels); outside any timed region
            t0 = time.perf_counter()
            pd = mz.Plan(p.n, p.src, p.dst, p.chain_id, device_build=True)
            dev_s = time.perf_counter() - t0
            same = all(pd.info[key] == info[key] for key in ("nnz", "levels", "ulevels", "device_bytes")) and \
                np.array_equal(pd.export(mz.MZ_EXPORT_ULEVEL), plan.export(mz.MZ_EXPORT_ULEVEL))
            variants["plan_build"] = {"host_s": round(build_s, 3), "device_s": round(dev_s, 3), "same_plan": bool(same)}
            pd.close()
        variants["plan_file"] = time_plan_file(mz, plan, info)
        pa = mz.Plan(p.n, p.src, p.dst, p.chain_id, mobius_schedule=mz.MZ_SCHED_ANTICHAIN)
        kta, tot, _, _, _, _ = time_transforms(mz, pa, x, 3, 1, torch, flush, anti=True)
        variants["mobius_antichain_schedule_" + args.dtype] = {
            "mobius_ms": round(kta["mob_init"] + kta["mob_wave"], 4), "levels": pa.info["levels"],
            "note": "Alg. 5/6 schedule (antichain levels) instead of U's dependency levels"}
        pa.close()
        variants["differentiation_c5"] = time_differentiation(mz, torch)
        variants["seeds_1_to_5"] = time_seeds(mz, torch, args.workload, args.dtype, flush)
        variants["paper_er_n2^20_deg4"] = time_single(mz, torch, "er1m4", args.dtype)
        variants["paper_er_n2^20_deg6"] = time_single(mz, torch, "er1m6", args.dtype)
        c3, p3, acc_c3 = time_c3(mz, torch, flush)
    del flush
    torch.cuda.empty_cache()
    c4 = None
    c4_samples = [(int(q), 31 if i == 0 else 0) for i, q in
                  enumerate(np.random.default_rng(5).choice(len(batch_posets), 6, replace=False))] \
        if batch_posets is not None else []
    if batch_posets is not None:
        plan.close()
        c4 = run_batch_workload(mz, "c4", batch_posets, max(3, args.steps // 4), 3, torch, e2e_steps=3,
                                samples=c4_samples, compare_builds=True)

    cpu = cpu_fast = accuracy = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(p, f_np, args.cpu_budget, 64)
        if args.dtype in ("f64", "i64") and not plan.handle:
            plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, host_only=True)
        if args.dtype in ("f64", "i64"):
            cpu_fast = cpu_paper_method(mz, plan, f_np, args.dtype, g.cpu().numpy())
        cases = [("c2", p, acc_c2, 6)]
        if not args.no_variants:
            cases += [("c3_uniform", p3, acc_c3["u"], 2), ("c3_lognormal", p3, acc_c3["ln"], 2)]
        if c4 is not None:
            for (pi, b), outs in c4.pop("_samples").items():
                n_, s_, d_, c_ = batch_posets[pi]
                cases.append(("c4", pg.Poset(n=n_, src=s_, dst=d_, chain_id=c_), outs, 3))
        try:
            accuracy = accuracy_leg(cases, args.accuracy_budget)
        except Exception as exc:          # keep the measured line; say what failed
            accuracy = {"error": f"{type(exc).__name__}: {exc}"}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"f64": "f64", "i64": "int64", "f32c": "f32c"}[args.dtype],
        "data": "synthetic",
        "config": {"workload": wl["desc"] + f"; f {fdesc}; B=1", "n": n, "k": k, "batch": B,
                   "nnz": info["nnz"], "levels": info["levels"], "ulevels": info["ulevels"],
                   "units": "2*n*B node-values per step (zeta output + Moebius output)",
                   "l2": "flushed between steps (512 MiB write), outside the timed events",
                   "parallelism": f"replicas x{world}", "host_build_s": round(build_s, 2)},
        "roofline": roof,
        "latency_roof": latency,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "cpu_paper_method": cpu_fast,
        "e2e": {"value": round(e2e_val, 1), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(e2e_ms / e2e_steps, 5),
                "copies": "pinned host memory; double-buffered: step i+1's H2D and step i's D2H overlap compute"},
        "gpu_launches": launches,
        "clocks": clocks,
        "tuning": tuned,
        "accuracy": accuracy,
        "c3_precision": c3,
        "c4_batched": c4,
        "variants": variants,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def batch_arm(args, posets):
    """--workload c4 / c4s: many posets in one plan, B functions each; one JSON line."""
    import torch
    import paper_2211_13706_gb300 as mz
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0"))))
    dk = args.dtype if args.dtype != "f64" or args.batch_dtype_f64 else "f32c"
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    res = run_batch_workload(mz, args.workload, posets, args.steps, args.warmup, torch,
                             dtypes=(dk, "f64") if dk != "f64" else ("f64",))
    clocks = sampler.stop()
    main = res[dk]
    tot_ms, value = reduce_over_ranks(main["ms_per_step"] * main["steps"],
                                      2 * res["n_total"] * res["batch"] * main["steps"], dist, "cuda")
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": main["steps"],
            "warmup": args.warmup, "ms_per_step": round(tot_ms / main["steps"], 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dk, "data": "synthetic",
            "config": {"workload": res["workload"], "posets": res["posets"], "n_total": res["n_total"],
                       "k_total": res["k_total"], "batch": res["batch"], "nnz": res["nnz"],
                       "max_ulevels": res["max_ulevels"], "l2": "inputs larger than L2",
                       "units": "2*n*B node-values per step", "device_build_s": res["device_build_s"],
                       "cuda_graph": main["cuda_graph"], "tuning": main["tuning"],
                       "parallelism": f"replicas x{world}"},
            "roofline": main["roofline"], "kernels": main["kernels"], "gather_alu": main.get("gather_alu"),
            "fp64_plain": res.get("f64"), "clocks": clocks, "gpu_launches": 6 * main["steps"]}
    print(json.dumps(line))


# ----------------------------------------------------------------------------- reference arm
def reference_arm(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    if args.workload in BATCH_WORKLOADS:
        # a batch workload: each step is one exact zeta row of one of its posets
        bw = BATCH_WORKLOADS[args.workload]
        specs = pg.planted_batch_specs(bw["count"], 1)
        n_, k_, sd = specs[0]
        p = pg.planted_chain_poset(n_, k_, sd, cross_deg=bw["cross_deg"])
        wl = {"desc": bw["desc"] + f" (rows of its first poset, n={n_}, k={k_})", "k": k_}
    else:
        wl = WORKLOADS[args.workload]
        p = make_poset(args.workload, 1)
    kind, fdesc = DTYPES[args.dtype]
    f_np = pg.function_values(p.n, 1, kind, 2)[:, 0]
    if args.dtype == "f32c":
        f_np = f_np.astype(np.float64)
    rng = np.random.default_rng(7)
    rows = rng.choice(p.n, args.steps + args.warmup, replace=False).tolist()
    csr_t0 = time.perf_counter()
    total = 0.0
    for i, r in enumerate(rows):
        t0 = time.perf_counter()
        oracle.zeta_rows(p.n, p.src, p.dst, f_np, [r])       # one step: one exact zeta row
        if i >= args.warmup:
            total += time.perf_counter() - t0
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64", "i64": "int64", "f32c": "f64"}[args.dtype], "data": "synthetic",
            "config": {"workload": wl["desc"] + f"; f {fdesc}; B=1", "n": p.n, "k": wl.get("k"), "batch": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one exact zeta row per step (BFS reachability + exact sum), single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.perf_counter() - csr_t0, 1)}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["mz", "reference"], default="mz")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS), default="c2")
    ap.add_argument("--batch-dtype-f64", action="store_true", help="batch workloads: time fp64 as the main line")
    ap.add_argument("--dtype", choices=sorted(DTYPES), default="f64")
    ap.add_argument("--variant-steps", type=int, default=50)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--accuracy-budget", type=float, default=90.0,
                    help="seconds of oracle rows for the accuracy figures (CPU-baseline leg)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)          # at least 3 untimed warm-up steps
    if args.impl == "reference":
        reference_arm(args)
    else:
        device_arm(args)


if __name__ == "__main__":
    main()
