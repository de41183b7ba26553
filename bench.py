"""Benchmark: sorted (uint64 key, uint32 index) pairs per second on GB300.

Workload (default): two arrays of n = 2^28 pairs each (3 GiB of pairs per
array), one lognormal floor(exp(N(30, 2))) and one 8-component Gaussian
mixture (means evenly spaced over [2^60, 2^63], sd 2^55), payload = original
index.  One step sorts both arrays in place with zsort_pairs_ex (learned
mapper by default, Eq. 1 z-score fallback).  Inputs are restored from a
pristine device copy between steps, outside the timed region; each restore
writes 6 GiB, far more than the 129 MB L2, so every step starts cold.

Printed: one JSON line (rank 0).  `value` = pairs sorted per second by the
device-timed sorts; `e2e` = the same through the C ABI with the inputs copied
from pinned host memory and the sorted pairs copied back inside the timed
region; `roofline` = algorithmic bytes of the persistent sort kernel (the
library's own count of bytes its passes read and write) over its measured
duration, against the measured HBM copy bandwidth; `cpu_baseline` = the
CPU oracle (plain sequential zSort in C) on a bounded sample of the same
workload on this host.

--impl reference runs the oracle as the reference arm on the same workload
shape (bounded sample per step) and prints its own JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_14419_gb300 import inputs  # noqa: E402

METRIC = "sorted 64-bit key+idx pairs/sec at 1 GB300 (plain vs learned/batched); % HBM roofline"
UNIT = "pairs/s"
BYTES_PER_PAIR = 12


KERNEL_SOURCES = [os.path.join(ROOT, "paper_2605_14419_gb300", "csrc", f)
                  for f in ("zsort.cu", "zsort_device.cuh", "zsort_tasks.cuh")]
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_persistent_bench_2p26.md")


def kernel_source_hash() -> str:
    """sha256 over the persistent kernel's sources (the code the DRAM counters describe)."""
    import hashlib

    h = hashlib.sha256()
    for path in KERNEL_SOURCES:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic_per_pair():
    """DRAM bytes per pair of k_persistent from the committed ncu summary, or
    None when the kernel sources changed since those counters were taken."""
    try:
        with open(TRAFFIC_PROFILE) as f:
            text = f.read()
    except OSError:
        return None, "no profile"
    fields = dict(line.split(":", 1) for line in text.splitlines() if line.startswith(("source_sha256:",
                                                                                          "dram_bytes_per_pair:")))
    if fields.get("source_sha256", "").strip() != kernel_source_hash():
        return None, "kernel changed since the ncu capture"
    try:
        return float(fields["dram_bytes_per_pair"]), "ncu capture at n=2^26, scaled by pairs"
    except (KeyError, ValueError):
        return None, "no figure"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_info():
    """Host cores and CPU model of this machine (the oracle's baseline runs here)."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model Name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def link_bandwidth(torch, dev, nbytes: int = 2 << 30, reps: int = 3):
    """Pinned host <-> device copy bandwidth on this machine: one large copy each
    way alone, then both directions at once (two streams), best of `reps`,
    CUDA events.  GB/s counts the bytes of one direction."""
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def timed(fn):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best

    def both():
        ev = torch.cuda.Event()
        ev.record()
        s1.wait_event(ev)
        s2.wait_event(ev)
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
        torch.cuda.current_stream().wait_stream(s1)
        torch.cuda.current_stream().wait_stream(s2)

    h2d = timed(lambda: d.copy_(h, non_blocking=True))
    d2h = timed(lambda: h2.copy_(d2, non_blocking=True))
    bi = timed(both)
    gb = nbytes / 1e9
    out = {"bytes": nbytes, "h2d_gbs": round(gb / (h2d / 1e3), 1), "d2h_gbs": round(gb / (d2h / 1e3), 1),
           "both_directions_gbs_each": round(gb / (bi / 1e3), 1)}
    del h, h2, d, d2
    torch.cuda.empty_cache()
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(n: int, rank: int = 0):
    """The two arrays of a rank (rank 0: seeds 30 and 31; other ranks their own)."""
    from paper_2605_14419_gb300 import replicas

    return [("lognormal", inputs.lognormal(n, replicas.rank_seed(30, rank))),
            ("gmm8", inputs.gaussian_mixture(n, replicas.rank_seed(31, rank)))]


def batched_measure(z, torch, dev, nseg: int, seed: int, steps: int, warmup: int, plain_segments: int,
                    tune_cache=None, tune_budget_ms: int = 60_000, cpu_segments: int = 0):
    """zsort_segmented on a batch of nseg log-uniform (32..2^20) segments, one
    persistent launch replayed from a CUDA graph, with the knobs chosen by the
    library's autotuner (untimed; served from tune_cache when it has the
    class); beside it the plain path, one zsort_pairs call per segment on the
    same data with default options (first plain_segments segments, scaled to
    pairs/s)."""
    keys, vals, off, _ = inputs.segmented_parallel(nseg, seed) if nseg >= 4000 else inputs.segmented(nseg, seed)
    n = keys.size
    kp = torch.from_numpy(keys.view(np.int64)).to(dev)
    vp = torch.from_numpy(vals.view(np.int32)).to(dev)
    od = torch.from_numpy(off.view(np.int64)).to(dev)
    kb, vb = torch.empty_like(kp), torch.empty_like(vp)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        z.reserve(n, nseg, stream)
        t0 = time.perf_counter()
        cached = tune_cache is not None and os.path.exists(tune_cache)
        opts = z.autotune(kp, vp, offsets=od, base=z.default_opts(flags=z.FLAG_GRAPH), cache_path=tune_cache,
                          budget_ms=tune_budget_ms, reps=1, stream=stream)
        tune_s = time.perf_counter() - t0
        tuned = {f: getattr(opts, f) for f in ("kmax", "leaf_target", "leaf_cap", "large_min", "chunks_per_cta")}
        tuned.update({"class": z.tune_class(kp, nseg=nseg, stream=stream), "tune_s": round(tune_s, 2),
                      "cache": tune_cache, "cache_existed": cached})
        times = []
        for i in range(warmup + steps):
            kb.copy_(kp)
            vb.copy_(vp)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            z.sort_segmented(kb, vb, od, opts=opts, stream=stream, check=False)
            e1.record(stream)
            rc = z.sync_status(stream)
            if rc != 0:
                raise z.ZsortError(rc, "bench batched")
            if i >= warmup:
                times.append(e0.elapsed_time(e1))
        st = z.last_stats(stream)
        # output check: sorted inside every segment, payload = position in segment
        seg_id = torch.repeat_interleave(torch.arange(nseg, device=dev),
                                         (od[1:] - od[:-1]).to(torch.int64))
        sk = kb ^ torch.tensor(-(2 ** 63), dtype=torch.int64, device=dev)
        same = seg_id[1:] == seg_id[:-1]
        assert bool((sk[1:][same] >= sk[:-1][same]).all()), "batched: not sorted"
        src = od[:-1][seg_id] + (vb.to(torch.int64) & 0xFFFFFFFF)
        assert bool(torch.equal(kp[src], kb)), "batched: payload does not follow its key"
        # stability: equal keys of a segment keep their input order
        eq = same & (kb[1:] == kb[:-1])
        assert bool((vb[1:][eq].to(torch.int64) > vb[:-1][eq].to(torch.int64)).all()), "batched: not stable"
        del seg_id, sk, same, src, eq
        # plain path: one zsort_pairs call per segment
        m = min(plain_segments, nseg)
        a, b = int(off[0]), int(off[m])
        kb[a:b].copy_(kp[a:b])
        vb[a:b].copy_(vp[a:b])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(m):
            s0, s1 = int(off[i]), int(off[i + 1])
            if s1 - s0 > 1:
                z.sort_pairs(kb[s0:s1], vb[s0:s1], stream=stream, check=False)
        e1.record(stream)
        stream.synchronize()
        plain_ms = e0.elapsed_time(e1)
    ms = sum(times) / len(times)
    out = {"segments": nseg, "pairs": n, "value": n / (ms / 1e3), "unit": UNIT, "ms": ms,
           "graph": True, "bytes_per_pair": st["bytes_algorithmic"] / n, "autotuned": tuned,
           "checked": "sorted, payload follows its key, stable, in every segment",
           "plain_per_segment_calls": {"segments": m, "pairs": b - a,
                                       "value": (b - a) / (plain_ms / 1e3), "unit": UNIT}}
    if cpu_segments:
        out["cpu_thread_pool"] = cpu_batched_rate(keys, vals, off, cpu_segments)
    return out


def _signed_order(torch, k, key_type: str):
    """int64 values whose signed order is the key order of k (int64 storage)."""
    sign = torch.tensor(-(2 ** 63), dtype=torch.int64, device=k.device)
    if key_type == "u64":
        return k ^ sign
    if key_type == "i64":
        return k
    return torch.where(k >= 0, k, k ^ torch.tensor(2 ** 63 - 1, dtype=torch.int64, device=k.device))  # totalOrder


def configs_measure(z, torch, dev, stream, reps: int = 3):
    """The other workloads at their stated sizes, one line each (pairs/s from
    CUDA events around each sort, inputs restored between sorts):
    five laws at n = 10^7 with Eq. 1 (the plain path at the paper's scale),
    and the adversarial laws at n = 10^8 with the learned map and its Eq. 1
    fallback at 4x the mean bucket load (u64 dense interval, int64 recentred,
    float64 N(0,1) with +-inf and +-0).  Each output is checked: ordered, and
    every payload still names its key."""
    def run(name, keys_np, key_type, opts):
        n = keys_np.size
        kd = torch.from_numpy(keys_np.view(np.int64)).to(dev)
        vd = torch.arange(n, dtype=torch.int32, device=dev)
        kb, vb = torch.empty_like(kd), torch.empty_like(vd)
        ts = []
        for r in range(reps + 1):
            kb.copy_(kd)
            vb.copy_(vd)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            z.sort_pairs(kb, vb, key_type=key_type, opts=opts, stream=stream, check=False)
            e1.record(stream)
            rc = z.sync_status(stream)
            if rc != 0:
                raise z.ZsortError(rc, f"bench {name}")
            if r:
                ts.append(e0.elapsed_time(e1))
        st = z.last_stats(stream)
        o = _signed_order(torch, kb, key_type)
        assert bool((o[1:] >= o[:-1]).all()), f"{name}: not sorted"
        assert bool(torch.equal(kd[vb.to(torch.int64) & 0xFFFFFFFF], kb)), f"{name}: payload does not follow its key"
        ms = statistics.median(ts)
        row = {"n": n, "key_type": key_type, "value": n / (ms / 1e3), "unit": UNIT, "ms": round(ms, 3),
               "bytes_per_pair": round(st["bytes_algorithmic"] / n, 2), "max_level": st["max_level"],
               "top_map": ["zscore", "learned_pwl", "range", "mlp", "learned_split"][st["top_map"]],
               "learned_accepted": st["learned_accepted"], "learned_rejected": st["learned_rejected"],
               "sampled_stats": st["sampled_stats"], "guard_levels": st["guard_levels"]}
        del kd, vd, kb, vb, o
        return row

    out = {"paper_scale_1e7_eq1": {}, "adversarial_1e8_learned": {}}
    plain = z.default_opts(mapper=z.MAP_ZSCORE)
    for fam, gen in inputs.FAMILIES.items():
        out["paper_scale_1e7_eq1"][fam] = run(fam, gen(10 ** 7, 2), "u64", plain)
    learned = z.default_opts(mapper=z.MAP_LEARNED, fallback_ratio=4.0)
    n4 = 10 ** 8
    out["adversarial_1e8_learned"]["u64_dense_interval"] = run("u64 dense", inputs.dense_interval_u64(n4, 4), "u64",
                                                                learned)
    out["adversarial_1e8_learned"]["i64_recentred"] = run("i64", inputs.dense_interval_i64(n4, 4).view(np.uint64),
                                                           "i64", learned)
    out["adversarial_1e8_learned"]["f64_specials"] = run("f64", inputs.normal_f64_specials(n4, 4).view(np.uint64),
                                                          "f64", learned)
    torch.cuda.empty_cache()
    return out


def cpu_oracle_rate(n_sample: int, budget_s: float = 12.0):
    """Oracle pairs/s on bounded samples of the same two distributions, and
    std::stable_sort (one thread) on the same samples."""
    import oracle

    samples = [inputs.lognormal(n_sample, 40), inputs.gaussian_mixture(n_sample, 41)]
    vals = inputs.index_payload(n_sample)
    done, t_total, reps = 0, 0.0, 0
    while True:
        for keys in samples:
            t0 = time.perf_counter()
            oracle.zsort_pairs(keys, vals)
            t_total += time.perf_counter() - t0
            done += n_sample
        reps += 1
        if t_total >= budget_s or reps >= 8:
            break
    sdone, st_total = 0, 0.0
    for keys in samples:
        t0 = time.perf_counter()
        oracle.stdsort_pairs(keys, vals)
        st_total += time.perf_counter() - t0
        sdone += n_sample
    return done / t_total, t_total, reps, sdone / st_total


def cpu_batched_rate(keys, vals, off, nseg_sample: int):
    """The oracle's zSort over the first nseg_sample segments of a batch,
    shared out over a pool of one std::thread per host core, and the same
    segments on one thread (the thread pool's baseline)."""
    import oracle

    m = min(nseg_sample, off.size - 1)
    a, b = 0, int(off[m])
    k, v, o = keys[a:b], vals[a:b], off[: m + 1]
    t0 = time.perf_counter()
    _, _, threads = oracle.zsort_segmented_mt(k, v, o)
    t_mt = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.zsort_segmented_mt(k, v, o, threads=1)
    t_1 = time.perf_counter() - t0
    return {"segments": m, "pairs": b - a, "threads": threads, "value": (b - a) / t_mt,
            "value_one_thread": (b - a) / t_1, "unit": UNIT, "seconds": round(t_mt + t_1, 2)}


def pairs_config(logn: int, mapper_name: str, world: int = 1) -> dict:
    """The config of the pairs workload (the same dict in both arms)."""
    return {
        "workload": f"zsort_pairs, 2 arrays x n=2^{logn} (u64 key, u32 index): lognormal "
                    f"floor(exp(N(30,2))) and 8-component Gaussian mixture; mapper={mapper_name}",
        "pairs_per_step": 2 * (1 << logn),
        "l2": f"inputs ({3 * (1 << logn) >> 28} GiB per array) far larger than L2; restored between steps",
        "parallelism": "replicas" if world > 1 else "single GPU",
    }


def run_reference(args):
    """Reference arm: the CPU oracle, timed on this host, on the workload shape."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    n_sample = args.sample
    arrays = [inputs.lognormal(n_sample, 40), inputs.gaussian_mixture(n_sample, 41)]
    vals = inputs.index_payload(n_sample)
    for _ in range(args.warmup):
        for a in arrays:
            oracle.zsort_pairs(a, vals)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for a in arrays:
            oracle.zsort_pairs(a, vals)
        t.append(time.perf_counter() - t0)
    total = sum(t)
    value = len(arrays) * n_sample * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded numpy PCG64)",
        "config": dict(pairs_config(args.logn, args.mapper), pairs_per_step=len(arrays) * n_sample,
                       sample=f"each step sorts n={n_sample} pairs of each of the two laws (the GPU arm sorts "
                              f"2^{args.logn} of each)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", **host_info(),
                         "sample": f"each step sorts the two arrays' laws at n={n_sample} (lognormal and "
                                   f"8-component mixture) with the sequential C oracle on one host core; "
                                   f"pairs/s of that sample stand for the 2 x 2^{args.logn} workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="zsort", choices=["zsort", "reference"])
    ap.add_argument("--logn", type=int, default=28, help="log2 of pairs per array")
    ap.add_argument("--mapper", default="learned", choices=["learned", "zscore"])
    ap.add_argument("--sample", type=int, default=1 << 22, help="CPU oracle sample size")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-lanes", type=int, default=1, help="copy streams per direction in the e2e measurement")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the z-score comparison run")
    ap.add_argument("--workload", default="pairs", choices=["pairs", "batched"],
                    help="pairs: 2 x 2^logn arrays; batched: segmented sort of --segments arrays")
    ap.add_argument("--segments", type=int, default=20_000)
    ap.add_argument("--tune-cache", default=os.environ.get("ZSORT_TUNE_CACHE"),
                    help="autotuner cache file for the batched workload (default: $ZSORT_TUNE_CACHE, else none)")
    ap.add_argument("--tune-budget-ms", type=int, default=60_000)
    ap.add_argument("--batched-side", type=int, default=20_000,
                    help="segments of the batched measurement reported beside the pairs workload (0: none)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 10^7 and 10^8 workload lines")
    ap.add_argument("--no-link", action="store_true", help="skip the pinned host-link bandwidth measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import paper_2605_14419_gb300 as z
    from paper_2605_14419_gb300 import build as zbuild
    from paper_2605_14419_gb300 import replicas

    rank, world, local = replicas.world_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        zbuild.build()
    if world > 1:
        dist.barrier()
    z.load()

    if args.workload == "batched":
        res = batched_measure(z, torch, dev, args.segments, replicas.rank_seed(5, rank), args.steps, args.warmup,
                              2000, args.tune_cache, args.tune_budget_ms)
        # every rank sorts its own batch; the job's time is the slowest rank's
        job_value = replicas.job_rate(res["pairs"], res["ms"] / 1e3, dev)
        if rank == 0:
            line = {
                "metric": METRIC, "value": job_value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic (seeded numpy PCG64)",
                "config": {"workload": f"zsort_segmented, {args.segments} arrays, log-uniform sizes 32..2^20, "
                                       "each from one of five families (uniform, normal, zipf, nearly sorted, "
                                       "descending), one persistent launch from a CUDA graph",
                           "pairs_per_step": res["pairs"], "l2": "inputs far larger than L2; restored between steps"},
                "batched": res, "gpu_launches": 3 * args.steps,
            }
            print(json.dumps(line), flush=True)
        return

    n = 1 << args.logn
    work = make_workload(n, rank)
    pristine = []
    for name, keys in work:
        kd = torch.from_numpy(keys.view(np.int64)).to(dev)
        vd = torch.arange(n, dtype=torch.int32, device=dev)
        pristine.append((name, kd, vd))
    del work
    bufs = [(torch.empty_like(kd), torch.empty_like(vd)) for _, kd, vd in pristine]
    stream = torch.cuda.current_stream()
    z.reserve(n, 1, stream)
    mapper = z.MAP_LEARNED if args.mapper == "learned" else z.MAP_ZSCORE

    def restore():
        for (_, kd, vd), (kb, vb) in zip(pristine, bufs):
            kb.copy_(kd)
            vb.copy_(vd)

    def timed_sorts(opts, keys_only=False):
        """Sorts both arrays (keys_only: the keys alone, vals = NULL); returns
        per-array (ms, bytes, stats)."""
        out = []
        for kb, vb in bufs:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            z.sort_pairs(kb, None if keys_only else vb, opts=opts, check=False)
            e1.record(stream)
            rc = z.sync_status(stream)
            if rc != 0:
                raise z.ZsortError(rc, "bench sort")
            st = z.last_stats(stream)
            out.append((e0.elapsed_time(e1), st["bytes_algorithmic"], st))
        return out

    def run(opts, steps, warmup, keys_only=False):
        for _ in range(warmup):
            restore()
            timed_sorts(opts, keys_only)
        res = []
        for _ in range(steps):
            restore()
            torch.cuda.synchronize()
            res.append(timed_sorts(opts, keys_only))
        return res

    opts = z.default_opts(mapper=mapper)
    # warm-up, then the timed steps, clocks sampled meanwhile
    for _ in range(args.warmup):
        restore()
        timed_sorts(opts)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    res = []
    for _ in range(args.steps):
        restore()
        torch.cuda.synchronize()
        res.append(timed_sorts(opts))
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    step_ms = [sum(a[0] for a in step) for step in res]
    total_ms = sum(step_ms)
    total_ms = replicas.max_over_ranks(total_ms, dev)  # the slowest rank
    n_arrays = len(bufs)
    pairs_per_step = n * n_arrays
    value = world * pairs_per_step * args.steps / (total_ms / 1e3)
    kernel_ms = [a[0] for step in res for a in step]
    kernel_bytes = [a[1] for step in res for a in step]
    avg_ms = sum(kernel_ms) / len(kernel_ms)
    avg_bytes = sum(kernel_bytes) / len(kernel_bytes)
    peak, peak_kind = load_peaks()
    achieved = avg_bytes / (avg_ms / 1e3) / 1e9
    traffic_pp, traffic_note = measured_traffic_per_pair()
    last_stats = [a[2] for a in res[-1]]
    # correctness of the last timed outputs (cheap device-side checks)
    for (name, kd, _), (kb, vb) in zip(pristine, bufs):
        s = kb ^ torch.tensor(-(2 ** 63), dtype=torch.int64, device=dev)
        assert bool((s[1:] >= s[:-1]).all()), f"{name}: not sorted"
        pos = vb.to(torch.int64) & 0xFFFFFFFF
        assert bool(torch.equal(kd[pos], kb)), f"{name}: payload does not follow its key"

    plain = None
    if not args.no_plain and mapper == z.MAP_LEARNED:
        pres = run(z.default_opts(mapper=z.MAP_ZSCORE), max(3, args.steps // 2), 1)
        pms = sum(sum(a[0] for a in step) for step in pres)
        plain = {"value": pairs_per_step * len(pres) / (pms / 1e3), "unit": UNIT,
                 "mapper": "zscore (Eq. 1)",
                 "bytes_per_pair": sum(a[1] for step in pres for a in step) / (n * len(bufs) * len(pres)),
                 "per_array_ms": [round(sum(step[i][0] for step in pres) / len(pres), 3)
                                  for i in range(len(bufs))]}

    mappers = None
    if not args.no_plain:
        # top-level bucket imbalance of each map on the full arrays (largest
        # bucket over the mean), and the MLP map's sort time beside the others
        imb = {}
        for name, kd, _ in pristine:
            row = {}
            for label, mp in (("zscore", z.MAP_ZSCORE), ("learned_pwl", z.MAP_LEARNED), ("mlp", z.MAP_MLP)):
                b, info = z.map_buckets(kd, z.default_opts(mapper=mp))
                cnt = torch.bincount(b.to(torch.int64), minlength=info.k)
                row[label] = {"map_used": ["zscore", "learned_pwl", "range", "mlp", "learned_split"][info.map], "k": info.k,
                              "max_over_mean": round(float(cnt.max()) * info.k / n, 2)}
                del b, cnt
            imb[name] = row
        torch.cuda.empty_cache()
        mres = run(z.default_opts(mapper=z.MAP_MLP), max(3, args.steps // 2), 1)
        mms = sum(sum(a[0] for a in step) for step in mres)
        mappers = {"mlp": {"value": pairs_per_step * len(mres) / (mms / 1e3), "unit": UNIT,
                           "per_array_ms": [round(sum(step[i][0] for step in mres) / len(mres), 3)
                                            for i in range(len(bufs))]},
                   "imbalance": imb}

    u128 = None
    if not args.no_plain:
        # 128-bit keys (one zSort of each key's 64-bit window, then a gather),
        # half as many keys
        n128 = n // 2
        rng = np.random.default_rng(replicas.rank_seed(77, rank))
        w = torch.from_numpy(rng.integers(0, 2 ** 63, 2 * n128, dtype=np.int64)).to(dev)
        wb = torch.empty_like(w)
        vb128 = torch.empty(n128, dtype=torch.int32, device=dev)
        times = []
        for i in range(4):
            wb.copy_(w)
            vb128.copy_(torch.arange(n128, dtype=torch.int32, device=dev))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            z.sort_pairs_u128(wb, vb128, check=False)
            e1.record(stream)
            rc = z.sync_status(stream)
            if rc != 0:
                raise z.ZsortError(rc, "bench u128")
            if i:
                times.append(e0.elapsed_time(e1))
        hi = wb[1::2] ^ torch.tensor(-(2 ** 63), dtype=torch.int64, device=dev)
        assert bool((hi[1:] >= hi[:-1]).all()), "u128 output not sorted by its high word"
        u128 = {"value": n128 / (sum(times) / len(times) / 1e3), "unit": "pairs/s", "keys": n128,
                "key_bits": 128, "ms": round(sum(times) / len(times), 3),
                "method": "one stable zSort of the 64-bit window (key - min) >> s, "
                          "s = max(0, bitlen(max - min) - 64); tied windows sorted by the bits below; a gather",
                "tied_runs": "none (random 126-bit keys: the top 64 significant bits differ)"}
        del w, wb, vb128, hi
        torch.cuda.empty_cache()

    keys_only = None
    if not args.no_plain:
        kres = run(opts, max(3, args.steps // 2), 1, keys_only=True)
        kms = sum(sum(a[0] for a in step) for step in kres)
        for (name, kd, _), (kb, _vb) in zip(pristine, bufs):
            s_ = kb ^ torch.tensor(-(2 ** 63), dtype=torch.int64, device=dev)
            assert bool((s_[1:] >= s_[:-1]).all()), f"{name}: keys-only output not sorted"
        keys_only = {"value": pairs_per_step * len(kres) / (kms / 1e3), "unit": "keys/s",
                     "mode": "vals = NULL (the paper's key-only workload), same arrays and mapper",
                     "bytes_per_key": sum(a[1] for step in kres for a in step) / (n * len(bufs) * len(kres)),
                     "per_array_ms": [round(sum(step[i][0] for step in kres) / len(kres), 3)
                                      for i in range(len(bufs))]}

    e2e = None
    if not args.no_e2e:
        hk = [torch.empty(n, dtype=torch.int64, pin_memory=True) for _ in pristine]
        hv = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in pristine]
        for (_, kd, vd), a, b in zip(pristine, hk, hv):
            a.copy_(kd)
            b.copy_(vd)
        ok_k = [torch.empty(n, dtype=torch.int64, pin_memory=True) for _ in pristine]
        ok_v = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in pristine]
        torch.cuda.synchronize()

        # the copies run on their own streams, one per direction, so that one
        # array's transfers overlap the other's sort and the two directions
        # overlap each other.  Steps alternate between two sets of device
        # buffers: the next step's upload of an array goes into the other set
        # while this step's result is still being read back, so neither
        # direction waits for the other (with one set, each array's upload,
        # sort and read-back formed one serial chain per step).  Each
        # direction's copies can also be split over --e2e-lanes streams.
        E2E_LANES = max(1, args.e2e_lanes)
        h2d_s = [torch.cuda.Stream(device=dev) for _ in range(E2E_LANES)]
        d2h_s = [torch.cuda.Stream(device=dev) for _ in range(E2E_LANES)]
        bufsets = [bufs, [(torch.empty_like(kb), torch.empty_like(vb)) for kb, vb in bufs]]
        free = [[torch.cuda.Event() for _ in bufs] for _ in bufsets]
        for row in free:
            for ev in row:
                ev.record(d2h_s[0])
        step_no = [0]

        def pieces(t):
            step = (t.numel() + E2E_LANES - 1) // E2E_LANES
            return [t[j * step:(j + 1) * step] for j in range(E2E_LANES)]

        def e2e_step():
            bset = step_no[0] % 2
            step_no[0] += 1
            for i, (kb, vb) in enumerate(bufsets[bset]):
                arrived = []
                for j, (cs, dk, hk_j, dv, hv_j) in enumerate(zip(h2d_s, pieces(kb), pieces(hk[i]), pieces(vb),
                                                                 pieces(hv[i]))):
                    cs.wait_event(free[bset][i])
                    with torch.cuda.stream(cs):
                        dk.copy_(hk_j, non_blocking=True)
                        dv.copy_(hv_j, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(cs)
                    arrived.append(ev)
                for ev in arrived:
                    stream.wait_event(ev)
                z.sort_pairs(kb, vb, opts=opts, stream=stream, check=False)
                sorted_ev = torch.cuda.Event()
                sorted_ev.record(stream)
                back = []
                for cs, hk_j, dk, hv_j, dv in zip(d2h_s, pieces(ok_k[i]), pieces(kb), pieces(ok_v[i]), pieces(vb)):
                    cs.wait_event(sorted_ev)
                    with torch.cuda.stream(cs):
                        hk_j.copy_(dk, non_blocking=True)
                        hv_j.copy_(dv, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(cs)
                    back.append(ev)
                for ev in back[1:]:  # the buffer is free once every piece is back
                    d2h_s[0].wait_event(ev)
                free[bset][i].record(d2h_s[0])

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e_steps = max(6, args.steps)  # enough steps that the pipeline fill and drain amortise
        e0.record(stream)
        for cs in h2d_s + d2h_s:
            cs.wait_event(e0)
        for _ in range(e_steps):
            e2e_step()
        for row in free:  # every result is back on the host
            for ev in row:
                stream.wait_event(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        rc = z.sync_status(stream)
        if rc != 0:
            raise z.ZsortError(rc, "bench e2e")
        for i, (name, kd, _) in enumerate(pristine):  # the host copies hold the sorted result
            hk_sorted = ok_k[i].numpy().view(np.uint64)
            assert bool(np.all(hk_sorted[1:] >= hk_sorted[:-1])), f"e2e {name}: not sorted"
            head = ok_v[i][:4096].to(dev).to(torch.int64) & 0xFFFFFFFF
            assert bool(torch.equal(kd[head], ok_k[i][:4096].to(dev))), f"e2e {name}: payload does not follow its key"
        ems = replicas.max_over_ranks(e0.elapsed_time(e1), dev)  # the slowest rank
        e2e = {"value": world * pairs_per_step * e_steps / (ems / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": pairs_per_step * BYTES_PER_PAIR,
               "d2h_bytes_per_step": pairs_per_step * BYTES_PER_PAIR}
        del hk, hv, ok_k, ok_v, bufsets

    link = None
    if not args.no_e2e and not args.no_link:
        link = link_bandwidth(torch, dev)
        if e2e is not None:
            # the bound the e2e step time has to respect: both arrays' pairs
            # each way per step over the measured link
            per_dir = pairs_per_step * BYTES_PER_PAIR / 1e9
            link["e2e_copy_bound_ms"] = round(1e3 * per_dir / min(link["h2d_gbs"], link["d2h_gbs"]), 2)
            link["e2e_ms_per_step"] = round(1e3 * pairs_per_step / e2e["value"] * world, 2)

    array_names = [name for name, _, _ in pristine]
    del bufs
    torch.cuda.empty_cache()
    configs = None
    if not args.no_configs:
        configs = configs_measure(z, torch, dev, stream)

    del pristine
    torch.cuda.empty_cache()
    batched = None
    if args.batched_side > 0:
        batched = batched_measure(z, torch, dev, args.batched_side, 5, 5, 3, min(args.batched_side, 2000),
                                  args.tune_cache, min(args.tune_budget_ms, 20_000),
                                  cpu_segments=4000 if (rank == 0 and not args.no_cpu) else 0)

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, secs, reps, std_rate = cpu_oracle_rate(args.sample)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"lognormal + gmm8, {args.sample} pairs each, {reps} rounds, {secs:.1f} s, one thread",
               "std_stable_sort": {"value": std_rate, "unit": UNIT, "cores": 1,
                                   "sample": "the same two samples, std::stable_sort by key, one thread"},
               **host_info()}
        if batched and "cpu_thread_pool" in batched:
            cpu["batched_thread_pool"] = batched["cpu_thread_pool"]

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded numpy PCG64)",
        "config": pairs_config(args.logn, args.mapper, world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": None if traffic_pp is None else traffic_pp * n, "traffic_note": traffic_note,
                     "peak_kind": peak_kind,
                     "kernel": "k_persistent (whole zsort_pairs call)",
                     "algorithmic_bytes_per_launch": avg_bytes, "avg_launch_ms": avg_ms},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": 3 * n_arrays * args.steps,
        "per_array": [{"array": name, "ms": round(sum(step[i][0] for step in res) / len(res), 3),
                       "bytes_per_pair": round(last_stats[i]["bytes_algorithmic"] / n, 2),
                       "max_level": last_stats[i]["max_level"],
                       "top_map": last_stats[i]["top_map"],
                       "leaves": last_stats[i]["leaves"],
                       "learned_accepted": last_stats[i]["learned_accepted"]}
                      for i, name in enumerate(array_names)],
        "plain_zscore": plain,
        "keys_only": keys_only,
        "u128": u128,
        "mappers": mappers,
        "batched": batched,
        "configs": configs,
        "link": link,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
