"""Benchmark of the GB300 load-balanced sample sort.

`python bench.py --gpus N --steps K --warmup W` sorts the 256M-key workload
(2^28 uint64 keys, half normal / half right-skewed lognormal, uint32 index
payload, P = 128 logical partitions) once per step, out of place, with inputs
resident in HBM, and prints one JSON line.  Under torchrun (N > 1) the ranks
sort ONE global array of N x 2^28 keys, shard r on rank r, with the paper's
distributed steps over NCCL (weak scaling); --replicas makes every rank sort
its own instance instead.

`--impl reference` times the CPU oracle instead, on a bounded sample of the same
workload, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1611_00463_gb300 import inputs  # noqa: E402

METRIC = "Gkeys/s & % HBM roofline; max/mean bucket load; learned vs sampled splitters"
L2_BYTES = 129 * 1000 * 1000          # GB300 L2
DEFAULT_WORKLOAD = "normal_lognormal_u64"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pgs", choices=["pgs", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(inputs.WORKLOADS) + ["batched"])
    ap.add_argument("--splitters", default="sampled", choices=["sampled", "learned"])
    ap.add_argument("--investigator", default="rank", choices=["rank", "equal", "off", "local"],
                    help="step 4 rule for duplicated splitters (local = the per-run division, not stable)")
    ap.add_argument("--guaranteed", action="store_true", help="oversample so every bucket < (1+eps) n/P")
    ap.add_argument("--instances", type=int, default=10000, help="batched workload: number of instances")
    ap.add_argument("--n", type=int, default=None, help="override the number of keys (smaller cases)")
    ap.add_argument("--P", type=int, default=None)
    ap.add_argument("--exchange", default="auto", choices=["auto", "scatter", "fused"])
    ap.add_argument("--merge-ways", type=int, default=0, choices=[0, 2, 4], help="lists merged per pass (0 = the library's choice: four-way from 2^23 keys)")
    ap.add_argument("--tile-variant", type=int, default=0, choices=[0, 1, 2, 3],
                    help="merge tile shape (0 = default; see pgs_config.tile_variant)")
    ap.add_argument("--samples-per-run", type=int, default=0, help="regular samples per run (0 = the paper's budget)")
    ap.add_argument("--search-queries", type=int, default=0,
                    help="time pgs_search of this many queries on the sorted workload instead")
    ap.add_argument("--sweep-samples", action="store_true",
                    help="time the sort at the paper's sample sizes 0.004X .. 1.4X (X = 256 KB / P) instead")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: every rank sorts its own array (default: one array sharded over the ranks)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-timer", action="store_true", help="skip per-launch events (profiling runs)")
    ap.add_argument("--no-comparator", action="store_true", help="skip the torch.sort(stable=True) context line")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region.

    Sampling starts on entry and the entry waits for the first sample, so the
    sampler is live before the timed region begins; every sample carries the
    host time it arrived at, and the summary keeps the samples taken between
    mark_start() and mark_end() (plus the first one after, which covers the
    region's last interval).  Without marks every sample counts."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms",
                 str(self.INTERVAL_MS), "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            deadline = time.perf_counter() + 5.0
            while not self.lines and time.perf_counter() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.perf_counter(), ln.strip()))

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()
        if self.proc is not None:                     # let the sample covering the last interval arrive
            time.sleep(self.INTERVAL_MS * 1.5e-3)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def window(self) -> list[str]:
        if self.t0 is None or self.t1 is None:
            return [ln for _, ln in self.lines]
        inside = [ln for t, ln in self.lines if self.t0 <= t <= self.t1]
        after = [ln for t, ln in self.lines if t > self.t1]
        return inside + after[:1]

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.window():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": self.INTERVAL_MS}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device, world: int) -> float:
    """The largest of every rank's value (a time: the job ends with its slowest rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(keys_per_rank: int, world: int, seconds: float) -> float:
    """Gkeys/s of the whole job: every rank's keys over the slowest rank's time (weak scaling)."""
    return keys_per_rank * world / seconds / 1e9


def kernel_source_hash(kernel: str = "k_merge_tile") -> str:
    """Hash of one kernel's source text (its template header to its closing
    brace) plus the PTX helpers it uses, so committed counters are used only
    for the kernel they were taken on."""
    src = open(os.path.join(ROOT, "paper_1611_00463_gb300", "csrc", "pgs_kernels.cuh")).read()
    start = src.index(kernel + "(")
    start = src.rfind("template", 0, start)
    end = src.index("\n}\n", start) + 3
    h = hashlib.sha256(src[start:end].encode())
    h.update(open(os.path.join(ROOT, "paper_1611_00463_gb300", "csrc", "pgs_ptx.cuh"), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str, n: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to n keys, or None if absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    src_kernel = {"merge": "k_merge_tile", "merge4": "k_merge4", "block_sort": "k_block_sort"}.get(kernel, kernel)
    vals = {}
    for ln in open(path):
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    try:
        if vals.get("source_hash") != kernel_source_hash(src_kernel):
            return None
        per_key = float(vals["dram_bytes_per_launch"]) / float(vals["keys_per_launch"])
        return per_key * n
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_step(keys, vals, P, dtype):
    from oracle import pgs_oracle as O
    O.stable_sort(keys, vals, dtype)
    O.buckets(keys, P, dtype)


def time_oracle(workload: str, P: int, sample_n: int, steps: int, warmup: int):
    dtype, keys, _ = inputs.workload(workload, n=sample_n)
    vals = inputs.index_payload(sample_n)
    for _ in range(warmup):
        oracle_step(keys, vals, P, dtype)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle_step(keys, vals, P, dtype)
    dt = (time.perf_counter() - t0) / steps
    return sample_n / dt / 1e9, dt, dtype


def cpu_parallel_sort_rate(workload: str, n: int, P: int, steps: int, warmup: int):
    """The oracle's stable sort on every host core (oracle/cpu_sort.c) over the
    workload's full keys: (Gkeys/s, seconds per sort, threads, dtype)."""
    from oracle import cpu_sort
    dtype, keys, _ = inputs.workload(workload, n=n)
    vals = inputs.index_payload(n)
    T = cpu_sort.threads_available()
    for _ in range(warmup):
        cpu_sort.stable_sort(keys, vals, dtype, T)
    t0 = time.perf_counter()
    for _ in range(steps):
        cpu_sort.stable_sort(keys, vals, dtype, T)
    dt = (time.perf_counter() - t0) / steps
    return n / dt / 1e9, dt, T, dtype


def cpu_baseline_block(args, n, P, steps=1, warmup=0):
    """cpu_baseline: the full workload on all host cores, with the one-thread
    numpy oracle on a bounded sample beside it."""
    from oracle import cpu_sort
    v, dt, T, dtype = cpu_parallel_sort_rate(args.workload, n, P, steps, warmup)
    sample_n = min(n, 1 << 24)
    v1, dt1, _ = time_oracle(args.workload, P, sample_n, 1, 0)
    return {"value": v, "unit": "Gkeys/s", "cores": T, "threads": T, "kind": "oracle",
            "cpu_model": cpu_sort.cpu_model(), "nproc": os.cpu_count(),
            "sample": f"the whole workload ({n} {dtype} keys + uint32 payload): the oracle's stable sort on "
                      f"(total-order key, input position), C, {T} threads (chunk merge sorts, then pairwise "
                      f"merges split by merge path over all threads), {dt:.2f} s per sort",
            "oracle_1thread": {"value": v1, "unit": "Gkeys/s",
                               "sample": f"first {sample_n} keys: numpy oracle stable sort + steps 1-4 "
                                         f"bucket vector, one thread, {dt1:.1f} s"}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "batched":
        return run_reference_batched(args)
    from oracle import cpu_sort
    dtype, n, P, _, _ = workload_shape(args)
    value, dt, T, _ = cpu_parallel_sort_rate(args.workload, n, P, args.steps, args.warmup)
    cpu = {"value": value, "unit": "Gkeys/s", "cores": T, "threads": T, "kind": "oracle",
           "cpu_model": cpu_sort.cpu_model(), "nproc": os.cpu_count(),
           "sample": f"the whole workload ({n} {dtype} keys + uint32 payload) every step: the oracle's stable "
                     f"sort, C, {T} threads"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": config_block(args, dtype, n, P, None),
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_batched(args):
    """The oracle on the first instances of the batched workload (bounded sample)."""
    from oracle import pgs_oracle as O
    sizes = inputs.batched_sizes(args.instances)
    P = inputs.batched_partitions(sizes)
    take, total = 0, 0
    while take < len(sizes) and total + sizes[take] <= (1 << 23):
        total += int(sizes[take])
        take += 1
    take = max(take, 1)
    inst = [inputs.batched_instance_keys(i, int(sizes[i])) for i in range(take)]
    n = sum(len(k) for k in inst)

    def step():
        for i, k in enumerate(inst):
            O.stable_sort(k, np.arange(len(k), dtype=np.uint32), "u64")
            O.buckets(k, int(P[i]), "u64")
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = n / dt / 1e9
    sample = f"first {take} instances of the batched workload ({n} keys): oracle stable sort + bucket vector, one thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "batched", "instances": args.instances},
            "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_shape(args):
    dtype, n0, P0, gen, seed = inputs.WORKLOADS[args.workload]
    n = args.n or n0
    P = args.P or P0
    return dtype, n, P, gen, seed


def l2_flush(n, keys):
    """True when the keys and payloads fit in L2, so the timed steps flush it."""
    return n * (keys.element_size() + 4) < L2_BYTES


def l2_note(n, key_bytes):
    if n * (key_bytes + 4) < L2_BYTES:
        return ("inputs smaller than L2: a write of twice the L2 evicts them before every timed step, "
                "each step timed alone")
    return "inputs larger than L2 (no flush between steps)"


def config_block(args, dtype, n, P, stats):
    c = {
        "workload": f"{args.workload}: {n} {dtype} keys + uint32 index payload, P={P} logical partitions, "
                    "stable ascending sort, out of place",
        "n": n, "P": P, "key": dtype, "payload": "u32 index",
        "l2": l2_note(n, 8 if dtype == "u64" else 4),
        "exchange": args.exchange,
        "merge_ways": args.merge_ways or (4 if n >= (1 << 23) else 2),
        "samples_per_run_option": getattr(args, "samples_per_run", 0) or "paper budget",
        "tile_variant": getattr(args, "tile_variant", 0),
        "splitters": args.splitters,
        "investigator": getattr(args, "investigator", "rank"),
        "guaranteed": bool(args.guaranteed),
    }
    if stats:
        c["passes"] = stats["passes"]
        c["samples_per_run"] = stats["samples_per_run"]
    return c


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_batched(args):
    """The batched workload: ~10,000 uneven uint64 instances with uint32
    payload in one CUDA-graph replay of the batched sort (tile shape chosen by
    the tuner), against per-instance pgs_sort_copy launches."""
    import torch
    import torch.distributed as dist

    from paper_1611_00463_gb300 import build as pbuild
    from paper_1611_00463_gb300 import pgs

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        pbuild.build()
    if world > 1:
        dist.barrier()
    pgs.load()
    t_gen = time.time()
    offsets, keys_np, P = inputs.batched(args.instances, seed=4 + 100 * rank)
    t_gen = time.time() - t_gen
    n = int(offsets[-1])
    vals_np = np.arange(n, dtype=np.uint32)
    kin = torch.from_numpy(keys_np.view(np.int64)).to(dev)
    vin = torch.from_numpy(vals_np.view(np.int32)).to(dev)
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    bt = pgs.Batch(offsets, P, dtype="u64", with_vals=True, device=dev)
    chosen, tune_ms = bt.tune(kout, vout)
    st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device=dev)
    cfg = bt.config(stats=st)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bt.sort_copy(kin, vin, kout, vout, stream=s, cfg=cfg)
    torch.cuda.synchronize(dev)
    for _ in range(max(args.warmup, 0)):
        g.replay()
    torch.cuda.synchronize(dev)
    stats = pgs.pgs_get_stats(st)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream(dev)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks.mark_start()
        ev0.record(cur)
        for _ in range(args.steps):
            g.replay()
        ev1.record(cur)
        torch.cuda.synchronize(dev)
        clocks.mark_end()
        if world > 1:
            dist.barrier()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev, world)
    value = whole_job_rate(n, world, ms_step * 1e-3)
    # The same instances, one pgs_sort_copy call (its own launch sequence) each.
    per = None
    if rank == 0:
        sizes = np.diff(offsets).astype(np.int64)
        ws = pgs.workspace(int(sizes.max()), int(P.max()), pgs.make_config(dtype="u64"), dev)
        cfgi = pgs.make_config(dtype="u64", workspace=ws)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for i in range(len(sizes)):
            a, b = int(offsets[i]), int(offsets[i + 1])
            pgs.pgs_sort_copy(kin[a:b], vin[a:b], kout[a:b], vout[a:b], int(P[i]), cfgi)
        e1.record(cur)
        torch.cuda.synchronize(dev)
        pms = e0.elapsed_time(e1)
        per = {"ms": pms, "value": n / (pms * 1e-3) / 1e9, "unit": "Gkeys/s",
               "speedup_of_batched": pms / ms_step}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"batched: {args.instances} instances, {n} uint64 keys + uint32 payload, "
                                   "lognormal sizes 1K..16M, per-instance distribution by seed, "
                                   "P_i = clamp(2^floor(log2(n_i/2^16)), 1, 256); one CUDA-graph replay "
                                   "of the batched sort per step, out of place",
                       "n": n, "instances": args.instances, "P_sum": int(P.sum()),
                       "tile_variant": chosen, "tune_ms": tune_ms, "generation_s": t_gen,
                       "passes": stats["passes"], "l2": "inputs larger than L2 (no flush between steps)"},
            "max_over_mean_bucket": stats["max_over_mean"],
            "gpu_launches": stats["launches"] * args.steps,
            "launches_per_step": stats["launches"],
            "per_instance_launches": per,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


SWEEP_FRACTIONS = [0.004, 0.04, 0.4, 1.0, 1.004, 1.04, 1.4]   # the sample sizes of Fig. 9 and 10


def run_sweep(args):
    """The sort at the paper's sample sizes f X, X = 256 KB / P of keys per run
    (Section V, Fig. 9 and 10): time per sort, per-step times, and the smallest
    and largest bucket, one point per size, in one JSON line."""
    import torch
    from paper_1611_00463_gb300 import build as pbuild
    from paper_1611_00463_gb300 import pgs
    pbuild.build()
    pgs.load()
    dev = torch.device("cuda", 0)
    dtype, n, P, gen, seed = workload_shape(args)
    keys_np = gen(n, seed)
    kin = pgs.as_device_keys(keys_np, dtype, dev)
    vin = torch.from_numpy(inputs.index_payload(n).view(np.int32)).to(dev)
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    w = kin.element_size()
    X = 262144 // (P * w)
    stream = torch.cuda.current_stream(dev)
    points = []
    with ClockSampler(0) as clocks:
        for f in SWEEP_FRACTIONS:
            s_run = max(1, int(f * X))
            opts = dict(dtype=dtype, exchange=args.exchange, merge_ways=args.merge_ways,
                        tile_variant=args.tile_variant, samples_per_run=s_run)
            ws = pgs.workspace(n, P, pgs.make_config(**opts), dev)
            st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device=dev)
            cfg = pgs.make_config(workspace=ws, stats=st, **opts)
            for _ in range(max(args.warmup, 0)):
                pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg, stream)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            ev0.record(stream)
            for _ in range(args.steps):
                pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg, stream)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            ms = ev0.elapsed_time(ev1) / args.steps
            timer = pgs.Timer(capacity=512)
            pgs.pgs_sort_copy(kin, vin, kout, vout, P, pgs.make_config(workspace=ws, stats=st, timer=timer, **opts),
                              stream)
            torch.cuda.synchronize(dev)
            recs, _ = timer.read()
            step_ms = {}
            for r in recs:
                step_ms[str(r["step"])] = step_ms.get(str(r["step"]), 0.0) + r["ms"]
            stv = pgs.pgs_get_stats(st, stream)
            mean = n / stv["P"]
            points.append({"fraction_of_X": f, "samples_per_run": s_run, "ms_per_sort": ms,
                           "Gkeys_per_s": n / (ms * 1e-3) / 1e9, "max_bucket": stv["max_bucket"],
                           "min_bucket": stv["min_bucket"], "max_over_mean": stv["max_bucket"] / mean,
                           "min_over_mean": stv["min_bucket"] / mean,
                           "load_difference": stv["max_bucket"] - stv["min_bucket"],
                           "per_step_ms": step_ms})
            del ws
    line = {"sweep": "samples_per_run", "workload": args.workload, "n": n, "P": P, "key": dtype,
            "X_keys_per_run": X, "steps": args.steps, "warmup": args.warmup, "points": points,
            "clocks": clocks.summary(),
            "note": "X = 256 KB / P of keys per run (Section V); per_step_ms keys are the steps of Section IV "
                    "(1 local sort, 2 sampling, 3 splitters, 4 cut search + investigator, 5 offsets/exchange, "
                    "6 bucket merge) from one extra timed sort"}
    print(json.dumps(line), flush=True)


def run_search(args):
    """pgs_search on the sorted workload: M queries (half of them keys of the
    array, half fresh draws of the same generator), lower bound plus bucket,
    CUDA-event time over the steps; checked against the oracle on a sample."""
    import torch
    from paper_1611_00463_gb300 import build as pbuild
    from paper_1611_00463_gb300 import pgs
    from oracle import pgs_oracle as O
    pbuild.build()
    pgs.load()
    dev = torch.device("cuda", 0)
    dtype, n, P, gen, seed = workload_shape(args)
    keys_np = gen(n, seed)
    kin = pgs.as_device_keys(keys_np, dtype, dev)
    kout = torch.empty_like(kin)
    cfg0 = pgs.make_config(dtype=dtype)
    ws = pgs.workspace(n, P, cfg0, dev)
    e = torch.zeros(P + 1, dtype=torch.int64, device=dev)
    pgs.pgs_sort_copy(kin, None, kout, None, P, pgs.make_config(dtype=dtype, workspace=ws, bucket_bounds=e))
    torch.cuda.synchronize(dev)
    del ws
    M = args.search_queries
    g = np.random.default_rng(seed + 99)
    hit_idx = torch.from_numpy(g.integers(0, n, size=M // 2)).to(dev)
    fresh = pgs.as_device_keys(gen(M - M // 2, seed + 100), dtype, dev)
    q = torch.cat([kout[hit_idx], fresh])
    q = q[torch.from_numpy(g.permutation(M)).to(dev)].contiguous()
    pos = torch.empty(M, dtype=torch.int64, device=dev)
    bkt = torch.empty(M, dtype=torch.int32, device=dev)
    sws = torch.empty(max(1, pgs.pgs_search_workspace_bytes(n, dtype)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # The plain bisection once, for comparison with the indexed search timed below.
    t_plain = []
    for k in range(max(args.warmup, 0) + 2):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pgs.pgs_search(kout, q, pos, dtype=dtype, bucket_bounds=e, bucket_out=bkt, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        t_plain.append(ev0.elapsed_time(ev1))
    for _ in range(max(args.warmup, 0)):
        pgs.pgs_search(kout, q, pos, dtype=dtype, bucket_bounds=e, bucket_out=bkt, workspace=sws, stream=stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        torch.cuda.synchronize(dev)
        clocks.mark_start()
        ev0.record(stream)
        for _ in range(args.steps):
            pgs.pgs_search(kout, q, pos, dtype=dtype, bucket_bounds=e, bucket_out=bkt, workspace=sws, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        clocks.mark_end()
    ms = ev0.elapsed_time(ev1) / args.steps
    # Oracle check on a sample of the queries (the sorted array is the CUDA sort's output).
    samp = torch.from_numpy(g.integers(0, M, size=min(M, 1 << 16))).to(dev)
    sorted_np = pgs.to_numpy_keys(kout, dtype)
    q_np = pgs.to_numpy_keys(q[samp].contiguous(), dtype)
    want = O.search(sorted_np, q_np, dtype, "left")
    ok = bool(np.array_equal(pos[samp].cpu().numpy(), want) and
              np.array_equal(bkt[samp].cpu().numpy(), O.bucket_of(want, e.cpu().numpy())))
    line = {"mode": "search", "metric": "Gqueries/s (pgs_search lower bound + bucket on the sorted workload)",
            "value": M / (ms * 1e-3) / 1e9, "unit": "Gqueries/s", "ms_per_step": ms, "queries": M, "n": n, "P": P,
            "key": dtype, "workload": args.workload, "steps": args.steps, "warmup": args.warmup,
            "sample_checked_against_oracle": ok, "clocks": clocks.summary(),
            "index": "every 64th key copied to the workspace (rebuilt every call, inside the timed region)",
            "plain_bisection": {"ms": min(t_plain[-2:]), "value": M / (min(t_plain[-2:]) * 1e-3) / 1e9},
            "queries_recipe": "half keys of the sorted array at random positions, half fresh draws of the same "
                              "generator, shuffled"}
    print(json.dumps(line), flush=True)


def order_as_signed(k, dtype: str):
    """Raw key bits (int64 for u64, int32 otherwise) -> a signed integer of the
    same width whose order is the key order (float32: IEEE totalOrder); the map
    is its own inverse."""
    import torch
    if dtype == "u64":
        return k ^ torch.iinfo(torch.int64).min
    if dtype == "u32":
        return k ^ torch.iinfo(torch.int32).min
    return k ^ ((k >> 31) & 0x7FFFFFFF)


def library_comparator(kin, vin, kout, vout, dtype, args, dev, world):
    """Context, not a baseline: the same stable sort through a library call,
    torch.sort(stable=True) on the order-mapped keys plus a gather of the
    payloads by the returned permutation, timed like the main arm; its output
    is compared with this library's bit for bit."""
    import torch
    stream = torch.cuda.current_stream(dev)

    def step():
        sk, idx = torch.sort(order_as_signed(kin, dtype), stable=True)
        return order_as_signed(sk, dtype), vin[idx]
    try:
        for _ in range(max(args.warmup, 1)):
            ko, vo = step()
        same = bool(torch.equal(ko, kout) and torch.equal(vo, vout))
        del ko, vo
        flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev) if l2_flush(kin.numel(), kin) else None
        torch.cuda.synchronize(dev)
        total = 0.0
        evs = []
        for i in range(args.steps if flush is not None else 1):
            if flush is not None:
                flush.fill_(i & 0xFF)                    # as the main arm: inputs evicted before every step
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(1 if flush is not None else args.steps):
                step()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        total = sum(a.elapsed_time(b) for a, b in evs)
        ms = max_over_ranks(total / args.steps, dev, world)
        return {"call": "torch.sort(order-mapped keys, stable=True) + payload gather by the permutation",
                "ms_per_step": ms, "value": whole_job_rate(kin.numel(), world, ms * 1e-3), "unit": "Gkeys/s",
                "outputs_equal": same}
    except RuntimeError as ex:                           # e.g. out of memory: report why, keep the line
        torch.cuda.empty_cache()
        return {"unavailable": str(ex).splitlines()[0][:200]}


def run_sharded(args):
    """--gpus N under torchrun: ONE global array of N x n keys, shard r (n keys,
    the workload's generator with seed + r) on rank r, sorted by the paper's
    distributed form (paper_1611_00463_gb300.sharded: local sort, sample and
    count all-gathers over NCCL, investigator cuts, all-to-all of segments,
    merge).  Rank b ends with bucket b.  Per-rank work is fixed as N grows
    (weak scaling); the whole-job rate is N x n keys over the slowest rank."""
    import torch
    import torch.distributed as dist

    from paper_1611_00463_gb300 import build as pbuild
    from paper_1611_00463_gb300 import pgs
    from paper_1611_00463_gb300.sharded import CudaSteps, sharded_sort

    world, rank, local = dist_env()
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        pbuild.build()
    dist.barrier()
    pgs.load()
    dtype, n, P, gen, seed = workload_shape(args)
    keys_np = gen(n, seed + rank)
    kin = pgs.as_device_keys(keys_np, dtype, dev)
    vin = torch.from_numpy((inputs.index_payload(n) + np.uint32((rank * n) & 0xFFFFFFFF)).view(np.int32)).to(dev)
    opts = dict(exchange=args.exchange, guaranteed=args.guaranteed, merge_ways=args.merge_ways,
                tile_variant=args.tile_variant, samples_per_run=args.samples_per_run, investigator=args.investigator)
    steps = CudaSteps(dtype, dev, **opts)
    for _ in range(max(args.warmup, 0)):
        out = sharded_sort(kin, vin, dtype=dtype, steps=steps)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        dist.barrier()
        torch.cuda.synchronize(dev)
        clocks.mark_start()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            out = sharded_sort(kin, vin, dtype=dtype, steps=steps)
        torch.cuda.synchronize(dev)
        dt = (time.perf_counter() - t0) / args.steps
        clocks.mark_end()
        dist.barrier()
    dt = max_over_ranks(dt, dev, world)
    e = out[2].cpu().numpy()
    if rank == 0:
        N = world * n
        sizes = np.diff(e)
        line = {
            "metric": METRIC, "value": whole_job_rate(n, world, dt), "unit": "Gkeys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": f"{args.workload}: one global array of {world} x {n} {dtype} keys + uint32 "
                                   f"payload, shard r on rank r (seed + r), sorted across the ranks",
                       "n_per_rank": n, "N": N, "P": world, "parallelism": f"sharded{world}",
                       "collectives": "NCCL all-gather (sizes, samples, counts), all-to-all-v (segments)",
                       "l2": "inputs larger than L2"},
            "max_over_mean_bucket": float(sizes.max() / (N / world)),
            "roofline": None, "e2e": None, "cpu_baseline": None,
            "clocks": clocks.summary(),
            "timing": "host clock around K steps between barriers and device synchronisation, max over ranks",
        }
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def main():
    args = parse()
    if args.sweep_samples:
        return run_sweep(args)
    if args.search_queries:
        return run_search(args)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if dist_env()[0] > 1 and not args.replicas:
        run_sharded(args)
        return
    import torch
    import torch.distributed as dist

    from paper_1611_00463_gb300 import build as pbuild
    from paper_1611_00463_gb300 import pgs

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        pbuild.build()
    if world > 1:
        dist.barrier()
    pgs.load()

    dtype, n, P, gen, seed = workload_shape(args)
    keys_np = gen(n, seed + rank)               # every rank sorts its own instance
    vals_np = inputs.index_payload(n)
    kin = pgs.as_device_keys(keys_np, dtype, dev)
    vin = torch.from_numpy(vals_np.view(np.int32)).to(dev)
    kout = torch.empty_like(kin)
    vout = torch.empty_like(vin)
    opts = dict(dtype=dtype, exchange=args.exchange, splitters=args.splitters, guaranteed=args.guaranteed,
                merge_ways=args.merge_ways, tile_variant=args.tile_variant, samples_per_run=args.samples_per_run,
                investigator=args.investigator)
    cfg0 = pgs.make_config(**opts)
    ws = pgs.workspace(n, P, cfg0, dev)
    st = torch.zeros(pgs.STATS_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    timer = None if args.no_timer else pgs.Timer(capacity=(1024 if args.splitters == "learned" else 256) * (args.steps + 1))
    cfg_plain = pgs.make_config(workspace=ws, stats=st, **opts)
    cfg_timed = pgs.make_config(workspace=ws, stats=st, timer=timer, **opts)

    for _ in range(max(args.warmup, 0)):
        pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg_plain, stream)
    torch.cuda.synchronize(dev)

    # The timed region: the steps exactly as a caller runs them.  Inputs
    # smaller than L2 would stay cached from one step to the next, so then a
    # write of twice the L2 evicts them before every step and each step is
    # timed alone.
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev) if l2_flush(n, kin) else None

    def timed_steps(cfg):
        if flush is None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg, stream)
            e1.record(stream)
            return lambda: e0.elapsed_time(e1)
        evs = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg, stream)
            e1.record(stream)
            evs.append((e0, e1))
        return lambda: sum(a.elapsed_time(b) for a, b in evs)

    with ClockSampler(torch.cuda.current_device()) as clocks:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks.mark_start()
        elapsed = timed_steps(cfg_plain)
        torch.cuda.synchronize(dev)
        clocks.mark_end()
        if world > 1:
            dist.barrier()
    ms_total = max_over_ranks(elapsed(), dev, world)
    ms_step = ms_total / args.steps
    value = whole_job_rate(n, world, ms_step * 1e-3)
    stats = pgs.pgs_get_stats(st, stream)                # every call writes the same statistics

    # The timed calls above replay the launch sequence that the library
    # captured on the warm-up's second identical call (pgs_graph_cache AUTO);
    # the same steps with every launch issued from the host are reported beside.
    cfg_direct = pgs.make_config(workspace=ws, stats=st, graph_cache="off", **opts)
    torch.cuda.synchronize(dev)
    elapsed_direct = timed_steps(cfg_direct)
    torch.cuda.synchronize(dev)
    dms = max_over_ranks(elapsed_direct() / args.steps, dev, world)
    direct = {"ms_per_step": dms, "value": whole_job_rate(n, world, dms * 1e-3), "unit": "Gkeys/s"}

    # The same steps again with a CUDA-event pair around every launch on the
    # sort's stream: the per-kernel durations of the roofline and the per-step
    # breakdown (the events themselves add a little time between launches).
    ms_instr = None
    if timer:
        timer.reset()
        torch.cuda.synchronize(dev)
        elapsed_instr = timed_steps(cfg_timed)
        torch.cuda.synchronize(dev)
        ms_instr = elapsed_instr() / args.steps

    # The same sort replayed from a CUDA graph (captured once): what the launch
    # sequence costs without the host's per-launch work, reported beside it.
    graph = None
    try:
        gs = torch.cuda.Stream(dev)
        gs.wait_stream(stream)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=gs):
            pgs.pgs_sort_copy(kin, vin, kout, vout, P, cfg_plain, gs)
        for _ in range(max(args.warmup, 1)):
            cg.replay()
        torch.cuda.synchronize(dev)
        gevs = []
        cur = torch.cuda.current_stream(dev)
        for i in range(args.steps if flush is not None else 1):
            if flush is not None:
                flush.fill_(i & 0xFF)
            gev0, gev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            gev0.record(cur)
            for _ in range(1 if flush is not None else args.steps):
                cg.replay()
            gev1.record(cur)
            gevs.append((gev0, gev1))
        torch.cuda.synchronize(dev)
        gms = max_over_ranks(sum(a.elapsed_time(b) for a, b in gevs) / args.steps, dev, world)
        graph = {"ms_per_step": gms, "value": whole_job_rate(n, world, gms * 1e-3), "unit": "Gkeys/s"}
        del cg
    except RuntimeError as ex:                           # capture unavailable: report why, keep the line
        graph = {"unavailable": str(ex).splitlines()[0][:200]}

    comparator = None if args.no_comparator else library_comparator(kin, vin, kout, vout, dtype, args, dev, world)

    # Dominant kernel and its roofline, from the launch timer of the timed region.
    peak, peak_src = peaks()
    roof, per_kernel, step_ms, kernel_roofs = None, {}, {}, {}
    if timer:
        recs, dropped = timer.read()
        for r in recs:
            d = per_kernel.setdefault(r["kernel"], {"launches": 0, "ms": 0.0, "bytes": 0})
            d["launches"] += 1
            d["ms"] += r["ms"]
            d["bytes"] += r["bytes"]
            step_ms[r["step"]] = step_ms.get(r["step"], 0.0) + r["ms"]
        # Each kernel that streams the whole data set once per launch (block
        # sort, pairwise and four-way merges, exchange) against the HBM peak;
        # the dominant one (most time) is the line's roofline.  A sort made
        # only of short launches has none.
        full_bytes = 2 * n * (kin.element_size() + 4)
        kernel_roofs = {}
        for k in per_kernel:
            sel = [r for r in recs if r["kernel"] == k and r["bytes"] >= full_bytes]
            if not sel:
                continue
            avg_ms = sum(r["ms"] for r in sel) / len(sel)
            per_launch = sum(r["bytes"] for r in sel) / len(sel)
            achieved = per_launch / (avg_ms * 1e-3) / 1e9
            kernel_roofs[k] = {"achieved": achieved, "frac": achieved / peak, "avg_launch_ms": avg_ms,
                               "bytes_per_launch": per_launch, "launches_counted": len(sel),
                               "ms_total": sum(r["ms"] for r in sel)}
        if kernel_roofs:
            top = max(kernel_roofs, key=lambda k: kernel_roofs[k]["ms_total"])
            kr = kernel_roofs[top]
            traffic = profiled_traffic(top, args.workload, n)
            roof = {"bound": "hbm", "kernel": top, "achieved": kr["achieved"], "peak": peak, "unit": "GB/s",
                    "frac": kr["frac"], "traffic": traffic, "bytes_per_launch": kr["bytes_per_launch"],
                    "avg_launch_ms": kr["avg_launch_ms"], "launches_counted": kr["launches_counted"],
                    "peak_source": peak_src,
                    # a pass that fits in L2 (129 MB) never waits on HBM: such a sort is bound by its
                    # kernels' latency chains, and the HBM fraction only says how far from HBM it is
                    "l2_resident": full_bytes < L2_BYTES,
                    "note": "achieved = algorithmic bytes (read + write of every key and payload) per "
                            "full-size launch / mean CUDA-event duration, events around every launch on the "
                            "sort's stream in a second pass of the timed steps"}
        for k in per_kernel:
            per_kernel[k]["share"] = per_kernel[k]["ms"] / sum(v["ms"] for v in per_kernel.values())
    bytes_per_pass = 2 * n * (kin.element_size() + 4)
    e2e_frac = stats["passes"] * bytes_per_pass / (ms_step * 1e-3) / 1e9 / peak

    # End to end through the public API with host buffers (pinned), copies included.
    e2e = None
    if not args.no_e2e:
        hk = torch.from_numpy(keys_np.view(np.int64 if dtype == "u64" else np.int32)).pin_memory()
        hv = torch.from_numpy(vals_np.view(np.int32)).pin_memory()
        ko = torch.empty_like(hk).pin_memory()              # the caller's output buffers, allocated once
        vo = torch.empty_like(hv).pin_memory()
        for _ in range(1):
            pgs.sort(hk, hv, P, out=(ko, vo), **opts)
        torch.cuda.synchronize(dev)
        k_e2e = max(1, min(args.steps, 5))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            pgs.sort(hk, hv, P, out=(ko, vo), **opts)
        torch.cuda.synchronize(dev)
        dt = max_over_ranks((time.perf_counter() - t0) / k_e2e, dev, world)
        # Steady state: two calls in flight, each on its own stream with its own
        # workspace and output buffers, so one call's copy to the device overlaps
        # the previous call's merge and copy back (the copy engines of the two
        # directions run at once).  Every step still moves its own input in and
        # its own result out inside the timed region.
        hws = pgs.pgs_host_workspace_bytes(n, P, pgs.make_config(**opts))
        lanes = []
        for _ in range(2):
            lanes.append((torch.cuda.Stream(dev), torch.empty(hws, dtype=torch.uint8, device=dev),
                          torch.empty_like(hk).pin_memory(), torch.empty_like(hv).pin_memory()))
        cfgs = [pgs.make_config(workspace=ln[1], **opts) for ln in lanes]

        def call(k):
            s_, _, ko_, vo_ = lanes[k % 2]
            pgs.pgs_sort_host(hk, hv, ko_, vo_, P, cfgs[k % 2], stream=s_)
        for k in range(2):
            call(k)
        torch.cuda.synchronize(dev)
        k_pipe = max(2, min(args.steps, 10))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(k_pipe):
            call(k)
        torch.cuda.synchronize(dev)
        dt_pipe = max_over_ranks((time.perf_counter() - t0) / k_pipe, dev, world)
        same = all(torch.equal(ln[2], ko) and torch.equal(ln[3], vo) for ln in lanes)
        del lanes, cfgs
        nbytes = n * (kin.element_size() + 4)
        e2e = {"value": whole_job_rate(n, world, dt_pipe), "unit": "Gkeys/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": dt_pipe * 1e3, "in_flight": 2,
               "outputs_equal_single_call": same,
               "single_call": {"value": whole_job_rate(n, world, dt), "ms": dt * 1e3},
               "api": "pgs_sort_host (C ABI, host buffers): pinned host keys/payloads in and out, "
                      "host-to-device copies in run groups overlapped with step 1, device-to-host copies "
                      "in bucket groups overlapped with step 6, all inside the call; two calls in flight "
                      "on two streams with their own workspaces and output buffers"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_block(args, n, P)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": config_block(args, dtype, n, P, stats),
            "roofline": roof,
            "hbm_frac_end_to_end": e2e_frac,
            "max_over_mean_bucket": stats["max_bucket"] / (n / stats["P"]),
            "splitters": {"mode": args.splitters, "fallback": stats["fallback"],
                          "learned_max_over_mean": stats["learned_over_mean"] if args.splitters == "learned" else None},
            "gpu_launches": stats["launches"] * args.steps,
            "launches_per_step": stats["launches"],
            "clocks": clocks.summary(),
            "e2e": e2e,
            "launch": "pgs_sort_copy calls; from the second identical call the library replays the launch "
                      "sequence it captured into a CUDA graph (pgs_graph_cache AUTO)",
            "direct_launches": direct,
            "graph_replay": graph,
            "library_comparator": comparator,
            "instrumented_ms_per_step": ms_instr,
            "cpu_baseline": cpu,
            "per_kernel": per_kernel,
            "kernel_rooflines": kernel_roofs if timer else None,
            "per_step_ms": {str(k): v / args.steps for k, v in sorted(step_ms.items())},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
