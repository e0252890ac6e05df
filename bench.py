"""Benchmark: uint32 keys sorted per second at n = 2^28 on GB300.

One step = one full bitonic sort (every launch of the plan) of one array of
uniform random uint32 keys already resident in HBM.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched by torch.distributed.run): every rank sorts its own array
(replicas, weak scaling; the sort has no cross-GPU exchange step).

--impl reference times the CPU oracle (the paper's network, plain C, one
core) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "uint32 Gkeys/s at n=2^28 (% HBM roofline); batched vs per-array speedup; p99"
UNIT = "Gkeys/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-log2", type=int, default=28, help="keys per array = 2^n_log2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e / per-kernel legs")
    ap.add_argument("--no-segmented", action="store_true", help="skip the batched segmented leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop leg")
    ap.add_argument("--serving-requests", type=int, default=20000)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner choices file: installed without measuring when it holds this size "
                         "(so a profiled run repeats a timed run's configuration), else written")
    ap.add_argument("--no-pairs", action="store_true", help="skip the key/value leg")
    ap.add_argument("--no-key-types", action="store_true", help="skip the int32/float32/64-bit key leg")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the paper's three GPU variants (Basic / Semi / Optimized) over its sizes")
    return ap.parse_args()


KERNEL_SOURCES = ("engine.cuh", "tile_pass.cuh", "tile_u32.cu", "desc.h", "patterns.h", "plan.cpp")


def kernel_source_hash():
    """Hash of the sources that define the tile-pass kernel and its plans."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1506_01446_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(n):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, scaled to n keys -- or None if the kernel changed since."""
    p = os.path.join(ROOT, "profiles", "traffic_global_pass.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d["bytes_per_launch"] * n / d["n"]


def segmented_leg(bt, torch, steps, tune_cache=None):
    """65,536 uint32 arrays (lengths log-uniform in [1, 8192]) sorted by one
    batched segmented call vs one bitonic_sort_u32 call per array.  With a
    tune_cache path the packed-tile launch is autotuned for the batch first."""
    keys_np, offs_np = workloads.segmented_u32(65536, seed=workloads.SEEDS["segmented"])
    tuned = None
    if tune_cache:
        from paper_1506_01446_gb300 import autotune
        tuned = autotune.tune_segmented(keys_np, offs_np, reps=3, cache_path=tune_cache)
        tuned = {k: v for k, v in tuned.items() if k != "tried"}
    src = torch.from_numpy(keys_np.view(np.int32)).cuda()
    buf = src.clone()
    offs = torch.from_numpy(offs_np).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        buf.copy_(src)
        bt.sort_segmented_(buf, offs)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        buf.copy_(src)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bt.sort_segmented_(buf, offs)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    batched_ms = statistics.median(times)
    # per-array form: one plain launch sequence per array, same stream
    lib = bt.load()
    saved = bt.get_options()
    bt.set_options(use_graph=0)
    base = buf.data_ptr()
    lens = np.diff(offs_np).tolist()
    ptrs = (base + 4 * offs_np[:-1].astype(np.int64)).tolist()
    sh = stream.cuda_stream
    f = lib.bitonic_sort_u32
    # every size class once outside any capture (plans, device state)
    for n_ in sorted(set(lens)):
        i_ = lens.index(n_)
        f(ptrs[i_], n_, 1, sh)
    buf.copy_(src)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for p, n_ in zip(ptrs, lens):
        f(p, n_, 1, sh)
    b.record(stream)
    torch.cuda.synchronize()
    host_loop_ms = a.elapsed_time(b)
    # the same 65,536 calls captured into one CUDA graph (the library enqueues
    # straight into the caller's capture), replayed: the device-side cost of
    # the per-array form without the host's per-call dispatch
    cap = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=cap, capture_error_mode="thread_local"):
        hc = cap.cuda_stream
        for p, n_ in zip(ptrs, lens):
            f(p, n_, 1, hc)
    graph_times = []
    for r in range(3):
        buf.copy_(src)
        torch.cuda.synchronize()
        # replay() launches the graph on the current stream: time it there
        rs = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(rs)
        g.replay()
        b.record(rs)
        torch.cuda.synchronize()
        graph_times.append(a.elapsed_time(b))
    per_array_ms = statistics.median(graph_times)
    bt.set_options(**saved)
    out = buf.cpu().numpy().view(np.uint32)
    ok = all(np.all(np.diff(out[offs_np[i]:offs_np[i + 1]].astype(np.int64)) >= 0) for i in range(0, 65536, 97))
    del g
    nkeys = int(offs_np[-1] - offs_np[0])
    return {"arrays": 65536, "keys": nkeys, "batched_ms": batched_ms, "batched_gkeys_s": nkeys / batched_ms / 1e6,
            "per_array_ms": per_array_ms, "speedup": per_array_ms / batched_ms,
            "per_array_host_loop_ms": host_loop_ms, "speedup_vs_host_loop": host_loop_ms / batched_ms,
            "sampled_sorted": bool(ok), "tuned": tuned,
            "note": "per-array form = 65,536 bitonic_sort_u32 calls on one stream, captured into one CUDA graph "
                    "and replayed (median of 3); per_array_host_loop_ms = the same calls issued from a Python "
                    "loop with plain launches"}


def long_segments_leg(bt, torch, steps):
    """A batch of segments longer than one tile (64 of 2^15 keys, 16 of 2^17,
    4 of 2^20: 8.4M keys), which run their own multi-pass plans in one
    persistent launch: keys only, and as pairs (values = index)."""
    lens = np.array([1 << 15] * 64 + [1 << 17] * 16 + [1 << 20] * 4, dtype=np.int64)
    offs_np = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=offs_np[1:])
    keys_np = workloads.uniform_u32(int(offs_np[-1]), seed=workloads.SEEDS["segmented"] + 1)
    src = torch.from_numpy(keys_np.view(np.int32)).cuda()
    buf = src.clone()
    vals = torch.arange(src.numel(), dtype=torch.int32, device="cuda")
    vbuf = vals.clone()
    offs = torch.from_numpy(offs_np.astype(np.int32)).cuda()
    out = {"segments": int(lens.size), "keys": int(offs_np[-1]),
           "lengths": "64 x 2^15, 16 x 2^17, 4 x 2^20"}
    for name, pairs in (("keys", False), ("pairs", True)):
        def run():
            if pairs:
                bt.sort_segmented_pairs_(buf, vbuf, offs)
            else:
                bt.sort_segmented_(buf, offs)
        times = []
        for i in range(steps + 2):
            buf.copy_(src)
            vbuf.copy_(vals)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run()
            b.record()
            torch.cuda.synchronize()
            if i >= 2:
                times.append(a.elapsed_time(b))
        ms = statistics.median(times)
        got = buf.cpu().numpy().view(np.uint32)
        ok = all(np.array_equal(got[offs_np[i]:offs_np[i + 1]], np.sort(keys_np[offs_np[i]:offs_np[i + 1]]))
                 for i in (0, 63, 64, 79, 80, 83))
        out[name] = {"ms": ms, "gkeys_s": int(offs_np[-1]) / ms / 1e6, "sampled_sorted": bool(ok)}
    return out


def pairs_leg(bt, torch, steps):
    """2^26 key/value pairs, keys uniform over [0, 2^20) (many ties), values =
    original index, ascending, ties by index."""
    n = 1 << 26
    k_np, v_np = workloads.pair_keys_u32(n, seed=workloads.SEEDS["pairs_n26"])
    ks, vs = torch.from_numpy(k_np.view(np.int32)).cuda(), torch.from_numpy(v_np.view(np.int32)).cuda()
    kb, vb = ks.clone(), vs.clone()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        kb.copy_(ks)
        vb.copy_(vs)
        bt.sort_pairs_(kb, vb)
    times = []
    for _ in range(steps):
        kb.copy_(ks)
        vb.copy_(vs)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bt.sort_pairs_(kb, vb)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = statistics.median(times)
    out_k = kb[:: 1 << 10].cpu().numpy().view(np.uint32)
    info = bt.plan_info(n, pairs=True)
    return {"n": n, "ms": ms, "gpairs_s": n / ms / 1e6, "plan": info, "sampled_sorted": bool(np.all(out_k[1:] >= out_k[:-1]))}


def distributions_leg(bt, torch, steps):
    """The network's compare-exchanges do not depend on the data (Section
    3.2), so a sort's time should not either: 2^24 uint32 keys of each of
    the five input distributions, ascending, median of `steps` sorts each
    (inputs restored by a device copy before each sort)."""
    n = 1 << 24
    stream = torch.cuda.current_stream()
    out = {}
    for dist in workloads.DISTRIBUTIONS:
        src = torch.from_numpy(workloads.keys_u32(dist, n, seed=workloads.SEEDS["n24"]).view(np.int32)).cuda()
        buf = src.clone()
        for _ in range(3):
            buf.copy_(src)
            bt.sort_(buf)
        times = []
        for _ in range(steps):
            buf.copy_(src)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bt.sort_(buf)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        out[dist] = statistics.median(times)
    return {"n": n, "ms": out, "max_over_min": max(out.values()) / min(out.values())}


def key_types_leg(bt, torch, steps, peak_gbs):
    """Keys-only sorts of the other key types, 512 MiB each (inputs larger
    than L2): 2^27 int32 / float32 keys, 2^26 uint64 / int64 / float64 keys,
    uniform random bit patterns without NaNs or -0 (so numpy can check the
    sampled output), ascending."""
    out = {}
    stream = torch.cuda.current_stream()
    for kind in workloads.TYPED_KEY_KINDS:
        wide = kind in ("uint64", "int64", "float64")
        n = 1 << (26 if wide else 27)
        keys = workloads.typed_keys(kind, n, seed=workloads.SEEDS["key_types"], specials=False)
        tdt = getattr(torch, {"uint64": "int64"}.get(kind, kind))
        src = torch.from_numpy(keys.view(np.int64 if wide else np.int32)).view(tdt).cuda()
        buf = src.clone()
        for _ in range(2):
            buf.copy_(src)
            bt.sort_typed_(buf, key_type=kind)
        times = []
        for _ in range(steps):
            buf.copy_(src)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bt.sort_typed_(buf, key_type=kind)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        ms = statistics.median(times)
        sample = buf[:: 1 << 10].cpu().view(torch.int64 if wide else torch.int32).numpy().view(keys.dtype)
        info = bt.plan_info(n, pairs=wide)
        design_ms = info["hbm_passes"] * 2 * keys.dtype.itemsize * n / (peak_gbs * 1e6)
        out[kind] = {"n": n, "ms": ms, "gkeys_s": n / ms / 1e6, "hbm_passes": info["hbm_passes"],
                     "design_roofline_frac": design_ms / ms,
                     "sampled_sorted": bool(np.all(sample[1:] >= sample[:-1]))}
        del src, buf
    return out


def ablation_leg(bt, torch):
    """Section 5, Table 1 in shape: the Basic (one kernel per step, Section 3.3),
    Semi (shared memory, Section 4.1) and Optimized (registers too, Section 4.2)
    variants over the paper's sizes 2^17..2^28."""
    saved = bt.get_options()
    rows = []
    for k in range(17, 29):
        n = 1 << k
        src = torch.from_numpy(workloads.uniform_u32(n, seed=k).view(np.int32)).cuda()
        buf = src.clone()
        row = {"n_log2": k}
        for name, var in (("basic", 1), ("semi", 2), ("optimized", 0)):
            bt.set_options(variant=var)
            buf.copy_(src)
            bt.sort_(buf)
            ts = []
            for _ in range(3):
                buf.copy_(src)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                bt.sort_(buf)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            row[name + "_ms"] = min(ts)
        rows.append(row)
    bt.set_options(**saved)
    return rows


def serving_leg(bt, requests):
    """Two offered loads, each a Poisson stream of `requests` requests, 30%
    with values, 16 GiB device budget, continuous batching:
      stated:  2,000 req/s, sizes log-uniform in [2^10, 2^22] keys (the
               workload the latency target is quoted at);
      batched_20k / batched_50k / batched_200k: 20,000, 50,000 and 200,000
               req/s, sizes log-uniform in [2^10, 2^14] keys, where requests
               overlap and the loop packs those that wait into one launch.
    The loop is the library's (bitonic_serve_run); batched_50k_python_loop
    repeats the 50,000 req/s point with the same loop written in Python."""
    from paper_1506_01446_gb300.serving import SortServer
    pool = workloads.uniform_u32(1 << 26, seed=7)
    pool_v = np.arange(1 << 26, dtype=np.uint32)
    srv = SortServer(pool, pool_v, budget_bytes=16 << 30, streams=4)
    out = {}
    for name, rate, hi_log2, engine in (("stated", 2000.0, 22, "native"), ("batched_20k", 20000.0, 14, "native"),
                                        ("batched_50k", 50000.0, 14, "native"),
                                        ("batched_200k", 200000.0, 14, "native"),
                                        ("batched_50k_python_loop", 50000.0, 14, "python")):
        arr, sizes, hv = workloads.serving_requests(requests, seed=workloads.SEEDS["serving"], rate=rate,
                                                    hi_log2=hi_log2)
        srv.warmup(int(sizes.max()))                     # workspaces and plans before the clock starts
        warm = min(200, requests)
        srv.run(arr[:warm], sizes[:warm], hv[:warm], engine=engine)
        stats = srv.run(arr, sizes, hv, engine=engine)
        stats["rate_req_s"] = rate
        stats["sizes"] = f"log-uniform [2^10, 2^{hi_log2}] keys, 30% with values"
        out[name] = stats
    # the stated point's numbers stay at the top level
    return {**out["stated"], "points": out}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def reduce_max(x: float, world: int) -> float:
    """Maximum of x over all ranks (the slowest rank sets the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int) -> int:
    """Each rank sorts its own array (replicas, no exchange between ranks)."""
    return workloads.SEEDS["n28_uniform"] + rank


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """The CPU oracle (Section 3.1 network, plain C, one core) on a bounded
    sample of the workload: each step sorts 2^20 uniform keys."""
    if rank != 0:
        return
    import oracle

    n_sample = 1 << 20
    keys = workloads.uniform_u32(n_sample, seed=workloads.SEEDS["n28_uniform"])
    for _ in range(args.warmup):
        oracle.bitonic_sort(keys)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.bitonic_sort(keys)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_sample * args.steps / total / 1e9
    sample = f"{args.steps} x 2^20 uniform uint32 keys (bounded sample of the 2^{args.n_log2} workload)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (splitmix64 uniform uint32)",
        # the arm's workload; each step times a bounded sample of it (cpu_baseline.sample)
        "config": {"workload": f"single uint32 array, n=2^{args.n_log2}, uniform random, ascending",
                   "n": 1 << args.n_log2, "parallelism": "replicas x1", "sample_keys_per_step": n_sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def _timed(fn, keys, budget_s, max_reps=8):
    """Runs fn(keys) until about budget_s seconds are spent; returns (out, seconds per call, calls)."""
    reps, total, out = 0, 0.0, None
    while (total < budget_s and reps < max_reps) or reps == 0:
        t0 = time.perf_counter()
        out = fn(keys)
        total += time.perf_counter() - t0
        reps += 1
    return out, total / reps, reps


def cpu_baseline(gpu_gkeys_s=None):
    """CPU sorts on the machine's host cores, each on a bounded sample of the
    workload (uniform uint32 keys from the same generator), every output
    checked against another CPU sort of the same input:
      oracle_network_1core  the oracle's Section 3.1 network, plain C (the
                            analogue of Table 1's CPU BitonicSort column);
      quicksort_1core       the oracle's median-of-three Hoare quicksort (the
                            CPU QuickSort column behind Section 5's speedups);
      std_sort_1core        std::sort;
      std_sort_all_cores    one std::sort per core, then parallel merges.
    The line's value is the oracle network's rate."""
    import oracle

    nproc = os.cpu_count() or 1
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = nproc
    full = workloads.uniform_u32(1 << 28, seed=workloads.SEEDS["n28_uniform"])
    legs = {}
    # oracle network on 2^22 keys (~10 s); quicksort of the same keys must agree
    s22 = full[: 1 << 22].copy()
    net, sec, reps = _timed(oracle.bitonic_sort, s22, 10.0)
    net = net[0]
    legs["oracle_network_1core"] = {"gkeys_s": s22.size / sec / 1e9, "n": s22.size, "calls": reps, "cores": 1}
    q22 = oracle.quicksort(s22)
    agree = bool(np.array_equal(net, q22))
    # quicksort and std::sort on 2^25 keys, one core each; they must agree
    s25 = full[: 1 << 25].copy()
    q25, sec, reps = _timed(oracle.quicksort, s25, 4.0, 3)
    legs["quicksort_1core"] = {"gkeys_s": s25.size / sec / 1e9, "n": s25.size, "calls": reps, "cores": 1}
    st25, sec, reps = _timed(oracle.std_sort, s25, 4.0, 3)
    legs["std_sort_1core"] = {"gkeys_s": s25.size / sec / 1e9, "n": s25.size, "calls": reps, "cores": 1}
    agree &= bool(np.array_equal(q25, st25))
    # every core on the full 2^28 array; its 2^25 prefix sort must agree too
    p28, sec, reps = _timed(lambda a: oracle.parallel_sort(a, usable), full, 3.0, 3)
    legs["std_sort_all_cores"] = {"gkeys_s": full.size / sec / 1e9, "n": full.size, "calls": reps, "cores": usable}
    agree &= bool(np.array_equal(oracle.parallel_sort(s25, usable), q25))
    agree &= bool(np.all(p28[1:] >= p28[:-1])) and int(p28.astype(np.uint64).sum()) == int(full.astype(np.uint64).sum())
    out = {"value": legs["oracle_network_1core"]["gkeys_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{legs['oracle_network_1core']['calls']} x 2^22 uniform uint32 keys, Section 3.1 network in "
                     "plain C; the other legs: quicksort and std::sort on 2^25 keys (one core), std::sort per "
                     "core plus parallel merges on the full 2^28",
           "cpu_model": cpu_model(), "nproc": nproc, "usable_cores": usable, "legs": legs,
           "outputs_agree": agree}
    if gpu_gkeys_s:
        out["gpu_vs_quicksort_1core"] = gpu_gkeys_s / legs["quicksort_1core"]["gkeys_s"]
        out["gpu_vs_std_sort_all_cores"] = gpu_gkeys_s / legs["std_sort_all_cores"]["gkeys_s"]
        out["paper_gpu_vs_quicksort"] = ("about 20x, up to 30x (Kepler K10 against one Xeon E5-2620 core, "
                                         "Section 5 / Table 1; context only)")
    return out


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    import torch.distributed as dist

    import paper_1506_01446_gb300 as bt

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = 1 << args.n_log2
    hbm_gbs, peak_src = load_peaks()
    keys_np = workloads.uniform_u32(n, seed=replica_seed(rank))
    tuned = None
    import tempfile
    seg_cache = os.path.join(tempfile.gettempdir(), f"bitonic_tune_seg_{rank}.json")
    if not args.no_tune:
        from paper_1506_01446_gb300 import autotune
        cache = args.tune_cache or os.path.join(tempfile.gettempdir(), f"bitonic_tune_{rank}.json")
        choices = autotune.load(cache) if args.tune_cache else None
        if choices is None or str(args.n_log2) not in choices.get("uint32", {}):
            choices = autotune.tune(classes=(args.n_log2,), pair_classes=(), reps=3, cache_path=cache)
        tuned = {k: v for k, v in choices["uint32"].get(str(args.n_log2), {}).items() if k != "tried"}
    pristine = torch.from_numpy(keys_np.view(np.int32)).cuda()
    buf = pristine.clone()
    stream = torch.cuda.current_stream()
    info = bt.plan_info(n)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also builds and caches the CUDA graph)
    for _ in range(args.warmup):
        buf.copy_(pristine)
        bt.sort_(buf)
    barrier()
    check = buf[:: max(1, n // 4096)].cpu().numpy().view(np.uint32)
    assert np.all(check[1:] >= check[:-1]), "output not sorted"

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        for i in range(args.steps):
            buf.copy_(pristine)  # restore the unsorted input (not timed)
            starts[i].record(stream)
            bt.sort_(buf)
            ends[i].record(stream)
        barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = reduce_max(sum(step_ms), world)
    ms_per_step = total_ms / args.steps
    value = n * world * args.steps / (total_ms / 1e3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (splitmix64 uniform uint32, input restored before every step, untimed)",
        "config": {"workload": f"single uint32 array, n=2^{args.n_log2}, uniform random, ascending",
                   "n": n, "l2": (f"inputs larger than L2 ({4 * n / 2**20:.0f} MiB per array)" if 4 * n > 129 << 20
                                  else "input restored by a copy before each step"),
                   "parallelism": f"replicas x{world}",
                   "plan": info, "tuned": tuned},
        "gpu_launches": bt.graph_kernels(n) * args.steps,
        "clocks": clk.summary(),
    }

    design_bytes = info["hbm_passes"] * 2 * 4 * n
    line["design_roofline"] = {
        "hbm_passes": info["hbm_passes"], "design_bytes": design_bytes,
        "roofline_ms": design_bytes / (hbm_gbs * 1e9) * 1e3,
        "frac": (design_bytes / (hbm_gbs * 1e9) * 1e3) / ms_per_step,
        "lower_bound_ms_8n": 8 * n / (hbm_gbs * 1e9) * 1e3,
        "peak_gbs": hbm_gbs, "peak_source": peak_src,
    }

    if not args.no_extras and rank == 0:
        # per-kernel times over K instrumented steps (plain launches, events
        # between launches) for the roofline of the dominant kernel
        L = info["launches"]
        per_kind = {}
        per_launch = [[] for _ in range(L)]
        for i in range(args.steps):
            buf.copy_(pristine)
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(L + 1)]
            kinds = bt.sort_profiled_(buf, evs)
            torch.cuda.synchronize()
            for j in range(L):
                t = evs[j].elapsed_time(evs[j + 1])
                per_kind.setdefault(kinds[j], []).append(t)
                per_launch[j].append(t)
        tot = {k: sum(v) for k, v in per_kind.items()}
        dom = max(tot, key=tot.get)
        # the same launches grouped by their register rounds (steps per round;
        # rounds are joined by shared-memory transposes), each group's mean
        # time against the HBM time of one read and write of every key
        shapes = bt.round_shapes(bt.debug_plan(n, 4))
        by_shape = {}
        for j in range(L):
            by_shape.setdefault((kinds[j], shapes[j]), []).extend(per_launch[j])
        hbm_ms = 2 * 4 * n / (hbm_gbs * 1e9) * 1e3
        line_shapes = []
        for (kd, shp), ts in sorted(by_shape.items(), key=lambda kv: -sum(kv[1])):
            mean = statistics.mean(ts)
            line_shapes.append({"kernel": bt.KIND_NAMES[kd], "steps_per_round": list(shp),
                                "launches": len(ts) // args.steps, "mean_ms": round(mean, 4),
                                "hbm_time_frac": round(hbm_ms / mean, 3)})
        avg_ms = statistics.mean(per_kind[dom])
        algo_bytes = 2 * 4 * n  # each launch reads and writes every key once
        achieved = algo_bytes / (avg_ms / 1e3) / 1e9
        traffic = measured_traffic(n)
        line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                            "frac": achieved / hbm_gbs, "traffic": traffic,
                            "kernel": bt.KIND_NAMES[dom], "launches_per_step": len(per_kind[dom]) // args.steps,
                            "avg_launch_ms": avg_ms, "peak_source": peak_src,
                            "share": {bt.KIND_NAMES[k]: v / sum(tot.values()) for k, v in tot.items()},
                            "by_round_shape": line_shapes,
                            "launch_timing": "CUDA events between the launches of the plan run as one sequence on "
                                             "the launching stream (the timed graph runs the leading launches as "
                                             "two concurrent tile ranges, the same kernels over the same tiles)"}

        # end to end through the C ABI on host buffers: one batched call
        # (bitonic_sort_u32_host_batch) sorts the K steps' arrays; every step
        # uploads its 1 GiB input from page-locked memory and reads its 1 GiB
        # result back.  The library overlaps step j+1's upload and step j-1's
        # download with step j's passes (two device buffers, one sort at a
        # time); inside a step the upload overlaps the tile sort and the
        # download the last pass.
        host_in = torch.from_numpy(keys_np.view(np.int32)).pin_memory()
        host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
        # the host link alone, just before: one 1 GiB copy each way from and to
        # page-locked memory (best of 3), so that a slow e2e step can be told
        # apart from a slow link
        def measure_link():
            link = {"h2d_gbs": 0.0, "d2h_gbs": 0.0}
            for _ in range(3):
                for name, dst, src_ in (("h2d_gbs", buf, host_in), ("d2h_gbs", host_out[0], buf)):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    dst.copy_(src_, non_blocking=True)
                    b.record(stream)
                    torch.cuda.synchronize()
                    link[name] = max(link[name], 4 * n / (a.elapsed_time(b) / 1e3) / 1e9)
            return link

        link = measure_link()
        # warm-up: buffers, streams, plan, and the graphs of the arrays between
        # the first and the last (one per device buffer)
        bt.sort_host_batch([host_in] * 4, [host_out[i % 2] for i in range(4)])
        torch.cuda.synchronize()
        # five timed batch calls, the median reported: the host link of a
        # shared machine occasionally slows for a while on its own (the link
        # is measured again after the calls)
        runs = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.sort_host_batch([host_in] * args.steps, [host_out[i % 2] for i in range(args.steps)])
            e1.record(stream)
            torch.cuda.synchronize()
            runs.append(e0.elapsed_time(e1) / args.steps)
        e2e_ms = statistics.median(runs)
        # one array alone: upload, sort and download with no neighbour to overlap
        la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        la.record(stream)
        bt.sort_host(host_in, host_out[0])
        lb.record(stream)
        torch.cuda.synchronize()
        line["e2e"] = {"value": n / (e2e_ms / 1e3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": 4 * n,
                       "d2h_bytes_per_step": 4 * n, "ms_per_step": e2e_ms,
                       "runs_ms_per_step": runs, "timing": "median of 5 batch calls of K steps",
                       "api": "bitonic_sort_u32_host_batch (one call for the K steps)",
                       "single_call_ms": la.elapsed_time(lb), "single_call_api": "bitonic_sort_u32_host",
                       "link_gbs": link,
                       "link_floor_ms": 4 * n / (link["h2d_gbs"] * 1e9) * 1e3 + 4 * n / (link["d2h_gbs"] * 1e9) * 1e3}
        out = host_out[0].numpy().view(np.uint32)
        assert np.all(out[1:] >= out[:-1])
        # the link again after the calls (overwrites host_out[0], checked above)
        line["e2e"]["link_gbs_after"] = measure_link()
    if not args.no_pairs and rank == 0:
        line["pairs"] = pairs_leg(bt, torch, max(3, args.steps))
    if not args.no_key_types and rank == 0:
        line["key_types"] = key_types_leg(bt, torch, max(3, args.steps), hbm_gbs)
        line["data_oblivious"] = distributions_leg(bt, torch, max(5, args.steps))
    if not args.no_ablation and rank == 0:
        line["ablation"] = ablation_leg(bt, torch)
    if not args.no_segmented and rank == 0:
        line["segmented"] = segmented_leg(bt, torch, max(3, args.steps), None if args.no_tune else seg_cache)
        line["segmented"]["long_segments"] = long_segments_leg(bt, torch, max(3, args.steps))
    if not args.no_serving and rank == 0:
        line["serving"] = serving_leg(bt, args.serving_requests)
    if not args.no_cpu_baseline and rank == 0:
        line["cpu_baseline"] = cpu_baseline(value)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
