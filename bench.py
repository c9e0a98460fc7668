"""Benchmark of the MPHF query path (one JSON line on rank 0).

Workload: n = 1e9 distinct u64 keys (seeded), Default parameters (gamma_3,
lambda 3.5, alpha 0.99, CacheLineEF), structure built on the GPU by the
library; one step = one query of all n keys in a seeded random order
(8 GB of keys in, 4 GB of u32 out, inputs far larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n N] [--impl reference]

--impl reference times the CPU oracle (one-by-one queries on the host
cores) on a bounded sample of the same workload.  Under torchrun every rank
holds a full replica and queries its own n keys (weak scaling, no
collective on the data path).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPHF ns/key & queries/s at n=1e9 u64; % of random-gather roofline; p99 lat"
UNIT = "queries/s"
QUERY_KERNEL_SOURCES = ["paper_2502_15539_gb300/csrc/mphf_window.cu", "paper_2502_15539_gb300/csrc/mphf_query.cu",
                        "paper_2502_15539_gb300/csrc/mphf_internal.cuh", "include/mphf_device.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "query_u64_windowed_n1e9.md")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=float, default=1e9)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=1 << 31,
                    help="keys of the oracle baseline leg (2^31: about 13 s on 16 host cores)")
    ap.add_argument("--ref-sample", type=int, default=1 << 26,
                    help="keys per step of the reference arm (the oracle), so that K + W steps take seconds")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-strings", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the PHF / Fast / Compact leg")
    ap.add_argument("--no-wide", action="store_true", help="skip the leg past 2^32 keys")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused-lookup leg")
    ap.add_argument("--wide-n", type=float, default=4.5e9, help="keys of the leg past 2^32 keys")
    ap.add_argument("--strings-n", type=float, default=3e8)
    ap.add_argument("--serve-requests", type=int, default=800)
    ap.add_argument("--batch-mphfs", type=int, default=256)
    ap.add_argument("--batch-config", default="",
                    help="keys_per_thread,threads,blocks_per_sm: fixed batch launch shape instead of autotuning")
    ap.add_argument("--l2-fetch-granularity", type=int, default=128,
                    help="L2 fetch granularity (bytes) set once for the whole run through "
                         "mphf_set_l2_fetch_granularity; 128 speeds up the random pilot gathers")
    ap.add_argument("--no-c1", action="store_true", help="skip the n = 1e6 leg")
    ap.add_argument("--c1-n", type=float, default=1e6)
    ap.add_argument("--structure", default="",
                    help="serialized structure file: loaded if it exists (no build in this process), else "
                         "built and written there (keeps profiled processes free of the builder)")
    ap.add_argument("--query-keys", type=int, default=0,
                    help="query a seeded sample of this many member keys per step instead of all n "
                         "(small profiling case against the full-size structure)")
    return ap.parse_args(argv)


def parse_defaults() -> dict:
    return vars(parse([]))


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in QUERY_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks() -> tuple[float, str]:
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(structure_n: int, keys_per_launch: int, l2_fetch_granularity: int = 128):
    """DRAM bytes of one query step from the committed ncu summary (the sum
    over the windowed passes of one chunk, per key, times the keys of the
    step), if it was taken on the current kernel sources, on a structure of
    the same n and at the same L2 fetch granularity; else None.  DRAM bytes
    per key depend on the structure (its pilot array against L2) and on the
    chunk size, not on how many chunks one step queries."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    sha = re.search(r"kernel_source_sha:\s*(\w+)", text)
    bpk = re.search(r"dram_bytes_per_key:\s*([0-9.]+)", text)
    gran = re.search(r"l2_fetch_granularity:\s*(\d+)", text)
    rec_n = re.search(r"structure_n:\s*(\d+)", text)
    if not sha or not bpk or not gran or not rec_n or sha.group(1) != kernel_source_sha():
        return None
    if int(gran.group(1)) != l2_fetch_granularity or int(rec_n.group(1)) != structure_n:
        return None
    return float(bpk.group(1)) * keys_per_launch


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self) -> dict:
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        busy = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)]
        return {"sm_mhz": statistics.median(busy or sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def aggregate_ranks(local_ms: float, keys_per_rank: int, steps: int, ws: int, device) -> tuple[float, float]:
    """Whole-job throughput over replicas: every rank's keys over the slowest
    rank's time (max over ranks of the timed region)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total = float(t.item())
    return total, ws * keys_per_rank * steps / (total / 1e3)


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2502_15539_gb300 import build_ext
    from paper_2502_15539_gb300 import native as N
    from paper_2502_15539_gb300 import workloads as W

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or not os.path.exists(N.LIB_PATH):
        build_ext.build()
    if ws > 1:
        dist.barrier()
    N.load()
    # One context-wide setting for every leg of the run (query, probe, builds).
    N.mphf_set_l2_fetch_granularity(args.l2_fetch_granularity)
    n = int(args.n)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    built_here = not (args.structure and os.path.exists(args.structure))
    # A loaded structure with a sampled query needs no full key set on the device.
    keys = W.u64_keys(n, seed=0, device=dev) if built_here or not 0 < args.query_keys < n else None
    if not built_here:
        with open(args.structure, "rb") as f:
            m = N.mphf_deserialize(f.read())
    else:
        m = N.mphf_build(keys)
        if args.structure:
            with open(args.structure, "wb") as f:
                f.write(N.mphf_serialize(m))
    info = N.mphf_info(m)
    if info["n"] != n:
        raise SystemExit(f"{args.structure} holds n={info['n']}, not {n}")
    if 0 < args.query_keys < n:
        mq = args.query_keys
        del keys
        torch.cuda.empty_cache()
        q = W.u64_keys_at(W.uniform_index(mq, n, seed=1 + rank, device=dev), seed=0)
    else:
        mq = n
        perm = W.permutation(n, seed=1 + rank, device=dev)
        q = keys[perm]
        del perm, keys
    torch.cuda.empty_cache()
    out = torch.empty(mq, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    # Fraction of keys whose slot is >= n (they read one CacheLineEF line).
    N.mphf_query_u64_phf(m, q, out)
    remapped = int(((out.to(torch.int64) & 0xFFFFFFFF) >= n).sum().item())

    def time_steps(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        barrier()
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        barrier()
        return [a.elapsed_time(b) for a, b in evs]

    run_query = lambda: N.mphf_query_u64(m, q, out, stream=stream)
    for _ in range(args.warmup):
        run_query()
    launches0 = N.mphf_launch_count()
    with ClockSampler(local) as clk:
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        per_step = time_steps(run_query, args.steps)
        t1.record(stream)
        barrier()
    launches = N.mphf_launch_count() - launches0
    clocks = clk.summary()
    total_ms, value = aggregate_ranks(sum(per_step), mq, args.steps, ws, dev)
    ms_per_step = total_ms / args.steps

    # Random-gather probes (the roofline of the pilot gathers), writing to
    # their own buffer so that `out` keeps the timed query's results.
    probe_out = torch.empty(mq, dtype=torch.int32, device=dev)
    # (a) matched: the query's own pilot accesses (its bucket indexes for the
    # same key stream, gathered from the structure's own pilot array).
    bidx = N.mphf_bucket_u64(m, q)
    pilots_ptr = N.mphf_device_view(m).pilots
    run_matched = lambda: N.mphf_gather_probe_at(bidx, pilots_ptr, info["pilot_bytes"], probe_out, stream=stream)
    for _ in range(args.warmup):
        run_matched()
    matched_ms = statistics.mean(time_steps(run_matched, args.steps))
    del bidx
    torch.cuda.empty_cache()
    # The single-pass kernel on the same stream (one window): the kernel the
    # matched probe bounds; the windowed path replaces its random DRAM reads.
    run_single = lambda: N.mphf_query_u64_windowed(m, q, probe_out, window_bytes=1 << 40, stream=stream)
    for _ in range(args.warmup):
        run_single()
    single_ms = statistics.mean(time_steps(run_single, args.steps))
    single_same = bool(torch.equal(probe_out, out))
    # (b) uniform: one byte at a uniformly random index of a table the size of the pilot array.
    table = torch.randint(0, 256, (info["pilot_bytes"],), dtype=torch.uint8, device=dev)
    run_probe = lambda: N.mphf_gather_probe(q, table, probe_out, stream=stream)
    for _ in range(args.warmup):
        run_probe()
    probe_ms = statistics.mean(time_steps(run_probe, args.steps))
    del table, probe_out

    # Roofline of the query step (HBM bound): algorithmic bytes per key =
    # 8 (key) + 4 (result) + 32 (the pilot's DRAM sector) + 64 per remapped key.
    # The library's automatic window count: ceil(pilot bytes / 100 MB), at
    # least 2, above 72 MiB of pilots and up to 6 windows, for >= 2^24 keys.
    pb = info["pilot_bytes"]
    W_passes = max(2, -(-pb // 100_000_000)) if pb > (72 << 20) and mq >= (1 << 24) else 1
    W_passes = W_passes if W_passes <= 6 else 1
    query_path = ("mphf_query_u64, windowed: window_first_kernel, "
                  f"{W_passes - 2} x window_mid_kernel, window_last_kernel per chunk of up to 2^28 keys"
                  if W_passes >= 2 else "mphf_query_u64, single pass: query_u64_kernel")
    peak, peak_kind = measured_peaks()
    alg_bytes = mq * (8 + 4 + 32) + remapped * 64
    kernel_ms = statistics.mean(per_step)
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    traffic = recorded_traffic(n, mq, args.l2_fetch_granularity)

    # End to end through the C ABI with pinned host buffers.
    e2e = None
    if not args.no_e2e:
        qh = torch.empty(mq, dtype=torch.int64, pin_memory=True)
        qh.copy_(q)
        oh = torch.empty(mq, dtype=torch.int32, pin_memory=True)
        for _ in range(max(1, args.warmup)):
            N.mphf_query_u64_host(m, qh, oh)
        barrier()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            N.mphf_query_u64_host(m, qh, oh)
        barrier()
        e2e_s = time.perf_counter() - w0
        tt = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e = {"value": ws * mq * args.steps / float(tt.item()), "unit": UNIT,
               "h2d_bytes_per_step": 8 * mq, "d2h_bytes_per_step": 4 * mq,
               "ms_per_step": 1e3 * float(tt.item()) / args.steps}
        del qh, oh

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(m, q, out, args.cpu_sample)
    variants = None if args.no_variants else run_variants(args, m, q, out, stream, time_steps)
    fused = None if args.no_fused else run_fused(args, m, q, out, stream, time_steps, remapped)
    del q, out, m
    torch.cuda.empty_cache()
    c1 = None if args.no_c1 else run_c1(args, dev, stream, rank == 0 and ws == 1 and not args.no_cpu_baseline)
    torch.cuda.empty_cache()
    wide = None if args.no_wide else run_wide(args, dev, stream)
    torch.cuda.empty_cache()
    batched = None if args.no_batched else run_batched(args, dev, stream)
    torch.cuda.empty_cache()
    torch.cuda.empty_cache()
    strings = None if args.no_strings else run_strings(args, dev, stream)
    torch.cuda.empty_cache()
    serving = None if args.no_serving else run_serving(args, dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": (f"plain at scale: n={n} distinct u64 keys, query all n in a seeded random order"
                                    if mq == n else f"profiling case: n={n} structure, {mq} sampled member keys"),
                       "n": n, "params": "Default (gamma_3, lambda 3.5, alpha 0.99, CacheLineEF)",
                       "P": info["P"], "S": info["S"], "B": info["B"], "bits_per_key": info["bits_per_key"],
                       "l2": (f"inputs larger than L2 ({8 * mq / 1e9:.3g} GB keys + {4 * mq / 1e9:.3g} GB out per "
                              f"step, {info['pilot_bytes'] / 1e6:.0f} MB pilots); no flush"),
                       "parallelism": f"replicas x{ws}", "l2_fetch_granularity": args.l2_fetch_granularity},
            "ns_per_key": 1e9 / (value / ws),
            "query_keys_per_step": mq,
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "alg_bytes_per_key": alg_bytes / mq,
                         "kernel": query_path,
                         "basis": "the whole query step (every pass) per 1e9 keys, as the step is timed"},
            "gather_roofline": {
                "frac": matched_ms / kernel_ms, "probe_ms": matched_ms, "query_ms": kernel_ms,
                "probe": "mphf_gather_probe_at: the query's own pilot gathers (its bucket indexes for the same "
                         "key stream, precomputed by mphf_bucket_u64, 8 B in) from the structure's pilot array, "
                         "u32 out",
                "probe_gathers_per_s": mq / (matched_ms / 1e3),
                "query_pilot_gathers_per_s": mq / (kernel_ms / 1e3),
                "single_pass": {"query_ms": single_ms, "queries_per_s": mq / (single_ms / 1e3),
                                "frac": matched_ms / single_ms, "outputs_identical": single_same,
                                "kernel": "query_u64_kernel (mphf_query_u64_windowed with one window)"},
                "note": "frac > 1: the windowed query reads each pilot from an L2-resident window, so it is not "
                        "bound by the random DRAM gathers the probe makes; the probe bounds the single pass",
                "uniform": {"probe_ms": probe_ms, "frac": probe_ms / kernel_ms,
                            "probe": "mphf_gather_probe: same key stream, 1 byte at a uniformly random index "
                                     f"of a {info['pilot_bytes']}-byte table per key (no skew)"},
                "key_stream_gbs": 8 * mq / (kernel_ms / 1e3) / 1e9,
                "result_stream_gbs": 4 * mq / (kernel_ms / 1e3) / 1e9},
            "remapped_fraction": remapped / mq,
            "build": {"ms": info["build_ms"], "ns_per_key": 1e6 * info["build_ms"] / n,
                      "evictions": info["evictions"], "hash_sort_ms": info["build_hash_sort_ms"],
                      "search_ms": info["build_search_ms"], "remap_ms": info["build_remap_ms"]},
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "structure": "built in this process" if built_here else f"loaded from {args.structure}",
            "c1": c1,
            "variants": variants,
            "fused": fused,
            "wide": wide,
            "batched": batched,
            "strings": strings,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_c1(args, dev, stream, with_oracle: bool):
    """The plain configuration: n = 1e6 distinct u64 keys (seed 0), Default
    parameters, GPU-built structure; all n keys queried once in a seeded
    random order (seed 1).  The query kernel alone, 20 launches, best and
    median, each timed with CUDA events and no host submission gap, both with
    L2 flushed before every launch (a 256 MB write) and back to back (inputs
    and structure L2-warm);
    host to host through mphf_query_u64_host with page-locked buffers; and
    two L2-regime gather probes over the same key stream as denominators:
    uniform over a table the size of the pilot array, and the query's own
    pilot gathers.  The oracle evaluates the same serialized structure on all
    n keys and the GPU's values must equal it."""
    import numpy as np
    import torch
    from paper_2502_15539_gb300 import native as N
    from paper_2502_15539_gb300 import workloads as W

    n = int(args.c1_n)
    keys = W.u64_keys(n, seed=0, device=dev)
    m = N.mphf_build(keys)
    info = N.mphf_info(m)
    q = keys[W.permutation(n, seed=1, device=dev)].contiguous()
    out = torch.empty(n, dtype=torch.int32, device=dev)
    probe_out = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    reps = 20

    def launches(fn, cold: bool) -> list[float]:
        """Per-launch device times of `reps` launches.  The GPU first runs a
        bounded sleep kernel (torch.cuda._sleep, about 4 ms) while the host
        enqueues every launch, so the launches run back to back and no
        interval includes host submission time."""
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda._sleep(8_000_000)
        for a, b in evs:
            if cold:
                flush.fill_(1)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    def summary(ts: list[float]) -> dict:
        return {"best_ms": min(ts), "median_ms": statistics.median(ts),
                "queries_per_s_best": n / (min(ts) / 1e3), "queries_per_s_median": n / (statistics.median(ts) / 1e3)}

    with torch.cuda.stream(stream):
        run_q = lambda: N.mphf_query_u64(m, q, out, stream=stream)
        cold, warm = summary(launches(run_q, True)), summary(launches(run_q, False))
        table = torch.randint(0, 256, (info["pilot_bytes"],), dtype=torch.uint8, device=dev)
        uni = summary(launches(lambda: N.mphf_gather_probe(q, table, probe_out, stream=stream), False))
        bidx = N.mphf_bucket_u64(m, q)
        ptr = N.mphf_device_view(m).pilots
        matched = summary(launches(lambda: N.mphf_gather_probe_at(bidx, ptr, info["pilot_bytes"], probe_out,
                                                                  stream=stream), False))
    torch.cuda.synchronize()
    qh = q.cpu().pin_memory()
    oh = torch.empty(n, dtype=torch.int32, pin_memory=True)
    for _ in range(3):
        N.mphf_query_u64_host(m, qh, oh)
    hts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        N.mphf_query_u64_host(m, qh, oh)
        hts.append(1e3 * (time.perf_counter() - t0))
    got = out.cpu().numpy().view(np.uint32)
    res = {"workload": f"plain: n={n} distinct u64 keys (seed 0), Default params, GPU-built structure "
                       f"(P={info['P']}, S={info['S']}, {info['pilot_bytes']} pilot bytes); all n keys once in a "
                       "seeded random order",
           "kernel_cold_l2": cold, "kernel_warm_l2": warm,
           "host_to_host": {"best_ms": min(hts), "median_ms": statistics.median(hts),
                            "queries_per_s_best": n / (min(hts) / 1e3), "h2d_bytes": 8 * n, "d2h_bytes": 4 * n,
                            "call": "mphf_query_u64_host, page-locked buffers, wall clock"},
           "gather_roofline": {
               "matched": dict(matched, frac=matched["median_ms"] / warm["median_ms"],
                               probe="the query's own pilot gathers (mphf_gather_probe_at)"),
               "uniform": dict(uni, frac=uni["median_ms"] / warm["median_ms"],
                               probe=f"uniform random byte of a {info['pilot_bytes']}-byte (L2-resident) table"),
               "basis": "median of the warm launches"},
           "host_outputs_equal_device": bool(np.array_equal(oh.numpy().view(np.uint32), got))}
    if with_oracle:
        from oracle import oracle as O
        ref = O.OracleMPHF.deserialize(N.mphf_serialize(m))
        want = ref.query_u64(W.as_uint64_numpy(q), threads=os.cpu_count() or 1)
        res["parity_checked_keys"] = n
        res["parity_ok"] = bool(np.array_equal(got, want))
    del flush, table, bidx, q, out, probe_out, keys, m
    return res


def run_fused(args, m, q, idx, stream, time_steps, remapped):
    """The device API inside an application kernel: out[i] = table[h(q[i])] for
    a seeded u32 table of n entries, fused into one kernel (mphf_lookup_u64)
    against the same result in two passes (mphf_query_u64 into an index
    array, then torch.index_select), on the main leg's query stream."""
    import torch
    from paper_2502_15539_gb300 import native as N

    n = N.mphf_info(m)["n"]
    mq = q.numel()
    if n > 2**31:
        return None   # the two-pass baseline indexes with int32 values
    gen = torch.Generator(device=q.device)
    gen.manual_seed(5)
    table = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device=q.device, generator=gen)
    fused_out = torch.empty(mq, dtype=torch.int32, device=q.device)
    two_out = torch.empty_like(fused_out)
    run_one = lambda: N.mphf_lookup_u64(m, q, table, fused_out, stream=stream)

    def run_two():
        N.mphf_query_u64(m, q, idx, stream=stream)
        torch.index_select(table, 0, idx, out=two_out)

    for _ in range(args.warmup):
        run_one()
        run_two()
    one_ms = statistics.mean(time_steps(run_one, args.steps))
    two_ms = statistics.mean(time_steps(run_two, args.steps))
    same = bool(torch.equal(fused_out, two_out))
    # The table reads alone: one byte of each result's 4-byte table entry, in
    # the query's order (idx holds the results of the last two-pass run), with
    # the same 8 B in and 4 B out per key and none of the query's work.
    tidx = idx.to(torch.int64) * 4
    probe_out = torch.empty(mq, dtype=torch.int32, device=q.device)
    run_tp = lambda: N.mphf_gather_probe_at(tidx, table.data_ptr(), 4 * n, probe_out, stream=stream)
    for _ in range(args.warmup):
        run_tp()
    table_probe_ms = statistics.mean(time_steps(run_tp, args.steps))
    del tidx, probe_out
    # 8 (key) + 4 (result) + 32 (pilot sector) + 32 (table sector) + 64 per remapped key.
    alg = mq * (8 + 4 + 32 + 32) + remapped * 64
    del table, fused_out, two_out
    peak, peak_kind = measured_peaks()
    achieved = alg / (one_ms / 1e3) / 1e9
    return {"workload": f"out[i] = table[h(q[i])]: {n}-entry u32 table, the main query stream ({mq} keys)",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "alg_bytes_per_key": alg / mq},
            "fused_ms": one_ms, "fused_queries_per_s": mq / (one_ms / 1e3),
            "two_pass_ms": two_ms, "speedup": two_ms / one_ms, "outputs_identical": same,
            "gather_roofline": {"probe_ms": table_probe_ms, "frac": table_probe_ms / one_ms,
                                "probe": "mphf_gather_probe_at: the lookup's table reads alone (each result's "
                                         "table entry, in query order, 8 B in, 4 B out per key)",
                                "rest_ms": one_ms - table_probe_ms},
            "fused_alg_bytes_per_key": alg / mq, "fused_achieved_gbs": alg / (one_ms / 1e3) / 1e9,
            "two_pass": "mphf_query_u64 into an int32 index array, then torch.index_select"}


def run_variants(args, m, q, out, stream, time_steps):
    """The other parameter sets of Table remap on the same keys and query
    stream: the PHF query of the Default structure (slots, no remap), Fast
    (gamma_1, lambda 3.0, plain remap array) and Compact (lambda 4.0), each
    built on the GPU and timed like the main leg."""
    from paper_2502_15539_gb300 import native as N

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        return statistics.mean(time_steps(fn, args.steps))

    mq = q.numel()
    peak, peak_kind = measured_peaks()

    def roofline(alg_per_key, ms_):
        achieved = alg_per_key * mq / (ms_ / 1e3) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind, "alg_bytes_per_key": alg_per_key}

    ms = timed(lambda: N.mphf_query_u64_phf(m, q, out, stream=stream))
    # PHF: 8 (key) + 4 (slot) + 32 (pilot sector), no remap read.
    res = {"default_phf": {"query_ms": ms, "queries_per_s": mq / (ms / 1e3), "roofline": roofline(44.0, ms)}}
    for name, prm in (("fast", {"lam": 3.0, "gamma": 1, "remap": 1}), ("compact", {"lam": 4.0})):
        mv = N.mphf_build(q, N.mphf_default_params(**prm))
        info = N.mphf_info(mv)
        ms = timed(lambda: N.mphf_query_u64(mv, q, out, stream=stream))
        # 8 + 4 + 32 per key, plus one remap sector (32 B Vec entry or 64 B CacheLineEF line) for the
        # remapped fraction (P S - n) / (P S) of the keys.
        frac_remap = (info["P"] * info["S"] - info["n"]) / (info["P"] * info["S"])
        alg = 44.0 + frac_remap * (32.0 if info["remap"] == 1 else 64.0)
        res[name] = {"params": prm, "query_ms": ms, "queries_per_s": mq / (ms / 1e3),
                     "bits_per_key": info["bits_per_key"], "build_ms": info["build_ms"], "roofline": roofline(alg, ms)}
        del mv
    return res


def run_wide(args, dev, stream):
    """Past 2^32 keys: wide_n distinct u64 keys, built on the GPU in shards of
    whole parts, queried in key order with 64-bit results.  The results are
    checked to be a bijection onto [0, n) on the device."""
    import torch
    from paper_2502_15539_gb300 import native as N
    from paper_2502_15539_gb300 import workloads as W

    n = int(args.wide_n)
    chunk = 1 << 28
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    for s0 in range(0, n, chunk):
        keys[s0:s0 + chunk] = W.u64_keys(min(chunk, n - s0), seed=3, device=dev, start=s0)
    m = N.mphf_build(keys)
    info = N.mphf_info(m)
    out = torch.empty(n, dtype=torch.int64, device=dev)
    N.mphf_query_u64_wide(m, keys, out, stream=stream)   # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 3))
    a.record(stream)
    for _ in range(steps):
        N.mphf_query_u64_wide(m, keys, out, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    # Matched probe: the query's own pilot reads (the bucket index of every
    # key of the same stream, gathered from the structure's pilot array),
    # without the hashing, slot and remap arithmetic; 8 B in and 4 B out per
    # key against the query's 8 B in and 8 B out.
    bidx = N.mphf_bucket_u64(m, keys)
    del keys
    probe_out = torch.empty(n, dtype=torch.int32, device=dev)
    pilots_ptr = N.mphf_device_view(m).pilots
    run_p = lambda: N.mphf_gather_probe_at(bidx, pilots_ptr, info["pilot_bytes"], probe_out, stream=stream)
    run_p()   # warm-up
    a.record(stream)
    for _ in range(steps):
        run_p()
    b.record(stream)
    torch.cuda.synchronize()
    probe_ms = a.elapsed_time(b) / steps
    del bidx, probe_out
    bijective = False
    if int(out.min().item()) >= 0 and int(out.max().item()) < n:   # in range: the fill stays in bounds
        seen = torch.zeros(n, dtype=torch.uint8, device=dev)
        seen.index_fill_(0, out, 1)
        bijective = int(seen.sum(dtype=torch.int64).item()) == n
        del seen
    del out, m
    # 8 (key) + 8 (value) + 32 (pilot sector) + a 64-byte CacheLineEF line for the remapped keys.
    peak, peak_kind = measured_peaks()
    alg = 48.0 + 64.0 * (info["P"] * info["S"] - n) / (info["P"] * info["S"])
    achieved = alg * n / (ms / 1e3) / 1e9
    return {"workload": f"{n} distinct u64 keys (> 2^32), query all in key order, 64-bit results",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "alg_bytes_per_key": alg},
            "P": info["P"], "S": info["S"], "bits_per_key": info["bits_per_key"],
            "build_ms": info["build_ms"], "build_ns_per_key": 1e6 * info["build_ms"] / n,
            "query_ms": ms, "queries_per_s": n / (ms / 1e3), "output_bijective": bijective,
            "gather_roofline": {"probe_ms": probe_ms, "frac": probe_ms / ms,
                                "probe": "mphf_gather_probe_at: the query's own pilot reads (mphf_bucket_u64 "
                                         "of the same key stream) from the structure's pilot array"}}


def run_batched(args, dev, stream):
    """Many structures in one persistent launch: 256 structures with n
    log-uniform in [1e3, 1e7] (seed 2), one request each of log-uniform size
    in [1, 1e6] (seed 3), 90% member and 10% non-member keys.  Timed: one
    graph-replayed persistent launch per step (autotuned shape) against one
    plain mphf_query_u64 launch per request."""
    import torch
    from paper_2502_15539_gb300 import native as N
    from paper_2502_15539_gb300 import workloads as W

    k = args.batch_mphfs
    ns = W.log_uniform_int(k, 1e3, 1e7, seed=2).tolist()
    qs = W.log_uniform_int(k, 1, 1e6, seed=3).tolist()
    # The structures are built concurrently: 64 host threads, one stream each
    # (a build synchronizes only its own stream).
    from concurrent.futures import ThreadPoolExecutor
    keys_all = [W.u64_keys(n, seed=1000 + i, device=dev) for i, n in enumerate(ns)]
    torch.cuda.synchronize()

    def build(i):
        return N.mphf_build(keys_all[i], stream=torch.cuda.Stream(device=dev))

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=64) as pool:
        structs = list(pool.map(build, range(k)))
    build_wall_ms = 1e3 * (time.perf_counter() - t0)
    build_ms = sum(N.mphf_info(m)["build_ms"] for m in structs)
    items = []
    for i, (m, n, qn) in enumerate(zip(structs, ns, qs)):
        nm = qn // 10
        q = torch.cat([keys_all[i][W.uniform_index(qn - nm, n, seed=2000 + i, device=dev)],
                       W.nonmember_u64_keys(nm, n, seed=1000 + i, device=dev)])
        items.append((m, q, torch.empty(qn, dtype=torch.int32, device=dev)))
    del keys_all
    torch.cuda.empty_cache()
    total = sum(qs)
    arr, keep = N.make_requests(items)
    b = N.Batch(k)
    if args.batch_config:
        kpt, thr, bps = (int(x) for x in args.batch_config.split(","))
        b.set_config(kpt, thr, bps, use_graph=True)
        tuned = b.config()
    else:
        tuned = b.autotune(arr, k, os.path.join(tempfile.gettempdir(), "mphf_batch_tune.jsonl"), stream=stream)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        reps = max(args.steps, 20)   # one batch is ~0.15 ms: average over enough of them
        a.record(stream)
        for _ in range(reps):
            fn()
        z.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(z) / reps

    batch_ms = timed(lambda: b.run(arr, k, stream=stream))
    plain_ms = timed(lambda: [N.mphf_query_u64(m, q, o, stream=stream) for m, q, o in items])
    # The batched outputs equal the per-request outputs (both parity-tested).
    b.run(arr, k, stream=stream)
    torch.cuda.synchronize()
    got = [o.clone() for _, _, o in items]
    for m, q, o in items:
        N.mphf_query_u64(m, q, o, stream=stream)
    torch.cuda.synchronize()
    same = all(torch.equal(g, o) for g, (_, _, o) in zip(got, items))
    # L2-regime gather roofline: the batch's whole key stream, one byte per key
    # at a uniformly random index of a table as large as all pilot arrays
    # together (the structures' pilots are L2-resident at this size).
    pilot_total = sum(N.mphf_info(m)["pilot_bytes"] for m in structs)
    allq = torch.cat([q for _, q, _ in items])
    pout = torch.empty(allq.numel(), dtype=torch.int32, device=dev)
    table = torch.randint(0, 256, (pilot_total,), dtype=torch.uint8, device=dev)
    probe_ms = timed(lambda: N.mphf_gather_probe(allq, table, pout, stream=stream))
    del allq, pout, table
    return {"workload": f"{k} structures, n log-uniform [1e3, 1e7] (sum {sum(ns)}), requests log-uniform "
                        f"[1, 1e6] (sum {total}), 90% members",
            "queries_per_s": total / (batch_ms / 1e3), "ms_per_batch": batch_ms,
            "gather_roofline": {"probe_ms": probe_ms, "frac": probe_ms / batch_ms,
                                "probe": f"the batch's {total} keys, 1 byte each at a uniformly random index of "
                                         f"a {pilot_total}-byte table (all pilot arrays together; L2 regime)"},
            "per_request_launches": {"queries_per_s": total / (plain_ms / 1e3), "ms_per_batch": plain_ms},
            "speedup": plain_ms / batch_ms, "autotuned": tuned, "outputs_identical": same,
            "build_ms_total": build_ms, "build_wall_ms": build_wall_ms,
            "build": "64 host threads, one stream each; build_ms_total sums the per-structure device times"}


def run_strings(args, dev, stream):
    """String keys: n = 3e8 random printable ASCII strings of length uniform in
    [16, 64], packed with u64 offsets; GPU build, then query passes over all n
    strings re-packed in a seeded random order."""
    import torch
    from paper_2502_15539_gb300 import native as N
    from paper_2502_15539_gb300 import workloads as W

    n = int(args.strings_n)
    data, off = W.strings(torch.arange(n, device=dev), seed=0)
    total_bytes = int(off[-1].item())
    m = N.mphf_build(data, offsets=off)
    info = N.mphf_info(m)
    del data, off
    torch.cuda.empty_cache()
    qd, qo = W.strings(W.permutation(n, seed=1, device=dev), seed=0)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        N.mphf_query_bytes(m, qd, qo, out, stream=stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    z = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        N.mphf_query_bytes(m, qd, qo, out, stream=stream)
    z.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(z) / args.steps
    # bijection of the full pass (a property that holds at any size)
    vals = out.to(torch.int64) & 0xFFFFFFFF
    bijective = False
    if int(vals.max().item()) < n:   # in range, so the fill below stays inside `seen`
        seen = torch.zeros(n, dtype=torch.int32, device=dev)
        seen.index_fill_(0, vals, 1)
        bijective = bool(seen.sum().item() == n)
        del seen
    del qd, qo, out, vals
    peak, peak_kind = measured_peaks()
    # Algorithmic bytes: the string, its u64 offset, the u32 result and one
    # 32-byte pilot sector per string.
    alg = total_bytes + n * (8 + 4 + 32)
    achieved = alg / (ms / 1e3) / 1e9
    return {"workload": f"{n} strings, length U[16,64] (mean {total_bytes / n:.1f} B), printable ASCII, "
                        "packed + u64 offsets; query order a seeded permutation, re-packed",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "alg_bytes_per_key": alg / n, "kernel": "query_bytes_kernel"},
            "build_ms": info["build_ms"], "build_ns_per_key": 1e6 * info["build_ms"] / n,
            "bits_per_key": info["bits_per_key"], "P": info["P"], "S": info["S"],
            "query_ms": ms, "queries_per_s": n / (ms / 1e3), "ns_per_key": 1e6 * ms / n,
            "key_bytes_per_s": (total_bytes + 8 * n) / (ms / 1e3), "output_bijective": bijective}


def run_serving(args, dev):
    """Serving: 16 resident structures (8 u64 with n log-uniform in [1e6, 5e8],
    8 string with n log-uniform in [1e6, 1e8], lengths 16..64), requests of
    log-uniform size in [1, 1e6] (90% members) on a uniformly chosen structure,
    HBM budget 60% of the structures' bytes (admission queues).  Capacity is
    measured with all requests arriving at once; then Poisson arrivals at 10%,
    50% and 90% of it give p50 / p99 latency (arrival to completion)."""
    import numpy as np
    import torch
    from paper_2502_15539_gb300 import native as N
    from paper_2502_15539_gb300 import workloads as W

    n_u64 = W.log_uniform_int(8, 1e6, 5e8, seed=4).tolist()
    n_str = W.log_uniform_int(8, 1e6, 1e8, seed=5).tolist()
    blobs, kinds, sizes = [], [], []
    for i, n in enumerate(n_u64):
        keys = W.u64_keys(n, seed=3000 + i, device=dev)
        m = N.mphf_build(keys)
        del keys
        blobs.append(N.mphf_serialize(m))
        info = N.mphf_info(m)
        sizes.append(info["pilot_bytes"] + info["remap_bytes"])
        kinds.append(("u64", n, 3000 + i))
        del m
        torch.cuda.empty_cache()
    for i, n in enumerate(n_str):
        data, off = W.strings(torch.arange(n, device=dev), seed=4000 + i)
        m = N.mphf_build(data, offsets=off)
        del data, off
        blobs.append(N.mphf_serialize(m))
        info = N.mphf_info(m)
        sizes.append(info["pilot_bytes"] + info["remap_bytes"])
        kinds.append(("bytes", n, 4000 + i))
        del m
        torch.cuda.empty_cache()
    def serve(budget):
        srv = N.Server(hbm_budget_bytes=budget, slots=4, max_batch_requests=1024, max_batch_keys=1 << 24)
        sids = [srv.add(b) for b in blobs]
        return srv, sids

    budget = int(0.6 * sum(sizes))
    srv, sids = serve(budget)

    R = args.serve_requests
    counts = W.log_uniform_int(R, 1, 1e6, seed=6).tolist()
    which = W.uniform_index(R, 16, seed=7).tolist()
    reqs, keep = [], []
    for r, (cnt, k) in enumerate(zip(counts, which)):
        kind, n, seed = kinds[k]
        nm = cnt // 10
        if kind == "u64":
            q = torch.cat([W.u64_keys_at(W.uniform_index(cnt - nm, n, 9000 + r, device=dev), seed=seed),
                           W.nonmember_u64_keys(nm, n, seed, device=dev)])
            out = torch.empty(cnt, dtype=torch.int32, device=dev)
            reqs.append(N.Server.request(sids[k], q, out))
            keep.append((q, out))
        else:
            ids = torch.cat([W.uniform_index(cnt - nm, n, 9000 + r, device=dev),
                             n + W.uniform_index(nm, n, 9500 + r, device=dev)])
            d, o = W.strings(ids, seed=seed)
            out = torch.empty(cnt, dtype=torch.int32, device=dev)
            reqs.append(N.Server.request(sids[k], d, out, o))
            keep.append((d, o, out))
    torch.cuda.synchronize()
    total_keys = sum(counts)

    def sweep(srv, seed):
        # Warm-up, then capacity: everything arrives at t = 0; then Poisson loads.
        srv.replay(reqs, [0.0] * R)
        srv.drain()
        srv.stats(reset=True)
        srv.replay(reqs, [0.0] * R)
        srv.drain()
        burst = srv.stats(reset=True)
        cap = burst["queries_per_s"]
        levels = {}
        rng = np.random.default_rng(seed)
        for load in (0.1, 0.5, 0.9):
            rate_req = load * cap / (total_keys / R)          # requests per second
            arrivals = np.cumsum(rng.exponential(1e6 / rate_req, R))
            srv.replay(reqs, arrivals)
            srv.drain()
            st = srv.stats(reset=True)
            levels[f"{int(load * 100)}%"] = {k: st[k] for k in ("p50_us", "p99_us", "max_us", "queries_per_s",
                                                               "mean_requests_per_batch", "evictions", "admissions")}
        return {"capacity_queries_per_s": cap, "burst_p50_us": burst["p50_us"], "burst_p99_us": burst["p99_us"],
                "poisson": levels}

    tight = sweep(srv, 8)
    srv.close()
    srv, sids_all = serve(2 * sum(sizes))
    # same requests, structure ids are assigned in the same order
    roomy = sweep(srv, 9)
    srv.close()
    return {"workload": f"16 structures (8 u64, n {min(n_u64)}..{max(n_u64)}; 8 string, n {min(n_str)}..{max(n_str)}, "
                        f"len 16..64), {R} requests of log-uniform size [1, 1e6] (sum {total_keys}), 4 slots",
            "budget_60pct": dict(tight, hbm_budget_bytes=budget, structure_bytes=sum(sizes)),
            "all_resident": roomy}


def cpu_baseline(m, q, out, sample: int):
    """The oracle, as it stands, on the host cores: one-by-one queries of a
    prefix of the same query stream against the same (serialized) structure.
    Its values are compared with the timed GPU query's output, key by key."""
    import numpy as np
    from oracle import oracle as O
    from paper_2502_15539_gb300 import native as N
    from paper_2502_15539_gb300 import workloads as W

    ref = O.OracleMPHF.deserialize(N.mphf_serialize(m))
    cnt = min(sample, q.numel())
    keys = W.as_uint64_numpy(q[:cnt])
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    want = ref.query_u64(keys, threads=cores)
    dt = time.perf_counter() - t0
    got = out[:cnt].cpu().numpy().view(np.uint32)
    mismatches = int(np.count_nonzero(got != want))
    del want, got
    one = min(cnt, 1 << 26)   # the one-thread loop on a shorter prefix (about 6 s)
    t0 = time.perf_counter()
    ref.query_u64(keys[:one], threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": cnt / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {cnt} keys of the query stream, same structure, {cores} threads",
            "parity_checked_keys": cnt, "parity_mismatches": mismatches, "parity_ok": mismatches == 0,
            "single_thread": {"value": one / dt1, "unit": UNIT, "ns_per_key": 1e9 * dt1 / one,
                              "sample": f"first {one} keys, 1 thread"}}


# ----------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_init()
    if rank != 0:
        return
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2502_15539_gb300 import workloads as W

    n = int(args.n)
    cores = os.cpu_count() or 1
    torch.set_num_threads(cores)
    keys = W.as_uint64_numpy(W.u64_keys(n, seed=0))
    ref = O.OracleMPHF.build_u64(keys, threads=cores)
    del keys
    sample = min(int(args.ref_sample), n)
    # A seeded sample of the query stream: keys of random indices.
    idx = W.uniform_index(sample, n, seed=1)
    qs = W.as_uint64_numpy(W.u64_keys_at(idx, seed=0))
    for _ in range(args.warmup):
        ref.query_u64(qs, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ref.query_u64(qs, threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * args.steps / total
    L = ref.layout
    clef_bytes = 64 * -(-(L.P * L.S - n) // 44)   # CacheLineEF: 44 values per 64-byte line
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"plain at scale: n={n} distinct u64 keys, oracle-built structure; each step "
                               f"queries a {sample}-key sample of member keys drawn with replacement (seed 1) "
                               "from the n keys",
                   "n": n, "params": "Default (gamma_3, lambda 3.5, alpha 0.99, CacheLineEF)",
                   "P": L.P, "S": L.S, "B": L.B, "bits_per_key": 8 * (L.P * L.B + clef_bytes) / n,
                   "l2": "host caches (the oracle runs on the host cores)",
                   "parallelism": f"oracle threads x{cores}", "l2_fetch_granularity": None},
        "ns_per_key": 1e9 / value,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} keys drawn from the n-key query stream per step, "
                                   f"oracle-built structure, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
