#!/usr/bin/env python
"""Benchmark of offloaded silicon-pixel local reconstruction on GB300.

One step = one pass of the whole reconstruction (decode, bucket, calibrate,
threshold, 8-connected clustering, charge/centroid reduction, ordered output,
labels) over one batch of the ``batched`` workload: 256 events of uneven size
(digi counts uniform in 10k-200k, ~27M digis) on the 64-module 160 x 416
geometry, seeded synthetic data.

  value        events/s, device-resident inputs (CUDA-event timed on the
               launching stream; inputs and working set exceed the 129 MB L2)
  e2e          the same through the public enqueue API with pinned host
               buffers: host-to-device copy of the inputs, the pass, and the
               results back in host memory, every step
  per_event    the plain per-event path on the ``full`` workload (one
               1856-module event of ~60k digis per launch, one stream)
  roofline     the dominant kernel's algorithmic bytes / its mean duration
  cpu_baseline the CPU oracle timed on this host's cores (reported baseline)

``--impl reference`` times the CPU oracle (the reference arm) instead.
Under torchrun each rank runs an independent replica on its own GPU (events
shard by rank, no collective on the data path); value sums over ranks.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2004_04334_gb300 import synth  # noqa: E402

METRIC = "events/s & Mdigis/s at 1 GB300 (batched vs per-event, % HBM peak); p50/p99 latency"
WORKLOAD = "batched"
# GB300 HBM3e, nominal (the roofline peak is the measured copy bandwidth; this is context)
NOMINAL_HBM_GBS = 8000.0
WORKLOAD_TEXT = {
    "batched": "uneven events, digi counts uniform in 10k-200k",
    "occupancy": "Poisson(80) clusters of 1-40 px per module, 10% 1x30 streaks, 2% hot modules at 20% occupancy",
    "full": "one full-size event (~60k digis)",
    "full_literal": "one event with 1% noise occupancy (~1.5M digis)",
    "tiny": "one 64-module event (~1.2k digis)",
    "serving": "lognormal sizes (median 80k, sigma 0.8, cap 500k)",
}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--events", type=int, default=0,
                   help="events of the workload (0: its defined count; smaller for profiler captures)")
    p.add_argument("--per-event-steps", type=int, default=200)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--device-only", action="store_true",
                   help="only the device-resident timed loop (for profiler captures)")
    p.add_argument("--serving-rates", default="1000,2000,5000,10000,20000,50000",
                   help="Poisson arrival rates (events/s) of the serving measurement")
    p.add_argument("--serving-events", type=int, default=100000,
                   help="most requests per serving rate (fewer at low rates, see --serving-seconds)")
    p.add_argument("--serving-seconds", type=float, default=8.0,
                   help="requests per rate: rate x this many seconds, at most --serving-events")
    p.add_argument("--no-extra-configs", action="store_true",
                   help="skip the per-event (cfg1, cfg2, cfg3 events one at a time) and high-occupancy lines")
    p.add_argument("--serving-only", action="store_true", help="only the serving measurement")
    p.add_argument("--e2e-depth", type=int, default=3, help="batches in flight in the end-to-end measurement")
    p.add_argument("--tuning", default="",
                   help="tile_slots,blocks_per_sm,ticket_items,warp_max[,label_store,item_threads]: use these "
                        "clustering settings instead of "
                        "autotuning (for profiler captures of one configuration)")
    p.add_argument("--serving-inflight", type=int, default=0, help="serving batches in flight (0: library default)")
    p.add_argument("--serving-max-batch", type=int, default=0, help="events per serving batch, at most (0: library "
                                                                      "default)")
    p.add_argument("--serving-profile", action="store_true",
                   help="diagnostic: stage timers on every serving batch (summed kernel time)")
    p.add_argument("--serving-staging", action="store_true",
                   help="serving inputs copied into pinned staging by hp_submit (default: submitted from pinned "
                        "buffers and copied by DMA)")
    return p.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank: int, world: int):
    """Seed of a rank's replica: the workload's own seed on one GPU, a
    distinct one per rank otherwise (replicas process different events)."""
    return None if world == 1 else synth.BASE_SEED + 3 + 1000 * rank


def max_over_ranks(t: float, world: int, device=None) -> float:
    """The slowest rank's time: a MAX all-reduce over the process group (no
    collective on one rank).  device: where the reduced tensor lives (the
    rank's GPU under NCCL, None for the CPU under gloo)."""
    if world == 1:
        return t
    import torch
    import torch.distributed as dist

    v = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def job_value(units_per_rank: int, steps: int, t: float, world: int) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank * steps / t


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(n_digis, n_events, n_modules, n_clusters, labels=True):
    """Bytes the method must move at least: inputs read once (word + module id),
    calibration read once per event, labels and cluster records written once."""
    return 6 * n_digis + 8 * n_modules * n_events + (4 * n_digis if labels else 0) + 24 * n_clusters


# Per-kernel algorithmic bytes (intermediates such as buckets are not counted).
def kernel_bytes(name, n_digis, n_events, n_modules, n_clusters):
    if name == "hist_kernel":
        return 2 * n_digis
    if name == "scatter_kernel":
        return 6 * n_digis
    if name == "cc_kernel":  # labels and calibration (its staged clusters are an intermediate)
        return 4 * n_digis + 8 * n_modules * n_events
    if name == "offsets_kernel":  # the per-event cluster offsets
        return 8 * (n_events + 1)
    if name == "copy_kernel":  # the cluster records, written once in order, and the event statuses
        return 24 * n_clusters + 4 * n_events
    if name == "hits_kernel":
        return 24 * n_clusters + 48 * n_modules + 8 * (n_events + 1)
    return 0


def _kernel_source_hash():
    """Hash of the kernels' code (comments and blank space stripped), which
    the committed ncu counters must match to be reported."""
    import re

    h = hashlib.sha256()
    for f in ("hp_kernels.cu", "hp_internal.h", "hp_hits.cu"):
        with open(os.path.join(ROOT, "paper_2004_04334_gb300", "csrc", f)) as fh:
            code = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def _traffic(kernel, n_units):
    """DRAM bytes per launch from the committed ncu summary (bytes per unit:
    per digi, or per hit for the hits kernel, scaled to n_units), if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:  # noqa: BLE001
        return None
    e = t.get(kernel)
    if not e or e.get("source_hash") != _kernel_source_hash():
        return None
    return int(e["dram_bytes_per_unit"] * n_units)


def _cpu_case(w, passes=3):
    """The library's CPU case (HP_FORCE_CPU: the same product on the host's
    cores) on the workload: events/s over `passes` whole batches, median."""
    from paper_2004_04334_gb300 import hp

    old = os.environ.get("HP_FORCE_CPU")
    os.environ["HP_FORCE_CPU"] = "1"
    try:
        ts = []
        with hp.Context(w.n_modules, w.gain, w.pedestal, want_labels=True) as ctx:
            for _ in range(passes + 1):
                t0 = time.perf_counter()
                ev = ctx.enqueue_batch(w.words, w.modules, w.offsets)
                assert ev.wait(600) == hp.HP_OK
                prov = ev.provenance()
                ev.release()
                ts.append(time.perf_counter() - t0)
    finally:
        if old is None:
            os.environ.pop("HP_FORCE_CPU", None)
        else:
            os.environ["HP_FORCE_CPU"] = old
    t = statistics.median(ts[1:])
    return {"value": w.n_events / t, "unit": "events/s", "mdigis_per_s": w.n_digis / t / 1e6,
            "host": prov["device_name"], "path": prov["path"],
            "what": f"hp_enqueue_batch on a CPU context (HP_FORCE_CPU), median of {passes} passes over the "
                    f"{w.n_events}-event workload, labels on"}


def cpu_oracle(w, events=None, threads=None):
    """Time the CPU oracle over events of w (one oracle call per event, run on
    `threads` host threads; the oracle releases the GIL)."""
    from oracle import oracle

    events = list(range(w.n_events)) if events is None else events
    threads = threads or os.cpu_count() or 1

    def one(e):
        words, mods = w.event(e)
        oracle.reconstruct_event(words, mods, w.n_modules, w.gain, w.pedestal)

    oracle.build()
    t0 = time.perf_counter()
    if threads == 1:
        for e in events:
            one(e)
    else:
        with cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(one, events))
    dt = time.perf_counter() - t0
    nd = sum(int(w.offsets[e + 1] - w.offsets[e]) for e in events)
    return len(events) / dt, nd / dt / 1e6, dt, threads


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    w = synth.workload(a.workload)
    sample = list(range(w.n_events))  # every event of the workload, each step (the same config as ours)
    for _ in range(a.warmup):
        cpu_oracle(w, sample[:16])
    vals = []
    t_all = 0.0
    for _ in range(a.steps):
        ev_s, md_s, dt, cores = cpu_oracle(w, sample)
        vals.append(ev_s)
        t_all += dt
    value = len(sample) * a.steps / t_all
    nd = sum(int(w.offsets[e + 1] - w.offsets[e]) for e in sample)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * t_all / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64",
            "data": "synthetic",
            "config": {"workload": f"{a.workload}: {WORKLOAD_TEXT.get(a.workload, '')}; {w.n_events} events, "
                                   f"{w.n_modules} modules of 160x416, {w.n_digis} digis, labels on",
                       "events_per_step": len(sample), "digis_per_step": nd, "n_modules": w.n_modules},
            "mdigis_per_s": nd * a.steps / t_all / 1e6,
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "sample": f"{len(sample)} events ({nd} digis) of the {a.workload} workload per step"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(a):
    import torch

    from paper_2004_04334_gb300 import build, hp

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    build.build()

    # each rank reconstructs its own shard of events (a replica), seeded by rank
    seed = rank_seed(rank, world)
    w = synth.workload(a.workload, n_events=a.events or None, seed=seed)
    E, N, M = w.n_events, w.n_digis, w.n_modules

    ctx = hp.Context(M, w.gain, w.pedestal, device=local, want_labels=True)
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    out = hp.DeviceOutputs(E, N, dev)
    stream = torch.cuda.Stream(dev)

    def step():
        ctx.reconstruct_device(E, N, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out,
                               stream.cuda_stream)

    # clocks sampled over the device work around the timed region (autotuning,
    # warm-up, the timed replays, the stage-timed passes and the hits chain):
    # the timed region alone is shorter than the sampling interval
    clocks = ClockSampler(local)
    clocks.start()

    # autotuner: pick the clustering kernel's settings for this launch shape (before any
    # other pass, so that every later launch, warm-up included, runs with them)
    if a.tuning:
        keys = ("tile_slots", "blocks_per_sm", "ticket_items", "warp_max", "label_store", "item_threads")
        ctx.set_tuning(E, N, dict(zip(keys, (int(x) for x in a.tuning.split(",")))))
        tuning = {"chosen": ctx.get_tuning(E, N), "candidates": "not searched (--tuning)"}
    else:
        tuned, tuned_ms, cand_ms = ctx.autotune(E, N, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(),
                                                out, reps=3)
        tuning = {"chosen": tuned, "candidates": [dict(c, ms=round(m, 4)) for c, m in
                                                  zip(ctx.tuning_candidates(), cand_ms)]}

    with torch.cuda.stream(stream):
        for _ in range(max(3, a.warmup)):
            step()
    torch.cuda.synchronize(dev)
    n_clusters = int(out.cluster_offsets[-1].item())
    assert int((out.event_status != 0).sum().item()) == 0, "device reported an error status"

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # device-resident timed region: the pass captured once in a CUDA graph, replayed per step
    graph = ctx.graph_capture(E, N, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out)
    for _ in range(3):
        graph.launch(stream.cuda_stream)
    barrier()
    launches0 = ctx.stats()["kernel_launches"]
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        graph.launch(stream.cuda_stream)
    e1.record(stream)
    barrier()
    t_dev = e0.elapsed_time(e1) / 1000.0
    gpu_launches = ctx.stats()["kernel_launches"] - launches0
    graph.destroy()
    # per-kernel durations: stage timers (CUDA events around each kernel, on the
    # launching stream) over the same number of directly launched passes
    ctx.profile_enable(a.steps)
    for _ in range(a.steps):
        step()
    barrier()
    prof = ctx.profile_read()
    ctx.profile_enable(0)
    t_dev = max_over_ranks(t_dev, world, dev)
    value = job_value(E, a.steps, t_dev, world)
    mdigis = world * N * a.steps / t_dev / 1e6

    # dominant kernel roofline
    name, (cnt, ms) = max(prof.items(), key=lambda kv: kv[1][1])
    per_launch_s = ms / max(cnt, 1) / 1000.0
    kb = kernel_bytes(name, N, E, M, n_clusters)
    peak, peak_kind = _peaks()
    achieved = kb / per_launch_s / 1e9
    path_bytes = algorithmic_bytes(N, E, M, n_clusters)
    shares = {k: round(v[1] / max(1e-12, sum(x[1] for x in prof.values())), 4) for k, v in prof.items()}

    chain = _chain(a, ctx, w, out, n_clusters, dev, stream, step, barrier, world)
    clk = clocks.stop()

    e2e = per_event = serving = occupancy = None
    if not a.device_only:
        e2e, per_event = _e2e_and_per_event(a, ctx, w, n_clusters, dev, stream, barrier, world)
    ctx.close()
    if not a.device_only and not a.no_extra_configs:
        # the batched workload's own events, one launch each: the same work as a batched step
        per_event["batched"] = _per_event(a, a.workload, dev, stream, barrier, n_events=E)
        occupancy = _device_config(a, "occupancy", dev, stream, barrier, world)
    if not a.device_only and rank == 0:
        serving = _serving_in_fresh_process(a, local)

    # the CPU case of the library (Sec. 3) and the CPU oracle last, after
    # every GPU measurement: their host threads and memory churn stay out of
    # the timed GPU and serving regions
    cpu_case = _cpu_case(w) if rank == 0 and not a.device_only else None
    cpu = None
    if rank == 0 and not a.no_cpu_baseline and not a.device_only:
        # whole passes over the workload until about 10-15 CPU-seconds of work
        # (0.75 s of wall time on all host threads), 20 passes at most
        passes, t_cpu, cores = 0, 0.0, 1
        while passes < 1 or (t_cpu < 0.75 and passes < 20):
            _, _, dt, cores = cpu_oracle(w)
            passes += 1
            t_cpu += dt
        cpu = {"value": passes * E / t_cpu, "unit": "events/s", "cores": cores, "kind": "oracle",
               "sample": f"{passes} passes over all {E} events ({N} digis a pass) of the {a.workload} workload, "
                         f"{cores} threads (one oracle call per event)",
               "mdigis_per_s": passes * N / t_cpu / 1e6, "seconds": t_cpu}
        # and on one core: the median of three passes over the first 8 events
        one = sorted((cpu_oracle(w, list(range(min(8, E))), threads=1) for _ in range(3)), key=lambda r: r[0])[1]
        cpu["single_core"] = {"value": one[0], "unit": "events/s", "mdigis_per_s": one[1],
                              "sample": f"first {min(8, E)} events, one thread, median of 3 passes"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000 * t_dev / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
            "config": {"workload": f"{a.workload}: {WORKLOAD_TEXT.get(a.workload, '')}; {E} events, {M} modules "
                                   f"of 160x416, {N} digis, labels on",
                       "events_per_step": E, "digis_per_step": N, "clusters_per_step": n_clusters,
                       "l2": "inputs (6 B/digi) and working set larger than the 129 MB L2; no flush",
                       "parallelism": f"replicas x{world}", "launch": "one CUDA graph replay per step"},
            "mdigis_per_s": mdigis,
            "path_algorithmic_GBps": path_bytes * a.steps / t_dev / 1e9,
            "roofline": {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "traffic": _traffic(name, N), "algorithmic_bytes_per_launch": kb,
                         "mean_launch_ms": per_launch_s * 1000, "kernel_shares": shares,
                         "timing": "stage timers over the same number of direct (non-graph) passes"},
            "e2e": e2e,
            "tuning": tuning,
            "chain": chain,
            "per_event": per_event,
            "batched_vs_per_event": (value / per_event["batched"]["value"])
            if per_event and "batched" in per_event else None,
            "batched_vs_per_event_note": "the batched step against the same 256 events launched one at a time "
                                         "(device-resident, one stream)",
            "occupancy": occupancy,
            "serving": serving,
            "gpu_launches": gpu_launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "cpu_case": cpu_case,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _chain(a, ctx, w, out, n_clusters, dev, stream, step, barrier, world):
    """raw -> clusters -> hits, device-resident on one stream: the chain's
    events/s and the hits kernel's own launch time (CUDA events around it)."""
    import torch

    E, M = w.n_events, w.n_modules
    origin, rot = synth.barrel_geometry(M)
    ctx.set_geometry(origin, rot, synth.PITCH_ROW, synth.PITCH_COL)
    cap = out.struct.capacity
    hxyz = [torch.empty(cap, dtype=torch.float32, device=dev) for _ in range(3)]

    def hits():
        ctx.hits_device(E, cap, out.cluster_offsets.data_ptr(), out.module.data_ptr(), out.x.data_ptr(),
                        out.y.data_ptr(), hxyz[0].data_ptr(), hxyz[1].data_ptr(), hxyz[2].data_ptr(),
                        stream.cuda_stream)

    for _ in range(max(3, a.warmup)):
        step()
        hits()
    barrier()
    marks = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for m0, m1 in marks:
        step()
        m0.record(stream)
        hits()
        m1.record(stream)
    c1.record(stream)
    barrier()
    t = c0.elapsed_time(c1) / 1000.0
    hits_s = sum(m0.elapsed_time(m1) for m0, m1 in marks) / 1000.0 / a.steps
    t = max_over_ranks(t, world, dev)
    kb = 24 * n_clusters + 48 * M + 8 * (E + 1)
    peak, peak_kind = _peaks()
    return {"value": job_value(E, a.steps, t, world), "unit": "events/s", "ms_per_step": 1000 * t / a.steps,
            "what": "hp_reconstruct_device + hp_hits_device per step on one stream",
            "hits_kernel": {"mean_launch_ms": hits_s * 1000, "hits_per_launch": n_clusters,
                            "algorithmic_bytes_per_launch": kb, "achieved": kb / hits_s / 1e9, "unit": "GB/s",
                            "peak": peak, "frac": kb / hits_s / 1e9 / peak, "peak_kind": peak_kind,
                            "traffic": _traffic("hits_kernel", n_clusters),
                            "note": "its inputs were just written by the clustering kernel and may be "
                                    "partly L2-resident"}}


def _e2e_and_per_event(a, ctx, w, n_clusters, dev, stream, barrier, world):
    import torch

    from paper_2004_04334_gb300 import hp

    E, N = w.n_events, w.n_digis
    # end to end through the public enqueue API: pinned host inputs, H2D, pass, results in host memory
    pw = torch.from_numpy(w.words.view(np.int32)).pin_memory()
    pm = torch.from_numpy(w.modules.view(np.int16)).pin_memory()
    depth = a.e2e_depth  # batches in flight: the next batch's copies overlap this one's kernels

    def run(flags):
        for _ in range(2):  # warm the pools at the timed depth (one device + pinned block per batch in flight)
            evs = [ctx.enqueue_batch(pw, pm, w.offsets, flags=flags) for _ in range(depth)]
            for ev in evs:
                ev.wait(120)
                ev.release()
        # three timed runs of K steps each (a run is tens of ms of host wall time, so
        # one scheduling hiccup moves it); the median run is reported
        runs = []
        for _ in range(3):
            barrier()
            t0 = time.perf_counter()
            inflight = []
            for _ in range(a.steps):
                inflight.append(ctx.enqueue_batch(pw, pm, w.offsets, flags=flags))
                if len(inflight) >= depth:
                    ev = inflight.pop(0)
                    ev.wait(120)
                    r = ev.fetch(copy=False)
                    nc, st = r.n_clusters, r.status
                    ev.release()
            for ev in inflight:
                ev.wait(120)
                r = ev.fetch(copy=False)
                nc, st = r.n_clusters, r.status
                ev.release()
            barrier()
            t_run = time.perf_counter() - t0
            assert st == hp.HP_OK and nc == n_clusters
            runs.append(max_over_ranks(t_run, world, dev))
        return sorted(runs)[1], runs

    # labels in the compact form (2 bytes a digi and 4 an item), then as int32 ids
    t_e2e, runs = run(hp.HP_INPUT_NOCOPY | hp.HP_LABELS_U16)
    t_i32, runs_i32 = run(hp.HP_INPUT_NOCOPY | hp.HP_WANT_LABELS)
    base_d2h = 24 * n_clusters + 8 * (E + 1) + 4 * E
    e2e = {"value": job_value(E, a.steps, t_e2e, world), "unit": "events/s", "batches_in_flight": depth,
           "labels": "compact (HP_LABELS_U16: rank in the module, item offsets)",
           "h2d_bytes_per_step": 6 * N + 8 * (E + 1),
           "d2h_bytes_per_step": 2 * N + 4 * E * w.n_modules + base_d2h,
           "mdigis_per_s": world * N * a.steps / t_e2e / 1e6,
           "runs_events_per_s": [job_value(E, a.steps, t, world) for t in runs], "reported": "median of the runs",
           "int32_labels": {"value": job_value(E, a.steps, t_i32, world), "unit": "events/s",
                            "d2h_bytes_per_step": 4 * N + base_d2h,
                            "runs_events_per_s": [job_value(E, a.steps, t, world) for t in runs_i32]}}

    per_event = {name: _per_event(a, name, dev, stream, barrier) for name in ("full", "tiny")}
    return e2e, per_event


def _per_event(a, name, dev, stream, barrier, n_events=1):
    """The plain per-event path on one workload: every event its own launch
    on one stream, device-resident (events/s), and every event through
    hp_enqueue_event one at a time (events/s and enqueue-to-completion
    p50/p99 from pinned host buffers)."""
    import torch

    from paper_2004_04334_gb300 import hp

    w = synth.workload(name, n_events=n_events if n_events > 1 else None)
    E = w.n_events
    ctx = hp.Context(w.n_modules, w.gain, w.pedestal, device=dev.index, want_labels=True)
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    sizes = (w.offsets[1:] - w.offsets[:-1]).astype(np.int64)
    per_offs = torch.from_numpy(np.stack([np.zeros(E, np.int64), sizes], 1).copy()).to(dev)
    out = hp.DeviceOutputs(1, int(sizes.max()), dev)

    def launch(e):
        o = int(w.offsets[e])
        ctx.reconstruct_device(1, int(sizes[e]), per_offs[e].data_ptr(), d_words.data_ptr() + 4 * o,
                               d_mods.data_ptr() + 2 * o, out, stream.cuda_stream)

    reps = max(1, a.per_event_steps // E)
    order = [e for _ in range(reps) for e in range(E)]
    with torch.cuda.stream(stream):
        for e in order[:max(10, E)]:
            launch(e)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for e in order:
        launch(e)
    e1.record(stream)
    barrier()
    t_dev = e0.elapsed_time(e1) / 1000.0
    pw = torch.from_numpy(w.words.view(np.int32).copy()).pin_memory().numpy().view(np.uint32)
    pm = torch.from_numpy(w.modules.view(np.int16).copy()).pin_memory().numpy().view(np.uint16)
    for e in range(min(E, 10)):  # warm the pools
        o = int(w.offsets[e])
        ev = ctx.enqueue_event(pw[o:o + int(sizes[e])], pm[o:o + int(sizes[e])])
        ev.wait(60)
        ev.release()
    lat = []
    t0 = time.perf_counter()
    for e in order:
        o = int(w.offsets[e])
        ev = ctx.enqueue_event(pw[o:o + int(sizes[e])], pm[o:o + int(sizes[e])])
        ev.wait(60)
        lat.append(ev.latency_ns / 1e6)
        ev.release()
    t_host = time.perf_counter() - t0
    ctx.close()
    nd = int(sizes.sum()) * reps
    return {"workload": f"{name}: {E} event(s) of {w.n_modules} modules, {int(sizes.mean())} digis on average",
            "events": len(order), "value": len(order) / t_dev, "unit": "events/s",
            "mdigis_per_s": nd / t_dev / 1e6, "what": "device-resident, one launch per event on one stream",
            "enqueue_one_at_a_time": {"value": len(order) / t_host, "unit": "events/s",
                                      "latency_ms_p50": float(np.percentile(lat, 50)),
                                      "latency_ms_p99": float(np.percentile(lat, 99)),
                                      "what": "hp_enqueue_event from pinned buffers, wait, release; one in flight"}}


def _device_config(a, name, dev, stream, barrier, world, n_events=0):
    """Another workload device-resident (autotuned, CUDA-graph replay), with
    its dominant kernel's roofline from the stage timers."""
    import torch

    from paper_2004_04334_gb300 import hp

    w = synth.workload(name, n_events=n_events or None)
    E, N, M = w.n_events, w.n_digis, w.n_modules
    ctx = hp.Context(M, w.gain, w.pedestal, device=dev.index, want_labels=True)
    d_words = torch.from_numpy(w.words.view(np.int32)).to(dev)
    d_mods = torch.from_numpy(w.modules.view(np.int16)).to(dev)
    d_offs = torch.from_numpy(w.offsets.view(np.int64)).to(dev)
    out = hp.DeviceOutputs(E, N, dev)
    tuned, _, _ = ctx.autotune(E, N, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out, reps=2)
    steps = max(3, a.steps // 4)
    graph = ctx.graph_capture(E, N, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out)
    for _ in range(3):
        graph.launch(stream.cuda_stream)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        graph.launch(stream.cuda_stream)
    e1.record(stream)
    barrier()
    t_dev = max_over_ranks(e0.elapsed_time(e1) / 1000.0, world, dev)
    graph.destroy()
    n_clusters = int(out.cluster_offsets[-1].item())
    assert int((out.event_status != 0).sum().item()) == 0, "device reported an error status"
    ctx.profile_enable(steps)
    for _ in range(steps):
        ctx.reconstruct_device(E, N, d_offs.data_ptr(), d_words.data_ptr(), d_mods.data_ptr(), out,
                               stream.cuda_stream)
    barrier()
    prof = ctx.profile_read()
    ctx.profile_enable(0)
    ctx.close()
    kname, (cnt, ms) = max(prof.items(), key=lambda kv: kv[1][1])
    per_launch_s = ms / max(cnt, 1) / 1000.0
    kb = kernel_bytes(kname, N, E, M, n_clusters)
    peak, peak_kind = _peaks()
    return {"workload": f"{name}: {WORKLOAD_TEXT.get(name, '')}; {E} events, {M} modules, {N} digis",
            "value": job_value(E, steps, t_dev, world), "unit": "events/s",
            "mdigis_per_s": world * N * steps / t_dev / 1e6, "ms_per_step": 1000 * t_dev / steps,
            "steps": steps, "clusters_per_step": n_clusters, "tuning": tuned,
            "path_algorithmic_GBps": algorithmic_bytes(N, E, M, n_clusters) * steps / t_dev / 1e9,
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": kb / per_launch_s / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": kb / per_launch_s / 1e9 / peak, "peak_kind": peak_kind,
                         "traffic": _traffic(kname, N), "algorithmic_bytes_per_launch": kb,
                         "mean_launch_ms": per_launch_s * 1000,
                         "kernel_shares": {k: round(v[1] / max(1e-12, sum(x[1] for x in prof.values())), 4)
                                           for k, v in prof.items()}}}


def run_serving(local, rates, n_requests, pool_events=200, submitters=4, budget=16 << 30, nocopy=False,
                profile=False, inflight=0, seconds=0.0, max_batch=0):
    """Serving workload: Poisson arrivals at each rate, event sizes lognormal
    (median 80k digis, sigma 0.8, capped at 500k), 4 native submitter threads
    with completion callbacks (hp_serve_replay), a 16 GB device budget,
    continuous batching; requests cycle over a pool of pre-generated events.
    Returns per-rate sustained events/s and p50/p99 submit-to-callback latency."""
    from paper_2004_04334_gb300 import hp

    import torch

    w = synth.workload("serving", n_events=pool_events)
    pool = [w.event(e) for e in range(w.n_events)]
    if nocopy:  # the data source's buffers: pinned, read by DMA in place
        pinned = [(torch.from_numpy(a.view(np.int32).copy()).pin_memory(),
                   torch.from_numpy(b.view(np.int16).copy()).pin_memory()) for a, b in pool]
        pool = [(a.numpy().view(np.uint32), b.numpy().view(np.uint16)) for a, b in pinned]
    out = []
    with hp.Context(w.n_modules, w.gain, w.pedestal, device=local, want_labels=True, n_streams=4) as ctx:
        tuned = pretune_batches(ctx, w, local)
        ctx.serve_start(budget_bytes=budget, want_labels=True, nocopy=nocopy, max_inflight_batches=inflight,
                        max_batch_events=max_batch)
        # warm the pools with every pool event, a few at a time and all at once
        ctx.serve_replay(pool, np.zeros(2 * len(pool)), np.arange(2 * len(pool)) % len(pool), submitters)
        n_max = n_requests
        for k, rate in enumerate(rates):
            # about `seconds` of arrivals at this rate, at most n_max requests
            n_requests = int(min(n_max, max(1000, rate * seconds))) if seconds > 0 else n_max
            gaps = synth.exponential(synth.child_seed(synth.BASE_SEED + 5, 1000 + k), n_requests, rate)
            arrival = np.cumsum(gaps) - gaps[0]
            idx = np.arange(n_requests) % len(pool)
            # steady state: a warm-up stretch at this rate first (pool bins of its batch sizes)
            nw = min(n_requests, 2000)
            ctx.serve_replay(pool, arrival[:nw], idx[:nw], submitters)
            s0 = ctx.stats()
            if profile:  # stage timers on every batch: summed kernel time (diagnostic; adds event records)
                ctx.profile_enable(1 << 20)
            lat, st, span = ctx.serve_replay(pool, arrival, idx, submitters)
            prof = ctx.profile_read() if profile else {}
            ctx.profile_enable(0)
            s1 = ctx.stats()
            nd = sum(len(pool[i][0]) for i in idx)
            nb = max(1, s1["serve_batches"] - s0["serve_batches"])
            out.append({"rate_offered": rate, "requests": n_requests,
                        "sustained_events_per_s": n_requests / span,
                        "mdigis_per_s": nd / span / 1e6,
                        "latency_ms_p50": float(np.percentile(lat, 50) * 1e3),
                        "latency_ms_p99": float(np.percentile(lat, 99) * 1e3),
                        "latency_ms_max": float(np.max(lat) * 1e3),
                        "errors": int((st != 0).sum()),
                        "mean_batch": n_requests / nb,
                        "submit_us_per_request": (s1["serve_submit_ns"] - s0["serve_submit_ns"]) / n_requests / 1e3,
                        "admitter_busy": (s1["serve_launch_ns"] - s0["serve_launch_ns"]) / 1e9 / span,
                        "completion_busy": (s1["serve_complete_ns"] - s0["serve_complete_ns"]) / 1e9 / span,
                        "kernel_busy": (sum(v[1] for v in prof.values()) / 1e3 / span) if profile else None,
                        "pool_backend_allocs": (s1["device_mallocs"] + s1["host_mallocs"]) -
                                               (s0["device_mallocs"] + s0["host_mallocs"])})
        stats = ctx.stats()
        ctx.serve_stop()
    return {"workload": f"serving: lognormal sizes (median 80k, sigma 0.8, cap 500k), pool of {pool_events} "
                        f"events, {submitters} native submitter threads, {budget >> 30} GB budget, "
                        f"inputs {'read in place from pinned buffers' if nocopy else 'copied into pinned staging'}",
            "batches": stats["serve_batches"], "requests": stats["serve_requests"], "pretuned_buckets": tuned,
            "rates": out}


def _serving_in_fresh_process(a, local):
    """The serving measurement in a process of its own, as a server runs:
    started from this script (--serving-only) on the same GPU, so that none
    of this process's earlier measurements (their contexts, pools, pinned
    buffers and caches) shares its address space.  Its JSON line is returned."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serving-only", "--serving-rates", a.serving_rates,
           "--serving-events", str(a.serving_events), "--serving-seconds", str(a.serving_seconds),
           "--serving-inflight", str(a.serving_inflight), "--serving-max-batch", str(a.serving_max_batch)]
    if a.serving_staging:
        cmd.append("--serving-staging")
    env = dict(os.environ, LOCAL_RANK=str(local))  # the same GPU, as a single process
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    p = subprocess.run(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=1800)
    if p.returncode != 0:
        raise RuntimeError("serving measurement failed: " + p.stderr[-2000:])
    line = [l for l in p.stdout.splitlines() if l.startswith("{")][-1]
    out = json.loads(line)
    out["process"] = "a fresh process of its own (bench.py --serving-only)"
    return out


def pretune_batches(ctx, w, local, sizes=(1, 2, 4, 8, 16, 32, 64, 128, 256), reps=2):
    """Autotune the shape buckets that serving batches fall in: for each batch
    size, random samples of the event pool as device-resident batches (the
    settings stay in the context for every later launch of those buckets).
    Returns, per (size, sample) pair tuned, the events, digis and the chosen
    setting (which label store, how many threads an item, tile and blocks)."""
    import torch

    from paper_2004_04334_gb300 import hp

    dev = torch.device(f"cuda:{local}")
    rng = np.random.default_rng(synth.child_seed(synth.BASE_SEED + 5, 77))
    chosen = []
    for E in sizes:
        for _ in range(reps):
            sub = w.subset(rng.integers(0, w.n_events, E))
            dw = torch.from_numpy(sub.words.view(np.int32)).to(dev)
            dm = torch.from_numpy(sub.modules.view(np.int16)).to(dev)
            do = torch.from_numpy(sub.offsets.view(np.int64)).to(dev)
            out = hp.DeviceOutputs(sub.n_events, sub.n_digis, dev, labels=False)
            best, best_ms, _ = ctx.autotune(sub.n_events, sub.n_digis, do.data_ptr(), dw.data_ptr(), dm.data_ptr(),
                                            out, reps=2)
            chosen.append(dict(best, events=int(sub.n_events), digis=int(sub.n_digis), ms=round(best_ms, 4)))
    torch.cuda.synchronize(dev)
    return chosen


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.serving_only:
        _, _, local = _dist()
        from paper_2004_04334_gb300 import build
        build.build()
        print(json.dumps(run_serving(local, [float(x) for x in a.serving_rates.split(",") if x],
                                     a.serving_events, nocopy=not a.serving_staging, profile=a.serving_profile,
                                     inflight=a.serving_inflight, seconds=a.serving_seconds,
                                     max_batch=a.serving_max_batch)), flush=True)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
