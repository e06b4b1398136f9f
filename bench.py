#!/usr/bin/env python3
"""Throughput of GB300-native ABEA on the large batched workload.

One step = one pass of the whole hot path (k-mer cache + input checks, band
loop, end cell, backtrack) over the workload "large_50k_ln8kb": 50,000
synthetic reads with log-normal lengths (median 8 kb, sigma_ln 0.5, at
least 500 b) of which 1 % are ultra-long (log-uniform 50-200 kb), k = 6,
W = 100; 1.35x10^11 in-matrix cells.  The metric is band-cell updates per
second (GCUPS: in-matrix cells filled, summed over reads), also reported as
reads/s.

  value : device-resident inputs (abea_align_batch_device); K steps spread
          round-robin over D contexts, each on its own stream (D = 2 batches
          in flight for this workload, about 62 GB of working memory each,
          so one batch's longest reads overlap the next batch's work), CUDA
          events around all K steps.
  e2e   : the same metric through abea_align_packed with page-locked host
          buffers, one host thread per context; each step copies its inputs
          host->device and its results device->host inside the timed region
          (the copies of one context overlap the other context's kernels).

Extra keys: the 4,096-read batch (median 5 kb, 6 batches in flight, and one
batch alone: its latency) and the wide k = 9 / W = 200 model, both
device-resident; the per-read scaling estimate, eventalign rows and event
detection on the 4,096-read batch; serving: serve_mix requests (70 % 400-base
prefixes, 30 % full reads) with seeded Poisson arrivals at 1x, 10x, 100x and
1000x the offered load of 512 channels x 450 bases/s through abea_server_*,
p50/p99 from submission to the result in host memory, per class.

cpu_baseline: the CPU oracle (oracle/, -O3) on bounded, evenly spaced samples
of the headline workload on the host cores (FP32 on all cores, FP32 on one
thread, FP64 on all cores); the FP64 run also gives the accuracy of the GPU
results on its sample (near-tie fraction, path mismatches on the other
reads, score error, FP64 score of the GPU paths against the FP64 optimum).

--impl reference runs the CPU oracle (FP32) on bounded samples of the same
workload.  With --gpus N > 1 each rank runs its own replica of the workload
(reads are independent; there is no data exchange).
"""
import argparse
import ctypes
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

WORKLOAD = "large_50k_ln8kb"
EXTRA_WORKLOADS = ("batch_4096_ln5kb", "wide_10k_ln10kb_k9_w200")
DEPTH = {"large_50k_ln8kb": 2, "batch_4096_ln5kb": 6, "wide_10k_ln10kb_k9_w200": 2}
METRIC = "ABEA band-cell updates/s (GCUPS) and reads/s on 1 GB300; p50/p99 latency served"
UNIT = "GCUPS"
# Issue slots of one cell update, the roofline's unit of work: 14, the budget of the canonical op sequence
# (10 FP32-pipe ops: x - mu', times 1/sigma', the emission, 5 FADD and 2 maxima; about 4 more for the
# 2-bit trace).  The kernel's own sequence is shorter (2 FFMA, 3 FADD, 2 compares and 2 selects for the
# two maxima with their directions, 2 votes for the trace, plus the band's bookkeeping shared over its
# cells), so the fraction quoted against 14 is the conservative one.
OPS_PER_CELL = 14
# DRAM bytes (read + write) per band of the core kernel from one ncu capture, valid only for the kernel
# source it was taken on; scaled to a launch by the batch's bands.
TRAFFIC_CAPTURE = {"source_sha1": "798a3581a806576aed2c2f22486da0b330c3a50d", "bytes_per_band": 85.147}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--reads", type=int, default=None, help="only the first N reads of the workload (profiling)")
    p.add_argument("--max-bases", type=int, default=None,
                   help="only the workload's reads of at most this many bases (profiling the full-load mix)")
    p.add_argument("--e2e-steps", type=int, default=None)
    p.add_argument("--cpu-seconds", type=float, default=8.0, help="target wall time of each CPU baseline leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the extra workloads")
    p.add_argument("--depth", type=int, default=None, help="batches in flight (one context and stream each)")
    p.add_argument("--event-reads", type=int, default=1024, help="reads whose raw signals event detection runs on")
    p.add_argument("--serve-requests", type=int, default=500,
                   help="serve_mix requests at 1x offered load (more at higher loads); 0 skips serving")
    p.add_argument("--block-theta", type=float, default=0.0,
                   help="reads above this multiple of the even per-warp share of bands run on a whole block "
                        "(<= 0: one warp per read)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
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
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 9]
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in rows:
            try:
                clk, cmax, util = float(r[1]), float(r[2]), float(r[4])
            except ValueError:
                continue
            mx.append(cmax)
            if util >= 50:
                sm.append(clk)
                for n, v in zip(names, r[6:10]):
                    if v.strip() == "Active":
                        reasons.add(n)
        if not sm:
            sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def max_over_ranks(x: float, world: int, dist=None, device=None) -> float:
    """The largest of every rank's x (all ranks call it; one rank: x itself)."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step: int, steps: int, seconds: float, world: int) -> float:
    """Whole-job rate: every rank processed its own copy of the workload (replicas), the job took
    the slowest rank's time."""
    return world * units_per_rank_step * steps / seconds


def geometry(W: int):
    """Offsets per lane C, whether lanes are partly filled, whether all 32 lanes are live, block-mode
    offsets per lane (the same choice as the library's)."""
    C = next((c for c in range((W + 31) // 32, 9) if W % c == 0), (W + 31) // 32)
    L = -(-W // C)
    cg = 0
    if W >= 32 and W % 4 == 0:
        cg = next((c for c in (1, 2) if (W // 4) % c == 0 and (W // 4) // c <= 31), 0)
    return C, C * L != W, L == 32, cg


def record_words(W: int) -> int:
    C, _, _, cg = geometry(W)
    return max((2 * C + 3) // 4 * 4, 8 * cg)


def kernel_name(W: int) -> str:
    C, mixed, full, cg = geometry(W)
    return f"align_kernel<{C},{str(mixed).lower()},{str(full).lower()},{cg}>"


def traffic_per_launch(bands: int):
    """DRAM bytes of one core-kernel launch over `bands` bands, from the ncu capture; None once the
    kernel source differs from the captured one (or none was taken)."""
    import hashlib
    if not TRAFFIC_CAPTURE["source_sha1"]:
        return None
    src = os.path.join(ROOT, "paper_2101_05012_gb300", "csrc", "abea_align.cu")
    with open(src, "rb") as f:
        if hashlib.sha1(f.read()).hexdigest() != TRAFFIC_CAPTURE["source_sha1"]:
            return None
    return int(TRAFFIC_CAPTURE["bytes_per_band"] * bands)


def make_workload_batch(synth, name, reads=None, max_bases=None):
    workers = max(1, min(16, os.cpu_count() or 1))
    if max_bases:
        L = synth.read_lengths(synth.WORKLOADS[name])
        return synth.make_batch(name, read_ids=np.nonzero(L <= max_bases)[0], workers=workers)
    return synth.make_batch(name, n_reads=reads, workers=workers)


def sample_ids(n: int, m: int) -> np.ndarray:
    return np.unique(np.linspace(0, n - 1, max(1, min(n, m)), dtype=np.int64))


def longest_first(batch, idx) -> np.ndarray:
    """idx ordered by decreasing band count: the oracle's threads take reads in this order, one at a
    time, so the longest ones start first and the threads finish together."""
    idx = np.asarray(idx, dtype=np.int64)
    bands = (batch.n_events() + batch.n_kmers())[idx]
    return idx[np.argsort(-bands, kind="stable")]


def oracle_rate(batch, seconds: float, threads: int, precision: str = "f32"):
    """The oracle on a bounded, evenly spaced sample of the batch (about `seconds` of wall time on
    `threads` threads): (GCUPS, reads/s, sample ids, results, description)."""
    from oracle import oracle
    n = batch.n
    cells_per_read = (batch.n_events() + batch.n_kmers() + 1).astype(np.float64) * batch.W
    pilot = batch.subset(sample_ids(n, 2 * threads))
    t = time.perf_counter()
    r = oracle.abea_batch(pilot, precision, n_threads=threads)
    dt = max(time.perf_counter() - t, 1e-3)
    rate = r["cells"].sum() / dt
    m = int(np.clip(rate * seconds / cells_per_read.mean(), threads, n))
    idx = longest_first(batch, sample_ids(n, m))
    sample = batch.subset(idx)
    t = time.perf_counter()
    r = oracle.abea_batch(sample, precision, n_threads=threads)
    dt = time.perf_counter() - t
    desc = (f"{len(idx)} of {n} reads, evenly spaced ({int(r['cells'].sum())} cells), {precision.upper()}, "
            f"{threads} thread{'s' if threads > 1 else ''}, {dt:.1f} s wall")
    return float(r["cells"].sum()) / dt / 1e9, len(idx) / dt, idx, r, desc


def serve_latency(binding, synth, device: int, load: float, n_req: int, theta: float):
    """serve_mix through the serving loop: seeded Poisson arrivals at `load` x the offered load of
    512 channels x 450 bases/s; latency from submission to the result in host memory, as the
    server stamps it."""
    batch, arrival, is_prefix = synth.serving_requests(n_req, load=load)
    ctx = binding.Context(device)
    ctx.set_model(batch.k, batch.model_mean, batch.model_stdv)
    srv = binding.Server(ctx, batch.W, max_batch_reads=256, max_wait_us=200, batches_in_flight=3,
                         block_theta=theta)
    reads = [batch.read(i) for i in range(batch.n)]
    warm = [srv.submit(*reads[i]) for i in range(min(32, batch.n))]
    for t in warm:
        while srv.poll(t, wait_us=100_000) is None:
            pass
    tickets = [None] * batch.n
    lat = np.zeros(batch.n)
    ready = threading.Semaphore(0)

    def poller():
        for i in range(batch.n):
            ready.acquire()
            while True:
                r = srv.poll(tickets[i], wait_us=100_000)
                if r is not None:
                    lat[i] = r[2]
                    break

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    for i in range(batch.n):
        d = t0 + arrival[i] - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tickets[i] = srv.submit(*reads[i])
        ready.release()
    th.join()
    wall = time.perf_counter() - t0
    srv.stop()
    ctx.close()
    ms = lat / 1e3
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    cls = {"prefix_400b": ms[is_prefix], "full_read": ms[~is_prefix]}
    return {"load": load, "requests": int(batch.n), "offered_req_per_s": float(batch.n / arrival[-1]),
            "served_req_per_s": float(batch.n / wall), "p50_ms": pct(ms, 50), "p99_ms": pct(ms, 99),
            **{f"{k}_p50_ms": pct(v, 50) for k, v in cls.items()},
            **{f"{k}_p99_ms": pct(v, 99) for k, v in cls.items()}}


def run_reference(args):
    """The FP32 CPU oracle on the host cores: each step aligns a core-balanced, evenly spaced sample of
    the workload (16 reads per thread, taken one at a time by the threads, longest first)."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    from paper_2101_05012_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    threads = os.cpu_count() or 1
    ids = sample_ids(w.n_reads, 16 * threads)
    sample = synth.make_batch(w, read_ids=ids)
    sample = sample.subset(longest_first(sample, np.arange(sample.n)))
    from oracle import oracle
    oracle.load()
    for _ in range(args.warmup):
        oracle.abea_batch(sample, "f32", n_threads=threads)
    times, cells = [], 0
    for _ in range(args.steps):
        t = time.perf_counter()
        r = oracle.abea_batch(sample, "f32", n_threads=threads)
        times.append(time.perf_counter() - t)
        cells = int(r["cells"].sum())
    total = sum(times)
    value = cells * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "reads": w.n_reads, "W": w.W, "k": w.k,
                       "step": f"FP32 CPU oracle over {len(ids)} evenly spaced reads of the workload"},
            "reads_per_s": len(ids) * args.steps / total,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{len(ids)} of {w.n_reads} reads per step ({cells} cells), "
                                       f"{threads} threads taking reads one at a time, longest first"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class Workload:
    """One workload's batch, contexts, streams and device buffers (device-resident leg)."""

    def __init__(self, torch, binding, batch, dev, D, theta):
        self.torch, self.binding, self.batch, self.dev, self.D = torch, binding, batch, dev, D
        n = batch.n
        self.pair_off = binding.pair_offsets(batch.n_events(), np.maximum(batch.n_kmers(), 1))
        n_pairs = int(self.pair_off[-1])
        self.ctxs = []
        for _ in range(D):
            c = binding.Context(dev.index)
            c.set_model(batch.k, batch.model_mean, batch.model_stdv)
            c.set_block_mode(theta)
            self.ctxs.append(c)
        self.d_seq = torch.from_numpy(batch.seq).to(dev)
        self.d_ev = torch.from_numpy(batch.events).to(dev)
        self.d_out = [torch.zeros(n * 24, dtype=torch.uint8, device=dev) for _ in range(D)]
        self.d_pairs = [torch.zeros(max(n_pairs, 1) * 2, dtype=torch.int32, device=dev) for _ in range(D)]
        self.streams = [torch.cuda.Stream(dev) for _ in range(D)]

    def step(self, i):
        b, j = self.batch, i % self.D
        self.ctxs[j].align_batch_device(b.n, b.W, self.d_seq, b.seq_off, self.d_ev, b.ev_off, b.scalings,
                                        self.d_out[j], self.d_pairs[j], self.pair_off,
                                        stream=self.streams[j].cuda_stream)

    def warm(self, warmup):
        torch, binding = self.torch, self.binding
        for i in range(max(warmup, self.D)):
            self.step(i)
        torch.cuda.synchronize(self.dev)
        res = binding.results_from_bytes(self.d_out[0].cpu().numpy())
        if not np.all(res["status"] == 0):
            raise SystemExit(f"bench: {int(np.sum(res['status'] != 0))} reads failed")
        for j in range(1, self.D):
            if not np.array_equal(binding.results_from_bytes(self.d_out[j].cpu().numpy()), res):
                raise SystemExit("bench: contexts disagree")
        self.res = res
        self.cells = int(res["cells"].sum())
        return res

    def latency(self, reps=3):
        torch = self.torch
        lat = []
        for _ in range(reps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(self.streams[0])
            self.step(0)
            a1.record(self.streams[0])
            a1.synchronize()
            lat.append(a0.elapsed_time(a1))
        return statistics.median(lat)

    def timed(self, steps):
        """ms of `steps` device-resident steps over the D streams, and the core kernels' launches and
        summed span."""
        torch = self.torch
        for c in self.ctxs:
            c.last_launch_stats()
        main = torch.cuda.Stream(self.dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for st in self.streams:
            st.wait_event(e0)
        for i in range(steps):
            self.step(i)
        for st in self.streams:
            ev = torch.cuda.Event()
            ev.record(st)
            main.wait_event(ev)
        e1.record(main)
        torch.cuda.synchronize(self.dev)
        launches, align_ms = 0, 0.0
        for c in self.ctxs:
            nl, ms = c.last_launch_stats()
            launches += nl
            align_ms += ms
        return e0.elapsed_time(e1), launches, align_ms

    def e2e(self, steps, world, dist):
        """Seconds of `steps` end-to-end steps through abea_align_packed (page-locked host buffers, one
        host thread per context), the launches they made, the bytes copied per step and the host pairs
        of context 0."""
        torch, binding, b = self.torch, self.binding, self.batch
        n = b.n
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        h_seq, h_ev = pin(b.seq), pin(b.events)
        n_pairs = int(self.pair_off[-1])
        h_out = [torch.zeros(n * 24, dtype=torch.uint8).pin_memory().numpy() for _ in range(self.D)]
        h_pairs = [torch.zeros(max(n_pairs, 1) * 2, dtype=torch.int32).pin_memory().numpy() for _ in range(self.D)]
        sc = np.ascontiguousarray(b.scalings, np.float32)
        errors = []

        def e2e_step(j):
            c = self.ctxs[j]
            rc = c.lib.abea_align_packed(c.h, n, b.W, binding._p(h_seq), binding._p(b.seq_off), binding._p(h_ev),
                                         binding._p(b.ev_off), binding._p(sc), binding._p(h_out[j]),
                                         binding._p(h_pairs[j]), binding._p(self.pair_off),
                                         ctypes.c_void_p(self.streams[j].cuda_stream))
            if rc != 0:
                errors.append(rc)

        for j in range(self.D):
            e2e_step(j)
        for c in self.ctxs:
            c.last_launch_stats()
        gate = threading.Barrier(self.D + 1)

        def worker(j):
            gate.wait()
            for _ in range(j, steps, self.D):
                e2e_step(j)

        threads = [threading.Thread(target=worker, args=(j,)) for j in range(self.D)]
        for th in threads:
            th.start()
        if world > 1:
            dist.barrier()
        gate.wait()
        t = time.perf_counter()
        for th in threads:
            th.join()
        secs = time.perf_counter() - t
        if errors:
            raise binding.AbeaError(errors[0], "abea_align_packed")
        launches = sum(c.last_launch_stats()[0] for c in self.ctxs)
        for j in range(self.D):
            if not np.array_equal(binding.results_from_bytes(h_out[j]), self.res):
                raise SystemExit("bench: host-memory results differ from device-resident results")
        h2d = int(b.seq.nbytes + b.events.nbytes + n * (112 + 4))
        d2h = int(n * 24 + n_pairs * 8)
        return secs, launches, h2d, d2h, h_pairs[0].reshape(-1, 2)

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []
        self.d_seq = self.d_ev = self.d_out = self.d_pairs = None
        self.torch.cuda.synchronize(self.dev)
        self.torch.cuda.empty_cache()


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2101_05012_gb300 import binding, synth

    rank, local_rank, world = dist_env()
    # synthetic inputs first (a process pool, started before any CUDA call)
    batch = make_workload_batch(synth, args.workload, args.reads, args.max_bases)
    extra_batches = {}
    if not args.no_extra and rank == 0 and world == 1 and not args.reads and not args.max_bases:
        for name in EXTRA_WORKLOADS:
            if name != args.workload:
                extra_batches[name] = make_workload_batch(synth, name)
    torch.cuda.set_device(local_rank)            # before the process group: NCCL binds the current device
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    n = batch.n
    D = args.depth or DEPTH.get(args.workload, 2)
    wl = Workload(torch, binding, batch, dev, D, args.block_theta)
    wl.warm(args.warmup)
    cells = wl.cells
    lat = wl.latency()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    ms_total, launches, align_ms = wl.timed(args.steps)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms_total = max_over_ranks(ms_total, world, dist, dev)
    ms_step = ms_total / args.steps
    value = job_rate(cells, args.steps, ms_total / 1e3, world) / 1e9
    reads_per_s = job_rate(n, args.steps, ms_total / 1e3, world)

    # end to end through the host-memory call
    e2e_steps = args.e2e_steps or max(3, min(args.steps, 10 if n > 10_000 else 60))
    e2e_s, e2e_launches, h2d, d2h, h_pairs = wl.e2e(e2e_steps, world, dist)
    e2e_s = max_over_ranks(e2e_s, world, dist, dev)
    e2e_value = job_rate(cells, e2e_steps, e2e_s, world) / 1e9

    # roofline of the core kernel: FP32-pipe issue.  With D batches in flight the launches overlap;
    # the kernel's rate is the cells of one launch over the launch period (timed region / launches);
    # the mean span of a single launch is reported beside it.
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    span_ms = align_ms / max(args.steps, 1)
    period_ms = ms_total / max(args.steps, 1)
    achieved = cells * OPS_PER_CELL / (period_ms / 1e3) / 1e12
    peak = sms * 128 * sm_max * 1e6 / 1e12
    bands = int((batch.n_events() + batch.n_kmers() + 1).sum())
    trace_bytes = bands * 4 * record_words(batch.W)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s", "frac": achieved / peak,
                "traffic": traffic_per_launch(bands), "kernel": kernel_name(batch.W),
                "launch_period_ms": period_ms, "launch_span_ms": span_ms, "batches_in_flight": D,
                "ops_per_cell": OPS_PER_CELL,
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (MEASURED_PEAKS.json sm_max_mhz)"}
    if clk and clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (sms * 128 * clk["sm_mhz"] * 1e6 / 1e12)
    config = {"workload": args.workload, "reads": n, "W": batch.W, "k": batch.k, "cells_per_step": cells,
              "bases_per_step": int(batch.seq.size), "events_per_step": int(batch.events.size),
              "parallelism": f"replicas x{world}" if world > 1 else "1 GPU", "batches_in_flight": D,
              "block_theta": args.block_theta,
              "l2": f"inputs ({batch.events.nbytes / 1e9:.1f} GB events) and the trace "
                    f"({trace_bytes / 1e9:.1f} GB per step) exceed the 129 MB L2"}
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s / e2e_steps, "gpu_launches": e2e_launches,
           "host_threads": D}
    h_res, h_pair_off = wl.res, wl.pair_off
    wl.close()

    # extra workloads (device-resident rate; the 4,096-read batch also alone, and the secondary kernels)
    extra, scal_line, ea_line, ev_line = {}, None, None, None
    for name, xb in extra_batches.items():
        xD = DEPTH.get(name, 2)
        x = Workload(torch, binding, xb, dev, xD, args.block_theta)
        x.warm(args.warmup)
        xlat = x.latency()
        xsteps = max(6, min(args.steps, 30 if xb.n <= 4096 else 10))
        xms, xl, _ = x.timed(xsteps)
        extra[name] = {"value": x.cells * xsteps / (xms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": xms / xsteps,
                       "steps": xsteps, "batches_in_flight": xD, "batch_latency_ms": xlat, "reads": xb.n,
                       "W": xb.W, "k": xb.k, "cells_per_step": x.cells, "gpu_launches": xl,
                       "kernel": kernel_name(xb.W)}
        if name == "batch_4096_ln5kb":
            extra[name]["autotune"] = autotune_leg(x)
            scal_line, ea_line, ev_line = secondary_kernels(torch, binding, synth, x, args)
        x.close()

    serving = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        serving = [serve_latency(binding, synth, local_rank, load, n_req, 1.0)
                   for load, n_req in ((1.0, args.serve_requests), (10.0, 4 * args.serve_requests),
                                       (100.0, 8 * args.serve_requests), (1000.0, 8 * args.serve_requests))]

    cpu, accuracy = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import rescore
        threads_n = os.cpu_count() or 1
        gc, rps, _, _, desc = oracle_rate(batch, args.cpu_seconds, threads_n, "f32")
        g1, r1, _, _, d1 = oracle_rate(batch, args.cpu_seconds, 1, "f32")
        g64, r64, idx64, o64, d64 = oracle_rate(batch, args.cpu_seconds, threads_n, "f64")
        sub = batch.subset(idx64)
        gp = [h_pairs[h_pair_off[i]:h_pair_off[i] + h_res["n_pairs"][i]] for i in idx64]
        sub_off = np.zeros(len(idx64) + 1, np.int64)
        np.cumsum([len(p) for p in gp], out=sub_off[1:])
        gpairs = np.concatenate(gp) if gp else np.zeros((0, 2), np.int32)
        accuracy = rescore.accuracy_against_fp64(sub, h_res[idx64], gpairs, sub_off, o64)
        accuracy["sample"] = f"the FP64 leg's {len(idx64)} reads"
        cpu = {"value": gc, "unit": UNIT, "cores": threads_n, "kind": "oracle", "sample": desc,
               "reads_per_s": rps, "flags": "gcc -O3 -ffp-contract=off",
               "threads_1": {"value": g1, "unit": UNIT, "reads_per_s": r1, "sample": d1},
               "fp64": {"value": g64, "unit": UNIT, "reads_per_s": r64, "sample": d64}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
                "reads_per_s": reads_per_s, "batch_latency_ms": lat, "kernel_launch_span_ms": span_ms,
                "gpu_launches": launches, "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
                "accuracy": accuracy, "clocks": clk, "extra_workloads": extra, "serving": serving,
                "scalings_estimate": scal_line, "event_detection": ev_line, "eventalign": ea_line}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def autotune_leg(x):
    """abea_autotune on a sample of the batch (its 32 longest reads and every 16th read), then the
    one-batch latency with the tuned launch geometry against per-warp mode alone (context 0)."""
    b, ctx = x.batch, x.ctxs[0]
    bands = b.n_events().astype(np.int64) + np.maximum(b.n_kmers(), 1) + 1
    ids = np.unique(np.concatenate([np.argsort(-bands)[:32], np.arange(0, b.n, 16)]))
    t0 = time.perf_counter()
    choices = ctx.autotune(b.subset(ids))
    tune_s = time.perf_counter() - t0
    tuned = x.latency()
    ctx.set_block_mode(0.0)                     # back to per-warp mode for the legs after this one
    per_warp = x.latency()
    return {"sample_reads": int(len(ids)), "tune_s": tune_s,
            "choices": [{k: (int(c[k]) if k not in ("gcups_per_warp", "gcups_block") else float(c[k]))
                         for k in c.dtype.names} for c in choices],
            "batch_latency_ms_tuned": tuned, "batch_latency_ms_per_warp": per_warp}


def secondary_kernels(torch, binding, synth, x, args):
    """The per-read scaling estimate, eventalign rows and event detection over the 4,096-read batch
    (context 0 of workload x, after its timed run)."""
    batch, dev, n = x.batch, x.dev, x.batch.n
    ctx, st = x.ctxs[0], x.streams[0]
    steps = max(6, min(args.steps, 30))
    hbm = float(measured_peaks().get("hbm_gbs") or 6800.0)

    def timed(fn):
        for _ in range(3):
            fn()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(st)
        for _ in range(steps):
            fn()
        s1.record(st)
        s1.synchronize()
        return s0.elapsed_time(s1) / steps

    d_sc = torch.zeros(n * 3, dtype=torch.float32, device=dev)
    d_sst = torch.zeros(n, dtype=torch.int32, device=dev)
    scal_ms = timed(lambda: ctx.estimate_scalings(n, x.d_seq, batch.seq_off, x.d_ev, batch.ev_off, d_sc, d_sst,
                                                  stream=st.cuda_stream))
    scal_bytes = int(batch.events.nbytes + batch.seq.nbytes)
    scal = {"kernel": "scalings_kernel", "ms_per_launch": scal_ms, "reads_per_s": n / (scal_ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": scal_bytes / (scal_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": scal_bytes / (scal_ms / 1e3) / 1e9 / hbm, "bytes_per_launch": scal_bytes},
            "ok_reads": int((d_sst == 0).sum().item())}

    ea_refs, ea_pos, ea_base = [], np.zeros(len(batch.seq), np.int32), 0
    for i in range(n):
        r_, p_ = synth.make_ref_alignment(batch.seq[batch.seq_off[i]:batch.seq_off[i + 1]].tobytes(), 9, i)
        ea_pos[batch.seq_off[i]:batch.seq_off[i + 1]] = np.where(p_ >= 0, p_ + ea_base, -1)
        ea_refs.append(r_)
        ea_base += len(r_)
    d_ref = torch.from_numpy(np.concatenate(ea_refs)).to(dev)
    d_rpos = torch.from_numpy(ea_pos).to(dev)
    d_rows = torch.empty(int(x.pair_off[-1]) * 40, dtype=torch.uint8, device=dev)
    ea_ms = timed(lambda: ctx.eventalign(n, x.d_seq, batch.seq_off, x.d_ev, batch.ev_off, batch.scalings, x.d_out[0],
                                         x.d_pairs[0], x.pair_off, d_rpos, d_ref, ea_base, False, d_rows,
                                         stream=st.cuda_stream))
    rows_n = int(x.res["n_pairs"].sum())
    ea_bytes = rows_n * (8 + 4 + 4 + 40)
    ea = {"kernels": ["eventalign_ranks_kernel", "eventalign_kernel"], "rows": rows_n, "ms_per_call": ea_ms,
          "launches_per_call": 2, "rows_per_s": rows_n / (ea_ms / 1e3),
          "roofline": {"bound": "hbm", "achieved": ea_bytes / (ea_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                       "frac": ea_bytes / (ea_ms / 1e3) / 1e9 / hbm, "bytes_per_launch": ea_bytes}}
    del d_ref, d_rpos, d_rows

    ev = None
    if args.event_reads > 0:
        rb = synth.make_raw_batch("batch_4096_ln5kb", n_reads=min(args.event_reads, n))
        d_raw = torch.from_numpy(rb.raw).to(dev)
        ev_cap = (rb.raw_off[1:] - rb.raw_off[:-1]) // 3 + 2
        ev_off = np.zeros(rb.n + 1, np.int64)
        np.cumsum(ev_cap, out=ev_off[1:])
        d_evs = torch.zeros(int(ev_off[-1]) * 16, dtype=torch.uint8, device=dev)
        d_nev = torch.zeros(rb.n, dtype=torch.int32, device=dev)
        det_ms = timed(lambda: ctx.detect_events(rb.n, d_raw, rb.raw_off, rb.calib, 3, 2.0, d_evs, ev_off, d_nev,
                                                 stream=st.cuda_stream))
        n_events = int(d_nev.sum().item())
        det_bytes = int(rb.raw.nbytes + n_events * 16)
        ev = {"kernels": ["event_tiles_kernel<3>", "event_scan_kernel", "event_emit_kernel"], "reads": rb.n,
              "samples": int(rb.raw.size), "events": n_events, "ms_per_call": det_ms, "launches_per_call": 3,
              "samples_per_s": rb.raw.size / (det_ms / 1e3),
              "roofline": {"bound": "hbm", "achieved": det_bytes / (det_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": det_bytes / (det_ms / 1e3) / 1e9 / hbm, "bytes_per_launch": det_bytes}}
        del d_raw, d_evs
    return scal, ea, ev


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
