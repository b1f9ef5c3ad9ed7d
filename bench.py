#!/usr/bin/env python
"""Throughput benchmark of the GPU receiver on the KK-16QAM workload.

Workload: a Kramers-Kronig 16QAM stream at 1 GBaud sampled at 4 GS/s, 12-bit,
buffers of 2^22 samples, RRC 0.1, CSPR 10 dB, 100 kHz linewidth, SNR 20 dB,
overlap-save Hilbert FFT 2^16 / 4096, downshift 0.55 GHz, 31-tap CMA -> DD-LMS
FIR at 2 samples/symbol, blind phase search 32 phases x 64 symbols, 16QAM Gray
demap, bit-error count.  One step runs the whole chain over a batch of
``--bufs-per-step`` consecutive buffers of one stream, drawn from a ring of
``--ring`` distinct synthetic buffers resident in HBM (the ring is larger than
L2).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (the method's plain restatement) on
the host cores, each step a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

# Each receiver handle pipelines its stages on five streams (plus a copy stream),
# and a group adds up to eight worker streams.  CUDA maps streams onto a limited
# set of hardware queues (8 unless raised); two pipeline stages that land on the
# same queue serialise behind each other.  Raise the limit before CUDA starts.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "KK-16QAM Rx GSa/s on 1 GB300 at oracle-matched BER; CNN-eq vs LMS BER & GSa/s"
FMT, NB, FS, BAUD = 4, 1 << 22, 4e9, 1e9
PROFILE_EVERY = 16          # stage events on one call in 16 of the timed run
WARMUP_MIN_S = 0.5          # untimed warm-up: at least this long, and at least --warmup steps
ALONE_REPS = 40            # single-buffer calls whose stages are timed alone (roofline)
GEN = dict(snr_db=20.0, cspr_db=10.0, linewidth=100e3)
STAGES = ["unpack", "kk_fwd", "kk_rows", "kk_inv", "mf", "eq", "demap"]
# algorithmic FP32 operations per ADC sample of each stage (5 N log2 N per FFT;
# the overlap-save factor N/(N-V) = 16/15 included)
OLS = 65536 / (65536 - 4096)
FLOPS_PER_SAMPLE = {"kk_fwd": 13.0 * OLS, "kk_rows": 60.0 * OLS, "kk_inv": 13.0 * OLS, "mf": 130.0,
                    "eq": 252.0, "kk_front": 86.0 * OLS}
BYTES_PER_SAMPLE = {"unpack": 1.5 + 2.0}   # packed read + 16-bit code write
LANES = 128                 # FP32 lanes per SM (the SM count is queried from the device)


def workload_config(args):
    return {"workload": "KK-16QAM single stream, 2^22-sample 12-bit buffers (synthetic)",
            "format": "KK-16QAM", "baud": BAUD, "fs": FS, "buf_len": NB, "ols_n": 65536, "ols_v": 4096,
            "fir_taps": 31, "bps_phases": 32, "bps_window": 64, "cspr_db": 10, "snr_db": 20,
            "linewidth_hz": 100e3, "bufs_per_step": args.bufs_per_step, "ring_buffers": args.ring,
            "l2": "inputs larger than L2: ring of %d distinct packed buffers = %.0f MiB" % (
                args.ring, args.ring * NB * 1.5 / 2 ** 20),
            "seed": 1}


def cpu_model():
    """The host CPU's model name (or its architecture where the kernel does not say)."""
    import platform
    arm = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                k = k.strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    return v.strip()
                if k in ("cpu implementer", "cpu part") and k not in arm:
                    arm[k] = v.strip()
    except OSError:
        pass
    if arm:   # Arm kernels give the implementer and part numbers only (0x41 / 0xd4f: Neoverse V2)
        return "%s, implementer %s, part %s" % (platform.machine(), arm.get("cpu implementer", "?"),
                                                 arm.get("cpu part", "?"))
    return platform.machine()


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------- clock sampler
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.period_ms = period_ms
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        inside = [l for (t, l) in self.samples if self.t0 is not None and self.t0 <= t <= self.t1]
        if not inside:   # fall back to the samples nearest the timed region
            inside = [l for (t, l) in self.samples][-3:]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in inside:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- reference
def reference_arm(args, rank):
    """FP64 oracle on the host cores; each step one bounded sample buffer."""
    import oracle
    import synth
    total = args.steps + args.warmup
    nb = NB   # the workload's own 2^22-sample buffer (about 3 s of oracle time each)
    while nb > 1 << 15 and total * nb / 1.2e6 > 240.0:   # only a very long run shrinks it
        nb //= 2
    g = synth.gen_kk_stream(FMT, nb, total, seed=1, truth=False,
                            workers=min(16, os.cpu_count() or 1), **GEN)
    o = oracle.Oracle(**oracle.default_cfg(FMT, nb))
    for b in range(args.warmup):
        o.process(g["packed"][b])
    t = time.perf_counter()
    for b in range(args.warmup, total):
        o.process(g["packed"][b])
    dt = time.perf_counter() - t
    value = args.steps * nb / dt / 1e9
    s = o.stats()
    cfg = workload_config(args)
    cfg.update(buf_len=nb, bufs_per_step=1, ring_buffers=total)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GSa/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "GSa/s", "cores": 1, "kind": "oracle",
                             "sample": f"one {nb}-sample buffer of the KK-16QAM stream per step",
                             "host_cpus": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "GSa/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "ber": s["ber"]}
    print(json.dumps(line), flush=True)


def _oracle_worker(bufs):
    """One independent oracle stream in a spawned process: (samples, seconds)."""
    import oracle
    o = oracle.Oracle(**oracle.default_cfg(FMT, len(bufs[0]) * 2 // 3))
    t = time.perf_counter()
    for b in bufs:
        o.process(b)
    return len(bufs) * len(bufs[0]) * 2 // 3, time.perf_counter() - t


def cpu_all_cores(packed, per_core: int = 2):
    """The oracle on every host core: one independent stream of `per_core`
    consecutive ring buffers per core, in spawned processes (the oracle itself stays
    single-threaded).  GSa/s = all samples over the wall time of the slowest core."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = [[packed[(per_core * i + j) % len(packed)] for j in range(per_core)] for i in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [[jobs[0][0][:3 * 8192]]] * cores)   # import and load in every worker first
        t = time.perf_counter()
        res = pool.map(_oracle_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t
    return {"cores": cores, "value": sum(n for n, _ in res) / wall / 1e9,
            "sample": f"{cores} independent streams of {per_core} buffers of 2^22 samples, one per core, "
                      "spawned processes, wall time of the slowest"}


def replica_throughput(ms_local, units_per_rank, dist=None, device="cpu"):
    """Replicas only: every rank runs its own stream; the job's time is the slowest
    rank's and its throughput is all ranks' units over that time (units per s)."""
    import torch
    world = 1
    ms = ms_local
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world / (ms * 1e-3)


# --------------------------------------------------------------------- GPU arm
def gpu_arm(args, rank, world, local):
    import torch
    import synth
    import paper_2010_14333_gb300 as rx

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    t_gen = time.perf_counter()
    g = synth.gen_kk_stream(FMT, NB, args.ring, seed=1 + rank, truth=False,
                            workers=min(16, os.cpu_count() or 1), **GEN)
    t_gen = time.perf_counter() - t_gen
    ring = [torch.from_numpy(p).cuda() for p in g["packed"]]
    r = rx.Receiver(FMT, NB, eq_warps=args.eq_warps, deadline_ms=args.deadline_ms)
    stream = torch.cuda.current_stream()

    # one step = one pipelined call over bufs_per_step consecutive buffers of the ring
    bits_out = [torch.zeros(r.max_bits // 8 + 16, dtype=torch.uint8, device="cuda")
                for _ in range(args.bufs_per_step)]
    out_ptrs = [b.data_ptr() for b in bits_out]
    sid = stream.cuda_stream

    host_s = [0.0]

    def run_steps(rcv, n):
        nbits = 0
        for _ in range(n):
            ins = [ring[(rcv.pos + j) % args.ring].data_ptr() for j in range(args.bufs_per_step)]
            t = time.perf_counter()
            nbits += sum(rx.rx_process_batch(rcv.h, ins, out_ptrs, sid))
            host_s[0] += time.perf_counter() - t
            rcv.pos += args.bufs_per_step
        return nbits

    # warm-up: at least W steps and at least WARMUP_MIN_S of back-to-back work, so
    # that the timed steps start from the clocks and pipeline state of a busy GPU
    # (the synthetic data generation before this leaves the GPU idle for seconds)
    clocks = Clocks(local, args.smi_ms)
    clocks.start()
    r.pos = 0
    warm_steps, t_w = 0, time.perf_counter()
    while warm_steps < args.warmup or time.perf_counter() - t_w < WARMUP_MIN_S:
        run_steps(r, 1)
        warm_steps += 1
        if warm_steps % 8 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    rx.rx_profile(r.h, max(1, min(PROFILE_EVERY, args.steps * args.bufs_per_step // 4)))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    if args.profile_range:
        torch.cuda.profiler.start()
    clocks.t0 = time.time()
    ev0.record(stream)
    host_s[0] = 0.0
    run_steps(r, args.steps)
    host_enqueue_ms = host_s[0] / args.steps * 1e3   # host time spent enqueueing one step
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.t1 = time.time()
    if args.profile_range:
        torch.cuda.profiler.stop()
    barrier()
    ms = ev0.elapsed_time(ev1)
    stage_ms, calls = rx.rx_profile_read(r.h)
    rx.rx_profile(r.h, False)
    time.sleep(0.1)
    clocks.stop()
    ms, value = replica_throughput(ms, args.steps * args.bufs_per_step * NB, dist, "cuda")
    value /= 1e9
    stats = r.stats()

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    host_ring = [torch.from_numpy(p).pin_memory() for p in g["packed"]]
    c2 = rx.rx_default_config(FMT)
    c2.eq_warps = args.eq_warps
    c2.deadline_ms = args.deadline_ms
    h2 = rx.rx_create(FMT, BAUD, FS, NB, c2)
    out_host = [torch.zeros(rx.rx_max_bits(h2) // 8 + 16, dtype=torch.uint8).pin_memory()
                for _ in range(args.bufs_per_step)]
    hout_ptrs = [t.data_ptr() for t in out_host]
    pos = 0
    e2e_steps = max(1, args.steps)
    h2d = d2h = 0
    # warm-up as for the device-resident steps: at least W steps and WARMUP_MIN_S of work
    e2e_warm, t_w = 0, time.perf_counter()
    while e2e_warm < args.warmup or time.perf_counter() - t_w < WARMUP_MIN_S:
        hin = [host_ring[(pos + j) % args.ring].data_ptr() for j in range(args.bufs_per_step)]
        rx.rx_process_host_batch(h2, hin, hout_ptrs, sid)
        pos += args.bufs_per_step
        e2e_warm += 1
        if e2e_warm % 8 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        hin = [host_ring[(pos + j) % args.ring].data_ptr() for j in range(args.bufs_per_step)]
        ns = rx.rx_process_host_batch(h2, hin, hout_ptrs, sid)
        pos += args.bufs_per_step
        h2d += args.bufs_per_step * NB * 3 // 2
        d2h += sum((n + 7) // 8 for n in ns)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    barrier()
    e2e_ms, e2e_value = replica_throughput(e2e_ms, e2e_steps * args.bufs_per_step * NB, dist, "cuda")
    e2e_value /= 1e9
    rx.rx_destroy(h2)
    # one step's host-to-device copies alone (pinned ring to the device, one copy per
    # buffer as the receiver issues them, best of three): the copy rate of this machine,
    # which bounds the end-to-end number
    nbytes = NB * 3 // 2
    h2d_gbs = None
    dst = torch.empty(nbytes * args.bufs_per_step, dtype=torch.uint8, device="cuda")
    best = None
    for _ in range(3):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for j in range(args.bufs_per_step):
            dst[j * nbytes:(j + 1) * nbytes].copy_(host_ring[j % args.ring], non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        t = c0.elapsed_time(c1)
        best = t if best is None else min(best, t)
    if best and best > 0:
        h2d_gbs = nbytes * args.bufs_per_step / (best * 1e-3) / 1e9
    del dst

    # ---- per-buffer latency, one buffer in flight at a time (the paper's budget:
    # five streams of 2^22 samples within 5 * 2^22 / 4 GS/s = 5.243 ms; one buffer
    # arrives every 1.049 ms)
    lat_dev, lat_host = [], []
    h3 = rx.rx_create(FMT, BAUD, FS, NB, rx.rx_default_config(FMT))
    try:
        for i in range(args.latency_reps + 5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rx.rx_process(r.h, ring[r.pos % args.ring].data_ptr(), out_ptrs[0], sid)
            b.record(stream)
            r.pos += 1
            c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c.record(stream)
            rx.rx_process_host(h3, host_ring[i % args.ring].data_ptr(), hout_ptrs[0], sid)
            d.record(stream)
            torch.cuda.synchronize()
            if i >= 5:
                lat_dev.append(a.elapsed_time(b))
                lat_host.append(c.elapsed_time(d))
    finally:
        rx.rx_destroy(h3)
    pct = lambda v, q: float(np.percentile(np.asarray(v), q))
    latency = {"reps": args.latency_reps, "budget_ms": 5.243, "arrival_interval_ms": NB / FS * 1e3,
               "device_p50_ms": pct(lat_dev, 50), "device_p99_ms": pct(lat_dev, 99),
               "host_p50_ms": pct(lat_host, 50), "host_p99_ms": pct(lat_host, 99),
               "note": "one buffer at a time; device = input resident in HBM, host = pinned H2D + chain + D2H"}

    # ---- the stages timed alone: one buffer in flight and a synchronize after each,
    # so no other kernel shares the SMs with the one timed
    rx.rx_profile(r.h, 1)
    for _ in range(ALONE_REPS):
        rx.rx_process(r.h, ring[r.pos % args.ring].data_ptr(), out_ptrs[0], sid)
        r.pos += 1
        torch.cuda.synchronize()
    alone_ms, alone_calls = rx.rx_profile_read(r.h)
    rx.rx_profile(r.h, 0)

    # ---- per-stage times (CUDA events on the launching stream) and roofline
    def per_stage(ms_by_stage, n):
        pc = {s: ms_by_stage[s] / max(n, 1) for s in STAGES}
        if pc["kk_rows"] < 1e-4 and pc["kk_inv"] < 1e-4:
            # 2^16-point blocks run as one fused cluster kernel, profiled in the first slot
            pc["kk_front"] = pc.pop("kk_fwd")
            del pc["kk_rows"], pc["kk_inv"]
        if pc.get("unpack", 0.0) == 0.0:
            pc.pop("unpack", None)      # the KK kernels read the packed input themselves
        return pc
    per_call = per_stage(stage_ms, calls)
    per_alone = per_stage(alone_ms, alone_calls)
    tot = sum(per_call.values())
    # the stages overlap on six streams, so their live times do not rank the
    # kernels: the equaliser, the top kernel of the serialised ncu launch list,
    # is the one reported
    dom = "eq" if per_call.get("eq", 0.0) > 0 else max(per_call, key=per_call.get)
    peaks = load_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * LANES * 2 * sm_max * 1e6 / 1e12        # FP32 TFLOP/s at the maximum SM clock
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    stages = {}
    tot_alone = sum(per_alone.values())
    for s in per_call:
        t, ta = per_call[s], per_alone.get(s, 0.0)
        d = {"ms_per_call": t, "share": t / tot if tot else 0.0,
             "alone_ms_per_call": ta, "alone_share": ta / tot_alone if tot_alone else 0.0}
        if s in FLOPS_PER_SAMPLE and ta > 0:
            d["tflops"] = FLOPS_PER_SAMPLE[s] * NB / (ta * 1e-3) / 1e12
            d["frac_alu"] = d["tflops"] / alu_peak
        if s in BYTES_PER_SAMPLE and ta > 0:
            d["gbs"] = BYTES_PER_SAMPLE[s] * NB / (ta * 1e-3) / 1e9
            d["frac_hbm"] = d["gbs"] / hbm_peak
        stages[s] = d
    traffic, traffic_src = None, None
    tr_path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if os.path.exists(tr_path):
        # ncu DRAM bytes of one launch, valid only while the kernel's source is the one
        # the capture was taken from (its sha256 is stored beside the figure)
        ent = json.load(open(tr_path)).get(dom)
        if isinstance(ent, dict):
            import hashlib
            src = os.path.join(ROOT, "paper_2010_14333_gb300", "csrc", ent.get("source", ""))
            cur = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] if os.path.isfile(src) else None
            if cur and cur == ent.get("source_sha16"):
                traffic = ent.get("bytes_per_launch")
                traffic_src = {k: ent.get(k) for k in ("capture", "source", "source_sha16", "profile")}
            else:
                traffic_src = {"stale": "kernel source changed since the capture", "capture": ent.get("capture")}
    timing = ("launches timed alone: CUDA events on the launching stream around each of %d launches, "
              "one buffer in flight (in the pipelined timed region the stages on five streams share the SMs, "
              "which stretches each launch: see pipelined)" % alone_calls)
    t_live = per_call.get(dom, 0.0)
    if alone_calls == 0 or tot_alone == 0 or not ("tflops" in stages[dom] or "gbs" in stages[dom]):
        roof = None
    elif dom in FLOPS_PER_SAMPLE:
        ach = stages[dom]["tflops"]
        live = FLOPS_PER_SAMPLE[dom] * NB / (t_live * 1e-3) / 1e12 if t_live > 0 else None
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": ach / alu_peak, "traffic": traffic, "traffic_source": traffic_src, "timing": timing,
                "pipelined": {"achieved": live, "frac": live / alu_peak if live else None,
                              "ms_per_launch": t_live},
                "peak_source": "FP32: %d SMs (queried) x 128 lanes x 2 flop x %.0f MHz (max SM clock of measured)" % (
                    sms, sm_max)}
        # cross-check of the derived peak: the library's FMA-rate self-test on this GPU now
        try:
            fma = rx.rx_selftest_fma_rate(1 << 16, sid)
            roof["fma_rate_measured"] = {"tflops": fma, "frac": ach / fma if fma > 0 else None,
                                         "kernel": "rx_selftest_fma_rate: 8 independent FMA chains per thread, "
                                                   "every SM filled, CUDA events"}
        except rx.RxError:
            roof["fma_rate_measured"] = None
    else:
        ach = stages[dom]["gbs"]
        live = BYTES_PER_SAMPLE[dom] * NB / (t_live * 1e-3) / 1e9 if t_live > 0 else None
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic, "traffic_source": traffic_src, "timing": timing,
                "pipelined": {"achieved": live, "frac": live / hbm_peak if live else None,
                              "ms_per_launch": t_live},
                "peak_source": "hbm_gbs of measured"}

    # ---- oracle on the host: CPU baseline and BER match on the same buffers
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        nref = 2
        o = oracle.Oracle(**oracle.default_cfg(FMT, NB))
        t = time.perf_counter()
        for b in range(nref):
            o.process(g["packed"][b])
        dt = time.perf_counter() - t
        so = o.stats()
        chk = rx.Receiver(FMT, NB)
        for b in range(nref):
            chk.process(ring[b])
        sg = chk.stats()
        allc = cpu_all_cores(g["packed"])
        cpu = {"value": nref * NB / dt / 1e9, "unit": "GSa/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {nref} buffers (2^22 samples each) of the same stream, single thread",
               "cores_all": allc["cores"], "value_all_cores": allc["value"], "sample_all_cores": allc["sample"],
               "host_cpus": os.cpu_count(), "cpu_model": cpu_model(),
               "ber_oracle": so["ber"], "ber_gpu_same_buffers": sg["ber"],
               "bit_errors_oracle": so["bit_errors"], "bit_errors_gpu": sg["bit_errors"], "bits": so["bits"]}

    cnn_line = None
    if rank == 0 and not args.no_cnn:
        cnn_line = cnn_leg(args, ring)
    prec_line = None
    if rank == 0 and not args.no_precision:
        prec_line = precision_leg(args, g, ring)
    fd_line = None
    if rank == 0 and not args.no_fd:
        fd_line = fd_leg(args, g, ring)
    rs_line = resampler_leg(args, ring) if rank == 0 and not args.no_rs else None
    sweep_line = sweep_leg(args) if rank == 0 and not args.no_sweep else None
    diff_line = diff_leg(args) if rank == 0 and not args.no_sweep else None
    dd_line = dd_leg(args) if rank == 0 and not args.no_dd else None
    stab_line = stability_leg(args) if rank == 0 and args.stability > 0 else None
    batched_line = None
    if rank == 0 and not args.no_batched:
        batched_line = batched_leg(args)

    clk = clocks.summary()
    launches_per_call = 6                 # KK front (three kernels), matched filter, equaliser, demap
    line = {"metric": METRIC, "value": value, "unit": "GSa/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "warmup_run": warm_steps, "ms_per_step": ms / args.steps,
            "host_enqueue_ms_per_step": host_enqueue_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args),
            "e2e": {"value": e2e_value, "unit": "GSa/s", "h2d_bytes_per_step": h2d // e2e_steps,
                    "d2h_bytes_per_step": d2h // e2e_steps, "steps": e2e_steps, "warmup_run": e2e_warm,
                    "h2d_gbs_copies_alone": h2d_gbs},
            "roofline": roof, "stages": stages, "latency": latency, "cpu_baseline": cpu, "cnn": cnn_line, "precision": prec_line,
            "fd_filter": fd_line, "batched": batched_line,
            "resampler": rs_line, "q_sweep": sweep_line, "stability": stab_line, "diff_coding": diff_line, "dd_symbol_equaliser": dd_line,
            "clocks": clk, "gpu_launches": launches_per_call * args.bufs_per_step * args.steps,
            "realtime_x": value / 4.0,
            # the whole chain against the HBM roofline: 1.625 algorithmic bytes per sample
            # (1.5 B of packed input, 0.125 B of bits out) at the measured copy bandwidth
            "chain_hbm": {"gbs": value * 1.625, "peak_gbs": peaks.get("hbm_gbs", 6800.0),
                          "frac": value * 1.625 / peaks.get("hbm_gbs", 6800.0),
                          "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"},
            "ber": cpu["ber_gpu_same_buffers"] if cpu else None,
            "ber_oracle": cpu["ber_oracle"] if cpu else None,
            "ber_note": "BER of the first 2 buffers of the stream, GPU and FP64 oracle on the same input; "
                        "the timed ring repeats its 32 buffers, so the PRBS reference is not aligned "
                        "after a wrap and the timed run's own BER is not meaningful",
            "device_error": stats["device_error"], "gen_s": t_gen}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


VOLT = dict(volterra=(0.05, 0.02), cspr_db=6.0, linewidth=0.0, phase_noise=False)


def cnn_leg(args, ring):
    """Learned equaliser against the adaptive FIR on the Volterra + SSBI channel
    (CSPR 6 dB, SNR 16..22 dB): train on 2^24 counter-based symbols, measure the BER on a
    fresh PRBS stream, and time the CNN receiver on the 2^22-sample buffers."""
    import torch
    import synth
    import paper_2010_14333_gb300 as rx
    from paper_2010_14333_gb300 import cnn
    t0 = time.perf_counter()
    nb, per_snr = NB, 4
    ys, syms, off = [], [], 0
    for i, snr in enumerate((16.0, 18.0, 20.0, 22.0)):
        sym = synth.random_symbols(FMT, per_snr * nb // 4 + 64, seed=1000 + i)
        g = synth.gen_kk_stream(FMT, nb, per_snr, seed=500 + i, symbols=sym, truth=False, snr_db=snr,
                                workers=min(16, os.cpu_count() or 1), **VOLT)
        ys.append(cnn.mf_output(g["packed"], nb))
        syms.append(sym[: len(ys[-1]) // 2])
    # one training set: the streams side by side (segments never cross a seam: a
    # 64-symbol gap of zeros is left between them and excluded)
    gap = 256
    y_all = np.concatenate([np.concatenate([y[: 2 * len(s)], np.zeros(2 * gap, np.complex64)]) for y, s in zip(ys, syms)])
    s_all = np.concatenate([np.concatenate([s, np.zeros(gap, np.complex64)]) for s in syms])
    n_train = sum(len(s) for s in syms)
    tr = cnn.CnnTrainer(batch=64, seed=7)
    tr.set_data(y_all, s_all, k_lo=64)
    steps = int(os.environ.get("RX_CNN_STEPS", "6000"))
    torch.cuda.synchronize()
    t_tr = time.perf_counter()
    tr.train(steps - steps // 4, lr=1e-3)
    tr.train(steps // 4, lr=2e-4)
    torch.cuda.synchronize()
    t_steps = time.perf_counter() - t_tr
    t_train = time.perf_counter() - t0
    # evaluation: fresh PRBS stream at 19 dB through both receivers
    gev = synth.gen_kk_stream(FMT, nb, 4, seed=777, truth=False, snr_db=19.0,
                              workers=min(16, os.cpu_count() or 1), **VOLT)
    lms, net = rx.Receiver(FMT, nb), rx.Receiver(FMT, nb)
    rx.rx_set_cnn(net.h, tr.h)
    for p in gev["packed"]:
        d = torch.from_numpy(p).cuda()
        lms.process(d)
        net.process(d)
    sl, sn = lms.stats(), net.stats()
    # throughput of the CNN receiver on the benchmark buffers
    r = rx.Receiver(FMT, nb)
    rx.rx_set_cnn(r.h, tr.h)
    r.process_batch(ring[:3])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nrun = 2 * len(ring)
    e0.record()
    r.process_batch(ring)
    r.process_batch(ring)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the same network with FP16 operands
    rb = rx.Receiver(FMT, nb, cnn_bf16=0)
    rx.rx_set_cnn(rb.h, tr.h)
    chk = rx.Receiver(FMT, nb, cnn_bf16=0)
    rx.rx_set_cnn(chk.h, tr.h)
    for p in gev["packed"]:
        chk.process(torch.from_numpy(p).cuda())
    rb.process_batch(ring[:3])
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    rb.process_batch(ring)
    rb.process_batch(ring)
    e3.record()
    torch.cuda.synchronize()
    fp16 = {"gsa_s": nrun * nb / (e2.elapsed_time(e3) * 1e-3) / 1e9, "ber": chk.stats()["ber"]}
    return {"gsa_s": nrun * nb / (ms * 1e-3) / 1e9, "ber_cnn": sn["ber"], "ber_lms": sl["ber"],
            "inference_operands": "bf16", "fp16_operands": fp16,
            "bits": sn["bits"], "train_symbols": int(n_train), "train_steps": steps, "batch_symbols": 64 * 64,
            "train_s": t_train, "train_steps_per_s": steps / t_steps,
            "train_symbols_per_s": steps * 64 * 64 / t_steps,
            "channel": "KK-16QAM, Volterra (0.05, 0.02), CSPR 6 dB, no laser phase noise; train SNR 16/18/20/22 dB "
                       "(counter-based symbols), test SNR 19 dB (PRBS-15)"}


def precision_leg(args, g, ring):
    """Precision forms of the equaliser on the KK-16QAM workload (eq_block 1024):
    the adaptive FP32 chain, the frozen-tap form in FP32, and the block-Toeplitz
    FIR on the tensor cores in BF16 / FP16 / FP8-E4M3.  Throughput over the ring;
    BER on the first two buffers of the stream (their soft-symbol error and BER
    against the FP64 oracle are asserted by the parity tests); the tensor-core FIR
    kernel timed alone."""
    import torch
    import paper_2010_14333_gb300 as rx
    nref = 2
    forms = [("adaptive_f32", rx.RX_FIR_ADAPTIVE), ("frozen_f32", rx.RX_FIR_FROZEN_F32),
             ("bf16", rx.RX_FIR_BF16), ("fp16", rx.RX_FIR_FP16), ("fp8_e4m3", rx.RX_FIR_FP8)]
    res = {}
    for name, prec in forms:
        d = rx.Receiver(FMT, NB, fir_prec=prec, eq_block=1024)
        for b in range(nref):
            d.process(ring[b])
        sd = d.stats()
        del d
        r = rx.Receiver(FMT, NB, fir_prec=prec, eq_block=1024)
        r.process_batch(ring[:3])
        torch.cuda.synchronize()
        rx.rx_profile(r.h, 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            r.process_batch(ring)
        e1.record()
        torch.cuda.synchronize()
        ms, calls = rx.rx_profile_read(r.h)
        rx.rx_profile(r.h, 0)
        # the equaliser stage alone: one buffer in flight, a synchronize after each
        sid = torch.cuda.current_stream().cuda_stream
        obuf = torch.empty(NB, dtype=torch.uint8, device="cuda")
        rx.rx_profile(r.h, 1)
        for i in range(10):
            rx.rx_process(r.h, ring[i % len(ring)].data_ptr(), obuf.data_ptr(), sid)
            torch.cuda.synchronize()
        ams, acalls = rx.rx_profile_read(r.h)
        rx.rx_profile(r.h, 0)
        res[name] = {"gsa_s": 2 * len(ring) * NB / (e0.elapsed_time(e1) * 1e-3) / 1e9,
                     "eq_us_per_buffer": ms["eq"] / max(calls, 1) * 1e3,
                     "eq_alone_us_per_buffer": ams["eq"] / max(acalls, 1) * 1e3,
                     "ber": sd["ber"], "bits": sd["bits"]}
        del r
    # the tensor-core FIR alone: 2^20 symbols (one buffer's payload), 31 taps
    nsym, nt = 1 << 20, 31
    rng = np.random.default_rng(3)
    ny = 2 * nsym + nt + 1
    yv = torch.from_numpy(rng.standard_normal(2 * ny).astype(np.float32)).cuda()
    wv = torch.zeros(2 * nt, dtype=torch.float32, device="cuda")
    wv[2 * (nt // 2)] = 1.0
    zv = torch.zeros(2 * nsym, dtype=torch.float32, device="cuda")
    stv = torch.zeros(1, dtype=torch.int32, device="cuda")
    sid = torch.cuda.current_stream().cuda_stream
    kern = {}
    for name, prec in forms[2:]:
        for _ in range(3):
            rx.rx_fir_block(yv.data_ptr(), ny, wv.data_ptr(), nt, prec, nsym, 1024, zv.data_ptr(), stv.data_ptr(), sid)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 50
        e0.record()
        for _ in range(reps):
            rx.rx_fir_block(yv.data_ptr(), ny, wv.data_ptr(), nt, prec, nsym, 1024, zv.data_ptr(), stv.data_ptr(), sid)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / reps * 1e3
        byt = nsym * (16 + 8)                    # 2 complex FP32 inputs + 1 complex output per symbol
        kern[name] = {"us_per_2e20_symbols": us, "gbs": byt / (us * 1e-6) / 1e9,
                      "algorithmic_tflops": 8 * nt * nsym / (us * 1e-6) / 1e12,
                      "tensor_tflops_issued": 2 * 128 * 32 * 128 * (nsym // 2048) / (us * 1e-6) / 1e12}
    return {"eq_block": 1024, "forms": res, "fir_kernel": kern,
            "sample": f"BER on the first {nref} buffers; throughput over the {len(ring)}-buffer ring x 2"}


def fd_leg(args, g, ring):
    """The paper's form of the reduction to 2 samples/symbol (Sec. 2): a static
    203-tap filter in the frequency domain on 1024-point overlap-save blocks (hop
    512, 8192 blocks per buffer) with a 512-point bin-truncation inverse, in place
    of the 65-tap time-domain matched filter.  Receiver throughput over the ring,
    the filter stage time, and the BER in that form on the first two buffers (its
    2-sps samples and BER against the FP64 oracle are asserted by the parity
    tests)."""
    import torch
    import paper_2010_14333_gb300 as rx
    nref = 2
    d = rx.Receiver(FMT, NB, mf_mode=1)
    for b in range(nref):
        d.process(ring[b])
    sd = d.stats()
    del d
    out = {"fd_n": 1024, "fd_taps": 203, "ber": sd["ber"], "bits": sd["bits"]}
    for mode in (1, 0):
        r = rx.Receiver(FMT, NB, mf_mode=mode)
        for _ in range(2):
            r.process_batch(ring)
        torch.cuda.synchronize()
        rx.rx_profile(r.h, 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            r.process_batch(ring)
        e1.record()
        torch.cuda.synchronize()
        ms, calls = rx.rx_profile_read(r.h)
        rx.rx_profile(r.h, 0)
        key = "frequency_domain" if mode else "time_domain_65_taps"
        out[key] = {"gsa_s": 2 * len(ring) * NB / (e0.elapsed_time(e1) * 1e-3) / 1e9,
                    "filter_us_per_buffer": ms["mf"] / max(calls, 1) * 1e3}
        del r
    out["pam4"] = pam_fd(args)
    return out


def resampler_leg(args, ring):
    """The receiver with the resampler to the transmitter's grid (ADC clock off the
    transmitter's): on two buffers of a stream generated through a -35 ppm ADC clock
    with a 0.4-sample delay, the clock estimated from the first buffer in the
    frequency-domain form, then the BER with the resampler set from the estimate
    (against the FP64 oracle set the same way in the parity tests) and without it;
    throughput over the benchmark ring (the resampler's work does not depend on the
    data)."""
    import torch
    import synth
    import paper_2010_14333_gb300 as rx
    st, ph = synth.clock_step(-35.0), int(0.4 * (1 << 32))
    t0 = time.perf_counter()
    g = synth.gen_kk_stream(FMT, NB, 2, seed=11, truth=False, clock_step=st, clock_phase0=ph, workers=2, **GEN)
    t_gen = time.perf_counter() - t0
    # the clock estimated from the first buffer in the frequency-domain form, then the
    # resampler configured with the estimate
    est = rx.Receiver(FMT, NB, mf_mode=1)
    est.process(torch.from_numpy(g["packed"][0]).cuda())
    e_ppm, e_delay = rx.rx_clock_estimate(est.h, torch.cuda.current_stream().cuda_stream)
    del est
    rs_step, rs_phase0 = rx.rx_resampler_from_clock(e_ppm, e_delay)
    d = rx.Receiver(FMT, NB, rs_step=rs_step, rs_phase0=rs_phase0)
    plain = rx.Receiver(FMT, NB)
    for p in g["packed"]:
        dv = torch.from_numpy(p).cuda()
        d.process(dv)
        plain.process(dv)
    out = {"ppm": -35.0, "delay_samples": 0.4, "estimated_ppm": e_ppm, "estimated_delay_samples": e_delay,
           "ber": d.stats()["ber"], "ber_without_resampler": plain.stats()["ber"], "gen_s": t_gen}
    del d, plain
    r = rx.Receiver(FMT, NB, rs_step=rs_step, rs_phase0=rs_phase0)
    for _ in range(2):
        r.process_batch(ring)
    torch.cuda.synchronize()
    rx.rx_profile(r.h, 4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(2):
        r.process_batch(ring)
    e1.record()
    torch.cuda.synchronize()
    ms, calls = rx.rx_profile_read(r.h)
    rx.rx_profile(r.h, 0)
    out["gsa_s"] = 2 * len(ring) * NB / (e0.elapsed_time(e1) * 1e-3) / 1e9
    out["resampler_and_filter_us_per_buffer"] = ms["mf"] / max(calls, 1) * 1e3
    return out


def pam_fd(args):
    """PAM-4 at 2 GBaud on 2^20-sample buffers: the 503-tap frequency-domain form
    against the 33-tap time-domain matched filter, with the BER of the
    frequency-domain form on the first two buffers, and the form's static taps
    fitted by least squares against its RRC taps."""
    import torch
    import synth
    import paper_2010_14333_gb300 as rx
    nb, nbufs, fmt = 1 << 20, 32, 1
    g = synth.gen_pam_stream(fmt, nb, nbufs, seed=5)
    ring = [torch.from_numpy(p).cuda() for p in g["packed"]]
    d = rx.Receiver(fmt, nb, mf_mode=1)
    for b in range(2):
        d.process(ring[b])
    res = {"buf_len": nb, "fd_taps": 503, "ber": d.stats()["ber"]}
    del d
    # static taps from a least-squares fit on the first buffer (the calibration the
    # paper's lab taps came from): normalised codes against the transmitted levels at
    # the symbol centres; then the filter output's error at the symbol centres of the
    # held-out third buffer (best gain for the RRC taps, none for the fitted ones) and
    # the BER of the three buffers, against the RRC taps
    codes = g["codes"][:nb].astype(np.float64)
    x = (codes - codes.mean()) / codes.std()
    k0, na = 126, 100000
    t0 = time.perf_counter()
    h = rx.rx_fd_ls_taps(x, 2 * k0, 2, g["symbols"][k0:k0 + na], 503)
    res["ls_fit_s"] = time.perf_counter() - t0
    for name, taps in (("rrc_taps", None), ("least_squares_taps", h)):
        d = rx.Receiver(fmt, nb, mf_mode=1, debug=1)
        if taps is not None:
            d.set_fd_taps(taps)
        for b in range(3):
            d.process(ring[b])
        y, y0 = d.debug(rx.RX_DBG_MF)
        y = np.asarray(y, np.float64)
        m = np.arange(y0 + (y0 & 1), y0 + len(y), 2)
        m = m[(m >= 2 * nb) & (m < 3 * nb - 600)]
        ys, a = y[m - y0], g["symbols"][m // 2]
        gain = float(ys @ a / (ys @ ys)) if taps is None else 1.0
        st = d.stats()
        res[name] = {"filter_rel_mse": float(np.mean((a - gain * ys) ** 2) / np.mean(a ** 2)),
                     "ber": st["ber"], "bit_errors": st["bit_errors"], "bits": st["bits"]}
        del d
    for mode in (1, 0):
        r = rx.Receiver(fmt, nb, mf_mode=mode)
        for _ in range(2):
            r.process_batch(ring)
        torch.cuda.synchronize()
        rx.rx_profile(r.h, 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(4):
            r.process_batch(ring)
        e1.record()
        torch.cuda.synchronize()
        ms, calls = rx.rx_profile_read(r.h)
        rx.rx_profile(r.h, 0)
        res["frequency_domain" if mode else "time_domain_33_taps"] = {
            "gsa_s": 4 * nbufs * nb / (e0.elapsed_time(e1) * 1e-3) / 1e9,
            "filter_us_per_buffer": ms["mf"] / max(calls, 1) * 1e3}
        del r
    return res


SWEEP = {0: (1 << 20, (6.0, 8.0, 10.0, 12.0, 14.0)),      # PAM-2
         1: (1 << 20, (12.0, 14.0, 16.0, 18.0, 20.0)),    # PAM-4
         2: (1 << 20, (18.0, 20.0, 22.0, 24.0, 26.0)),    # PAM-8
         3: (1 << 22, (6.0, 8.0, 10.0, 12.0, 14.0)),      # KK-QPSK
         4: (1 << 22, (14.0, 16.0, 18.0, 20.0, 22.0))}    # KK-16QAM
FMT_NAMES = ["PAM-2", "PAM-4", "PAM-8", "KK-QPSK", "KK-16QAM"]


def sweep_leg(args):
    """Synthetic analogue of the paper's Q-factor versus OSNR curves (Fig. 2a, b):
    every format over five SNR points (in-band Es/N0 of the generator), BER and
    Q = 20 log10(sqrt(2) erfcinv(2 BER)) of the GPU receiver over a few buffers
    per point."""
    import torch
    import synth
    import paper_2010_14333_gb300 as rx
    nb_per = 4
    res = {}
    for fmt, (nb, snrs) in SWEEP.items():
        pts = []
        for i, snr in enumerate(snrs):
            if fmt >= 3:
                g = synth.gen_kk_stream(fmt, nb, nb_per, seed=40 + i, snr_db=snr, truth=False,
                                        workers=min(nb_per, os.cpu_count() or 1))
            else:
                g = synth.gen_pam_stream(fmt, nb, nb_per, seed=40 + i, snr_db=snr)
            r = rx.Receiver(fmt, nb)
            for p in g["packed"]:
                r.process(torch.from_numpy(p).cuda())
            st = r.stats()
            pt = {"snr_db": snr, "bits": st["bits"], "ber": st["ber"],
                  "q_db": st["q_db"] if np.isfinite(st["q_db"]) else None,
                  "slip_windows": st["slip_windows"]}
            pts.append(pt)
            del r
        res[FMT_NAMES[fmt]] = {"buf_len": nb, "buffers_per_point": nb_per, "points": pts}
    return res


def stability_leg(args):
    """Synthetic analogue of the paper's 6-second Q time series (Fig. 2c): one
    continuous KK-16QAM stream of --stability buffers of 2^22 samples (5720 = 6 s of
    signal at 4 GS/s), generated on the GPU (synth.gpu, the KK recipe of the
    workload), each window of 20 buffers (20.97 ms of signal) copied to pinned host
    memory as the ADC's DMA would leave it, then run through the end-to-end host
    path (copies in and out).  Per window: Q-factor and the device time of the
    window against its real-time budget; per buffer: the receiver's own latency
    record (rx_stats) against the paper's 5.243 ms."""
    import torch
    import paper_2010_14333_gb300 as rx
    from synth.gpu import KKStreamGPU
    nbufs, win = args.stability, 20
    gen = KKStreamGPU(FMT, NB, seed=77, snr_db=GEN["snr_db"], cspr_db=GEN["cspr_db"], linewidth=GEN["linewidth"])
    ring = [torch.zeros(NB * 3 // 2, dtype=torch.uint8).pin_memory() for _ in range(win)]
    c = rx.rx_default_config(FMT)
    h = rx.rx_create(FMT, BAUD, FS, NB, c)
    outs = [torch.zeros(rx.rx_max_bits(h) // 8 + 16, dtype=torch.uint8).pin_memory() for _ in range(win)]
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    series, prev = [], None
    budget_ms = win * NB / FS * 1e3
    t_gen = 0.0
    t0 = time.perf_counter()
    try:
        for w0 in range(0, nbufs - win + 1, win):
            tg = time.perf_counter()
            for j in range(win):   # the window's ADC buffers land in pinned host memory
                ring[j].copy_(gen.next(), non_blocking=True)
            torch.cuda.synchronize()
            t_gen += time.perf_counter() - tg
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rx.rx_process_host_batch(h, [t.data_ptr() for t in ring], [o.data_ptr() for o in outs], sid)
            e1.record(stream)
            torch.cuda.synchronize()
            st = rx.rx_stats(h, sid)
            bits = st["bits"] - (prev["bits"] if prev else 0)
            errs = st["bit_errors"] - (prev["bit_errors"] if prev else 0)
            ber = errs / bits if bits else None
            series.append({"window": w0 // win, "bits": bits, "ber": ber,
                           "q_db": (None if not ber else float(oracle_free_q_db(ber))),
                           "device_ms": e0.elapsed_time(e1)})
            prev = st
        fb = torch.zeros(rx.rx_max_bits(h) // 8 + 16, dtype=torch.uint8, device="cuda")
        nflush = rx.rx_flush(h, fb.data_ptr(), sid)
        st = rx.rx_stats(h, sid)
    finally:
        rx.rx_destroy(h)
    qs = [x["q_db"] for x in series[1:] if x["q_db"] is not None]
    ms = [x["device_ms"] for x in series[1:]]
    return {"buffers": nbufs, "seconds_of_signal": nbufs * NB / FS, "window_buffers": win,
            "window_ms_of_signal": budget_ms, "gen": "synth.gpu (torch on the GPU), seed 77", "gen_s": t_gen,
            "wall_s": time.perf_counter() - t0,
            "q_db_mean": float(np.mean(qs)) if qs else None, "q_db_min": float(np.min(qs)) if qs else None,
            "q_db_max": float(np.max(qs)) if qs else None, "device_ms_max": float(np.max(ms)) if ms else None,
            "window_deadline_misses": int(sum(m > budget_ms for m in ms)),
            "ber_total": st["ber"], "bits_total": st["bits"], "flushed_bits": nflush,
            "per_buffer_latency": {"calls": st["lat_calls"], "budget_ms": st["deadline_ms"],
                                   "deadline_misses": st["deadline_misses"], "p50_ms": st["lat_p50_ms"],
                                   "p99_ms": st["lat_p99_ms"], "max_ms": st["lat_max_ms"],
                                   "note": "the receiver's own record: device time from the start of a buffer's "
                                           "first kernel to the end of its demap (GPU global timer), 20 buffers "
                                           "enqueued at a time"},
            "note": "the first window holds the training symbols and is excluded from the summary",
            "series": [{"w": x["window"], "q": None if x["q_db"] is None else round(x["q_db"], 3),
                        "ms": round(x["device_ms"], 3)} for x in series]}


def diff_leg(args):
    """Plain Gray mapping against differential quadrant coding on the workload's
    KK-16QAM stream (20 dB, 100 kHz laser phase noise: the blind phase search slips
    by pi/2 now and then): the BER-tester view (each window scored under its best
    rotation) and the raw BER of the delivered bits, for 8 buffers of 2^22 samples."""
    import torch
    import synth
    import paper_2010_14333_gb300 as rx
    nb, nbufs, out = NB, 8, {}
    for diff in (0, 1):
        g = synth.gen_kk_stream(FMT, nb, nbufs, seed=31, truth=False, diff=bool(diff),
                                workers=min(8, os.cpu_count() or 1), **GEN)
        r = rx.Receiver(FMT, nb, diff_code=diff)
        for p in g["packed"]:
            r.process(torch.from_numpy(p).cuda())
        st = r.stats()
        out["differential" if diff else "gray"] = {
            "bits": st["bits"], "ber_tester_view": st["ber"],
            "raw_ber_delivered": st["raw_bit_errors"] / st["bits"] if st["bits"] else None,
            "slip_windows": st["slip_windows"]}
        del r
    return out


def dd_leg(args):
    """The paper's short KK equaliser (4-tap decision-directed LMS updated after every
    symbol, no phase search; eq_mode = RX_EQ_DD_SYMBOL) against the workload's 31-tap
    window equaliser with the 32-phase search, on a KK-16QAM stream at 20 dB without
    relative laser phase noise (the paper's self-coherent link; with 100 kHz of it the
    short form loses the phase between blocks): BER over 16 consecutive 2^22-sample
    buffers generated on the GPU, receiver throughput over them, and the equaliser
    stage timed alone."""
    import torch
    import paper_2010_14333_gb300 as rx
    from synth.gpu import KKStreamGPU
    t0 = time.perf_counter()
    gen = KKStreamGPU(FMT, NB, seed=41, snr_db=20.0, linewidth=0.0)
    ring = [gen.next().clone() for _ in range(16)]
    torch.cuda.synchronize()
    out = {"buffers": len(ring), "gen_s": time.perf_counter() - t0,
           "stream": "KK-16QAM 20 dB, CSPR 10 dB, no relative laser phase noise (synth.gpu, seed 41)"}
    sid = torch.cuda.current_stream().cuda_stream
    for name, cfg in (("window_31_taps_phase_search", {}),
                      ("dd_symbol_4_taps", dict(eq_mode=rx.RX_EQ_DD_SYMBOL, ntaps=4))):
        r = rx.Receiver(FMT, NB, **cfg)
        r.process_batch(ring)
        st = r.stats()
        del r
        r = rx.Receiver(FMT, NB, **cfg)
        r.process_batch(ring)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            r.process_batch(ring)
        e1.record()
        torch.cuda.synchronize()
        gsa = 2 * len(ring) * NB / (e0.elapsed_time(e1) * 1e-3) / 1e9
        obuf = torch.empty(NB, dtype=torch.uint8, device="cuda")
        rx.rx_profile(r.h, 1)
        for i in range(8):
            rx.rx_process(r.h, ring[i].data_ptr(), obuf.data_ptr(), sid)
            torch.cuda.synchronize()
        ms, calls = rx.rx_profile_read(r.h)
        rx.rx_profile(r.h, 0)
        out[name] = {"ber": st["ber"], "bits": st["bits"], "bit_errors": st["bit_errors"],
                     "slip_windows": st["slip_windows"], "gsa_s": gsa,
                     "eq_alone_us_per_buffer": ms["eq"] / max(calls, 1) * 1e3}
        del r
    return out


def oracle_free_q_db(ber: float) -> float:
    """Q = 20 log10(sqrt(2) erfcinv(2 BER)) by bisection on math.erfc."""
    import math
    lo, hi = 0.0, 30.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.erfc(mid) > 2.0 * ber:
            lo = mid
        else:
            hi = mid
    return 20.0 * math.log10(math.sqrt(2.0) * 0.5 * (lo + hi))


def _gen_member(job):
    """One member stream of the batched workload (runs in a spawned worker)."""
    import synth
    fmt, nb, nbufs, seed, snr = job
    if fmt >= 3:
        g = synth.gen_kk_stream(fmt, nb, nbufs, seed=seed, snr_db=snr, truth=False)
    else:
        g = synth.gen_pam_stream(fmt, nb, nbufs, seed=seed, snr_db=snr)
    return g["packed"]


def batched_leg(args):
    """Many streams at once: 64 receivers with buffer lengths drawn from
    {2^18 .. 2^22}, formats mixed (PAM-2/4/8 at 2 GBaud, KK-QPSK/16QAM at
    1 GBaud), SNR 14..22 dB.  Aggregate GSa/s over rounds of one buffer per
    stream: one stream after another on one CUDA stream, then as a group (worker
    streams), as a group captured into an updated CUDA graph, and with the
    autotuned implementation choices; per-round latency percentiles."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import torch
    import paper_2010_14333_gb300 as rx
    rng = np.random.default_rng(2022)
    nmem = args.batched_streams
    fmts = rng.integers(0, 5, nmem)
    lens = 1 << (18 + rng.integers(0, 5, nmem))
    snrs = rng.uniform(14.0, 22.0, nmem)
    nbufs = 2
    t0 = time.perf_counter()
    jobs = [(int(f), int(n), nbufs, 5000 + m, float(sn)) for m, (f, n, sn) in enumerate(zip(fmts, lens, snrs))]
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        packed = list(ex.map(_gen_member, jobs))
    t_gen = time.perf_counter() - t0
    dev = [[torch.from_numpy(p).cuda() for p in pk] for pk in packed]
    samples_round = int(np.sum(lens))
    st = torch.cuda.Stream()
    sid = st.cuda_stream

    def make():
        rs = [rx.Receiver(int(f), int(n)) for f, n in zip(fmts, lens)]
        outs = [torch.zeros(r.max_bits // 8 + 16, dtype=torch.uint8, device="cuda") for r in rs]
        return rs, outs

    def ev():
        return torch.cuda.Event(enable_timing=True)

    res = {}
    for mode in ("serial", "group", "group_graph", "group_graph_tuned"):
        rs, outs = make()
        g = None
        if mode != "serial":
            flags = {"group": 0, "group_graph": rx.RX_GROUP_GRAPH,
                     "group_graph_tuned": rx.RX_GROUP_GRAPH | rx.RX_GROUP_TUNE}[mode]
            tt = time.perf_counter()
            g = rx.rx_group_create([r.h for r in rs], flags)
            t_create = time.perf_counter() - tt
        optr = [o.data_ptr() for o in outs]

        def round_(k):
            ins = [dev[m][k % nbufs].data_ptr() for m in range(nmem)]
            if g is None:
                for m in range(nmem):
                    rx.rx_process(rs[m].h, ins[m], optr[m], sid)
            else:
                rx.rx_group_process(g, ins, optr, sid)

        with torch.cuda.stream(st):
            for k in range(3):
                round_(k)
            st.synchronize()
            e0, e1 = ev(), ev()
            e0.record(st)
            for k in range(args.batched_rounds):
                round_(k)
            e1.record(st)
            st.synchronize()
            ms = e0.elapsed_time(e1)
            lat = []
            for k in range(args.batched_rounds):
                a, b = ev(), ev()
                a.record(st)
                round_(k)
                b.record(st)
                st.synchronize()
                lat.append(a.elapsed_time(b))
        errs = sum(r.stats()["device_error"] != 0 for r in rs)
        d = {"gsa_s": samples_round * args.batched_rounds / (ms * 1e-3) / 1e9,
             "ms_per_round": ms / args.batched_rounds,
             "round_latency_p50_ms": float(np.percentile(lat, 50)),
             "round_latency_p99_ms": float(np.percentile(lat, 99)),
             "members_with_device_error": int(errs)}
        if g is not None:
            d["create_s"] = t_create
            if mode == "group_graph_tuned":
                tun = [rx.rx_group_tuning(g, m) for m in range(nmem)]
                d["tuned_kk_front_1"] = int(sum(1 for f, t in zip(fmts, tun) if f >= 3 and t[0] == 1))
                d["tuned_eq_warps"] = {str(w): int(sum(1 for t in tun if t[1] == w)) for w in (2, 4, 8)}
            rx.rx_group_destroy(g)
        res[mode] = d
        del rs, outs
    names = ["PAM-2", "PAM-4", "PAM-8", "KK-QPSK", "KK-16QAM"]
    return {"streams": nmem, "samples_per_round": samples_round, "rounds": args.batched_rounds,
            "formats": {n: int(np.sum(fmts == i)) for i, n in enumerate(names)},
            "lengths": {str(int(l)): int(np.sum(lens == l)) for l in sorted(set(lens.tolist()))},
            "budget_ms": 5.243, "gen_s": t_gen, "modes": res,
            "note": "each stream cycles 2 buffers of its own synthetic stream; latency = one round "
                    "(one buffer of every stream) from an idle GPU"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--bufs-per-step", type=int, default=64)
    ap.add_argument("--ring", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cnn", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-fd", action="store_true")
    ap.add_argument("--no-rs", action="store_true")
    ap.add_argument("--smi-ms", type=int, default=10, help="clock sampling period (ms) during the timed steps")
    ap.add_argument("--no-sweep", action="store_true", help="skip the Q-factor versus SNR sweep of every format")
    ap.add_argument("--no-dd", action="store_true", help="skip the leg of the paper's short symbol-by-symbol equaliser")
    ap.add_argument("--stability", type=int, default=5720,
                    help="buffers of the Q time series (5720 = the paper's 6 s at 4 GS/s; 0: off)")
    ap.add_argument("--batched-streams", type=int, default=64)
    ap.add_argument("--batched-rounds", type=int, default=10)
    ap.add_argument("--latency-reps", type=int, default=1000)
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop, for a range profile of the "
                         "pipelined chain (DRAM bytes of all its kernels as they overlap)")
    ap.add_argument("--eq-warps", type=int, default=0, help="equaliser blocks per CTA (0: library default)")
    ap.add_argument("--deadline-ms", type=float, default=0.0,
                    help="per-buffer latency budget of the timed receivers (0: the library default, five buffer "
                         "durations; < 0: no latency record)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args, rank)
        return
    gpu_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
