"""Throughput benchmark of the fused LS/MRC receiver on GB300.

One step = one ``lsas_run_frame`` over a batch of 1000 frames of the "scale"
workload (64 antennas, N = 1024, CP 128, 1 pilot + 13 16-QAM data symbols,
sc16 input; 4.13 GB of samples, larger than L2), i.e. the whole hot path:
CP removal, FFT, LS estimate, MRC combine, demap and bit packing.

Prints one JSON line (rank 0):
  value      antenna*subcarrier samples/s  (F * M * S * N per step / time),
             whole job over all ranks (each rank processes its own frames)
  roofline   the fused kernel's algorithmic bytes (input + H + packed bits)
             per launch / its CUDA-event time, against the measured HBM peak
  e2e        the same metric through lsas_run_frame_host with pinned host
             buffers, host<->device copies inside the timed region
  cpu_baseline  the FP64 oracle timed on the host cores on a bounded sample
  latency_ms p50/p99 of single-frame calls
``--impl reference`` times the oracle instead (the CPU reference arm).
"""

from __future__ import annotations

import argparse
import gc
import hashlib
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

import synth  # noqa: E402

FALLBACK_HBM_GBS = 6800.0
CSRC = os.path.join(ROOT, "paper_1901_07499_gb300", "csrc")
# the sources of each fused kernel (its own file, the shared helpers and the
# per-warp kernel's item walk), whose hash keys a committed traffic capture
KERNEL_SRC = {
    "twin_kernel": ("lsas_kernels.cuh", "lsas_warp.cuh", "lsas_twin.cuh"),
    "warp_kernel": ("lsas_kernels.cuh", "lsas_warp.cuh"),
    "hyb_kernel": ("lsas_kernels.cuh", "lsas_warp.cuh", "lsas_hyb.cuh"),
    "pair_kernel": ("lsas_kernels.cuh", "lsas_warp.cuh", "lsas_pair.cuh"),
    "twinpair_kernel": ("lsas_kernels.cuh", "lsas_warp.cuh", "lsas_twin.cuh", "lsas_twinpair.cuh"),
    "frame_kernel": ("lsas_kernels.cuh",),
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fused_kernel_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lsas", choices=["lsas", "reference"])
    ap.add_argument("--config", default="scale")
    ap.add_argument("--frames", type=int, default=0, help="frames per step (default: config)")
    ap.add_argument("--pool", type=int, default=32, help="distinct seeded frames tiled")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--latency-calls", type=int, default=1000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fma-peak", action="store_true",
                    help="skip the FP32 FMA peak measurement (roofline_fp32 then nominal)")
    ap.add_argument("--sweep", action="store_true",
                    help="throughput over the antenna x FFT-length grid (one JSON line per shape)")
    ap.add_argument("--sweep-steps", type=int, default=10, help="timed steps per sweep shape")
    ap.add_argument("--host-link", action="store_true",
                    help="host<->device copy bandwidth report (one JSON line per path)")
    ap.add_argument("--serving", action="store_true",
                    help="serving-loop report: latency vs offered load (one JSON line per load)")
    ap.add_argument("--serving-loads", default="1,5,10,20,40", help="offered loads, G samples/s")
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--serving-forms", default="plain,learned",
                    help="receiver forms to serve: plain (FP32 LS), learned (LS + refinement)")
    ap.add_argument("--denoiser", action="store_true",
                    help="learned LS refinement: train, then MSE/BER against plain LS per SNR")
    ap.add_argument("--denoiser-rows", type=int, default=200_000)
    ap.add_argument("--denoiser-ckpt", default="")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_frame_ids(rank, pool):
    """Seeded frame indices owned by a rank: independent units, no exchange."""
    return range(rank * pool, (rank + 1) * pool)


def max_over_ranks(value, world, device):
    """Largest value over all ranks (the slowest rank's time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_samples(world, frames, cfg):
    """Antenna*subcarrier samples processed by the whole job in one step."""
    return world * frames * cfg.M * cfg.S * cfg.N


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash(kernel):
    """Hash of the sources of one fused kernel (a name of KERNEL_SRC)."""
    h = hashlib.sha256()
    for name in KERNEL_SRC[kernel]:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(cfg, frames):
    """DRAM bytes per launch from a committed ncu capture of this kernel
    source on this workload (the file holds one entry per workload), scaled
    by frames; None when absent or the kernel changed."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
        for e in (d if isinstance(d, list) else [d]):
            if (e.get("workload") == cfg.name and
                    e.get("kernel_sha") == kernel_hash(fused_kernel_name(cfg).split(" ")[0])):
                return float(e["dram_bytes_per_frame"]) * frames
        return None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons sampled during a window."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t0 = time.time()
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [c.strip() for c in line.split(",")]))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle

def time_oracle(cfg, seconds, min_frames=1):
    """Run the FP64 oracle on seeded frames until ``seconds`` have elapsed;
    returns (samples/s, frames, threads)."""
    import oracle
    frames = 0
    t_used = 0.0
    fid = 0
    while t_used < seconds or frames < min_frames:
        b = synth.generate(cfg, frame_ids=[fid])
        t0 = time.perf_counter()
        oracle.receive(b.frames, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, b.pilot,
                       keep_Y=False)
        t_used += time.perf_counter() - t0
        frames += 1
        fid += 1
    rate = frames * cfg.M * cfg.S * cfg.N / t_used
    return rate, frames, blas_threads(), t_used


ORACLE_ONE_CORE = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import oracle, synth
cfg = synth.config_by_name(sys.argv[2])
seconds = float(sys.argv[3])
frames, used, fid = 0, 0.0, 0
while used < seconds or frames < 1:
    b = synth.generate(cfg, frame_ids=[fid])
    t0 = time.perf_counter()
    oracle.receive(b.frames, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, b.pilot, keep_Y=False)
    used += time.perf_counter() - t0
    frames += 1
    fid += 1
print(json.dumps({"rate": frames * cfg.M * cfg.S * cfg.N / used, "frames": frames, "seconds": used}))
"""


def time_oracle_one_core(cfg, seconds):
    """The oracle on one core: a fresh interpreter with its BLAS held to one
    thread (set before numpy loads).  Returns the parsed JSON or None."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", ORACLE_ONE_CORE, ROOT, cfg.name, str(seconds)],
                             env=env, capture_output=True, text=True, timeout=120 + 4 * seconds)
        return json.loads(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    except Exception:
        return None


def cpu_model():
    """CPU model name from lscpu (or /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return os.uname().machine


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads", 1) for d in threadpool_info() if d.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


def measure_fma_peak(lsas, torch, index, reps=5):
    """The CUDA cores' FP32 FMA throughput measured on this GPU
    (lsas_fma_peak_run: independent packed-FMA chains on every SM), best of
    ``reps`` launches timed with CUDA events, with the SM clock sampled
    during the launches."""
    import ctypes
    sms = torch.cuda.get_device_properties(index).multi_processor_count
    blocks, threads, iters = 4 * sms, 512, 1 << 15
    out = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    flops = ctypes.c_double(0.0)

    def run():
        lsas.check(lsas.lsas_fma_peak_run(blocks, threads, iters, out.data_ptr(),
                                          ctypes.byref(flops), stream.cuda_stream),
                   "lsas_fma_peak_run")
    run()
    torch.cuda.synchronize()
    clk = ClockSampler(index)
    clk.start()
    time.sleep(0.3)
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(20):
            run()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) / 20)
    clocks = clk.stop()
    tflops = flops.value / (best * 1e-3) / 1e12
    return {"tflops": tflops, "ms_per_launch": best, "clocks": clocks,
            "launch": f"{blocks} blocks x {threads} threads x {iters} iterations x 8 chains "
                      "of packed FMAs (lsas_fma_peak_run)"}


def fp32_roofline(cfg, F, ms_step, clocks, fma=None, sms=None):
    """The FFT's FP32 rate against the CUDA cores' FP32 peak: nominal
    5 N log2 N flop per FFT (every symbol of every antenna).  The peak is the
    FMA throughput measured in the same run (``fma``, from
    measure_fma_peak); without it, SMs x 128 FP32 lanes x 2 flop x the
    maximum SM clock, marked nominal."""
    import math
    flops = F * cfg.M * cfg.S * 5.0 * cfg.N * math.log2(cfg.N)
    achieved = flops / (ms_step * 1e-3) / 1e12
    if fma is not None:
        peak = fma["tflops"]
        src = "measured"
        how = fma["launch"] + f", SM clock median {fma['clocks'].get('sm_mhz')} MHz"
    else:
        if sms is None:
            import torch
            sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        src = "nominal"
        how = f"{sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "flop_per_frame": flops / F,
            "peak_source": src, "peak_how": how}


def fused_kernel_name(cfg):
    """The fused kernel lsas_run_frame launches for this workload (aligned
    rows, as the benchmark's input is)."""
    choice = os.environ.get("LSAS_FUSED_KERNEL")
    if cfg.N == 1024 and cfg.fmt == "sc16" and choice == "tensor":
        return ("hyb_kernel (fused CP strip + FFT + LS + MRC + demap; first FFT pass on the "
                "CUDA cores, second on tcgen05)")
    twin_n = cfg.N == 1024 or (cfg.N == 512 and cfg.M >= 32) or (cfg.N == 256 and cfg.M >= 128)
    if twin_n and cfg.fmt == "sc16" and choice not in ("warp", "tensor"):
        return ("twin_kernel (fused CP strip+FFT+LS+MRC+demap, per-warp pipelines, two "
                "symbols per step in split real/imaginary form)")
    if cfg.N <= 1024:
        return "warp_kernel (fused CP strip+FFT+LS+MRC+demap, per-warp pipelines)"
    if cfg.fmt == "sc16" and choice not in ("warp", "tensor"):
        return ("twinpair_kernel (fused CP strip+FFT+LS+MRC+demap, pipelines of warp pairs, two "
                "symbols per step in split real/imaginary form)")
    if cfg.fmt == "sc16":
        return "pair_kernel (fused CP strip+FFT+LS+MRC+demap, pipelines of warp pairs)"
    return "frame_kernel (fused CP strip+FFT+LS+MRC+demap)"


def workload_config(cfg, F, pool):
    return {"workload": f"{cfg.name}: {F} frames x {cfg.M} antennas x N={cfg.N} "
                        f"(CP {cfg.cp}, {cfg.S} symbols, {cfg.Q}-QAM, {cfg.fmt})",
            "frames": F, "M": cfg.M, "N": cfg.N, "cp": cfg.cp, "n_sym": cfg.S,
            "qam": cfg.Q, "input": cfg.fmt, "distinct_frames": pool,
            "l2": "inputs larger than L2 (no flush needed)"}


def reference_arm(args, cfg):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    per_step = 2
    F = args.frames or cfg.F
    times = []
    for i in range(args.warmup + args.steps):
        import oracle
        b = synth.generate(cfg, frame_ids=range(i * per_step, (i + 1) * per_step))
        t0 = time.perf_counter()
        oracle.receive(b.frames, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, b.pilot,
                       keep_Y=False)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    t = sum(times)
    value = args.steps * per_step * cfg.M * cfg.S * cfg.N / t
    line = {
        "impl": "reference", "metric": "antenna*subcarrier samples/s", "value": value,
        "unit": "samples/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
        # the same workload as the GPU arm; each step times a bounded sample of it
        "config": workload_config(cfg, F, min(args.pool, F)),
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": blas_threads(),
                         "kind": "oracle",
                         "sample": f"{per_step} of the workload's {F} frames per step "
                                   f"({args.steps} timed steps), generation excluded"},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_report(args):
    """Serving loop (lsas_server_*) under Poisson arrivals of frames of mixed
    configurations: M in {16, 32, 64, 128}, N in {256, 512, 1024, 2048},
    CP = N/8, 14 symbols, QAM in {4, 16, 64}, 8 taps, SNR U[5, 30] dB.  Six
    seeded configurations are registered; each arrival picks one uniformly
    and one of its 4 pooled frames (pinned host memory).  Per offered load
    (antenna*subcarrier samples/s): achieved throughput and p50/p99 latency
    from submit to results in host memory."""
    import threading
    import torch
    import paper_1901_07499_gb300.lsas as lsas
    # the load generator busy-waits for arrival times while the waiter thread
    # collects results: switch between them every 0.2 ms, not every 5 ms
    sys.setswitchinterval(2e-4)
    rng = np.random.default_rng(0x5E5)
    combos = []
    while len(combos) < 6:
        c = (int(rng.choice([16, 32, 64, 128])), int(rng.choice([256, 512, 1024, 2048])),
             int(rng.choice([4, 16, 64])))
        if c not in combos:
            combos.append(c)
    cfgs = [synth.frames.sweep_config(M, N).replace(Q=Q, taps=8, snr_db=(5.0, 30.0), F=4,
                                              name=f"serve_M{M}_N{N}_Q{Q}") for M, N, Q in combos]
    pools = [synth.generate(c, frame_ids=range(4)) for c in cfgs]
    max_batch, max_wait = 16, 200.0
    for form in args.serving_forms.split(","):
        serving_sweep(args, lsas, torch, form, cfgs, pools, max_batch, max_wait, rng)


def serving_sweep(args, lsas, torch, form, cfgs, pools, max_batch, max_wait, rng):
    """One form of the receiver ("plain": lsas_run_frame; "learned": LS ->
    tensor-core refinement -> MRC) over the offered loads."""
    import threading
    pb = None
    weights = None
    if form == "learned":
        import paper_1901_07499_gb300.denoiser as dnm
        if args.denoiser_ckpt:
            dn = dnm.Denoiser.load(args.denoiser_ckpt)
            weights = f"checkpoint {os.path.basename(args.denoiser_ckpt)}"
        else:
            # the refinement's cost does not depend on its weights' values
            dn = dnm.Denoiser(seed=1)
            weights = "initial weights (timing does not depend on their values)"
        pb = dn.bf16_params()
    elif form != "plain":
        raise ValueError(f"unknown serving form {form!r}")
    srv = lsas.Server(mem_budget=24 << 30, max_batch=max_batch, max_wait_us=max_wait)
    ids = [srv.register(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, pilot=b.pilot,
                        refine_params_bf16=pb)
           for c, b in zip(cfgs, pools)]
    xs = [[torch.from_numpy(np.ascontiguousarray(b.frames[i])).pin_memory() for i in range(4)]
          for b in pools]
    ring = 512
    outs = [[(torch.empty((c.M, c.N), dtype=torch.complex64).pin_memory(),
              torch.empty(c.D * c.N * c.q // 8, dtype=torch.uint8).pin_memory())
             for _ in range(ring)] for c in cfgs]
    samples = [c.M * c.S * c.N for c in cfgs]
    mean_samples = float(np.mean(samples))
    # warm-up, not measured: a few frames of every configuration (first
    # launches, host-side first touches)
    warm = [srv.submit(ids[ci], xs[ci][k % 4], *outs[ci][k]) for ci in range(len(cfgs))
            for k in range(8)]
    srv.wait_many(warm)
    for load in [float(v) for v in args.serving_loads.split(",")]:
        rate = load * 1e9 / mean_samples          # frames per second
        lat, lat_ci, lat_t, done_samples = [], [], [], [0]
        tickets = []
        cv = threading.Condition()
        finished = [False]

        def waiter():
            # collects results in groups of up to 64 tickets (one call each)
            i = 0
            while True:
                with cv:
                    while i >= len(tickets) and not finished[0]:
                        cv.wait()
                    if i >= len(tickets):
                        return
                    chunk = tickets[i:i + 64]
                got = srv.wait_many([t for t, _, _ in chunk])
                done_samples[0] += sum(samples[ci] for _, ci, _ in chunk)
                lat.extend(got)
                lat_ci.extend(ci for _, ci, _ in chunk)
                lat_t.extend(ts for _, _, ts in chunk)
                i += len(chunk)

        th = threading.Thread(target=waiter)
        th.start()
        # a garbage-collector pause in the generator would turn ~10 ms of
        # Poisson arrivals into one burst; collect now, not during the window
        gc.collect()
        gc.disable()
        st0 = srv.stats()
        t0 = time.perf_counter()
        t_next = t0
        n = 0
        max_lag = 0.0   # how late the generator submitted an arrival
        while t_next - t0 < args.serving_seconds:
            while time.perf_counter() < t_next:
                pass
            # every arrival that is due goes to the server in one call
            now = time.perf_counter()
            max_lag = max(max_lag, now - t_next)
            batch, cis = [], []
            while t_next <= now and t_next - t0 < args.serving_seconds and len(batch) < 64:
                ci = int(rng.integers(len(cfgs)))
                slot = n % ring
                if n >= ring:   # the slot's previous result must be home before reuse
                    while len(lat) <= n - ring:
                        time.sleep(0)
                H, bits = outs[ci][slot]
                batch.append((ids[ci], xs[ci][n % 4], H, bits))
                cis.append(ci)
                n += 1
                t_next += rng.exponential(1.0 / rate)
            t_sub = time.perf_counter() - t0
            ts = srv.submit_many(batch)
            with cv:
                tickets.extend((t, c, t_sub) for t, c in zip(ts, cis))
                cv.notify()
        with cv:
            finished[0] = True
            cv.notify()
        th.join()
        wall = time.perf_counter() - t0
        gc.enable()
        st1 = srv.stats()
        lat_us = np.array(lat)
        lat_c = np.array(lat_ci)
        lat_s = np.array(lat_t)
        # frames slower than 4x the median: how many, and when they were
        # submitted (one burst of a few ms, or spread over the window)
        slow = lat_us > 4 * np.percentile(lat_us, 50)
        slow_rec = {"frames": int(slow.sum())}
        if slow.any():
            st = np.sort(lat_s[slow])
            gaps = np.diff(st)
            slow_rec.update({"first_ms": float(st[0] * 1e3), "last_ms": float(st[-1] * 1e3),
                             "bursts": int(1 + np.sum(gaps > 0.05)),
                             "max_us": float(lat_us[slow].max())})
        per_config = {}
        for ci, c in enumerate(cfgs):
            sel = lat_us[lat_c == ci]
            if sel.size:
                per_config[c.name] = {"frames": int(sel.size),
                                      "p50": float(np.percentile(sel, 50)),
                                      "p99": float(np.percentile(sel, 99))}
        print(json.dumps({
            "mode": "serving", "form": form, "weights": weights,
            "offered_gsps": load, "achieved_gsps": done_samples[0] / wall / 1e9,
            "frames": n, "launches": st1["launches"] - st0["launches"],
            "latency_us": {"p50": float(np.percentile(lat_us, 50)),
                           "p99": float(np.percentile(lat_us, 99)),
                           "max": float(lat_us.max())},
            "max_batch": max_batch, "max_wait_us": max_wait,
            "per_config_latency_us": per_config,
            "slow_frames": slow_rec,
            "generator_max_lag_ms": max_lag * 1e3,
            "configs": [c.name for c in cfgs], "data": "synthetic (seeded generator)"}))
        sys.stdout.flush()
    code = srv.close()
    if code != lsas.LSAS_OK:
        raise RuntimeError(f"server reported {lsas.lsas_status_str(code).decode()}")


def denoiser_report(args):
    """Train the LS refinement on LS-domain rows (N = 1024, 4..16 taps,
    1..3 dB/tap, SNR U[0, 30] dB), then per SNR in {0, 5, 10, 20, 30} dB run
    16 frames of 64 antennas, N = 1024, 16-QAM (8 taps, 2 dB/tap, sc16)
    through lsas_run_frame (plain LS) and through lsas_estimate -> refinement
    (bf16 weights; CUDA-core and tensor-core forms) -> lsas_demodulate; report
    channel MSE against the true channel, bit error rate against the
    transmitted bits, and device time of each refinement per frame."""
    import torch
    import paper_1901_07499_gb300.lsas as lsas
    import paper_1901_07499_gb300.denoiser as dnm
    nets = {}
    for form in ("fp32", "bf16-tc"):
        t0 = time.perf_counter()
        losses = []
        net = dnm.train(rows=args.denoiser_rows, N=1024, batch=256, epochs=1, lr=1e-3, seed=1,
                        log=lambda ep, rows, loss: losses.append(loss),
                        tensor_cores=(form == "bf16-tc"))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        # device time of one gradient + Adam step on a 256-row batch
        Hs, Hl, _ = synth.ls_pairs(256, 1024, seed=99)
        Ht_ = torch.from_numpy(Hs.astype(np.complex64)).cuda()
        Hl_ = torch.from_numpy(Hl.astype(np.complex64)).cuda()
        probe = dnm.Denoiser(seed=2)
        probe.train_step(Hl_, Ht_, 1e-3, tensor_cores=(form == "bf16-tc"))
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        for _ in range(10):
            probe.train_step(Hl_, Ht_, 1e-3, tensor_cores=(form == "bf16-tc"))
        e[1].record()
        torch.cuda.synchronize()
        print(json.dumps({"mode": "denoiser-train", "form": form, "rows": net.rows_seen,
                          "steps": net.step, "final_loss": losses[-1] if losses else None,
                          "first_chunk_loss": losses[0] if losses else None,
                          "seconds": wall, "step_ms_256_rows": e[0].elapsed_time(e[1]) / 10,
                          "params": lsas.LSAS_DN_PARAMS,
                          "data": "synthetic LS-domain pairs (synth.ls_pairs)"}))
        sys.stdout.flush()
        nets[form] = net
    dn = nets["fp32"]
    if args.denoiser_ckpt:
        dn.save(args.denoiser_ckpt)
    pb = dn.bf16_params()
    pb_tc = nets["bf16-tc"].bf16_params()
    F = 16
    for snr in (0.0, 5.0, 10.0, 20.0, 30.0):
        cfg = synth.frames.sweep_config(64, 1024).replace(Q=16, taps=8, decay_db=2.0, snr_db=snr, F=F,
                                                           name=f"denoiser_eval_{int(snr)}dB")
        b = synth.generate(cfg, frame_ids=range(F))
        plan = lsas.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                         max_frames=F, pilot=b.pilot)
        x = torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()
        H_ls, bits_ls, _ = plan.run_frame(x)
        H_dn = dn.apply(H_ls, params_bf16=pb)
        bits_dn, _ = plan.demodulate(x, H_dn)
        H_tc = dn.apply(H_ls, params_bf16=pb, tensor_cores=True)
        bits_tc, _ = plan.demodulate(x, H_tc)
        # the refinement fused after LS, then MRC (one call)
        work = dn.work(F * cfg.M, cfg.N)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        H_fu, bits_fu, _ = plan.run_frame_refined(x, pb, work, st)
        # the network trained in BF16 on the tensor cores, fused after LS
        H_bt, bits_bt, _ = plan.run_frame_refined(x, pb_tc, work, st)
        plan.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        ev[0].record()
        for _ in range(5):
            dn.apply(H_ls, out=H_dn, params_bf16=pb)
        ev[1].record()
        ev[2].record()
        for _ in range(5):
            dn.apply(H_ls, out=H_tc, params_bf16=pb, tensor_cores=True)
        ev[3].record()
        ev[4].record()
        for _ in range(5):
            plan.run_frame_refined(x, pb, work, st, H=H_fu, bits=bits_fu)
        ev[5].record()
        ev[6].record()
        for _ in range(5):
            plan.run_frame(x, H_ls, bits_ls)
        ev[7].record()
        torch.cuda.synchronize()
        if int(st.item()) != 0:
            raise RuntimeError("fused refinement reported a timeout")
        if int(dn.status().item()) != 0:
            raise RuntimeError("tensor-core refinement reported a timeout")
        Htrue = np.fft.fft(b.taps, cfg.N, axis=-1) * b.gain[:, None, None]
        def mse(Hg):
            return float(np.mean(np.abs(Hg.cpu().numpy() - Htrue) ** 2) / np.mean(np.abs(Htrue) ** 2))
        def ber(bits):
            got = np.unpackbits(bits.cpu().numpy(), axis=-1, bitorder="big")[:, :cfg.D * cfg.N * cfg.q]
            return float(np.mean(got != b.bits.reshape(F, -1)))
        print(json.dumps({"mode": "denoiser-eval", "snr_db": snr, "frames": F, "M": cfg.M, "N": cfg.N,
                          "qam": cfg.Q, "nmse_ls": mse(H_ls), "nmse_dn": mse(H_dn),
                          "nmse_dn_tc": mse(H_tc), "nmse_fused": mse(H_fu),
                          "nmse_bf16_trained": mse(H_bt), "ber_bf16_trained": ber(bits_bt),
                          "ber_ls": ber(bits_ls), "ber_dn": ber(bits_dn),
                          "ber_dn_tc": ber(bits_tc), "ber_fused": ber(bits_fu),
                          "refine_us_per_frame": 1e3 * ev[0].elapsed_time(ev[1]) / 5 / F,
                          "refine_tc_us_per_frame": 1e3 * ev[2].elapsed_time(ev[3]) / 5 / F,
                          "fused_receiver_us_per_frame": 1e3 * ev[4].elapsed_time(ev[5]) / 5 / F,
                          "plain_receiver_us_per_frame": 1e3 * ev[6].elapsed_time(ev[7]) / 5 / F}))
        sys.stdout.flush()


def sweep_shapes():
    """The antenna x FFT-length grid of the scale workload (CP = N/8) and the
    paper's own (N, CP) shapes (64, 16) and (1024, 72) at 16 antennas."""
    grid = [synth.frames.sweep_config(M, N) for M in (8, 16, 32, 64, 128)
            for N in (64, 256, 512, 1024, 2048)]
    return grid + [synth.frames.paper_config(16, 64), synth.frames.paper_config(16, 1024)]


def sweep_report(args):
    """Throughput of lsas_run_frame over the sweep shapes, one JSON line per
    shape.  A step is one call over four waves of frames (4 x SMs, one block
    per frame, so no batch split), tiled from 4 seeded frames; the L2 is
    flushed (a 256 MB write) before each timed step, and each step is timed
    alone with CUDA events on the launching stream; the line reports the
    median of the steps."""
    import torch
    import paper_1901_07499_gb300.lsas as lsas
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    F = args.frames or 4 * sms
    steps = args.sweep_steps
    peak, peak_src = measured_peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for cfg in sweep_shapes():
        b = synth.generate(cfg.replace(F=4), frame_ids=range(4))
        plan = lsas.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                         max_frames=F, pilot=b.pilot)
        xp = torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()
        x = xp.repeat((F + 3) // 4, 1, 1, 1)[:F].contiguous()
        del xp
        H, bits = plan.empty_H(F), plan.empty_bits(F)
        for _ in range(max(args.warmup, 3)):
            plan.run_frame(x, H, bits)
        plan.sync()
        times = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.run_frame(x, H, bits)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        plan.sync()
        ms = statistics.median(times)
        in_b, h_b, bit_b, _ = lsas.frame_bytes(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.Q, cfg.fmt)
        alg = F * (in_b + h_b + bit_b)
        print(json.dumps({
            "mode": "sweep", "shape": cfg.name, "M": cfg.M, "N": cfg.N, "cp": cfg.cp,
            "n_sym": cfg.S, "qam": cfg.Q, "input": cfg.fmt, "frames": F,
            "kernel": fused_kernel_name(cfg).split(" ")[0], "launches": plan.run_frame_launches(F),
            "ms_per_step": ms, "metric": "antenna*subcarrier samples/s",
            "value": F * cfg.M * cfg.S * cfg.N / (ms * 1e-3),
            "us_per_frame": ms * 1e3 / F,
            "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": alg / (ms * 1e-3) / 1e9 / peak,
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_frame": in_b + h_b + bit_b},
            "l2": "flushed before each timed step"}), flush=True)
        plan.close()
        del x, H, bits
        torch.cuda.empty_cache()
    return 0


def host_link_report(args):
    """Bandwidth of this machine's host<->device link, which bounds the e2e
    figure: 1 GiB from pinned host memory to the device through the copy
    engines in 1, 2, 4 and 8 concurrent streams, and device to pinned host in
    one, best of five, CUDA events.  One JSON line per path."""
    import torch
    n = 1 << 30
    h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    h.fill_(1)
    d = torch.empty(n, dtype=torch.uint8, device="cuda")

    def best_ms(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    for ns in (1, 2, 4, 8):
        streams = [torch.cuda.Stream() for _ in range(ns)]

        def up():
            cur = torch.cuda.current_stream()
            part = n // ns
            for i, st in enumerate(streams):
                st.wait_stream(cur)
                with torch.cuda.stream(st):
                    d[i * part:(i + 1) * part].copy_(h[i * part:(i + 1) * part], non_blocking=True)
            for st in streams:
                cur.wait_stream(st)
        print(json.dumps({"mode": "host-link", "path": "h2d copy engines", "streams": ns,
                          "GB/s": n / best_ms(up) / 1e6}), flush=True)
    print(json.dumps({"mode": "host-link", "path": "d2h copy engine", "streams": 1,
                      "GB/s": n / best_ms(lambda: h.copy_(d, non_blocking=True)) / 1e6}), flush=True)
    return 0


def main():
    args = parse()
    cfg = synth.config_by_name(args.config)
    if args.host_link:
        return host_link_report(args)
    if args.sweep:
        return sweep_report(args)
    if args.serving:
        return serving_report(args)
    if args.denoiser:
        return denoiser_report(args)
    if args.impl == "reference":
        return reference_arm(args, cfg)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1901_07499_gb300.lsas as lsas

    F = args.frames or cfg.F
    pool = min(args.pool, F)
    # each rank owns its own seeded frames (independent units, no exchange)
    b = synth.generate(cfg, frame_ids=rank_frame_ids(rank, pool))
    plan = lsas.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                     max_frames=F, pilot=b.pilot)
    xp = torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()
    reps = (F + pool - 1) // pool
    x = xp.repeat(reps, 1, 1, 1)[:F].contiguous()
    del xp
    H = plan.empty_H(F)
    bits = plan.empty_bits(F)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        plan.run_frame(x, H, bits)
    plan.sync()
    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)   # let the sampler start before the timed region
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.run_frame(x, H, bits)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier()
    plan.sync()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    ms_step = ms / args.steps
    samples = job_samples(world, F, cfg)
    value = samples / (ms_step * 1e-3)

    in_b, h_b, bit_b, eq_b = lsas.frame_bytes(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.Q, cfg.fmt)
    launches = plan.run_frame_launches(F)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    full = (F // sms) * sms
    dominant = None
    if launches > 1 and full > 0:
        # the frames after the last whole wave run split (shard launch +
        # combine): the dominant kernel is the whole-wave launch, timed alone
        # here on the same stream (a batch of whole waves runs unsplit)
        xf, Hf, bf = x[:full], H[:full], bits[:full]
        for _ in range(args.warmup):
            plan.run_frame(xf, Hf, bf)
        torch.cuda.synchronize()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            plan.run_frame(xf, Hf, bf)
        c.record(stream)
        torch.cuda.synchronize()
        ms_main = max_over_ranks(a.elapsed_time(c), world, "cuda") / args.steps
        dominant = {"frames": full, "ms": ms_main, "share_of_step": ms_main / ms_step,
                    "tail_frames": F - full, "tail_shards": plan.batch_split_shards(F)}
    dom_frames = dominant["frames"] if dominant else F
    dom_ms = dominant["ms"] if dominant else ms_step
    alg_bytes = dom_frames * (in_b + h_b + bit_b)
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9
    peak, peak_src = measured_peaks()
    traffic = ncu_traffic(cfg, dom_frames)

    # single-frame latency
    lat = []
    x1, H1, b1 = x[:1], H[:1], bits[:1]
    for i in range(args.latency_calls + 10):
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.run_frame(x1, H1, b1)
        c.record(stream)
        c.synchronize()
        if i >= 10:
            lat.append(a.elapsed_time(c))
    lat.sort()
    # the same single frame with its antennas split into equal shards that
    # run side by side (8 antennas per shard keeps every warp of a block busy)
    shards = max([g for g in range(1, cfg.M + 1) if cfg.M % g == 0 and cfg.M // g >= 8] or [1])
    lat_s = []
    if shards > 1:
        for i in range(args.latency_calls + 10):
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.run_frame_split(x1, shards, H1, b1)
            c.record(stream)
            c.synchronize()
            if i >= 10:
                lat_s.append(a.elapsed_time(c))
        lat_s.sort()

    # the CUDA cores' FP32 peak on this GPU, for the ALU roofline
    fma = measure_fma_peak(lsas, torch, local) if not args.no_fma_peak else None

    # end to end through the host-buffer entry point
    xh = x[:F].cpu().pin_memory()
    Hh = torch.empty((F, cfg.M, cfg.N), dtype=torch.complex64).pin_memory()
    bh = torch.empty((F, bits.shape[1]), dtype=torch.uint8).pin_memory()
    plan.run_frame_host(xh, Hh, bh)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.run_frame_host(xh, Hh, bh)
    t_e2e = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, world, "cuda")
    plan.sync()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, nfr, threads, used = time_oracle(cfg, args.cpu_seconds)
        cpu = {"value": rate, "unit": "samples/s", "cores": threads, "kind": "oracle",
               "sample": f"{nfr} frames of the same workload ({used:.1f} s), "
                         "generation excluded",
               "cpu_model": cpu_model()}
        one = time_oracle_one_core(cfg, args.cpu_seconds / 2)
        if one is not None:
            cpu["one_core"] = {"value": one["rate"], "unit": "samples/s",
                               "sample": f"{one['frames']} frames ({one['seconds']:.1f} s), "
                                         "BLAS held to one thread"}

    if rank == 0:
        line = {
            "metric": "antenna*subcarrier samples/s", "value": value, "unit": "samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generator)",
            "config": workload_config(cfg, F, pool),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src,
                         "kernel": fused_kernel_name(cfg),
                         "algorithmic_bytes_per_frame": in_b + h_b + bit_b,
                         "frames_per_launch": dom_frames,
                         "step_frac": F * (in_b + h_b + bit_b) / (ms_step * 1e-3) / 1e9 / peak,
                         "dominant_launch": dominant},
            "roofline_fp32": fp32_roofline(cfg, F, ms_step, clocks, fma),
            "e2e": {"value": samples / t_e2e, "unit": "samples/s",
                    "h2d_bytes_per_step": F * plan.host_input_bytes_per_frame(),
                    "d2h_bytes_per_step": F * (h_b + bit_b)},
            "latency_ms": {"frames_per_call": 1, "p50": lat[len(lat) // 2],
                           "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "antenna_split": ({"shards": shards, "p50": lat_s[len(lat_s) // 2],
                                              "p99": lat_s[min(len(lat_s) - 1, int(0.99 * len(lat_s)))]}
                                             if lat_s else None)},
            "gpu_launches": args.steps * launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    plan.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
