"""Benchmark of the streaming connectivity push on GB300.

Default workload (one pushed trial per step): large all-to-all source space, 5124 nodes,
window W = 100 trials x 500 samples at 1 kHz, Hann taper, 40 bins (4-44 Hz, nfft 1000),
the 7 spectral metrics, streaming mode with resident accumulators (27.8 GB, larger than
L2, so no L2 flush is needed between steps). A step = one fc_push_trial of a new trial
through taper + band spectrum, per-node PSD sums, the streaming add/subtract update with
fused finalize and band average (plus the periodic re-sum when it falls due).

Metric: pair-bin updates/s = P * B / (time per push), P = n(n-1)/2 pairs, B bins.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs an independent session (weak scaling, no collective on
the data path); rank 0 prints one JSON line with the max-over-ranks time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "large_stream": dict(n=5124, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=100,
                         desc="large all-to-all source space, streaming push: 5124 nodes, "
                              "W=100 trials x 500 samples @1 kHz, Hann, 40 bins (4-44 Hz, nfft 1000), "
                              "7 spectral metrics, FP32 terms + double-float accumulators"),
    "source_stream": dict(n=2000, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=50,
                          desc="source space streaming push: 2000 nodes, W=50 trials x 500 samples, "
                               "40 bins (4-44 Hz), 7 spectral metrics"),
    # profiling case: same kernel shapes, 1.1 GB of state (> L2) so that an ncu capture stays small
    "profile_stream": dict(n=1024, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=20,
                           desc="profiling case: 1024 nodes, W=20 trials x 500 samples, 40 bins, "
                                "7 spectral metrics (1.1 GB of accumulators)"),
}
METRIC = "pair-bin updates/s per pushed trial"
UNIT = "pair-bin updates/s"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------- environment


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_bf16_tflops():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("bf16_tflops", 0.0)) or None
    return 1900.0


def stream_kernel_hash():
    h = hashlib.sha256()
    for f in ("k_stream.cu", "pair_common.cuh", "df32.cuh", "terms.cuh", "mbar.cuh"):
        with open(os.path.join(ROOT, "paper_2303_03279_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_hash, workload):
    """DRAM bytes per launch of the streaming kernel from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "k_stream_traffic.txt")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 3 and not line.startswith("#") and parts[0] == workload and parts[1] == kernel_hash:
                return float(parts[2])
    return None


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's value (the whole job ends when its last rank ends)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms_per_step: float) -> float:
    """Units all ranks processed per second: every rank runs its own session (weak scaling)."""
    return world * units_per_rank / (ms_per_step / 1000.0)


# ----------------------------------------------------------------- trial pool


def make_trials(w, count, seed=42):
    from synth import ar2_source_model, ar2_source_trials
    model = ar2_source_model(seed, w["n"], fs=w["fs"])
    return ar2_source_trials(model, 0, count, w["N"])


# ----------------------------------------------------------------- CPU oracle leg


def _oracle_sample_job(args):
    """One full-window oracle evaluation on a node subset (runs in a spawned process)."""
    n_sub, N, fs, band, W, seed = args
    import numpy as np  # noqa: F811
    import oracle as O
    from synth import ar2_source_model, ar2_source_trials
    model = ar2_source_model(seed, n_sub, fs=fs)
    x = ar2_source_trials(model, 0, W, N)
    bins = O.band_bins(fs, band[2], band[0], band[1])
    t0 = time.perf_counter()
    X = O.spectra(x, bins, band[2], "hann")
    nets = O.spectral_networks_dense(X)
    dt = time.perf_counter() - t0
    assert np.isfinite(nets["COH"]).all()
    P = n_sub * (n_sub - 1) // 2
    return dt, P * len(bins)


def host_cpu():
    """CPU model and logical core count of this host."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    return {"model": model or "unknown", "nproc": os.cpu_count() or 1}


def cpu_oracle_time(w, n_sub, reps=1, threads=1):
    """Time the oracle in a spawned process; BLAS threads pinned to ``threads`` (the numpy
    oracle's only multithreaded steps are its library matmuls)."""
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = str(threads)
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(1) as pool:
            res = [pool.apply(_oracle_sample_job, ((n_sub, w["N"], w["fs"], w["band"], w["W"], 7 + r),))
                   for r in range(reps)]
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return res


def run_reference(args, w, wname):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n_sub = args.ref_nodes
    for _ in range(args.warmup):
        cpu_oracle_time(w, n_sub)
    times, units = [], 0
    for _ in range(args.steps):
        (dt, pb), = cpu_oracle_time(w, n_sub)
        times.append(dt)
        units = pb
    ms = 1000.0 * sum(times) / len(times)
    value = units / (ms / 1000.0)
    sample = (f"{n_sub}-node subset of the {w['n']}-node workload: one full-window oracle evaluation "
              f"per step (FP64 DFT of W={w['W']} trials, pair sums, 7 spectral metrics)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "description": w["desc"], "oracle_nodes": n_sub},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU leg


SERVING = dict(N=500, fs=1000.0, pool=4,
               desc="16 concurrent sessions (4x60, 4x128, 4x306, 3x1000, 1x5124 nodes), windows "
                    "W ~ U{20..100} trials x 500 samples @1 kHz, 7 spectral metrics; sensor-size sessions "
                    "(<= 306 nodes) nfft 512, 1-50 Hz (25 bins), source-size sessions nfft 1000, 4-44 Hz "
                    "(40 bins); Poisson arrivals at U[5, 50] trials/s per session; N(0,1) trials")


def serving_band(n_nodes):
    """Sensor-size sessions: 1-50 Hz at nfft 512; source-size sessions: 4-44 Hz at nfft 1000."""
    return (1.0, 50.0, 512) if n_nodes <= 306 else (4.0, 44.0, 1000)


def band_bin_count(band, fs):
    return sum(1 for k in range(band[2] // 2 + 1) if band[0] * band[2] <= k * fs < band[1] * band[2])


def serving_leg(fc, plain, duration_s, seed, saturate=False, precision=0):
    """Replay the serving trace through one fc_server (batched streaming, or plain FP32).

    Every session gets one untimed trial first (calibration, module load). In replay mode
    each trial is submitted at its Poisson arrival time; with ``saturate`` every trial of
    the trace is submitted at once (peak aggregate throughput). Latency = completion time
    of the trial's network - its arrival time (host clock).
    """
    from synth import serving_trace, white_trials

    trace = serving_trace(seed, duration_s)
    N, fs = SERVING["N"], SERVING["fs"]
    pools = {n: white_trials(1000 + n, SERVING["pool"], n, N) for n in sorted({s.n_nodes for s in trace})}
    sv = fc.fc_server_create(plain=plain, precision=precision)
    try:
        ids = [fc.fc_server_open(sv, s.n_nodes, N, fs, serving_band(s.n_nodes), "hann", fc.FC_SPECTRAL_METRICS,
                                 s.window) for s in trace]
        for k, s in enumerate(trace):
            fc.fc_server_submit(sv, ids[k], pools[s.n_nodes][SERVING["pool"] - 1], fc.fc_server_now_ms())
        fc.fc_server_drain(sv, 600000)
        fc.fc_server_poll(sv, len(trace) + 8)
        st0 = fc.fc_server_stats_get(sv)
        events = sorted((float(t), k) for k, s in enumerate(trace) for t in s.arrivals_s)
        units = {ids[k]: (s.n_nodes * (s.n_nodes - 1) // 2) * band_bin_count(serving_band(s.n_nodes), fs)
                 for k, s in enumerate(trace)}
        t0 = fc.fc_server_now_ms()
        for i, (t, k) in enumerate(events):
            if not saturate:
                target = t0 + 1000.0 * t
                while True:
                    d = target - fc.fc_server_now_ms()
                    if d <= 0:
                        break
                    time.sleep(min(d, 2.0) / 1000.0)
            fc.fc_server_submit(sv, ids[k], pools[trace[k].n_nodes][i % (SERVING["pool"] - 1)], fc.fc_server_now_ms())
        fc.fc_server_drain(sv, 600000)
        res = fc.fc_server_poll(sv, len(events) + 8)
        st1 = fc.fc_server_stats_get(sv)
    finally:
        fc.fc_server_destroy(sv)
    assert len(res) == len(events) and all(r[2] == fc.FC_OK for r in res), "serving trace did not complete"
    lat = sorted(r[4] - r[3] for r in res)
    span_ms = max(r[4] for r in res) - t0
    upd = sum(units[r[0]] for r in res)
    launches = st1["launches"] - st0["launches"]
    return {"trials": len(res), "value": upd / (span_ms / 1000.0), "unit": UNIT, "span_ms": span_ms,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))],
                           "max": lat[-1], "what": "trial arrival to network ready (host clock)"},
            "ticks": launches, "trials_per_tick": (st1["batched_trials"] - st0["batched_trials"]) / max(1, launches),
            "sessions_per_stream_launch": float(np.mean([r[5] for r in res])),
            "hbm_used_bytes": st1["hbm_used"],
            "windows": [s.window for s in trace], "rates_per_s": [round(s.rate_hz, 2) for s in trace]}


CASES = {
    # small, self-contained launches for profiler captures (a few GB at most)
    "meg_bf16_window": dict(n=306, N=1000, fs=1000.0, band=(1.0, 100.0, 1024), W=100, prec="bf16", pushes=0,
                            desc="306 MEG-shaped channels, one bulk push of 100 x 1000 samples, 101 bins, BF16 "
                                 "tensor-core full window"),
    "window_1024_fp32": dict(n=1024, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=100, prec="fp32", pushes=3,
                             desc="1024 nodes, W = 100, 40 bins, full-window FP32 recompute: bulk fill + 3 pushes"),
    "window_1024_bf16": dict(n=1024, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=100, prec="bf16", pushes=3,
                             desc="1024 nodes, W = 100, 40 bins, BF16 tensor-core full window: bulk fill + 3 pushes"),
    "window_5124_bf16": dict(n=5124, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=100, prec="bf16", pushes=1,
                             desc="5124 nodes, W = 100, 40 bins, BF16 tensor-core full window (about 1.5 GB on the "
                                  "device): bulk fill + 1 push"),
    "window_1024_tf32x3": dict(n=1024, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=100, prec="tf32x3", pushes=3,
                               desc="1024 nodes, W = 100, 40 bins, split-TF32 tensor-core full window: bulk fill + "
                                    "3 pushes"),
    "window_5124_tf32x3": dict(n=5124, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=100, prec="tf32x3", pushes=1,
                               desc="5124 nodes, W = 100, 40 bins, split-TF32 tensor-core full window (FP32-class "
                                    "linear metrics; about 4 GB on the device): bulk fill + 1 push"),
    "xcor_meg_window": dict(n=306, N=1000, fs=1000.0, band=(1.0, 100.0, 1024), W=100, prec="fp32", pushes=2,
                            metrics="XCOR",
                            desc="XCOR only, 306 MEG-sized channels, W = 100 trials x 1000 samples (2048-point "
                                 "transforms), full-window recompute: bulk fill + 2 pushes"),
    "xcor_306_window": dict(n=306, N=500, fs=600.0, band=(8.0, 12.0, 600), W=20, prec="fp32", pushes=2,
                            metrics="XCOR",
                            desc="XCOR only, 306 nodes, W = 20 trials x 500 samples (1024-point transforms), "
                                 "full-window recompute: bulk fill + 2 pushes"),
    "cor_1000_window": dict(n=1000, N=1000, fs=600.0, band=(8.0, 12.0, 1200), W=50, prec="fp32", pushes=3,
                            metrics="COR",
                            desc="COR only, 1000 nodes, W = 50 trials x 1000 samples, full-window recompute on "
                                 "the tensor cores (split TF32): bulk fill + 3 pushes"),
}


CONFIG_LEGS = {
    # the other workloads of the benchmark, measured beside the headline in the default run
    "eeg_full_window": dict(n=60, N=500, fs=1000.0, band=(1.0, 50.0, 512), W=20, gen="eeg", mode="full", reps=10,
                            desc="sensor-space EEG, plain method: 60 channels, 20 trials x 500 samples @1 kHz "
                                 "(N(0,1) + 10 Hz sinusoids coupled at lags 0, pi/4, pi/2 on 10 seeded pairs), "
                                 "Hann, nfft 512, 1-50 Hz (25 bins), all 9 metrics once over the full trial set"),
    "meg_full_window": dict(n=306, N=1000, fs=1000.0, band=(1.0, 100.0, 1024), W=100, gen="meg", mode="full", reps=4,
                            desc="MEG sensor space, full-window GPU path: 306 channels, 100 trials x 1000 samples "
                                 "@1 kHz (1/f Gaussian noise + 40 coupled pairs at 8-30 Hz), Hann, nfft 1024, "
                                 "1-100 Hz (101 bins), all 9 metrics; one new trial per push, whole window "
                                 "recomputed"),
    "source_stream": dict(n=2000, N=500, fs=1000.0, band=(4.0, 44.0, 1000), W=50, gen="ar2", mode="stream",
                          pushes=500,
                          desc="source space, streaming: 2000 AR(2) alpha sources with a 200-edge coupling "
                               "graph, W = 50 trials x 500 samples @1 kHz, one new trial per push (98 % overlap), "
                               "500 pushes, Hann, nfft 1000, 4-44 Hz (40 bins), 7 spectral metrics"),
}


def config_legs(fc, torch, stream):
    """Device time per push of the other workloads (CUDA events on the session stream).

    Full-window legs: one bulk fill, then ``reps`` single-trial pushes, each recomputing the
    whole window (the EEG leg instead repeats its one evaluation of all 20 trials). Streaming
    leg: one bulk fill of the window, then ``pushes`` single-trial pushes, exact and in the
    mixed-precision streaming form (BF16, TF32 drift re-sum); beside it pushes through the
    mixed-precision full window (BF16, TF32 tensor-core linear sums).
    """
    from synth import ar2_source_model, ar2_source_trials, eeg_sinusoid_trials, meg_pink_trials

    def timed(sess, xs, count=1):
        ev = []
        for x in xs:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if count == 1:
                fc.fc_push_trial(sess.handle, x)
            else:
                fc.fc_push_trials(sess.handle, x, count)
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    out = {}
    for name, c in CONFIG_LEGS.items():
        n, N, W = c["n"], c["N"], c["W"]
        if c["gen"] == "eeg":
            x = eeg_sinusoid_trials(21, W, n, N, fs=c["fs"])[0]
        elif c["gen"] == "meg":
            x = meg_pink_trials(22, W + c["reps"], n, N, fs=c["fs"])[0]
        else:
            x = ar2_source_trials(ar2_source_model(23, n, fs=c["fs"]), 0, W + 16, N)
        dev = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
        leg = {"description": c["desc"]}
        precs = [("fp32", fc.FC_PREC_FP32, c["mode"])] + (
            [("bf16", fc.FC_PREC_BF16, "full"), ("tf32", fc.FC_PREC_TF32, "full")] if c["gen"] != "eeg"
            else [("bf16", fc.FC_PREC_BF16, "full")])
        if c["mode"] == "stream":  # the mixed-precision streaming form (tensor-core drift re-sum)
            precs += [("bf16_stream", fc.FC_PREC_BF16, "stream"), ("tf32_stream", fc.FC_PREC_TF32, "stream")]
        for pname, prec, pmode in precs:
            mode = fc.FC_MODE_STREAM if pmode == "stream" else fc.FC_MODE_FULL
            mask = fc.FC_ALL_METRICS if (c["mode"] == "full" and prec == fc.FC_PREC_FP32) else fc.FC_SPECTRAL_METRICS
            with fc.Session(n, N, c["fs"], c["band"], "hann", mask, W, mode=mode, precision=prec,
                            stream=stream.cuda_stream) as s:
                P, B = s.P, s.B
                fc.fc_set_profiling(s.handle, True)
                if c["gen"] == "eeg":
                    ts = timed(s, [dev] * (c["reps"] + 1), count=W)[1:]  # one evaluation of the 20 trials each
                else:
                    fc.fc_push_trials(s.handle, dev[:W].contiguous(), W)
                    fc.fc_sync(s.handle)
                    fc.fc_kernel_times(s.handle, reset=True)
                    k = c.get("pushes", c.get("reps")) if mode == fc.FC_MODE_STREAM else c.get("reps", 4)
                    pool = dev.shape[0] - W
                    ts = timed(s, [dev[W + (i % pool)] for i in range(k)])
                kt = fc.fc_kernel_times(s.handle, reset=True)
            ms = sum(ts) / len(ts)
            ts_sorted = sorted(ts)
            leg[pname] = {
                "path": (("streaming add/subtract update" + ("" if prec == fc.FC_PREC_FP32 else
                          f", drift re-sum with tcgen05 {pname[:4].upper()} linear sums"))
                         if mode == fc.FC_MODE_STREAM else
                         ("full-window recompute, CUDA cores" if prec == fc.FC_PREC_FP32 else
                          f"full-window recompute, tcgen05 {pname.upper()} linear sums + CUDA-core non-linear sums")),
                "metrics": "all 9" if mask == fc.FC_ALL_METRICS else "7 spectral",
                "pushes_timed": len(ts), "ms_per_push": ms,
                "p50_ms": ts_sorted[len(ts) // 2], "p99_ms": ts_sorted[min(len(ts) - 1, int(round(0.99 * (len(ts) - 1))))],
                "pair_bins_per_push": P * B, "value": P * B / (ms / 1000.0), "unit": UNIT,
                "contributions_per_s": (P * B * W / (ms / 1000.0)) if mode == fc.FC_MODE_FULL else None,
                "kernels_ms_per_push": {k2: round(v[1] / len(ts), 4) for k2, v in kt.items() if v[0]},
            }
        out[name] = leg
        del dev
    return out


def run_project_case(args):
    """Source projection of sensor trials (the paper's source-level pipeline): 306 MEG-sized
    channels onto 5124 sources, 500-sample trials, 40 bins, W = 20, streaming pushes. The
    spectral-only session projects band spectra (frequency domain); a session that also
    holds COR projects the time series. Per push: device time of the projection and
    spectrum kernels of each path."""
    import torch
    from paper_2303_03279_gb300 import fc
    from synth import white_trials

    fc.load()
    n, C, N, W, pushes = 5124, 306, 500, 20, 5
    M = (np.random.default_rng(9).standard_normal((n, C)) / np.sqrt(C)).astype(np.float32)
    x = torch.from_numpy(white_trials(7, W + pushes, C, N)).cuda()
    out = {"case": "project_5124", "description": run_project_case.__doc__.split("\n\n")[0].replace("\n    ", " ")}
    for name, mask in (("frequency_domain (spectral metrics)", fc.FC_SPECTRAL_METRICS),
                       ("time_domain (spectral metrics + COR)", fc.FC_SPECTRAL_METRICS | fc.FC_COR)):
        with fc.Session(n, N, 1000.0, (4.0, 44.0, 1000), "hann", mask, W) as s:
            fc.fc_set_projection(s.handle, torch.from_numpy(M).cuda())
            fc.fc_push_trials(s.handle, x[:W].contiguous(), W)
            fc.fc_sync(s.handle)
            fc.fc_set_profiling(s.handle, True)
            fc.fc_kernel_times(s.handle, reset=True)
            for k in range(pushes):
                fc.fc_push_trial(s.handle, x[W + k])
            fc.fc_sync(s.handle)
            kt = fc.fc_kernel_times(s.handle, reset=True)
        out[name] = {k: round(v[1] / pushes, 4) for k, v in kt.items() if k in ("project", "spectrum") and v[0]}
    out["flops_per_trial"] = {"frequency_domain": 2 * n * C * 2 * 40, "time_domain": 2 * n * C * N}
    print(json.dumps(out))
    return 0


def run_case(args):
    """One small named case (the profiler captures' workloads); prints its timing per push."""
    if args.case == "spectrum_methods":
        return run_spectrum_case(args)
    if args.case == "project_5124":
        return run_project_case(args)
    import torch
    from paper_2303_03279_gb300 import fc
    from synth import meg_pink_trials, white_trials

    c = CASES[args.case]
    fc.load()
    n, N, W = c["n"], c["N"], c["W"]
    if args.case.startswith("meg"):
        x = meg_pink_trials(3, W + c["pushes"], n, N)
        x = x[0] if isinstance(x, tuple) else x
    else:
        x = white_trials(5, W + c["pushes"], n, N)
    x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    prec = {"fp32": fc.FC_PREC_FP32, "bf16": fc.FC_PREC_BF16, "tf32x3": fc.FC_PREC_TF32X3}[c["prec"]]
    mask = {"COR": fc.FC_COR, "XCOR": fc.FC_XCOR}.get(c.get("metrics"), fc.FC_SPECTRAL_METRICS)
    with fc.Session(n, N, c["fs"], c["band"], "hann", mask, W, mode=fc.FC_MODE_FULL, precision=prec) as s:
        fc.fc_push_trials(s.handle, x[:W].contiguous(), W)
        fc.fc_sync(s.handle)
        fc.fc_set_profiling(s.handle, True)
        fc.fc_kernel_times(s.handle, reset=True)
        t0 = time.perf_counter()
        for k in range(c["pushes"]):
            fc.fc_push_trial(s.handle, x[W + k])
        fc.fc_sync(s.handle)
        dt = (time.perf_counter() - t0) * 1000.0 / max(1, c["pushes"])
        kt = fc.fc_kernel_times(s.handle, reset=True)
    print(json.dumps({"case": args.case, "description": c["desc"], "ms_per_push": dt if c["pushes"] else None,
                      "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in kt.items() if v[0]}}))
    return 0


def run_spectrum_case(args):
    """Band spectra by the band DFT and by the real FFT (Methods 2.4: per-trial spectra),
    device time of the spectrum kernel per trial, for sensor-, source- and wide-band shapes
    (bulk pushes of 8 white-noise trials into full-window sessions, three pushes per method)."""
    import torch
    from paper_2303_03279_gb300 import fc
    from synth import white_trials

    fc.load()
    shapes = [  # n, N, fs, (f_lo, f_hi, nfft)
        (60, 500, 1000.0, (1.0, 50.0, 512)),
        (60, 600, 600.0, (8.0, 12.0, 600)),
        (5124, 500, 1000.0, (4.0, 44.0, 1000)),
        (306, 1000, 1000.0, (1.0, 100.0, 1024)),
        (5124, 500, 1000.0, (4.0, 44.0, 512)),
        (5124, 1000, 1000.0, (1.0, 100.0, 1024)),
        (2000, 1000, 1000.0, (0.0, 501.0, 1024)),
        (1000, 4000, 1000.0, (1.0, 100.0, 4096)),
    ]
    K, reps = 8, 3
    rows = []
    for n, N, fs, band in shapes:
        x = torch.from_numpy(white_trials(n + N, K, n, N)).cuda()
        row = {"n": n, "N": N, "nfft": band[2], "band_hz": [band[0], band[1]]}
        for name, sp in (("dft", fc.FC_SPECTRUM_DFT), ("fft", fc.FC_SPECTRUM_FFT), ("auto", fc.FC_SPECTRUM_AUTO)):
            with fc.Session(n, N, fs, band, "hann", fc.FC_COH, K, mode=fc.FC_MODE_FULL, spectrum=sp) as s:
                row["bins"] = s.B
                fc.fc_push_trials(s.handle, x, K)
                fc.fc_sync(s.handle)
                fc.fc_set_profiling(s.handle, True)
                fc.fc_kernel_times(s.handle, reset=True)
                for _ in range(reps):
                    fc.fc_push_trials(s.handle, x, K)
                fc.fc_sync(s.handle)
                kt = fc.fc_kernel_times(s.handle, reset=True)
                if name == "auto":
                    row["auto_picks"] = "fft" if s.info().spectrum == fc.FC_SPECTRUM_FFT else "dft"
                else:
                    row[f"{name}_us_per_trial"] = round(kt["spectrum"][1] * 1000.0 / (reps * K), 3)
        rows.append(row)
        del x
        torch.cuda.empty_cache()
    print(json.dumps({"case": "spectrum_methods", "description": run_spectrum_case.__doc__.split("\n\n")[0]
                      .replace("\n    ", " "), "rows": rows}))
    return 0


def run_sweep(args):
    """Secondary sweep shaped like the paper's performance evaluation (Results 3.1: fs = nfft
    = 600 Hz, 8-12 Hz = 4 bins, storage mode off so that every evaluation recomputes the
    window; node counts x window sizes for one trial, node counts x trial counts at 1,000
    samples). Each row: device time of one full evaluation (bulk push of the K trials through
    the full-window path, FP32) and its network read into device memory."""
    import torch
    from paper_2303_03279_gb300 import fc
    from synth import white_trials

    fc.load()
    stream = torch.cuda.Stream()
    nodes = [60, 128, 306, 1000, 2000]
    shapes = [(1, ns) for ns in (500, 1000, 2000, 4000, 8000)] + [(k, 1000) for k in (10, 50, 100)]
    metrics = {"COR": fc.FC_COR, "XCOR": fc.FC_XCOR, "spectral (COH ... DSWPLI)": fc.FC_SPECTRAL_METRICS}
    rows = []
    for n in nodes:
        for K, N in shapes:
            x = torch.from_numpy(white_trials(n + K + N, K, n, N)).cuda()
            for mname, mask in metrics.items():
                if mname == "XCOR" and (n * (n - 1) // 2 * K * N > 2e10 or N > 8192):
                    continue  # bounded run time; XCOR sessions take N <= 8192 samples
                nfft = 600 * ((N + 599) // 600)  # 600 (1 Hz bins) or the next multiple that holds the window
                with fc.Session(n, N, 600.0, (8.0, 12.0, nfft), "hann", mask, K, mode=fc.FC_MODE_FULL,
                                stream=stream.cuda_stream) as sess:
                    out = torch.empty(n * (n - 1) // 2, device="cuda")
                    bit = fc.FC_COR if mask == fc.FC_COR else (fc.FC_XCOR if mask == fc.FC_XCOR else fc.FC_COH)
                    reps, t = 3, []
                    for r in range(reps + 1):
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        fc.fc_push_trials(sess.handle, x, K)
                        fc.fc_get_network(sess.handle, bit, 1, out)
                        b.record(stream)
                        b.synchronize()
                        if r:
                            t.append(a.elapsed_time(b))
                rows.append({"metric": mname, "nodes": n, "samples": N, "trials": K, "nfft": nfft,
                             "ms": round(sum(t) / len(t), 4)})
    print(json.dumps({"sweep": "paper-style performance sweep (fs = 600 Hz, nfft 600 or the next multiple of 600 "
                               "that holds the window, 8-12 Hz, full recompute, FP32)",
                      "unit": "ms per evaluation", "rows": rows}), flush=True)
    return 0


def run_ours(args, w, wname):
    import torch
    from paper_2303_03279_gb300 import fc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fc.load()
    n, N, W, B_band = w["n"], w["N"], w["W"], w["band"]
    steps, warmup = args.steps, args.warmup
    pool_n = min(W + warmup + steps, args.pool)
    t0 = time.time()
    host = make_trials(w, pool_n, seed=42 + rank)
    log(f"[rank {rank}] generated {pool_n} trials in {time.time() - t0:.1f}s")
    dev = torch.from_numpy(host).cuda()
    stream = torch.cuda.Stream()
    mask = fc.FC_SPECTRAL_METRICS
    sess = fc.Session(n, N, w["fs"], B_band, "hann", mask, W, mode=fc.FC_MODE_STREAM,
                      stream=stream.cuda_stream, resum_period=args.resum_period)
    P, B = sess.P, sess.B
    units = P * B
    torch.cuda.synchronize()

    def trial(k):
        return dev[k % pool_n]

    # fill the window (bulk push: one re-sum from the stored spectra), then warm up
    fc.fc_push_trials(sess.handle, dev[:W].contiguous() if pool_n >= W else dev, W)
    fc.fc_sync(sess.handle)
    for k in range(warmup):
        fc.fc_push_trial(sess.handle, trial(W + k))
    fc.fc_sync(sess.handle)

    # timed region: device-resident inputs
    fc.fc_set_profiling(sess.handle, True)
    fc.fc_kernel_times(sess.handle, reset=True)
    launches0 = fc.fc_launch_count(sess.handle)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(steps):
            ev[k][0].record(stream)
            fc.fc_push_trial(sess.handle, trial(W + warmup + k))
            ev[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    fc.fc_sync(sess.handle)
    launches = fc.fc_launch_count(sess.handle) - launches0
    ktimes = fc.fc_kernel_times(sess.handle, reset=True)
    fc.fc_set_profiling(sess.handle, False)
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world, "cuda")
    ms_per_step = total_ms / steps
    lat = sorted(a.elapsed_time(b) for a, b in ev)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))]
    value = whole_job_rate(units, world, ms_per_step)

    # roofline of the dominant kernel (streaming update)
    launches_k, tot_k = ktimes["stream"]
    hbm, peak_kind = measured_peaks()
    roofline = None
    if launches_k:
        avg_ms = tot_k / launches_k
        alg_bytes = 104.0 * units + 28.0 * P  # state read + write, 7 network planes written
        achieved = alg_bytes / (avg_ms / 1000.0) / 1e9
        roofline = {"kernel": "k_stream", "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "peak_source": peak_kind, "avg_launch_ms": avg_ms,
                    "algorithmic_bytes_per_launch": alg_bytes,
                    "traffic": ncu_traffic(stream_kernel_hash(), wname)}
    kernel_share = {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in ktimes.items() if v[0]}
    if "window" in kernel_share:  # the exact re-sum slice runs on a side stream beside the update
        kernel_share["window"]["note"] = ("drift re-sum slice on the session's side stream, timed from its "
                                          "fork: includes waiting for the SMs the update holds")

    # e2e: host trial in (pinned), one metric's network out, through the public API. Each
    # step pushes its trial from pinned host memory and reads its COH network back into
    # pinned host memory; the reads are started asynchronously and waited for one step
    # later, so copies in and out overlap the next push (the per-step time is the interval
    # between completed results in the steady state).
    e2e = None
    if not args.no_e2e:
        pinned_in = torch.from_numpy(host[: min(pool_n, 8)].copy()).pin_memory()
        outs = [torch.empty(P, dtype=torch.float32).pin_memory() for _ in range(2)]
        e2e_steps = max(3, min(steps, args.e2e_steps))
        fc.fc_sync(sess.handle)
        tt = []
        t_prev = None
        for k in range(e2e_steps + 3):
            fc.fc_push_trial(sess.handle, pinned_in[k % pinned_in.shape[0]].numpy())
            fc.fc_get_network_async(sess.handle, fc.FC_COH, outs[k % 2].numpy())
            if k >= 1:
                fc.fc_network_wait(sess.handle)  # step k - 1's network is in host memory
                now = time.perf_counter()
                if k >= 3:
                    tt.append(now - t_prev)
                t_prev = now
        fc.fc_network_wait(sess.handle)
        fc.fc_sync(sess.handle)
        e2e_ms = 1000.0 * sum(tt) / len(tt)
        e2e = {"value": world * units / (e2e_ms / 1000.0), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": n * N * 4, "d2h_bytes_per_step": P * 4,
               "interval_ms": {"p50": sorted(tt)[len(tt) // 2] * 1000.0, "max": max(tt) * 1000.0},
               "steps": e2e_steps,
               "how": "fc_push_trial from pinned host memory + fc_get_network_async into pinned host "
                      "memory every step, each result waited for one step later"}
    sess.close()
    del sess
    torch.cuda.synchronize()

    # plain FP32 comparator: CUDA-core full-window recompute per push, no accumulators
    plain = None
    mixed = None
    mixed_stream = None
    mixed_stream_split = None
    if not args.no_plain:
        ps = fc.Session(n, N, w["fs"], B_band, "hann", mask, W, mode=fc.FC_MODE_FULL, stream=stream.cuda_stream)
        fc.fc_push_trials(ps.handle, dev[:W].contiguous(), W)
        fc.fc_sync(ps.handle)
        pst = max(2, min(args.plain_steps, steps))
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(pst)]
        for k in range(pst):
            pev[k][0].record(stream)
            fc.fc_push_trial(ps.handle, trial(W + k))
            pev[k][1].record(stream)
        torch.cuda.synchronize()
        pl = sorted(a.elapsed_time(b) for a, b in pev)
        pms = sum(pl) / len(pl)
        plain = {"value": world * units / (pms / 1000.0), "unit": UNIT, "ms_per_step": pms,
                 "contributions_per_s": world * units * W / (pms / 1000.0),
                 "latency_ms": {"p50": pl[len(pl) // 2], "p99": pl[-1]}, "steps": pst,
                 "path": "CUDA-core full-window recompute per push (FC_MODE_FULL), FP32"}
        ps.close()
        del ps
        # mixed precision full window: tensor-core linear sums (BF16) + CUDA-core non-linear sums
        ms = fc.Session(n, N, w["fs"], B_band, "hann", mask, W, mode=fc.FC_MODE_FULL, precision=fc.FC_PREC_BF16,
                        stream=stream.cuda_stream)
        fc.fc_push_trials(ms.handle, dev[:W].contiguous(), W)
        fc.fc_sync(ms.handle)
        fc.fc_set_profiling(ms.handle, True)
        fc.fc_kernel_times(ms.handle, reset=True)
        mst = max(3, min(args.plain_steps * 3, steps))
        mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(mst)]
        for k in range(mst):
            mev[k][0].record(stream)
            fc.fc_push_trial(ms.handle, trial(W + k))
            mev[k][1].record(stream)
        torch.cuda.synchronize()
        mkt = fc.fc_kernel_times(ms.handle, reset=True)
        ml = sorted(a.elapsed_time(b) for a, b in mev)
        mms = sum(ml) / len(ml)
        tc_launches, tc_ms = mkt["herk_tc"]
        mixed = {"value": world * units / (mms / 1000.0), "unit": UNIT, "ms_per_step": mms,
                 "contributions_per_s": world * units * W / (mms / 1000.0),
                 "latency_ms": {"p50": ml[len(ml) // 2], "p99": ml[-1]}, "steps": mst,
                 "path": "full-window recompute per push: tcgen05 BF16 Hermitian products (COH, IMAGCOHY, PLV) "
                         "+ CUDA-core non-linear sums (PLI, USPLI, WPLI, DSWPLI)",
                 "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in mkt.items() if v[0]}}
        if tc_launches:
            # algorithmic tensor work: 16 flop per pair-bin-trial (the CSD and phasor complex
            # multiply-adds); the launched GEMMs (4 real 128 x 128 x Kp per 128-node tile pair and
            # bin, Kp = 2W padded to the 16-element K-step of the resident-operand products,
            # full diagonal tiles) are larger
            nt128 = (n + 127) // 128
            kp = ((2 * W + 15) // 16) * 16
            flops_alg = 16 * P * B * W
            flops_padded = 4 * 2 * 128 * 128 * kp * (nt128 * (nt128 + 1) // 2) * B
            herk_ms = tc_ms / tc_launches * 2
            achieved = flops_alg / (herk_ms / 1000.0) / 1e12
            bf16_peak = measured_bf16_tflops()
            mixed["tensor"] = {"flops_per_push": flops_alg, "launched_flops_per_push": flops_padded,
                               "herk_ms_per_push": herk_ms,
                               "achieved_tflops": achieved, "peak_tflops": bf16_peak,
                               "frac": achieved / bf16_peak if bf16_peak else None,
                               "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)" if bf16_peak else None,
                               "note": "algorithmic flops (16 per pair-bin-trial) over the operand pack + MMA "
                                       "kernel time per push"}
        ms.close()
        del ms
        # mixed-precision streaming: the exact streaming update, drift re-sum slices with the
        # linear sums on the tensor cores (BF16 operand ring; split TF32: high and low parts)
        for key, sprec, label in (("bf16", fc.FC_PREC_BF16, "BF16"),
                                  ("tf32x3", fc.FC_PREC_TF32X3, "split-TF32 (hi hi + hi lo + lo hi)")):
            torch.cuda.synchronize()
            ss = fc.Session(n, N, w["fs"], B_band, "hann", mask, W, mode=fc.FC_MODE_STREAM, precision=sprec,
                            stream=stream.cuda_stream)
            fc.fc_push_trials(ss.handle, dev[:W].contiguous(), W)
            for k in range(warmup):
                fc.fc_push_trial(ss.handle, trial(W + k))
            fc.fc_sync(ss.handle)
            fc.fc_set_profiling(ss.handle, True)
            fc.fc_kernel_times(ss.handle, reset=True)
            sst = max(3, steps)
            sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(sst)]
            for k in range(sst):
                sev[k][0].record(stream)
                fc.fc_push_trial(ss.handle, trial(W + warmup + k))
                sev[k][1].record(stream)
            torch.cuda.synchronize()
            skt = fc.fc_kernel_times(ss.handle, reset=True)
            sl = sorted(a.elapsed_time(b) for a, b in sev)
            sms_ = sum(sl) / len(sl)
            kms = {k: v[1] / sst for k, v in skt.items() if v[0]}
            leg = {"value": world * units / (sms_ / 1000.0), "unit": UNIT, "ms_per_step": sms_,
                   "latency_ms": {"p50": sl[len(sl) // 2], "p99": sl[-1]}, "steps": sst,
                   "path": f"exact streaming update (FP32 terms, double-float sums); drift re-sum slice: "
                           f"tcgen05 {label} linear sums over the operand ring + CUDA-core non-linear sums "
                           f"(exact signs; the update's own terms added exactly into double words)",
                   "kernels_ms_per_push": {k: round(v, 4) for k, v in kms.items()},
                   "tensor_core_share_of_push": kms.get("herk_tc", 0.0) / sms_,
                   # the slice's non-linear sums run beside the update on a side stream: their
                   # event times include waiting for SMs, so the push time beyond the update is
                   # what the re-sum costs
                   "push_beyond_update_ms": sms_ - kms.get("stream", 0.0),
                   "side_stream_note": "window: the slice's non-linear sums, timed on the side "
                                       "stream from the fork (includes waiting for the update's SMs)"}
            if key == "bf16":
                mixed_stream = leg
            else:
                mixed_stream_split = leg
            ss.close()
            del ss

    # serving: many concurrent sessions, continuous batching vs plain FP32 one trial at a time
    serving = None
    if world == 1 and not args.no_serving:
        del dev
        torch.cuda.empty_cache()
        rep_b = serving_leg(fc, False, args.serving_seconds, 11)
        rep_m = serving_leg(fc, False, args.serving_seconds, 11, precision=fc.FC_PREC_BF16)
        rep_p = serving_leg(fc, True, args.serving_seconds, 11)
        burst = serving_leg(fc, False, args.serving_seconds, 11, saturate=True)
        serving = {"trace": SERVING["desc"], "seconds": args.serving_seconds,
                   "summary": {
                       "what": "Poisson replay of the trace; latency = trial arrival to network ready (host clock); "
                               "value = pair-bin updates of all completed pushes / span",
                       "batched": {"p50_ms": rep_b["latency_ms"]["p50"], "p99_ms": rep_b["latency_ms"]["p99"],
                                   "value": rep_b["value"], "unit": UNIT},
                       "batched_mixed_bf16": {"p50_ms": rep_m["latency_ms"]["p50"], "p99_ms": rep_m["latency_ms"]["p99"],
                                              "value": rep_m["value"], "unit": UNIT},
                       "plain_fp32": {"p50_ms": rep_p["latency_ms"]["p50"], "p99_ms": rep_p["latency_ms"]["p99"],
                                      "value": rep_p["value"], "unit": UNIT},
                       "p99_ratio_plain_over_batched": rep_p["latency_ms"]["p99"] / max(1e-9, rep_b["latency_ms"]["p99"]),
                       "burst_peak_value": burst["value"],
                   },
                   "batched_replay": rep_b,
                   "batched_mixed_bf16_replay": rep_m,
                   "plain_fp32_replay": rep_p,
                   "burst_all_submitted_at_once": burst,
                   "batched_path": "streaming add/subtract update, up to 32 sessions per launch of the persistent kernel",
                   "batched_mixed_path": "the same with BF16 sessions: exact streaming update, drift re-sum slices "
                                         "with tcgen05 linear sums",
                   "plain_path": "one trial at a time, full-window FP32 recompute (FC_MODE_FULL), no batching",
                   "burst_note": "every trial of the trace submitted at t = 0: peak aggregate throughput; its "
                                 "latencies are queueing behind the whole burst, not the serving latency"}

    configs = None
    if world == 1 and not args.no_configs:
        torch.cuda.empty_cache()
        configs = config_legs(fc, torch, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        res = cpu_oracle_time(w, args.cpu_nodes)
        dt, pb = res[0]
        cpu = {"value": pb / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_nodes}-node subset of the workload, one full-window FP64 oracle "
                         f"evaluation (W={W} trials, {B} bins, 7 spectral metrics); the oracle has no "
                         f"streaming form, so one push costs a full window", "seconds": dt,
               "host": host_cpu()}
        if not args.no_cpu_all_core:
            nproc = cpu["host"]["nproc"]
            (dta, pba), = cpu_oracle_time(w, args.cpu_nodes, threads=nproc)
            cpu["all_core"] = {"value": pba / dta, "threads": nproc, "seconds": dta,
                               "note": "same sample; BLAS threads = nproc (the oracle's matmuls)"}

    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded AR(2) alpha sources + 200-edge coupling graph)",
        "config": {"workload": wname, "description": w["desc"], "n_nodes": n, "n_samples": N,
                   "window": W, "n_bins": B, "pairs": P, "pair_bins_per_push": units,
                   "resum_period": args.resum_period or W, "metrics": "COH,IMAGCOHY,PLV,PLI,USPLI,WPLI,DSWPLI",
                   "l2": "inputs larger than L2 (27.8 GB resident state), no flush",
                   "parallelism": f"{world} independent session(s), one per GPU"},
        "latency_ms": {"p50": p50, "p99": p99, "what": "device time from push enqueue to network ready"},
        "plain_fp32": plain, "mixed_bf16_full_window": mixed, "mixed_bf16_stream": mixed_stream,
        "mixed_tf32x3_stream": mixed_stream_split,
        "serving": serving, "configs": configs,
        "roofline": roofline, "kernels": kernel_share, "cpu_baseline": cpu, "e2e": e2e,
        "clocks": clocks.summary(), "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="large_stream", choices=sorted(WORKLOADS))
    ap.add_argument("--resum-period", type=int, default=0)
    ap.add_argument("--pool", type=int, default=128)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--cpu-nodes", type=int, default=512)
    ap.add_argument("--ref-nodes", type=int, default=96)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the EEG, MEG and source-space legs")
    ap.add_argument("--no-cpu-all-core", action="store_true")
    ap.add_argument("--sweep", action="store_true", help="print the paper-style performance sweep instead")
    ap.add_argument("--case", choices=sorted(CASES) + ["project_5124", "spectrum_methods"],
                    help="run one small named case (profiler captures)")
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    w = WORKLOADS[args.workload]
    if args.sweep:
        return run_sweep(args)
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args, w, args.workload)
    return run_ours(args, w, args.workload)


if __name__ == "__main__":
    sys.exit(main())
