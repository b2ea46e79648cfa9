#!/usr/bin/env python
"""Throughput benchmark of the GB300 FX correlator hot path.

One step = the whole hot path (F-engine: PFB + real FFT + coarse/fine delay
and phase; X-engine with integration; MAD flagging) over one synthetic
stream shaped like the four-antenna dual-pol L-band streaming workload:
8 inputs x 2^28 int8 samples, 4096 channels, 4-tap PFB, 1024-spectrum
integrations (32 per stream), sigma = 5 over 64-channel windows.

  value : input GB/s with the stream resident in HBM (corr_run_dev), timed
          with CUDA events on the launching stream; inputs (2 GiB) exceed L2.
  e2e   : the same metric through corr_push from pinned host memory in
          64 MiB chunks, plus corr_get_vis / corr_get_flags, per step.

Multi-GPU: replicas only -- each rank correlates its own stream, no
collective on the data path; value = all ranks' bytes / max rank time.
``--impl reference`` times the FP64 CPU oracle on host cores instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sustained input GB/s (PFB+X+flag, 1 GB300) vs plain FP32 path at stated vis error"

WORKLOADS = {
    "c2": dict(n_ant=4, n_pol=2, n_chan=4096, taps=4, n_int=1024, samples=1 << 28, chunk=1 << 24,
               desc="4 ant x 2 pol int8 real, 2^28 samples/input (2 GiB), 4-tap Hann-sinc PFB, "
                    "4096 ch, n_int 1024, 3 tones +20 dB, 1% bursts +10 dB, delays 0-40 smp, "
                    "MAD sigma 5 / 64 ch"),
    "c1": dict(n_ant=4, n_pol=1, n_chan=1024, taps=4, n_int=512, samples=1 << 22, chunk=1 << 22,
               desc="4 ant x 1 pol int8 real, 2^22 samples/input, 4-tap PFB, 1024 ch, n_int 512"),
    "c4": dict(n_ant=0, n_pol=2, n_chan=0, taps=4, n_int=0, samples=1 << 24, chunk=1 << 22,
               desc="8 sub-array streams (n_ant, n_chan, n_int) = " + str([(4, 512, 4096), (6, 1024, 2048),
                    (8, 2048, 1024), (12, 4096, 512), (16, 8192, 256), (24, 512, 1024), (32, 1024, 512),
                    (32, 2048, 256)]) + " x 2 pols, 2^24 int8 samples/input (4.5 GB), one captured graph, "
                    "autotuned rings vs separate ungraphed runs"),
    "c5": dict(n_ant=32, n_pol=1, n_chan=4096, taps=4, n_int=256, samples=64 * 256 * 8192, chunk=1 << 22,
               desc="32 inputs int8 real, 64 rows x 256 spectra x 8192 samples/input (4 GiB), 4-tap PFB, "
                    "4096 ch, dynamic spectra of 256-spectrum rows in 64 x 256 tiles (512 tiles), learned "
                    "flagger (5x5 conv 1-32-32-32-1, BF16 tcgen05) with MAD fallback below confidence 0.9; "
                    "noise + tones / chirps 0-30 dB + bursts 0-8 dB"),
    "c3": dict(n_ant=32, n_pol=2, n_chan=1024, taps=4, n_int=4096, samples=1 << 26, chunk=1 << 24,
               desc="32 ant x 2 pol int8 real, 2^26 samples/input (4 GiB), 4-tap PFB, 1024 ch, n_int 4096, "
                    "requantised to int8 (tensor-core X, BF16 MMA) vs the plain FP32 path"),
}

# Stages reported by corr_stage_times, their kernels, and the algorithmic bytes
# each moves per input sample (see the design notes):
#   FIR  reads 1 B int8, writes z = (y_a, y_b) as FP32: 4 B;
#   FFT  reads z (4 B) and writes one complex64 per channel per input (4 B);
#   X    reads the channelised spectra (4 B); finalise / flag: per integration.
#   requant reads the spectra (4 B) and writes one code per component (1 B
#   e4m3, 2 B int8-as-BF16); the tensor-core Gram reads the codes.
STAGES = ["fir", "fft", "xengine", "finalize", "flag", "requant", "gram"]
KERNELS = {"fir": "fir_kernel<4>", "fft": "fft_kernel<M,0>", "xengine": "xengine_kernel",
           "finalize": "finalize_kernel", "flag": "mad_flag_kernel", "requant": "requant_kernel",
           "gram": "gram_kernel (tcgen05)"}
BYTES_PER_SAMPLE = {"fir": 5.0, "fft": 8.0, "xengine": 4.0, "finalize": 0.0, "flag": 0.0, "requant": 6.0,
                    "gram": 2.0}


# DRAM read + write per input sample of a kernel, from one ncu capture of the
# same launch shape and the same kernel code (profiles/fir_fft_c2_small_ncu.md:
# fft_kernel<8192,3>, 268.5 MB read + 215.7 MB written per launch of 1024
# spectra x 4 pairs = 67.1 M samples with 256 MiB rings, cold cache).
# Reported as the roofline's `traffic` only for the workload and kernel it
# was taken on.
TRAFFIC_PER_SAMPLE = {("c2", "fft"): 484.27e6 / 67108864}


def _spec(wl, rank, samples):
    from fxsynth import config_c1, config_c2, config_c3
    from paper_2604_20640_gb300.replicas import rank_seed
    if wl == "c2":
        return config_c2(seed=rank_seed(2000, rank, 1), n_samples=samples, M=2 * WORKLOADS[wl]["n_chan"])
    if wl == "c3":
        return config_c3(seed=rank_seed(3000, rank, 1), n_samples=samples)
    return config_c1(seed=rank_seed(1000, rank, 1), n_samples=samples)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
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
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(wl, n_integrations=None):
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload:
    the first integrations of one stream (about 10-30 s of work), one thread."""
    W = WORKLOADS[wl]
    M = 2 * W["n_chan"]
    if n_integrations is None:
        n_integrations = 4
    samples = M * W["n_int"] * n_integrations
    partial = False
    if wl == "c3":
        # 64-input integrations take minutes in the oracle: time 256 spectra
        # (one partial integration; the work per sample is the same)
        samples, partial = M * 256, True
    code = (
        "import sys, time, json, numpy as np\n"
        "sys.path.insert(0, %r)\n"
        "from fxsynth import config_c1, config_c2, config_c3, make_stream\n"
        "from oracle import fx_oracle as fx\n"
        "wl = %r\n"
        "spec = (config_c2(seed=2000, n_samples=%d, M=%d) if wl == 'c2' else\n"
        "        config_c3(seed=3000, n_samples=%d) if wl == 'c3' else config_c1(seed=1000, n_samples=%d))\n"
        "x = make_stream(spec)\n"
        "t0 = time.perf_counter()\n"
        "R, F, T = fx.correlate(x, %d, %d, %d, spec.tau, spec.phi, partial=%r)\n"
        "dt = time.perf_counter() - t0\n"
        "print(json.dumps({'seconds': dt, 'bytes': int(x.size), 'n_int': int(R.shape[0])}))\n"
    ) % (ROOT, wl, samples, M, samples, samples, W["n_chan"], W["taps"], W["n_int"], partial)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["bytes"] / d["seconds"] / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "first %d spectra of one stream (%d MiB int8), FP64 numpy oracle, 1 thread, %.1f s"
                      % (samples // M, d["bytes"] >> 20, d["seconds"])}


def c4_cpu_baseline():
    """The FP64 oracle, as it stands, on the first 64 spectra of every
    sub-array stream of the batching workload (one thread), per input byte."""
    code = (
        "import sys, time, json\n"
        "sys.path.insert(0, %r)\n"
        "from fxsynth import config_c4_streams, make_stream\n"
        "from fxsynth.streams import C4_SHAPES\n"
        "from oracle import fx_oracle as fx\n"
        "secs, nbytes = 0.0, 0\n"
        "for spec, (na, nc, ni) in zip(config_c4_streams(seed=4000, n_samples=64 * 2 * 8192), C4_SHAPES):\n"
        "    spec.n_samples = 64 * 2 * nc\n"
        "    x = make_stream(spec)\n"
        "    t0 = time.perf_counter()\n"
        "    fx.correlate(x, nc, 4, ni, spec.tau, spec.phi, partial=True)\n"
        "    secs += time.perf_counter() - t0\n"
        "    nbytes += int(x.size)\n"
        "print(json.dumps({'seconds': secs, 'bytes': nbytes}))\n"
    ) % (ROOT,)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "failed"}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["bytes"] / d["seconds"] / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "first 64 spectra of each of the 8 sub-array streams (%d MiB int8), FP64 numpy "
                      "oracle, 1 thread, %.1f s" % (d["bytes"] >> 20, d["seconds"])}


def run_reference_c5(args):
    W = WORKLOADS["c5"]
    secs = []
    for i in range(args.warmup + args.steps):
        d, spb = c5_cpu_sample()
        if d is None:
            print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + spb}))
            return
        if i >= args.warmup:
            secs.append(spb)
    spb = sum(secs) / len(secs)
    val = 1.0 / spb / 1e9
    ms = spb * 32 * W["samples"] * 1e3
    sample = ("per step: dynamic spectrum of one input over 16 rows + FP64 net forward and MAD on one tile, "
              "scaled to the 32-input batch, FP64 numpy oracle, 1 thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c5: " + W["desc"], "sample": sample, "l2": "host CPU path"},
        "cpu_baseline": {"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload == "c5":
        run_reference_c5(args)
        return
    W = WORKLOADS[args.workload]
    M = 2 * W["n_chan"]
    samples = M * W["n_int"]
    code = (
        "import sys, time, json, numpy as np\n"
        "sys.path.insert(0, %r)\n"
        "from fxsynth import config_c1, config_c2, make_stream\n"
        "from oracle import fx_oracle as fx\n"
        "spec = (config_c2(seed=2000, n_samples=%d, M=%d) if %r == 'c2' else config_c1(seed=1000, n_samples=%d))\n"
        "x = make_stream(spec)\n"
        "ts = []\n"
        "for i in range(%d):\n"
        "    t0 = time.perf_counter()\n"
        "    fx.correlate(x, %d, %d, %d, spec.tau, spec.phi)\n"
        "    ts.append(time.perf_counter() - t0)\n"
        "print(json.dumps({'times': ts[%d:], 'bytes': int(x.size)}))\n"
    ) % (ROOT, samples, M, args.workload, samples, args.warmup + args.steps, W["n_chan"], W["taps"],
         W["n_int"], args.warmup)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " +
                          (r.stderr.strip().splitlines() or ["?"])[-1]}))
        return
    d = json.loads(r.stdout.strip().splitlines()[-1])
    ms = 1e3 * sum(d["times"]) / len(d["times"])
    val = d["bytes"] / (ms * 1e-3) / 1e9
    out = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + ": " + W["desc"], "sample": "one integration per step",
                   "l2": "host CPU path"},
        "cpu_baseline": {"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "one integration (%d MiB int8) per step, FP64 numpy oracle, 1 thread"
                                   % (d["bytes"] >> 20)},
        "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


TENSOR_MIN_INPUTS = 24


def run_batched(args, rank, world, local):
    """Eight uneven sub-array streams: one captured graph (autotuned) vs the
    same streams run one after another without a graph (default tuning)."""
    import tempfile
    import torch
    import torch.distributed as dist
    from paper_2604_20640_gb300 import Correlator, Group
    from paper_2604_20640_gb300.replicas import rank_seed, max_over_ranks, job_rate
    from fxsynth import config_c4_streams
    from fxsynth.streams_torch import make_stream_torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    S = args.samples or WORKLOADS["c4"]["samples"]
    specs = config_c4_streams(seed=rank_seed(4000, rank), n_samples=S)
    from fxsynth.streams import C4_SHAPES
    members, plains, xs, vis, flags, precs = [], [], [], [], [], []
    for spec, (na, nc, ni) in zip(specs, C4_SHAPES):
        # chosen form: tensor-core X-engine (int8 codes) once N is large
        prec = 1 if 2 * na >= TENSOR_MIN_INPUTS else 0
        precs.append(prec)
        c = Correlator(na, 2, nc, 4, ni, precision=prec)
        c.set_delays(spec.tau, spec.phi)
        cp = Correlator(na, 2, nc, 4, ni)
        cp.set_delays(spec.tau, spec.phi)
        x = make_stream_torch(spec, device=dev)
        n = max(1, c.n_integrations(S))
        members.append(c)
        plains.append(cp)
        xs.append(x)
        vis.append(torch.empty((n, nc, 2 * na, 2 * na), dtype=torch.complex64, device=dev))
        flags.append(torch.empty((n, nc, 2 * na, 2 * na), dtype=torch.uint8, device=dev))
    bytes_step = sum(x.numel() for x in xs)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        ms = max_over_ranks(ms, dist if world > 1 else None, dev)
        return ms

    # plain: one stream after another, no graph, default tuning
    def plain():
        for c, x, v, f in zip(plains, xs, vis, flags):
            c.run_dev(x, v, f)
    ms_plain = timed(plain, args.steps)
    # chosen: autotuned rings, one captured graph of all eight pipelines
    cache = os.path.join(tempfile.gettempdir(), "corr_tune_%d.txt" % os.getpid())
    for c, x in zip(members, xs):
        c.autotune(x, cache)
    g = Group(members)
    g.run_dev(xs, vis, flags)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    l0 = g._L.corr_kernel_launches(g._h)
    ms = timed(lambda: g.run_dev(xs, vis, flags), args.steps)
    launches = (g._L.corr_kernel_launches(g._h) - l0) * args.steps // (args.steps + args.warmup)
    clk = clocks.stop()
    value = job_rate(bytes_step, world, ms)

    # --- roofline: a captured graph carries no per-kernel events, so the
    # members run once more one by one (untimed) with every stage bracketed
    st_ms, st_n, st_bytes = [0.0] * len(STAGES), [0] * len(STAGES), [0.0] * len(STAGES)
    for c, x, v, f, prec in zip(members, xs, vis, flags, precs):
        bps = dict(BYTES_PER_SAMPLE)
        if prec == 2:
            bps.update(requant=5.0, gram=1.0)
        c.set_option("stage_timing", 1)
        c.stage_times()
        c.run_dev(x, v, f)
        m_ms, m_n = c.stage_times()
        c.set_option("stage_timing", 0)
        n_used = (x.shape[1] // c.M) * c.M * c.n_in
        for i, k in enumerate(STAGES):
            st_ms[i] += m_ms[i]
            st_n[i] += m_n[i]
            st_bytes[i] += bps[k] * n_used if m_n[i] else 0.0
    tot = sum(st_ms) or 1.0
    share = {k: st_ms[i] / tot for i, k in enumerate(STAGES)}
    di = max((i for i, k in enumerate(STAGES) if BYTES_PER_SAMPLE[k] > 0), key=lambda i: st_ms[i])
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    avg_ms = st_ms[di] / max(1, st_n[di])
    bpl = st_bytes[di] / max(1, st_n[di])
    roofline = {"kernel": KERNELS[STAGES[di]], "bound": "hbm", "achieved": bpl / (avg_ms * 1e-3) / 1e9,
                "peak": hbm, "unit": "GB/s", "frac": bpl / (avg_ms * 1e-3) / 1e9 / hbm, "traffic": None,
                "peak_source": "measured" if peaks else "fallback", "bytes_per_launch": bpl,
                "avg_launch_ms": avg_ms, "launches": st_n[di], "stage_share": share,
                "source": "members run one by one outside the graph (untimed), every stage bracketed"}

    # --- end to end: every step copies the eight streams from pinned host
    # memory into the graph's input buffers, replays the graph and reads the
    # visibilities and flags back into pinned host buffers
    e2e = None
    if not args.no_e2e:
        hosts = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in xs]
        for h, x in zip(hosts, xs):
            h.copy_(x)
        vis_h = [torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for v in vis]
        flags_h = [torch.empty(f.shape, dtype=f.dtype, pin_memory=True) for f in flags]

        def e2e_step():
            for h, x in zip(hosts, xs):
                x.copy_(h, non_blocking=True)
            g.run_dev(xs, vis, flags)
            for a, b in zip(vis_h, vis):
                a.copy_(b, non_blocking=True)
            for a, b in zip(flags_h, flags):
                a.copy_(b, non_blocking=True)
            stream.synchronize()

        for _ in range(max(1, args.warmup)):
            e2e_step()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        ems = (time.perf_counter() - t0) * 1e3 / args.steps
        ems = max_over_ranks(ems, dist if world > 1 else None, dev)
        d2h = sum(v.numel() * v.element_size() for v in vis) + sum(f.numel() for f in flags)
        e2e = {"value": job_rate(bytes_step, world, ems), "unit": "GB/s", "h2d_bytes_per_step": bytes_step,
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ems,
               "note": "copies, graph and read-back in sequence (the graph's input buffers are fixed)"}
        del hosts, vis_h, flags_h
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c4: " + WORKLOADS["c4"]["desc"], "samples_per_input": S,
                       "l2": "inputs (%d MiB/step) larger than L2" % (bytes_step >> 20),
                       "tuning": [c.tuning() for c in members],
                       "path": "one captured graph; tensor-core X (int8) for members with >= %d inputs, "
                               "CUDA-core FP32 X below" % TENSOR_MIN_INPUTS},
            "gpu_launches": int(launches), "clocks": clk, "roofline": roofline, "e2e": e2e,
            "cpu_baseline": None if args.no_cpu else c4_cpu_baseline(),
            "plain_fp32": {"value": job_rate(bytes_step, world, ms_plain), "ms_per_step": ms_plain,
                           "ratio": ms_plain / ms},
        }
        print(json.dumps(out))
    g.close()
    if world > 1:
        dist.destroy_process_group()


C5_C_MIN = 0.9
C5_TRAIN_STEPS = 1500


def c5_cpu_sample():
    """Oracle time per input byte of the flagging workload on a bounded
    sample: the dynamic spectrum of one input over 16 rows (33.5 M samples),
    then the net's FP64 forward pass and the MAD rule on one tile (a tile
    covers 8.4 M samples of one input), one thread."""
    code = (
        "import sys, time, json, numpy as np\n"
        "sys.path.insert(0, %r)\n"
        "from fxsynth.streams import StreamSpec, make_stream\n"
        "from oracle import flagnet_oracle as fn\n"
        "x = make_stream(StreamSpec(n_ant=1, n_pol=1, n_samples=16 * 256 * 8192, seed=5, src_frac=0.0))\n"
        "t0 = time.perf_counter()\n"
        "P = fn.dynamic_spectrum(x, 4096, 4, 256)\n"
        "t1 = time.perf_counter()\n"
        "tile = np.concatenate([P[0]] * 4, axis=0)[:, :256]\n"
        "z, _ = fn.forward(fn.init_params(0), fn.tile_input(tile)[None, None])\n"
        "f = fn.mad_tile_flags(tile[None])\n"
        "t2 = time.perf_counter()\n"
        "print(json.dumps({'spec_s': t1 - t0, 'spec_samples': int(x.size), 'tile_s': t2 - t1}))\n"
    ) % ROOT
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return None, (r.stderr.strip().splitlines() or ["?"])[-1]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    sec_per_byte = d["spec_s"] / d["spec_samples"] + d["tile_s"] / (64 * 256 * 8192 / 16)
    return d, sec_per_byte


def run_flagger(args, rank, world, local):
    """Dynamic spectra + learned flagger: F-engine (PFB + FFT) -> 256-spectrum
    power rows -> 64 x 256 tiles -> net (MAD on tiles below confidence 0.9)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2604_20640_gb300 import Correlator, FlagNet
    from paper_2604_20640_gb300 import flagger, train_flagnet
    from paper_2604_20640_gb300.replicas import rank_seed, max_over_ranks, job_rate
    from fxsynth.rfi_torch import RfiSpec, make_rfi_batch, noise_only

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    W = WORKLOADS["c5"]
    n_row = 256
    spec = RfiSpec(n_in=32, n_chan=W["n_chan"], n_row=n_row, seed=rank_seed(5000, rank))
    S = spec.n_samples
    # --- the net: trained here on F-engine tiles of other seeds (8-input batches)
    t_train = time.time()
    src = train_flagnet.TileSource(n_in=8, n_chan=W["n_chan"], n_row=n_row, seed=rank_seed(7000, rank), device=dev)
    net = FlagNet(train_flagnet.init_params(0))
    losses = train_flagnet.train(net, src, args.train_steps, 32, 1e-3)
    t_train = time.time() - t_train
    del src
    # --- the measured batch and its truth (held out)
    # 512 MiB rings: 256-spectrum launches (the dynamic spectra take 12.1 ms
    # per 4 GiB batch against 15.1 ms with the 64 MiB default's 32-spectrum
    # launches; no spectra ring is written in this mode)
    corr = Correlator(W["n_ant"], W["n_pol"], W["n_chan"], W["taps"], W["n_int"], ring_mb=args.ring_mb or 512)
    one = Correlator(1, 1, W["n_chan"], W["taps"], W["n_int"])
    level = flagger.noise_level(one, noise_only(spec, S, dev), n_row)
    one.close()
    b = make_rfi_batch(spec, 0, dev)
    x = b["total"]
    truth, t_nb, t_bb = flagger.truth_tiles(corr, b["nb"], b["bb"], b["g_nb"], b["g_bb"], level, n_row,
                                            train_flagnet.TRUTH_FRACTION)
    del b["nb"], b["bb"]
    power = flagger.power_tiles(corr, x, n_row)
    quality = train_flagnet.evaluate(net, power, truth, t_nb, t_bb, C5_C_MIN)
    quality.update({"train_steps": args.train_steps, "train_tiles": 32 * args.train_steps,
                    "train_seconds": round(t_train, 1),
                    "loss_first_last": [float(np.mean(losses[:10])), float(np.mean(losses[-50:]))]})
    B = power.shape[0]
    flags = torch.empty((B, 64, 256), dtype=torch.uint8, device=dev)
    conf = torch.empty(B, device=dev)
    stream = torch.cuda.current_stream(dev)

    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(max(args.steps, 1))]

    def step(i=None):
        flagger.power_tiles(corr, x, n_row, out=power)
        if i is not None:
            fev[i][0].record(stream)
        net.flag(power, flags, conf, c_min=C5_C_MIN)
        if i is not None:
            fev[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    # --- stage shares from one untimed step with every F-engine stage
    # bracketed; the timed steps bracket only the dominant kernel's launches
    corr.set_option("stage_timing", 1)
    corr.stage_times()
    step(0)
    torch.cuda.synchronize(dev)
    share_ms, _ = corr.stage_times()
    share = {k: share_ms[i] for i, k in enumerate(STAGES) if share_ms[i] > 0}
    share["flagger"] = fev[0][0].elapsed_time(fev[0][1])
    tot = sum(share.values()) or 1.0
    share = {k: v / tot for k, v in share.items()}
    dom = max((k for k in ("fir", "fft")), key=lambda k: share.get(k, 0.0))
    di = STAGES.index(dom)
    corr.set_option("stage_mask", 1 << di)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    l0 = corr.launches + net.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    launches = corr.launches + net.launches - l0
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, dist if world > 1 else None, dev)
    bytes_step = spec.n_in * S
    value = job_rate(bytes_step, world, ms)
    stage_ms, stage_n = corr.stage_times()
    corr.set_option("stage_timing", 0)
    corr.set_option("stage_mask", 127)
    flag_ms = sum(a.elapsed_time(b) for a, b in fev[:args.steps]) / max(1, args.steps)
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    bf16 = peaks.get("bf16_tflops") or 1900.0
    flops_tile = 2.0 * 64 * 256 * 25 * (1 * 32 + 32 * 32 + 32 * 32 + 32 * 1)
    n_samples_pass = bytes_step * args.steps
    # in the flagging pass the FFT reads z (4 B/sample) and keeps only the
    # powers (no spectra written)
    bps_c5 = {"fir": 5.0, "fft": 4.0}
    bytes_per_launch = bps_c5[dom] * n_samples_pass / max(1, stage_n[di])
    avg_ms = stage_ms[di] / max(1, stage_n[di])
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    kname = "fft_kernel<%d,2> (power mode)" % (2 * W["n_chan"]) if dom == "fft" else KERNELS[dom]
    roofline = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "peak_source": "measured" if peaks else "fallback",
                "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms, "launches": stage_n[di],
                "stage_share": share,
                "flagger": {"bound": "tensor", "ms": flag_ms, "tiles": B,
                            "achieved_tflops": flops_tile * B / (flag_ms * 1e-3) / 1e12, "peak": bf16,
                            "unit": "TFLOP/s", "frac": flops_tile * B / (flag_ms * 1e-3) / 1e12 / bf16,
                            "flop_per_tile": flops_tile}}
    # --- end to end: pinned host input, H2D + dynamic spectra + flagger + D2H
    # flags every step; two device input buffers let the copy of step i+1
    # overlap the processing of step i
    e2e = None
    if not args.no_e2e:
        host = torch.empty((spec.n_in, S), dtype=torch.int8, pin_memory=True)
        host.copy_(x)
        fh = torch.empty((B, 64, 256), dtype=torch.uint8, pin_memory=True)
        bufs = [x, torch.empty_like(x)]
        copy_stream = torch.cuda.Stream(dev)
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        freed = [torch.cuda.Event(), torch.cuda.Event()]
        for e in freed:
            e.record(stream)

        def e2e_steps(k):
            for i in range(k):
                b = i % 2
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(freed[b])
                    bufs[b].copy_(host, non_blocking=True)
                    copied[b].record(copy_stream)
                stream.wait_event(copied[b])
                flagger.power_tiles(corr, bufs[b], n_row, out=power)
                net.flag(power, flags, conf, c_min=C5_C_MIN)
                freed[b].record(stream)
                fh.copy_(flags, non_blocking=True)
            stream.synchronize()

        e2e_steps(max(1, args.warmup))
        t0 = time.perf_counter()
        e2e_steps(args.steps)
        ems = (time.perf_counter() - t0) * 1e3 / args.steps
        ems = max_over_ranks(ems, dist if world > 1 else None, dev)
        e2e = {"value": job_rate(bytes_step, world, ems), "unit": "GB/s",
               "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": int(fh.numel()), "ms_per_step": ems}
        del host, bufs
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            d, spb = c5_cpu_sample()
            if d is None:
                cpu = {"error": spb}
            else:
                cpu = {"value": 1.0 / spb / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                       "sample": "dynamic spectrum of one input over 16 rows (%d MiB int8, %.1f s) + FP64 net "
                                 "forward and MAD on one tile (%.1f s), scaled per input byte, 1 thread"
                                 % (d["spec_samples"] >> 20, d["spec_s"], d["tile_s"])}
        out = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
            "config": {"workload": "c5: " + W["desc"], "samples_per_input": S, "tiles": B,
                       "ring_mb": args.ring_mb or 512,
                       "l2": "inputs (%d MiB/step) larger than L2" % (bytes_step >> 20),
                       "parallelism": "replicas" if world > 1 else "single"},
            "gpu_launches": int(launches), "clocks": clk, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
            "flagger_quality": quality,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--samples", type=int, default=0, help="override samples per input")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision", type=int, default=None,
                    help="0 FP32 CUDA-core X, 1 int8 / 2 e4m3 tensor-core X (default: FP32, int8 for c3)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison run")
    ap.add_argument("--train-steps", type=int, default=C5_TRAIN_STEPS, help="c5: Adam steps before timing")
    ap.add_argument("--ring-mb", type=int, default=0, help="c1-c3: spectrum ring size (MiB, 0 = autotuned)")
    ap.add_argument("--chunk", type=int, default=0, help="c1-c3 e2e: samples per input per push (0 = workload default)")
    ap.add_argument("--bits", type=int, default=8, choices=[8, 16],
                    help="c1-c3: 16 = the 16-bit padded recorder mode (the same stream scaled to 14-bit values)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "c4":
        run_batched(args, rank, world, local)
        return
    if args.workload == "c5":
        run_flagger(args, rank, world, local)
        return

    import torch
    import torch.distributed as dist
    from paper_2604_20640_gb300 import Correlator
    from paper_2604_20640_gb300.replicas import max_over_ranks, job_rate
    from fxsynth.streams_torch import make_stream_torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    W = WORKLOADS[args.workload]
    S = args.samples or W["samples"]
    n_in = W["n_ant"] * W["n_pol"]
    spec = _spec(args.workload, rank, S)
    x = make_stream_torch(spec, device=dev)
    if args.bits == 16:
        x = x.to(torch.int16) * 64          # 14-bit values in int16 containers
    prec = args.precision if args.precision is not None else (1 if args.workload == "c3" else 0)
    ring = {"ring_mb": args.ring_mb} if args.ring_mb else {}
    c = Correlator(W["n_ant"], W["n_pol"], W["n_chan"], W["taps"], W["n_int"], precision=prec,
                   sample_bits=args.bits, **ring)
    if not args.ring_mb:
        # ring size and FIR run length from the library's autotuner (untimed)
        c.autotune(x)
    tuning = c.tuning()
    c.set_delays(spec.tau, spec.phi)
    n_intg = c.n_integrations(S)
    vis = torch.empty((n_intg, W["n_chan"], n_in, n_in), dtype=torch.complex64, device=dev)
    flags = torch.empty((n_intg, W["n_chan"], n_in, n_in), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        c.run_dev(x, vis, flags)
    torch.cuda.synchronize(dev)
    # One untimed step with every stage bracketed by events gives the stage
    # shares and the dominant kernel; the timed steps bracket only that
    # kernel's launches (fewer events disturb the pipeline less).
    bps = dict(BYTES_PER_SAMPLE)
    if args.bits == 16:
        bps["fir"] += 1.0          # the FIR reads 2 bytes per sample
    if prec == 2:
        bps.update(requant=5.0, gram=1.0)
    c.set_option("stage_timing", 1)
    c.stage_times()
    c.run_dev(x, vis, flags)
    share_ms, _ = c.stage_times()
    total_stage = sum(share_ms) or 1.0
    share = {k: share_ms[i] / total_stage for i, k in enumerate(STAGES)}
    dom = max((k for k in STAGES if bps[k] > 0), key=lambda k: share[k])
    di = STAGES.index(dom)
    c.set_option("stage_mask", 1 << di)
    barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    l0 = c.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        c.run_dev(x, vis, flags)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    launches = c.launches - l0
    ms = e0.elapsed_time(e1) / args.steps
    stage_ms, stage_n = c.stage_times()
    c.set_option("stage_timing", 0)
    c.set_option("stage_mask", 127)
    ms = max_over_ranks(ms, dist if world > 1 else None, dev)
    bytes_step = n_in * S * (args.bits // 8)
    value = job_rate(bytes_step, world, ms)

    # ---- the plain FP32 path on the same stream (the metric's denominator) ----
    plain = None
    if prec != 0 and not args.no_plain:
        cp = Correlator(W["n_ant"], W["n_pol"], W["n_chan"], W["taps"], W["n_int"], sample_bits=args.bits)
        cp.set_delays(spec.tau, spec.phi)
        for _ in range(max(1, args.warmup)):
            cp.run_dev(x, vis, flags)
        torch.cuda.synchronize(dev)
        barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            cp.run_dev(x, vis, flags)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        pms = p0.elapsed_time(p1) / args.steps
        pms = max_over_ranks(pms, dist if world > 1 else None, dev)
        pval = job_rate(bytes_step, world, pms)
        plain = {"value": pval, "ms_per_step": pms, "ratio": value / pval}
        cp.close()

    # ---- end to end through the public host API ----
    e2e = None
    if not args.no_e2e:
        # The host issues every launch of the push path, once per ring pass,
        # so it takes a ring of at least 128 MiB whatever the device-resident
        # tuning chose (small rings make the pushes launch-bound).
        ring_e2e = args.ring_mb or max(tuning[0], 128)
        ce = Correlator(W["n_ant"], W["n_pol"], W["n_chan"], W["taps"], W["n_int"], chunk=args.chunk or W["chunk"],
                        precision=prec, sample_bits=args.bits, ring_mb=ring_e2e, fir_spt=tuning[1])
        ce.set_delays(spec.tau, spec.phi)
        host = torch.empty((n_in, S), dtype=x.dtype, pin_memory=True)
        host.copy_(x)
        chunk = args.chunk or W["chunk"]
        # results land by DMA in pinned buffers the loop reuses
        vis_h = torch.empty((n_intg + 1, W["n_chan"], n_in, n_in), dtype=torch.complex64, pin_memory=True)
        flags_h = torch.empty((n_intg + 1, W["n_chan"], n_in, n_in), dtype=torch.uint8, pin_memory=True)

        phase = [0.0, 0.0]          # host seconds in the pushes / in flush + pops

        def e2e_step():
            ta = time.perf_counter()
            for p in range(0, S, chunk):
                ce.push(host[:, p:p + chunk])
            tb = time.perf_counter()
            ce.flush()
            v = ce.get_vis(out=vis_h)
            f = ce.get_flags(out=flags_h)
            assert v.shape[0] == f.shape[0] >= n_intg
            ce.reset()
            phase[0] += tb - ta
            phase[1] += time.perf_counter() - tb
            return v, f

        for _ in range(max(1, args.warmup)):
            e2e_step()
        barrier()
        phase[:] = [0.0, 0.0]
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v, f = e2e_step()
        t1 = time.perf_counter()
        barrier()
        ems = (t1 - t0) * 1e3 / args.steps
        ems = max_over_ranks(ems, dist if world > 1 else None, dev)
        e2e = {"value": job_rate(bytes_step, world, ems), "unit": "GB/s", "ring_mb": ring_e2e,
               "h2d_bytes_per_step": bytes_step,
               "d2h_bytes_per_step": int(v.numel() * v.element_size() + f.numel() * f.element_size()),
               "ms_per_step": ems, "push_ms": phase[0] * 1e3 / args.steps,
               "flush_pop_ms": phase[1] * 1e3 / args.steps}
        ce.close()
        del host

    # ---- roofline of the dominant kernel, from the live per-stage events ----
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    n_spec = S // (2 * W["n_chan"])
    samples_timed = args.steps * n_spec * 2 * W["n_chan"] * n_in
    bytes_per_launch = bps[dom] * samples_timed / max(1, stage_n[di])
    avg_ms = stage_ms[di] / max(1, stage_n[di])
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    tps = TRAFFIC_PER_SAMPLE.get((args.workload, dom))
    traffic = tps * samples_timed / max(1, stage_n[di]) if tps and prec == 0 else None
    kname = KERNELS[dom]
    if dom == "fft":
        # mode 3: spectra ring pair-major (FP32 path with n_in_pad <= 8); 0: channel-major
        kname = "fft_kernel<%d,%d>" % (2 * W["n_chan"], 3 if prec == 0 and (n_in + 3) // 4 * 4 <= 8 else 0)
    roofline = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src,
                "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms, "launches": stage_n[di],
                "stage_share": share}

    if rank == 0:
        cpu = None if args.no_cpu else cpu_baseline(args.workload)
        out = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload + ": " + W["desc"],
                       "path": ["plain FP32 (CUDA-core X)", "int8 requantised, tcgen05 X (BF16 MMA)",
                                "e4m3 requantised, tcgen05 X"][prec],
                       "samples_per_input": S, "sample_bits": args.bits,
                       "tuning": {"ring_mb": tuning[0], "fir_spt": tuning[1]},
                       "l2": "inputs (%d MiB/step) larger than L2" % (bytes_step >> 20),
                       "parallelism": "replicas" if world > 1 else "single"},
            "gpu_launches": launches, "clocks": clk, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
        }
        if plain is not None:
            out["plain_fp32"] = plain
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
