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

# Stages reported by corr_stage_times and their kernels.
STAGES = ["fir", "fft", "xengine", "finalize", "flag", "requant", "gram"]
KERNELS = {"fir": "fir_kernel<4>", "fft": "fft_kernel<M,3>", "xengine": "xengine_kernel",
           "finalize": "finalize_kernel", "flag": "mad_flag_kernel", "requant": "words_from_spectra_kernel",
           "gram": "gram_w_kernel (tcgen05 over the F-engine's code words, visibilities in its epilogue)"}
# Algorithmic bytes per input sample of each hot-path kernel, in the unit the
# scope table's measurement section fixes: the whole hot path (PFB, FFT,
# delays, X-engine, flagging) reads each int8 input sample once (1 B); on the
# reduced-precision path the F-engine also writes one code per real sample
# (1 B) and the tensor-core X-engine reads it back.  Every kernel of a stage
# is credited with the bytes of the samples it processes.
ALG_BYTES_PER_SAMPLE = {"fir": 1.0, "fft": 1.0, "xengine": 1.0, "finalize": 0.0, "flag": 0.0,
                        "requant": 1.0, "gram": 1.0}
# Bytes each kernel of this build actually moves per input sample, rings
# included (FIR: 1 B in + 4 B of z = (y_a, y_b) out; FFT: 4 B of z in + one
# complex64 per channel per input out; X-engine: the spectra back in;
# requantiser (a stream's first ring fill): spectra in, one 1-byte code
# (int8 or e4m3) per sample out as code words; Gram: the codes).
# Reported beside the algorithmic figure, not used for it.
INTERMEDIATE_BYTES_PER_SAMPLE = {"fir": 5.0, "fft": 8.0, "xengine": 4.0, "finalize": 0.0, "flag": 0.0,
                                 "requant": 5.0, "gram": 1.0}


# DRAM read + write per input sample of a kernel, from one ncu capture of the
# same launch shape and the same kernel code (profiles/fused_fengine_c2_ncu.md:
# pfb_fft_kernel<8192,3,4>, 74.8 MB read + 206.9 MB written per launch of
# 1024 spectra x 4 pairs = 67.1 M samples with 256 MiB rings, cold cache).
# Reported as the roofline's `traffic` only for the workload and kernel it
# was taken on.
TRAFFIC_PER_SAMPLE = {("c2", "fused"): 281.71e6 / 67108864}

# Inputs below this size are timed step by step with L2 flushed in between
# (L2 is 129 MB on a GB300; twice that is written).
L2_FLUSH_BYTES = 256 << 20


def _spec(wl, rank, samples):
    from fxsynth import config_c1, config_c2, config_c3
    from paper_2604_20640_gb300.replicas import rank_seed
    if wl == "c2":
        return config_c2(seed=rank_seed(2000, rank, 1), n_samples=samples, M=2 * WORKLOADS[wl]["n_chan"])
    if wl == "c3":
        return config_c3(seed=rank_seed(3000, rank, 1), n_samples=samples)
    return config_c1(seed=rank_seed(1000, rank, 1), n_samples=samples)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms; the
    constructor returns once the first sample is in, so the samples cover
    the region timed after it."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.p.poll() is None:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)
        self.n0 = 0
        try:
            self.n0 = len(open(self.f.name).read().strip().splitlines())
        except OSError:
            pass

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        lines = open(self.f.name).read().strip().splitlines()
        # samples taken after the first one (the timed region started then)
        rows = [r.split(",") for r in lines[max(0, getattr(self, "n0", 0) - 1):] if r.strip()]
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


def _oracle_job(job):
    """One unit of oracle work in a spawned worker (the oracle runs only
    here, on the host cores, never on the product path).

    ("integration", path, i, n_chan, taps, n_int, tau, phi, compare):
        fx.correlate on the samples integration i of the stream reads (one
        extra frame behind it for the coarse advance), timed; with compare =
        (vis, flags) of the GPU for integration 0, also the visibility error
        (max relative Frobenius per channel) and the flags that differ
        outside the 1e-4 T band.
    ("rho", path, f_lo, s0, s1, n_chan, taps, tau, phi, inputs, chans, vis):
        normalised coefficients of spectra [s0, s1) on the sampled inputs and
        channels from the oracle F-engine over the slice the spectra read
        (frames f_lo ...); returns max |rho_gpu - rho_oracle|.
    """
    import numpy as np
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import fx_oracle as fx
    kind = job[0]
    if kind == "integration":
        _, path, i, n_chan, taps, n_int, tau, phi, compare = job
        M = 2 * n_chan
        x = np.load(path, mmap_mode="r")
        xs = np.ascontiguousarray(x[:, i * n_int * M:(i + 1) * n_int * M + M])
        t0 = time.perf_counter()
        R, F, T = fx.correlate(xs, n_chan, taps, n_int, tau, phi)
        dt = time.perf_counter() - t0
        out = {"seconds": dt, "bytes": int(n_int * M * xs.shape[0])}
        if compare is not None:
            vis, flags = compare
            err = fx.rel_frobenius_per_channel(vis[None].astype(np.complex128), R[:1])
            A = np.abs(R[:1])
            bad = (flags[None] != F[:1]) & ~(np.abs(A - T[:1]) < 1e-4 * T[:1])
            out.update({"vis_rel_frobenius_max": float(err.max()), "flags_differing_outside_band": int(bad.sum()),
                        "flags_set": int(F[:1].sum())})
        return out
    if kind == "c5sample":
        # the flagging workload's oracle on a bounded sample: the dynamic
        # spectrum of one input over 16 rows, then the net's FP64 forward
        # pass and the MAD rule on one tile
        from fxsynth.streams import StreamSpec, make_stream
        from oracle import flagnet_oracle as fn
        x = make_stream(StreamSpec(n_ant=1, n_pol=1, n_samples=16 * 256 * 8192, seed=5 + job[1], src_frac=0.0))
        t0 = time.perf_counter()
        P = fn.dynamic_spectrum(x, 4096, 4, 256)
        t1 = time.perf_counter()
        tile = np.concatenate([P[0]] * 4, axis=0)[:, :256]
        fn.forward(fn.init_params(0), fn.tile_input(tile)[None, None])
        fn.mad_tile_flags(tile[None])
        t2 = time.perf_counter()
        return {"spec_s": t1 - t0, "spec_samples": int(x.size), "tile_s": t2 - t1}
    if kind == "c4stream":
        # the first 64 spectra of sub-array stream i of the batching workload
        from fxsynth import config_c4_streams, make_stream
        from fxsynth.streams import C4_SHAPES
        i = job[1]
        spec = config_c4_streams(seed=4000, n_samples=64 * 2 * 8192)[i]
        na, nc, ni = C4_SHAPES[i]
        spec.n_samples = 64 * 2 * nc
        x = make_stream(spec)
        t0 = time.perf_counter()
        fx.correlate(x, nc, 4, ni, spec.tau, spec.phi, partial=True)
        return {"seconds": time.perf_counter() - t0, "bytes": int(x.size)}
    if kind == "rho":
        _, path, f_lo, s0, s1, n_chan, taps, tau, phi, inputs, chans, vis = job
        x = np.load(path, mmap_mode="r")
        V = []
        for a in inputs:
            Va = fx.f_engine(np.ascontiguousarray(x[a:a + 1]), n_chan, taps, tau[a:a + 1], phi[a:a + 1])[0]
            V.append(Va[s0 - f_lo:s1 - f_lo][:, chans])
        V = np.stack(V)
        R = np.einsum('ask,bsk->kab', V, V.conj()) / (s1 - s0)
        rho_o = fx.normalised_coefficients(R)
        rho_g = fx.normalised_coefficients(vis.astype(np.complex128))
        return {"rho_abs_err_max": float(np.abs(rho_g - rho_o).max())}
    raise ValueError(kind)


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_pool(n):
    """Spawned workers with one BLAS/OpenMP thread each (spawn, so that no
    worker inherits a CUDA context)."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    return mp.get_context("spawn").Pool(n)


def _save_host(x_dev, lo, hi):
    """Samples [lo, hi) of every input of a device stream, saved for the
    oracle workers; returns the file path."""
    import numpy as np
    f = tempfile.NamedTemporaryFile(suffix=".npy", delete=False)
    f.close()
    np.save(f.name, x_dev[:, lo:hi].cpu().numpy())
    return f.name


def oracle_leg(wl, x_dev, spec, vis0, flags0):
    """CPU baseline and visibility / flag error of a single-stream workload.

    The FP64 oracle, as it stands, on the first integrations of the timed
    stream itself: one integration on one thread (which also gives the error
    of the GPU's integration 0), then one integration per host core at once
    (throughput of all cores).  The 64-input workload's integrations take
    minutes in the oracle's O(N^2 T) correlation, so it times a 256-spectrum
    partial integration instead and takes no error here."""
    import numpy as np
    W = WORKLOADS[wl]
    M, n_int = 2 * W["n_chan"], W["n_int"]
    cores = _host_cores()
    n_avail = x_dev.shape[1] // (n_int * M)
    tau, phi = np.asarray(spec.tau, np.float64), np.asarray(spec.phi, np.float64)
    if wl == "c3":
        n_int_s = 256
        path = _save_host(x_dev, 0, n_int_s * M + M)
        pool = _oracle_pool(cores)
        try:
            one = pool.apply(_oracle_job, (("integration", path, 0, W["n_chan"], W["taps"], n_int_s, tau, phi, None),))
            t0 = time.perf_counter()
            outs = pool.map(_oracle_job, [("integration", path, 0, W["n_chan"], W["taps"], n_int_s, tau, phi, None)]
                            * cores, chunksize=1)
            wall = time.perf_counter() - t0
        finally:
            pool.close()
            pool.join()
            os.unlink(path)
        return {"value": sum(o["bytes"] for o in outs) / wall / 1e9, "unit": "GB/s", "cores": cores,
                "kind": "oracle", "value_1_core": one["bytes"] / one["seconds"] / 1e9,
                "sample": "first 256 spectra of the timed stream (%d MiB int8) per core, %d cores at once "
                          "(%.1f s wall); FP64 numpy oracle, one thread per process" % (one["bytes"] >> 20, cores, wall)}, None
    n_par = max(1, min(cores, n_avail))
    path = _save_host(x_dev, 0, min(x_dev.shape[1], n_par * n_int * M + M))
    pool = _oracle_pool(n_par)
    try:
        cmp = (vis0, flags0)
        one = pool.apply(_oracle_job, (("integration", path, 0, W["n_chan"], W["taps"], n_int, tau, phi, cmp),))
        t0 = time.perf_counter()
        outs = pool.map(_oracle_job, [("integration", path, i, W["n_chan"], W["taps"], n_int, tau, phi, None)
                                      for i in range(n_par)], chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
        os.unlink(path)
    cpu = {"value": sum(o["bytes"] for o in outs) / wall / 1e9, "unit": "GB/s", "cores": n_par, "kind": "oracle",
           "value_1_core": one["bytes"] / one["seconds"] / 1e9,
           "sample": "integrations 0-%d of the timed stream (%d MiB int8 each), one per process on %d host "
                     "cores at once (%.1f s wall; one integration on one core: %.1f s); FP64 numpy oracle"
                     % (n_par - 1, one["bytes"] >> 20, n_par, wall, one["seconds"])}
    err = {"integration": 0, "vis_rel_frobenius_max": one["vis_rel_frobenius_max"], "vis_bar": 1e-5,
           "flags_differing_outside_band": one["flags_differing_outside_band"], "flags_set": one["flags_set"],
           "flag_band": "|A - T| < 1e-4 T"}
    return cpu, err


def e4m3_vis(args, x, spec):
    """Visibilities of the 64-input workload's stream through the e4m3
    pipeline (one untimed run, autotuned like the timed one)."""
    import torch
    from paper_2604_20640_gb300 import Correlator
    W = WORKLOADS["c3"]
    n_in = W["n_ant"] * W["n_pol"]
    c = Correlator(W["n_ant"], W["n_pol"], W["n_chan"], W["taps"], W["n_int"], precision=2,
                   **({"ring_mb": args.ring_mb} if args.ring_mb else {}))
    if not args.ring_mb:
        c.autotune(x)
    c.set_delays(spec.tau, spec.phi)
    n = c.n_integrations(x.shape[1])
    vis = torch.empty((n, W["n_chan"], n_in, n_in), dtype=torch.complex64, device=x.device)
    flags = torch.empty((n, W["n_chan"], n_in, n_in), dtype=torch.uint8, device=x.device)
    c.run_dev(x, vis, flags)
    torch.cuda.synchronize()
    c.close()
    return vis


def rho_error(x_dev, spec, n_chan, taps, n_int, vis_dev, ints, n_inputs=16, chans=(0, 3, 100, 511, 512, 900, 1023)):
    """max |rho_gpu - rho_oracle| on the first n_inputs inputs and sampled
    channels of the given integrations, from the oracle F-engine over the
    slice of the timed stream each integration reads (spawned workers)."""
    import numpy as np
    M = 2 * n_chan
    tau, phi = np.asarray(spec.tau, np.float64), np.asarray(spec.phi, np.float64)
    inputs = list(range(n_inputs))
    chans = [c for c in chans if c < n_chan]
    jobs, paths = [], []
    for i in ints:
        s0, s1 = i * n_int, (i + 1) * n_int
        f_lo = max(0, s0 - taps)
        path = _save_host(x_dev[:n_inputs], f_lo * M, min(x_dev.shape[1], (s1 + 2) * M))
        paths.append(path)
        vis = vis_dev[i, chans][:, :n_inputs, :n_inputs].cpu().numpy()
        jobs.append(("rho", path, f_lo, s0, s1, n_chan, taps, tau, phi, inputs, chans, vis))
    pool = _oracle_pool(len(jobs))
    try:
        outs = pool.map(_oracle_job, jobs, chunksize=1)
    finally:
        pool.close()
        pool.join()
        for p in paths:
            os.unlink(p)
    return {"integrations": list(ints), "inputs": n_inputs, "channels": chans,
            "rho_abs_err_max": max(o["rho_abs_err_max"] for o in outs), "rho_bar": 5e-3}


def c4_cpu_baseline():
    """The FP64 oracle, as it stands, on the first 64 spectra of every
    sub-array stream of the batching workload, per input byte: the eight
    streams spread over one process per host core (each stream at least
    once), and the one-core figure from each job's own time."""
    cores = _host_cores()
    jobs = [("c4stream", i % 8) for i in range(max(8, cores))]
    pool = _oracle_pool(min(cores, len(jobs)))
    try:
        t0 = time.perf_counter()
        outs = pool.map(_oracle_job, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    nbytes = sum(o["bytes"] for o in outs)
    secs = sum(o["seconds"] for o in outs)
    return {"value": nbytes / wall / 1e9, "unit": "GB/s", "cores": min(cores, len(jobs)), "kind": "oracle",
            "value_1_core": nbytes / secs / 1e9,
            "sample": "first 64 spectra of each of the 8 sub-array streams, %d jobs (%d MiB int8) on %d host "
                      "cores at once (%.1f s wall); FP64 numpy oracle"
                      % (len(jobs), nbytes >> 20, min(cores, len(jobs)), wall)}


def run_reference_c5(args):
    W = WORKLOADS["c5"]
    vals = []
    cores = 1
    for i in range(args.warmup + args.steps):
        d, spb, all_gbs, cores = c5_cpu_sample()
        if d is None:
            print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + spb}))
            return
        if i >= args.warmup:
            vals.append(all_gbs)
    val = sum(vals) / len(vals)
    ms = 32 * W["samples"] / (val * 1e9) * 1e3
    sample = ("per step and host core at once: dynamic spectrum of one input over 16 rows + FP64 net forward "
              "and MAD on one tile, scaled to the 32-input batch, FP64 numpy oracle, one thread per process")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "c5: " + W["desc"], "sample": sample, "l2": "host CPU path"},
        "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    Each step correlates one integration of the workload's stream per host
    core, all cores at once (one process each, one BLAS thread each)."""
    if rank != 0:
        return
    if args.workload == "c5":
        run_reference_c5(args)
        return
    import numpy as np
    from fxsynth import config_c1, config_c2, config_c3, make_stream
    wl = args.workload if args.workload in ("c1", "c2", "c3") else "c2"
    W = WORKLOADS[wl]
    M = 2 * W["n_chan"]
    n_int = W["n_int"] if wl != "c3" else 256
    samples = M * n_int + M
    spec = (config_c2(seed=2000, n_samples=samples, M=M) if wl == "c2" else
            config_c3(seed=3000, n_samples=samples) if wl == "c3" else config_c1(seed=1000, n_samples=samples))
    x = make_stream(spec)
    f = tempfile.NamedTemporaryFile(suffix=".npy", delete=False)
    f.close()
    np.save(f.name, x)
    cores = _host_cores()
    tau, phi = np.asarray(spec.tau, np.float64), np.asarray(spec.phi, np.float64)
    job = ("integration", f.name, 0, W["n_chan"], W["taps"], n_int, tau, phi, None)
    try:
        pool = _oracle_pool(cores)
        try:
            walls, nbytes = [], 0
            for i in range(args.warmup + args.steps):
                t0 = time.perf_counter()
                outs = pool.map(_oracle_job, [job] * cores, chunksize=1)
                if i >= args.warmup:
                    walls.append(time.perf_counter() - t0)
                nbytes = sum(o["bytes"] for o in outs)
        finally:
            pool.close()
            pool.join()
    except Exception as e:            # the arm reports, it does not crash the driver
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: %s" % e}))
        return
    finally:
        os.unlink(f.name)
    ms = 1e3 * sum(walls) / len(walls)
    val = nbytes / (ms * 1e-3) / 1e9
    sample = ("per step: one %s (%d MiB int8) per host core, %d cores at once, FP64 numpy oracle, one thread "
              "per process" % ("integration" if wl != "c3" else "256-spectrum partial integration",
                               (nbytes // cores) >> 20, cores))
    out = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl + ": " + W["desc"], "sample": sample, "l2": "host CPU path"},
        "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
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
        prec = 1 if 2 * na >= args.tensor_min_inputs else 0
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

    # plain: one FP32 stream after another, no graph, each at its own
    # autotuned ring (the same tuning step the chosen form gets)
    cache_plain = os.path.join(tempfile.gettempdir(), "corr_tune_plain_%d.txt" % os.getpid())
    for c, x in zip(plains, xs):
        c.autotune(x, cache_plain)

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
    st_flops = [0.0] * len(STAGES)
    fused_m, plain_m = [], []
    for c, x, v, f, prec in zip(members, xs, vis, flags, precs):
        bps = dict(ALG_BYTES_PER_SAMPLE)
        c.set_option("stage_timing", 1)
        c.stage_times()
        c.run_dev(x, v, f)
        m_ms, m_n = c.stage_times()
        c.set_option("stage_timing", 0)
        n_used = (x.shape[1] // c.M) * c.M * c.n_in
        fused_c = m_n[STAGES.index("fir")] == 0       # the fused F-engine runs no FIR launches
        (fused_m if fused_c else plain_m).append(c.M)
        for i, k in enumerate(STAGES):
            st_ms[i] += m_ms[i]
            st_n[i] += m_n[i]
            st_bytes[i] += bps[k] * n_used if m_n[i] else 0.0
            st_flops[i] += flops_per_sample(k, fused_c, c.M, c.taps, c.n_in) * n_used if m_n[i] else 0.0
    tot = sum(st_ms) or 1.0
    share = {k: st_ms[i] / tot for i, k in enumerate(STAGES)}
    di = max((i for i, k in enumerate(STAGES) if ALG_BYTES_PER_SAMPLE[k] > 0), key=lambda i: st_ms[i])
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    avg_ms = st_ms[di] / max(1, st_n[di])
    bpl = st_bytes[di] / max(1, st_n[di])
    inter = sum(INTERMEDIATE_BYTES_PER_SAMPLE[STAGES[di]] * (x.shape[1] // c.M) * c.M * c.n_in
                for c, x in zip(members, xs)) / max(1, st_n[di])
    kname = KERNELS[STAGES[di]]
    if STAGES[di] == "fft":
        kname = "; ".join(["pfb_fft_kernel<M,3,4> (fused PFB + FFT, M = %s)" % sorted(set(fused_m))]
                          * bool(fused_m) +
                          ["fft_kernel<M,3> after fir_kernel (M = %s)" % sorted(set(plain_m))] * bool(plain_m))
    roofline = {"kernel": kname, "bound": "hbm", "achieved": bpl / (avg_ms * 1e-3) / 1e9,
                "bytes_per_sample": ALG_BYTES_PER_SAMPLE[STAGES[di]], "intermediate_bytes_per_launch": inter,
                "peak": hbm, "unit": "GB/s", "frac": bpl / (avg_ms * 1e-3) / 1e9 / hbm, "traffic": None,
                "peak_source": "measured" if peaks else "fallback", "bytes_per_launch": bpl,
                "avg_launch_ms": avg_ms, "launches": st_n[di], "stage_share": share,
                "source": "members run one by one outside the graph (untimed), every stage bracketed"}
    if st_flops[di] > 0:
        fp = fp32_peak()
        tf = st_flops[di] / (st_ms[di] * 1e-3) / 1e12
        alu = {"achieved": tf, "peak": fp["scalar"], "unit": "TFLOP/s", "frac": tf / fp["scalar"],
               "flop_per_sample_avg": st_flops[di] / max(1.0, st_bytes[di] / ALG_BYTES_PER_SAMPLE[STAGES[di]]),
               "peak_source": "measured (corr_peak_fp32, scalar FMA chains)"}
        if alu["frac"] > roofline["frac"]:
            hbm_part = {k: roofline[k] for k in ("achieved", "peak", "unit", "frac", "peak_source")}
            roofline.update({k: alu[k] for k in ("achieved", "peak", "unit", "frac", "peak_source")})
            roofline.update(bound="alu", hbm=hbm_part, alu={"flop_per_sample_avg": alu["flop_per_sample_avg"]})
        else:
            roofline["alu"] = alu

    # --- end to end: every step copies the eight streams from pinned host
    # memory, runs the group and reads the visibilities and flags back into
    # pinned host memory.  Two groups (two member sets with their own input
    # and result buffers, tuned alike) alternate, so one step's host->device
    # copies and the previous step's read-back run on copy streams while the
    # other group's graph runs.
    e2e = None
    if not args.no_e2e:
        sets = [(g, xs, vis, flags)]
        members_b = []
        for spec, (na, nc, ni), prec in zip(specs, C4_SHAPES, precs):
            c = Correlator(na, 2, nc, 4, ni, precision=prec)
            c.set_delays(spec.tau, spec.phi)
            members_b.append(c)
        for c, x in zip(members_b, xs):
            c.autotune(x, cache)
        xs_b = [torch.empty_like(x) for x in xs]
        vis_b = [torch.empty_like(v) for v in vis]
        flags_b = [torch.empty_like(f) for f in flags]
        g_b = Group(members_b)
        sets.append((g_b, xs_b, vis_b, flags_b))
        hosts = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in xs]
        for h, x in zip(hosts, xs):
            h.copy_(x)
        res_h = [([torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for v in vis],
                  [torch.empty(f.shape, dtype=f.dtype, pin_memory=True) for f in flags]) for _ in range(2)]
        h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        for b in range(2):
            ev_done[b].record(stream)
            ev_out[b].record(stream)

        def e2e_steps(k):
            for i in range(k):
                b = i % 2
                gb, xb, vb, fb = sets[b]
                with torch.cuda.stream(h2d):
                    h2d.wait_event(ev_done[b])            # this set's last run has read its inputs
                    for h, x in zip(hosts, xb):
                        x.copy_(h, non_blocking=True)
                    ev_in[b].record(h2d)
                stream.wait_event(ev_in[b])
                stream.wait_event(ev_out[b])              # this set's last results are read out
                gb.run_dev(xb, vb, fb, stream=stream)
                ev_done[b].record(stream)
                with torch.cuda.stream(d2h):
                    d2h.wait_event(ev_done[b])
                    for a, v in zip(res_h[b][0], vb):
                        a.copy_(v, non_blocking=True)
                    for a, f in zip(res_h[b][1], fb):
                        a.copy_(f, non_blocking=True)
                    ev_out[b].record(d2h)
            torch.cuda.synchronize(dev)

        e2e_steps(max(2, args.warmup))
        reps = []
        for _ in range(3):      # median of three windows (the host's copies vary)
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            e2e_steps(args.steps)
            reps.append((time.perf_counter() - t0) * 1e3 / args.steps)
        ems = sorted(reps)[1]
        ems = max_over_ranks(ems, dist if world > 1 else None, dev)
        ok = all(torch.equal(a, b) for a, b in zip(vis, vis_b)) and all(torch.equal(a, b) for a, b in zip(flags, flags_b))
        d2h_bytes = sum(v.numel() * v.element_size() for v in vis) + sum(f.numel() for f in flags)
        e2e = {"value": job_rate(bytes_step, world, ems), "unit": "GB/s", "h2d_bytes_per_step": bytes_step,
               "d2h_bytes_per_step": int(d2h_bytes), "ms_per_step": ems,
               "note": "two groups alternate: copies in, graph, read-back overlapped across steps",
               "sets_agree": bool(ok), "repetitions_ms_per_step": [round(r, 3) for r in reps]}
        g_b.close()
        for c in members_b:
            c.close()
        del hosts, res_h, xs_b, vis_b, flags_b
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c4: " + WORKLOADS["c4"]["desc"], "samples_per_input": S,
                       "l2": "inputs (%d MiB/step) larger than L2" % (bytes_step >> 20),
                       "tuning": [c.tuning() for c in members],
                       "path": "one captured graph; tensor-core X (int8) for members with >= %d inputs, "
                               "CUDA-core FP32 X below" % args.tensor_min_inputs},
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
    covers 8.4 M samples of one input).  Returns (the first job's figures,
    its seconds per byte, the throughput of one job per host core run at
    once in GB/s, the cores)."""
    cores = _host_cores()
    pool = _oracle_pool(cores)
    tile_bytes = 64 * 256 * 8192 / 16
    try:
        t0 = time.perf_counter()
        outs = pool.map(_oracle_job, [("c5sample", i) for i in range(cores)], chunksize=1)
        wall = time.perf_counter() - t0
    except Exception as e:   # noqa: BLE001 -- reported in the line instead
        return None, str(e), None, cores
    finally:
        pool.close()
        pool.join()
    spb = [o["spec_s"] / o["spec_samples"] + o["tile_s"] / tile_bytes for o in outs]
    # bytes each job covered: its seconds over its seconds per byte
    done = sum((o["spec_s"] + o["tile_s"]) / b for o, b in zip(outs, spb))
    return outs[0], spb[0], done / wall / 1e9, cores


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
    # algorithmic: each input sample read once (1 B); this build's kernels
    # move more: the FIR writes z (4 B/sample), the FFT reads it back and
    # keeps only the powers (no spectra written)
    bps_c5 = {"fir": 5.0, "fft": 4.0}
    bytes_per_launch = ALG_BYTES_PER_SAMPLE[dom] * n_samples_pass / max(1, stage_n[di])
    avg_ms = stage_ms[di] / max(1, stage_n[di])
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    fused = dom == "fft" and share.get("fir", 0.0) == 0.0
    M = 2 * W["n_chan"]
    kname = (("pfb_fft_kernel<%d,2,%d> (fused PFB + FFT, power mode)" % (M, W["taps"])) if fused else
             ("fft_kernel<%d,2> (power mode)" % M)) if dom == "fft" else KERNELS[dom]
    if fused:
        bps_c5["fft"] = 1.0              # samples in; powers accumulate into the tiles
    fl = flops_per_sample(dom, fused, M, W["taps"], spec.n_in)
    fp = fp32_peak()
    tf = fl * n_samples_pass / max(1, stage_n[di]) / (avg_ms * 1e-3) / 1e12
    roofline = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "peak_source": "measured" if peaks else "fallback",
                "bytes_per_launch": bytes_per_launch, "bytes_per_sample": ALG_BYTES_PER_SAMPLE[dom],
                "intermediate_bytes_per_launch": bps_c5[dom] * n_samples_pass / max(1, stage_n[di]),
                "avg_launch_ms": avg_ms, "launches": stage_n[di], "stage_share": share,
                "alu": {"achieved": tf, "peak": fp["scalar"], "unit": "TFLOP/s", "frac": tf / fp["scalar"],
                        "flop_per_sample": fl, "peak_source": "measured (corr_peak_fp32, scalar FMA chains)"},
                "flagger": {"bound": "tensor", "ms": flag_ms, "tiles": B,
                            "achieved_tflops": flops_tile * B / (flag_ms * 1e-3) / 1e12, "peak": bf16,
                            "unit": "TFLOP/s", "frac": flops_tile * B / (flag_ms * 1e-3) / 1e12 / bf16,
                            "flop_per_tile": flops_tile}}
    if roofline["alu"]["frac"] > roofline["frac"]:
        hbm_part = {k: roofline[k] for k in ("achieved", "peak", "unit", "frac", "peak_source")}
        alu = roofline.pop("alu")
        roofline.update({"bound": "alu", "achieved": alu["achieved"], "peak": alu["peak"], "unit": "TFLOP/s",
                         "frac": alu["frac"], "peak_source": alu["peak_source"], "hbm": hbm_part,
                         "flop_per_sample": alu["flop_per_sample"]})
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
        reps = []
        for _ in range(3):      # median of three windows (the host's copies vary)
            t0 = time.perf_counter()
            e2e_steps(args.steps)
            reps.append((time.perf_counter() - t0) * 1e3 / args.steps)
        ems = sorted(reps)[1]
        ems = max_over_ranks(ems, dist if world > 1 else None, dev)
        e2e = {"value": job_rate(bytes_step, world, ems), "unit": "GB/s",
               "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": int(fh.numel()), "ms_per_step": ems,
               "repetitions_ms_per_step": [round(r, 3) for r in reps]}
        del host, bufs
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            d, spb, all_gbs, cores = c5_cpu_sample()
            if d is None:
                cpu = {"error": spb}
            else:
                cpu = {"value": all_gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                       "value_1_core": 1.0 / spb / 1e9,
                       "sample": "per host core at once: the dynamic spectrum of one input over 16 rows (%d MiB "
                                 "int8, %.1f s) + FP64 net forward and MAD on one tile (%.1f s), scaled per input "
                                 "byte; FP64 numpy oracle, one thread per process"
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
    ap.add_argument("--tensor-min-inputs", type=int, default=TENSOR_MIN_INPUTS,
                    help="c4: members with at least this many inputs use the tensor-core X-engine (int8)")
    ap.add_argument("--no-e4m3", action="store_true",
                    help="c3 at int8: skip the timed e4m3 run beside it (its error is still reported)")
    ap.add_argument("--no-chosen", action="store_true",
                    help="c2: skip the 64-input tensor-core form added to the line (chosen_form)")
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
    from paper_2604_20640_gb300.replicas import max_over_ranks, job_rate
    from fxsynth.streams_torch import make_stream_torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    wl = args.workload
    W = WORKLOADS[wl]
    S = args.samples or W["samples"]
    n_in = W["n_ant"] * W["n_pol"]
    spec = _spec(wl, rank, S)
    x = make_stream_torch(spec, device=dev)
    if args.bits == 16:
        x = x.to(torch.int16) * 64          # 14-bit values in int16 containers
    prec = args.precision if args.precision is not None else (1 if wl == "c3" else 0)
    m = measure_stream(args, wl, prec, x, spec, dev, world, barrier, clocks=True)
    bytes_step = n_in * S * (args.bits // 8)
    ms = max_over_ranks(m["ms"], dist if world > 1 else None, dev)
    value = job_rate(bytes_step, world, ms)

    # ---- the plain FP32 path on the same stream, at its own autotuned ring ----
    plain = None
    if prec != 0 and not args.no_plain:
        mp_ = measure_stream(args, wl, 0, x, spec, dev, world, barrier, clocks=False, stages=False)
        pms = max_over_ranks(mp_["ms"], dist if world > 1 else None, dev)
        plain = {"value": job_rate(bytes_step, world, pms), "ms_per_step": pms, "ratio": ms and pms / ms,
                 "tuning": mp_["tuning"]}
    elif prec == 0:
        plain = {"value": value, "ms_per_step": ms, "ratio": 1.0,
                 "note": "this workload is defined on the FP32 path (CUDA-core X-engine): the chosen form and "
                         "the plain path are the same here; see chosen_form for the tensor-core form"}

    # ---- the other code type the 64-input workload names, timed the same way ----
    e4m3, e4m3_v = None, None
    if wl == "c3" and prec == 1 and not args.no_e4m3:
        me = measure_stream(args, wl, 2, x, spec, dev, world, barrier, clocks=False, stages=True)
        ems = max_over_ranks(me["ms"], dist if world > 1 else None, dev)
        e4m3 = {"value": job_rate(bytes_step, world, ems), "ms_per_step": ems,
                "ratio_to_plain": plain and ems and plain["ms_per_step"] / ems,
                "tuning": me["tuning"], "path": "e4m3 requantised, tcgen05 X (kind::f8f6f4)",
                "x_engine": (me["roofline"] or {}).get("x_engine")}
        e4m3_v = me["vis"]
        del me["flags"]

    # ---- end to end through the public host API ----
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(args, wl, prec, x, spec, m["tuning"], dev, world, dist)

    # ---- oracle: CPU baseline and the error of the timed stream's results ----
    cpu, error = None, None
    if rank == 0 and not args.no_cpu:
        if wl == "c3":
            cpu, _ = oracle_leg(wl, x, spec, None, None)
            error = rho_error(x, spec, W["n_chan"], W["taps"], W["n_int"], m["vis"], (0, m["vis"].shape[0] - 1))
            error["dtype"] = ["fp32", "int8", "e4m3"][prec]
            if prec == 1:
                # the other code type the workload names: the same stream
                # through the e4m3 pipeline (the timed run's results, else
                # one untimed run), its error too
                ev = e4m3_v if e4m3_v is not None else e4m3_vis(args, x, spec)
                error["e4m3"] = rho_error(x, spec, W["n_chan"], W["taps"], W["n_int"], ev,
                                          (0, m["vis"].shape[0] - 1))
        else:
            cpu, error = oracle_leg(wl, x, spec, m["vis"][0].cpu().numpy(), m["flags"][0].cpu().numpy())
    del m["vis"], m["flags"]
    e4m3_v = None

    # ---- the tensor-core form on the 64-input workload beside its plain path ----
    chosen = None
    if wl == "c2" and args.bits == 8 and not args.no_chosen:
        chosen = chosen_form(args, rank, dev, world, barrier, dist)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl + ": " + W["desc"],
                       "path": ["plain FP32 (CUDA-core X)", "int8 requantised, tcgen05 X (BF16 MMA)",
                                "e4m3 requantised, tcgen05 X"][prec],
                       "samples_per_input": S, "sample_bits": args.bits,
                       "tuning": {"ring_mb": m["tuning"][0], "fir_spt": m["tuning"][1], "x_depth": m["tuning"][2]},
                       "l2": m["l2"],
                       "parallelism": "replicas" if world > 1 else "single"},
            "gpu_launches": m["launches"], "clocks": m["clocks"], "roofline": m["roofline"], "e2e": e2e,
            "cpu_baseline": cpu, "error": error, "plain_fp32": plain,
        }
        if e4m3 is not None:
            out["e4m3"] = e4m3
        if chosen is not None:
            out["chosen_form"] = chosen
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def measure_stream(args, wl, prec, x, spec, dev, world, barrier, clocks=True, stages=True):
    """Time corr_run_dev over the device-resident stream x (autotuned ring
    unless --ring-mb is given): warm-up, one untimed step with every stage
    bracketed (stage shares, dominant kernel), then the timed steps with only
    the dominant kernel's launches bracketed.  Returns the timing, tuning,
    roofline entry and the last step's results."""
    import torch
    from paper_2604_20640_gb300 import Correlator
    W = WORKLOADS[wl]
    S = x.shape[1]
    n_in = W["n_ant"] * W["n_pol"]
    ring = {"ring_mb": args.ring_mb} if args.ring_mb else {}
    c = Correlator(W["n_ant"], W["n_pol"], W["n_chan"], W["taps"], W["n_int"], precision=prec,
                   sample_bits=args.bits, **ring)
    if not args.ring_mb:
        c.autotune(x)                  # ring size and FIR run length (untimed)
    tuning = c.tuning()
    c.set_delays(spec.tau, spec.phi)
    n_intg = c.n_integrations(S)
    vis = torch.empty((n_intg, W["n_chan"], n_in, n_in), dtype=torch.complex64, device=dev)
    flags = torch.empty((n_intg, W["n_chan"], n_in, n_in), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        c.run_dev(x, vis, flags)
    torch.cuda.synchronize(dev)
    share, di = None, None
    if stages:
        c.set_option("stage_timing", 1)
        c.stage_times()
        c.run_dev(x, vis, flags)
        share_ms, share_n = c.stage_times()
        total_stage = sum(share_ms) or 1.0
        share = {k: share_ms[i] / total_stage for i, k in enumerate(STAGES)}
        dom = max((k for k in STAGES if ALG_BYTES_PER_SAMPLE[k] > 0), key=lambda k: share[k])
        di = STAGES.index(dom)
        c.set_option("stage_mask", 1 << di)
    barrier()
    torch.cuda.synchronize(dev)
    # an input that fits in L2 (c1) is timed step by step with L2 flushed
    # between the steps (a 256 MiB write, outside the events)
    flush = x.numel() * x.element_size() < L2_FLUSH_BYTES
    scratch = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev) if flush else None
    sampler = ClockSampler(dev.index) if clocks else None
    l0 = c.launches
    if flush:
        ms_sum = 0.0
        for i in range(args.steps):
            scratch.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.run_dev(x, vis, flags)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms_sum += e0.elapsed_time(e1)
        ms = ms_sum / args.steps
    else:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            c.run_dev(x, vis, flags)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
    barrier()
    clk = sampler.stop() if sampler else None
    launches = c.launches - l0
    l2 = ("L2 flushed between timed steps (%d MiB write outside the events)" % (L2_FLUSH_BYTES >> 20) if flush
          else "inputs (%d MiB/step) larger than L2" % (x.numel() * x.element_size() >> 20))
    roofline = None
    if stages:
        stage_ms, stage_n = c.stage_times()
        c.set_option("stage_timing", 0)
        c.set_option("stage_mask", 127)
        roofline = _roofline(wl, prec, args, dom, di, share, stage_ms, stage_n, S, n_in)
        if prec != 0:
            roofline["x_engine"] = _gram_roofline(wl, prec, share_ms, share_n, n_in)
    c.close()
    return {"ms": ms, "tuning": tuning, "launches": launches, "clocks": clk, "roofline": roofline,
            "vis": vis, "flags": flags, "l2": l2}


def _gram_roofline(wl, prec, stage_ms, stage_n, n_in):
    """The tensor-core X-engine's rate from the step with every stage
    bracketed (live CUDA events): the algorithmic 2 (2N)^2 K flop of each
    channel's Gram matrix (N inputs, K spectra an integration) per launch
    against the measured BF16 tensor peak (e4m3: times the nominal ratio 2)."""
    gi = STAGES.index("gram")
    if not stage_n[gi]:
        return None
    W = WORKLOADS[wl]
    ms = stage_ms[gi] / stage_n[gi]
    flop = 2.0 * (2 * n_in) ** 2 * W["n_int"] * W["n_chan"]
    peaks = _peaks()
    burst = peaks.get("bf16_tflops") or 1900.0
    sust = peaks.get("bf16_tflops_sustained") or 1700.0
    scale = 2.0 if prec == 2 else 1.0
    tf = flop / (ms * 1e-3) / 1e12
    return {"kernel": "gram_w_kernel<%d> (%s)" % (prec == 2, "e4m3, kind::f8f6f4" if prec == 2 else
                                                   "int8 widened to BF16, kind::f16"),
            "bound": "tensor", "avg_launch_ms": ms, "launches": stage_n[gi], "flop_per_launch": flop,
            "achieved": tf, "peak": burst * scale, "unit": "TFLOP/s", "frac": tf / (burst * scale),
            "frac_of_sustained": tf / (sust * scale),
            "peak_source": ("measured BF16 burst x nominal ratio 2" if prec == 2 else "measured BF16 burst"),
            "input_gbs": n_in * 2 * W["n_chan"] * W["n_int"] / (ms * 1e-3) / 1e9}


def flops_per_sample(dom, fused, M, taps, n_in):
    """Algorithmic FP32 work per input sample of a hot-path kernel, in the
    scope table's operation counts: PFB FIR 2P, real FFT 2.5 log2 M (the
    conventional 5 N log2 N of an N-point complex transform carrying two real
    inputs), X-engine 2 (n_in + 1)."""
    import math
    fir, fft = 2.0 * taps, 2.5 * math.log2(M)
    if dom == "fft":
        return fir + fft if fused else fft
    return {"fir": fir, "xengine": 2.0 * (n_in + 1)}.get(dom, 0.0)


_FP32_PEAK = {}


def fp32_peak():
    """Measured FP32 FMA rate of this device (corr_peak_fp32, scalar and
    packed f32x2 forms), once per process."""
    if not _FP32_PEAK:
        from paper_2604_20640_gb300.corr import peak_fp32
        s, _ = peak_fp32(False, 4096)
        p, _ = peak_fp32(True, 4096)
        _FP32_PEAK.update(scalar=s, packed=p)
    return dict(_FP32_PEAK)


def _roofline(wl, prec, args, dom, di, share, stage_ms, stage_n, S, n_in):
    """Roofline entry of the dominant kernel from its live CUDA-event times:
    algorithmic bytes (and FP32 operations) per launch -- the samples the
    timed launches processed x the per-sample figure -- over the average
    launch duration.  The bound is the resource the kernel is closer to:
    HBM (measured copy peak) or FP32 arithmetic (measured FMA peak)."""
    W = WORKLOADS[wl]
    # the fused F-engine runs no FIR launches (shares come from the untimed
    # step with every stage bracketed)
    fused = dom == "fft" and share.get("fir", 0.0) == 0.0
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    es = args.bits // 8
    n_spec = S // (2 * W["n_chan"])
    samples_timed = args.steps * n_spec * 2 * W["n_chan"] * n_in
    launches = max(1, stage_n[di])
    alg = ALG_BYTES_PER_SAMPLE[dom] * (es if dom in ("fir", "fft", "xengine") else 1)
    inter = dict(INTERMEDIATE_BYTES_PER_SAMPLE)
    if fused:
        inter["fft"] = 1.0 + 4.0        # samples in, spectra out (no z ring)
        if prec != 0:
            # reduced precision: 4-byte code words per pair and channel out,
            # read by the Gram as they are (int8 and e4m3)
            inter.update(fft=1.0 + 1.0, requant=0.0)
    if es == 2:
        inter["fir"] += 1.0
    bytes_per_launch = alg * samples_timed / launches
    avg_ms = stage_ms[di] / launches
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    tps = TRAFFIC_PER_SAMPLE.get((wl, "fused" if fused else dom))
    traffic = tps * samples_timed / launches if tps and prec == 0 and es == 1 else None
    kname = KERNELS[dom]
    M = 2 * W["n_chan"]
    if dom == "fft":
        # pair-major spectra (mode 3); with reduced precision the F-engine
        # writes int8 (6) / e4m3 (7) code words from the second ring fill on
        mode = 3 if prec == 0 else (6 if prec == 1 else 7)
        kname = ("pfb_fft_kernel<%d,%d,%d> (fused PFB + FFT)" % (M, mode, W["taps"]) if fused
                 else "fft_kernel<%d,%d>" % (M, mode))
    fl = flops_per_sample(dom, fused, M, W["taps"], n_in)
    hbm_part = {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "peak_source": peak_src}
    out = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
           "frac": achieved / hbm, "traffic": traffic, "peak_source": peak_src,
           "bytes_per_launch": bytes_per_launch, "bytes_per_sample": alg,
           "intermediate_bytes_per_launch": inter[dom] * samples_timed / launches,
           "avg_launch_ms": avg_ms, "launches": stage_n[di], "stage_share": share}
    if fl > 0:
        fp = fp32_peak()
        tf = fl * samples_timed / launches / (avg_ms * 1e-3) / 1e12
        alu = {"achieved": tf, "peak": fp["scalar"], "unit": "TFLOP/s", "frac": tf / fp["scalar"],
               "flop_per_sample": fl, "peak_source": "measured (corr_peak_fp32, scalar FMA chains)",
               "peak_packed_f32x2": fp["packed"],
               "peak_nominal": 152 * 128 * 2 * 2.07e9 / 1e12}
        if alu["frac"] > out["frac"]:
            out.update({"bound": "alu", "achieved": tf, "peak": fp["scalar"], "unit": "TFLOP/s",
                        "frac": alu["frac"], "peak_source": alu["peak_source"], "hbm": hbm_part})
            out["alu"] = {k: alu[k] for k in ("flop_per_sample", "peak_packed_f32x2", "peak_nominal")}
        else:
            out["alu"] = alu
    return out


def end_to_end(args, wl, prec, x, spec, tuning, dev, world, dist):
    """The same samples through the host API as a continuing stream: each
    step pushes the next S samples per input from pinned host memory
    (corr_push) and pops every integration completed so far (corr_get_vis /
    corr_get_flags into pinned buffers), as a real-time correlator runs; the
    stream is flushed once after the timed steps."""
    import torch
    from paper_2604_20640_gb300 import Correlator
    from paper_2604_20640_gb300.replicas import max_over_ranks, job_rate
    W = WORKLOADS[wl]
    S = x.shape[1]
    n_in = W["n_ant"] * W["n_pol"]
    bytes_step = n_in * S * (args.bits // 8)
    # The host issues every launch of the push path, once per ring pass, so
    # it takes a ring of at least 128 MiB whatever the device-resident tuning
    # chose (small rings make the pushes launch-bound).
    ring_e2e = args.ring_mb or max(tuning[0], 128)
    chunk = args.chunk or W["chunk"]
    ce = Correlator(W["n_ant"], W["n_pol"], W["n_chan"], W["taps"], W["n_int"], chunk=chunk,
                    precision=prec, sample_bits=args.bits, ring_mb=ring_e2e, fir_spt=tuning[1], x_depth=tuning[2])
    ce.set_delays(spec.tau, spec.phi)
    host = torch.empty((n_in, S), dtype=x.dtype, pin_memory=True)
    host.copy_(x)
    n_intg = S // (2 * W["n_chan"]) // W["n_int"]
    # results land by DMA in pinned buffers the loop reuses
    vis_h = torch.empty((n_intg + 1, W["n_chan"], n_in, n_in), dtype=torch.complex64, pin_memory=True)
    flags_h = torch.empty((n_intg + 1, W["n_chan"], n_in, n_in), dtype=torch.uint8, pin_memory=True)
    phase = [0.0, 0.0]          # host seconds in the pushes / in flush + pops

    popped = [0]

    def e2e_step():
        ta = time.perf_counter()
        for p in range(0, S, chunk):
            ce.push(host[:, p:p + chunk])
        tb = time.perf_counter()
        v = ce.get_vis(out=vis_h)
        f = ce.get_flags(out=flags_h)
        assert v.shape[0] == f.shape[0]
        popped[0] += v.shape[0]
        phase[0] += tb - ta
        phase[1] += time.perf_counter() - tb
        return v, f

    for _ in range(max(1, args.warmup)):
        e2e_step()
    # the host->device copies of this shared host vary between windows of
    # time: the timed steps run three times over and the median counts
    reps = []
    timed_ints = 0
    for _ in range(3):
        if world > 1:
            dist.barrier()
        phase[:] = [0.0, 0.0]
        popped[0] = 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v, f = e2e_step()
        t1 = time.perf_counter()
        if world > 1:
            dist.barrier()
        reps.append(((t1 - t0) * 1e3 / args.steps, phase[0] * 1e3 / args.steps, phase[1] * 1e3 / args.steps))
        timed_ints = max(timed_ints, popped[0])
    ce.flush()
    ce.get_vis(out=vis_h)
    ce.get_flags(out=flags_h)
    # every step's integrations were read back: n_intg per step, the stream's
    # last one (held back one spectrum for the delays) popped by the next step
    assert timed_ints >= args.steps * n_intg - 1, (timed_ints, args.steps, n_intg)
    med = sorted(reps)[1]
    ems = med[0]
    ems = max_over_ranks(ems, dist if world > 1 else None, dev)
    out = {"value": job_rate(bytes_step, world, ems), "unit": "GB/s", "ring_mb": ring_e2e,
           "h2d_bytes_per_step": bytes_step,
           "d2h_bytes_per_step": int(v.numel() * v.element_size() + f.numel() * f.element_size()),
           "ms_per_step": ems, "push_ms": med[1], "pop_ms": med[2], "integrations_read_back": timed_ints,
           "repetitions_ms_per_step": [round(r[0], 3) for r in reps],
           "mode": "continuing stream: each step pushes %d MiB from pinned memory and pops the integrations "
                   "completed so far; flushed after the timed steps" % (bytes_step >> 20)}
    ce.close()
    del host
    return out


def chosen_form(args, rank, dev, world, barrier, dist):
    """The metric's chosen form where the X-engine is a dense contraction:
    the 64-input workload (2^26 int8 samples per input, 1024 channels,
    n_int 4096) with int8 codes on the tcgen05 X-engine, against the plain
    FP32 path on the same stream, both at their own autotuned rings, with the
    normalised-coefficient error of the chosen form against the oracle."""
    from paper_2604_20640_gb300.replicas import max_over_ranks, job_rate
    from fxsynth.streams_torch import make_stream_torch
    W = WORKLOADS["c3"]
    S = W["samples"]
    n_in = W["n_ant"] * W["n_pol"]
    spec = _spec("c3", rank, S)
    x = make_stream_torch(spec, device=dev)
    sub = argparse.Namespace(**vars(args))
    sub.bits = 8
    mc = measure_stream(sub, "c3", 1, x, spec, dev, world, barrier, clocks=False)
    mp_ = measure_stream(sub, "c3", 0, x, spec, dev, world, barrier, clocks=False, stages=False)
    bytes_step = n_in * S
    ms = max_over_ranks(mc["ms"], dist if world > 1 else None, dev)
    pms = max_over_ranks(mp_["ms"], dist if world > 1 else None, dev)
    out = {"workload": "c3: " + W["desc"], "value": job_rate(bytes_step, world, ms), "ms_per_step": ms,
           "plain_fp32": {"value": job_rate(bytes_step, world, pms), "ms_per_step": pms,
                          "tuning": mp_["tuning"]},
           "ratio": pms / ms, "tuning": mc["tuning"], "gpu_launches": mc["launches"],
           "roofline": mc["roofline"]}
    if rank == 0 and not args.no_cpu:
        out["error"] = rho_error(x, spec, W["n_chan"], W["taps"], W["n_int"], mc["vis"], (0, mc["vis"].shape[0] - 1))
    del mc["vis"], mc["flags"], mp_["vis"], mp_["flags"], x
    return out


if __name__ == "__main__":
    main()
