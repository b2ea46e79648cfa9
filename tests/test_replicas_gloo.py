"""Multi-process replica mode on CPU (gloo, world size 2): per-rank seeds are
distinct, each rank's correlation (the FP64 oracle here, no GPU) equals what
a single process computes for that seed, the timing reduction takes the
slowest rank, and the job rate counts every rank's bytes."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_result(rank):
    from fxsynth import config_c1, make_stream
    from oracle import fx_oracle as fx
    from paper_2604_20640_gb300.replicas import rank_seed
    spec = config_c1(seed=rank_seed(1000, rank), n_samples=2 * 64 * 16 * 2)
    x = make_stream(spec)
    R, F, _ = fx.correlate(x, 64, 4, 16, spec.tau, spec.phi)
    return R, F


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2604_20640_gb300.replicas import max_over_ranks, job_rate
    R, F = _rank_result(rank)
    # gather every rank's visibilities on rank 0 (test only: the product has
    # no data-path collective)
    t = torch.from_numpy(np.ascontiguousarray(R.view(np.float64)))
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    ms = max_over_ranks(10.0 + rank, dist)
    if rank == 0:
        out.put((([p.numpy() for p in parts]), ms, job_rate(1 << 20, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts, ms, rate = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ms == 11.0
    assert abs(rate - 2 * (1 << 20) / 11e-3 / 1e9) < 1e-12
    for r in range(2):
        R, _ = _rank_result(r)
        assert np.array_equal(parts[r].view(np.complex128).reshape(R.shape), R)
    assert not np.array_equal(parts[0], parts[1])      # distinct per-rank streams
