"""Batched sub-array streams (one captured CUDA graph with a persistent tail
kernel) and the autotuner.

Each member of a group must produce exactly what its own corr_run_dev
produces (and match the FP64 oracle); replaying the graph must repeat the
result; new buffers must be picked up by a fresh capture.  The group's tail
kernel (finalisation and MAD flags of every member, from a device work
queue) waits on per-integration dependency counters with a bounded wait: a
withheld dependency must end in CORR_ETIMEDOUT, not a hang.  Tuning changes
only speed: results stay bit-identical.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from fxsynth import StreamSpec, make_stream, delays_for  # noqa: E402
from oracle import fx_oracle as fx  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SHAPES = [(2, 64, 40), (3, 128, 20), (6, 32, 64), (8, 256, 12)]   # (n_ant, n_chan, n_int), 2 pols


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def _member(i, n_ant, n_chan, n_int, extra=0):
    from paper_2604_20640_gb300 import Correlator
    n_in = 2 * n_ant
    S = 2 * n_chan * n_int * 3 + 17 + extra
    tau, phi = delays_for(n_in, 100 + i)
    x = make_stream(StreamSpec(n_ant=n_ant, n_pol=2, n_samples=S, seed=100 + i, tau=tau, phi=phi))
    c = Correlator(n_ant, 2, n_chan, 4, n_int)
    c.set_delays(tau, phi)
    n = c.n_integrations(S)
    vis = torch.zeros((n, n_chan, n_in, n_in), dtype=torch.complex64, device=DEV)
    flags = torch.zeros((n, n_chan, n_in, n_in), dtype=torch.uint8, device=DEV)
    return c, x, torch.from_numpy(x).to(DEV), vis, flags, tau, phi


def test_group_graph_matches_members_and_oracle():
    from paper_2604_20640_gb300 import Group
    ms = [_member(i, *sh) for i, sh in enumerate(SHAPES)]
    solo = []
    for c, x, xd, vis, flags, tau, phi in ms:
        v2, f2 = torch.zeros_like(vis), torch.zeros_like(flags)
        c.run_dev(xd, v2, f2)
        solo.append((v2, f2))
    g = Group([m[0] for m in ms])
    outs = g.run_dev([m[2] for m in ms], [m[3] for m in ms], [m[4] for m in ms])
    torch.cuda.synchronize()
    first = [(m[3].clone(), m[4].clone()) for m in ms]
    for (c, x, xd, vis, flags, tau, phi), (v2, f2), n in zip(ms, solo, outs):
        assert n == vis.shape[0]
        assert torch.equal(vis, v2) and torch.equal(flags, f2)
        Ro, Fo, To = fx.correlate(x, c.n_chan, 4, c.n_int, tau, phi)
        err = fx.rel_frobenius_per_channel(vis.cpu().numpy().astype(np.complex128), Ro).max()
        assert err < 1e-5
    # replay the captured graph into zeroed outputs
    for m in ms:
        m[3].zero_()
        m[4].zero_()
    g.run_dev([m[2] for m in ms], [m[3] for m in ms], [m[4] for m in ms])
    torch.cuda.synchronize()
    for m, (v1, f1) in zip(ms, first):
        assert torch.equal(m[3], v1) and torch.equal(m[4], f1)
    # new output buffers -> new capture, same results
    new_vis = [torch.zeros_like(m[3]) for m in ms]
    g.run_dev([m[2] for m in ms], new_vis, [m[4] for m in ms])
    torch.cuda.synchronize()
    for v, (v1, _) in zip(new_vis, first):
        assert torch.equal(v, v1)
    g.close()


def test_autotune_is_bit_identical_and_cached(tmp_path):
    c, x, xd, vis, flags, tau, phi = _member(9, 4, 512, 32)
    c.run_dev(xd, vis, flags)
    ref_v, ref_f = vis.clone(), flags.clone()
    cache = str(tmp_path / "tune.txt")
    c.autotune(xd, cache)
    ring, spt, depth = c.tuning()
    assert ring in (32, 64, 128, 256) and spt in (0, 8, 16) and depth in (4, 6)
    assert os.path.exists(cache) and len(open(cache).read().strip().splitlines()) == 1
    vis.zero_()
    flags.zero_()
    c.run_dev(xd, vis, flags)
    torch.cuda.synchronize()
    assert torch.equal(vis, ref_v) and torch.equal(flags, ref_f)
    # a second handle of the same shape takes the cached choice without timing
    c2, *_ = _member(9, 4, 512, 32)
    c2.autotune(xd, cache)
    assert c2.tuning() == (ring, spt, depth)
    # the X-engine depth alone does not change the results either
    for d in (4, 6):
        c.set_option("x_depth", d)
        vis.zero_()
        c.run_dev(xd, vis, flags)
        torch.cuda.synchronize()
        assert torch.equal(vis, ref_v)
    assert len(open(cache).read().strip().splitlines()) == 1


def test_group_tail_wait_expires_on_a_withheld_dependency():
    """Fault injection: the tail kernel's first finalise item does not count
    itself done, so the flag items of that (member, integration) wait for a
    counter that never completes; after tc_wait_ms they record
    CORR_ETIMEDOUT and skip.  Everything else is computed; without the
    injection (a new capture) the group matches its members' own runs."""
    from paper_2604_20640_gb300 import Group, CORR_ETIMEDOUT
    ms = [_member(i, *sh) for i, sh in enumerate(SHAPES[:2])]
    solo = []
    for c, x, xd, vis, flags, tau, phi in ms:
        v2, f2 = torch.zeros_like(vis), torch.zeros_like(flags)
        c.run_dev(xd, v2, f2)
        solo.append((v2, f2))
    g = Group([m[0] for m in ms])
    g.set_option("tc_wait_ms", 5)
    g.set_option("inject_stall", 1)
    for m in ms:
        m[4].fill_(7)                                  # flags: 7 = never written
    g.run_dev([m[2] for m in ms], [m[3] for m in ms], [m[4] for m in ms])
    torch.cuda.synchronize()
    assert g.device_status() == CORR_ETIMEDOUT
    f0 = ms[0][4]
    assert torch.all(f0[0] == 7)                       # member 0, integration 0: flags skipped
    assert torch.all(f0[1:] <= 1)                      # its later integrations are flagged
    assert torch.all(ms[1][4] <= 1)
    assert torch.equal(ms[1][3], solo[1][0]) and torch.equal(ms[1][4], solo[1][1])
    g.set_option("inject_stall", 0)
    g.run_dev([m[2] for m in ms], [m[3] for m in ms], [m[4] for m in ms])
    torch.cuda.synchronize()
    assert g.device_status() == 0
    for m, (v2, f2) in zip(ms, solo):
        assert torch.equal(m[3], v2) and torch.equal(m[4], f2)
    g.close()
