"""Checkpoint / resume of a stream and host-side failure handling.

A stream pushed in ragged pieces into handle A, checkpointed at an arbitrary
point (mid-integration, mid partial-sum group, with results still queued and
a delay change pending), restored into a new handle B that receives the rest:
the results popped from A before the checkpoint and from B after it equal an
uninterrupted stream bit for bit, for the FP32 and the int8 tensor-core paths.
Failures are made on the host: an injected device-allocation failure must
fail the push with CORR_ENOMEM and leave the handle usable; a full result
queue (max_pending) refuses pushes with CORR_EAGAIN until results are popped.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from fxsynth import StreamSpec, delays_for, make_stream  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_20640_gb300.build import build_library
    build_library()


def _push_all(c, x, sizes, pos=0):
    for n in sizes:
        n = min(n, x.shape[1] - pos)
        if n <= 0:
            break
        c.push(x[:, pos:pos + n])
        pos += n
    return pos


@pytest.mark.parametrize("prec,n_ant,n_chan,n_int,cut", [(0, 4, 256, 100, 0.37), (0, 4, 256, 100, 0.81),
                                                        (1, 8, 128, 300, 0.55)])
def test_resume_from_a_checkpoint_is_bit_identical(prec, n_ant, n_chan, n_int, cut):
    from paper_2604_20640_gb300 import Correlator
    n_in = 2 * n_ant
    M = 2 * n_chan
    S = M * (n_int * 4 + 13) + 71
    tau, phi = delays_for(n_in, 17)
    x = make_stream(StreamSpec(n_ant=n_ant, n_pol=2, n_samples=S, seed=17, tau=tau, phi=phi))
    opts = dict(precision=prec, chunk=20000)
    ref = Correlator(n_ant, 2, n_chan, 4, n_int, **opts)
    ref.set_delays(tau, phi)
    _push_all(ref, x, [S])
    ref.set_delays(np.asarray(tau) + 0.3, phi)            # no effect: after the last push
    ref.flush()
    v_ref, f_ref = ref.get_vis(), ref.get_flags()
    ref.close()

    a = Correlator(n_ant, 2, n_chan, 4, n_int, **opts)
    a.set_delays(tau, phi)
    cut_at = int(S * cut)
    _push_all(a, x[:, :cut_at], [12345, 3, 50000, cut_at])
    v1 = a.get_vis(max_int=1)                              # pop one, leave the rest queued
    state = a.save_state()
    a.close()
    b = Correlator(n_ant, 2, n_chan, 4, n_int, **opts)
    b.load_state(state)
    _push_all(b, x, [7777, S], pos=cut_at)
    b.flush()
    v2, f2 = b.get_vis(), b.get_flags()
    b.close()
    v = np.concatenate([v1, v2]) if v1.shape[0] else v2
    assert v.shape == v_ref.shape
    assert np.array_equal(v, v_ref)
    assert np.array_equal(f2, f_ref)                      # no flags were popped before the checkpoint


def test_pending_delay_change_survives_a_checkpoint():
    from paper_2604_20640_gb300 import Correlator
    n_ant, n_chan, n_int = 2, 128, 50
    M = 2 * n_chan
    S = M * (n_int * 3 + 5)
    tau, phi = delays_for(4, 3)
    tau2 = np.asarray(tau) + np.array([0.0, 1.7, -2.2, 0.4])
    x = make_stream(StreamSpec(n_ant=n_ant, n_pol=2, n_samples=S, seed=3, tau=tau, phi=phi))
    cut = M * (n_int + 20) + 9                             # inside the second integration
    ref = Correlator(n_ant, 2, n_chan, 4, n_int)
    ref.set_delays(tau, phi)
    ref.push(x[:, :cut])
    ref.set_delays(tau2, phi)                              # applies at the third integration
    ref.push(x[:, cut:])
    ref.flush()
    v_ref = ref.get_vis()
    ref.close()
    a = Correlator(n_ant, 2, n_chan, 4, n_int)
    a.set_delays(tau, phi)
    a.push(x[:, :cut])
    a.set_delays(tau2, phi)
    state = a.save_state()
    a.close()
    b = Correlator(n_ant, 2, n_chan, 4, n_int)
    b.load_state(state)
    b.push(x[:, cut:])
    b.flush()
    assert np.array_equal(b.get_vis(), v_ref)
    b.close()


def test_states_of_other_shapes_and_started_handles_are_refused():
    from paper_2604_20640_gb300 import Correlator, CorrError, CORR_EINVAL, CORR_ESTATE
    a = Correlator(2, 1, 64, 4, 10)
    x = make_stream(StreamSpec(n_ant=2, n_pol=1, n_samples=5000, seed=1))
    a.push(x)
    st = a.save_state()
    b = Correlator(2, 1, 128, 4, 10)
    with pytest.raises(CorrError) as e:
        b.load_state(st)
    assert e.value.code == CORR_EINVAL
    with pytest.raises(CorrError) as e:
        b.load_state(st[:100])
    assert e.value.code == CORR_EINVAL
    with pytest.raises(CorrError) as e:
        a.load_state(st)
    assert e.value.code == CORR_ESTATE
    a.close()
    b.close()


def test_injected_allocation_failure_leaves_the_handle_usable():
    from paper_2604_20640_gb300 import Correlator, CorrError, CORR_ENOMEM
    n_ant, n_chan, n_int = 2, 128, 40
    S = 2 * n_chan * n_int * 2 + 3
    tau, phi = delays_for(4, 8)
    x = make_stream(StreamSpec(n_ant=n_ant, n_pol=2, n_samples=S, seed=8, tau=tau, phi=phi))
    ref = Correlator(n_ant, 2, n_chan, 4, n_int)
    ref.set_delays(tau, phi)
    ref.push(x)
    ref.flush()
    v_ref = ref.get_vis()
    ref.close()
    for k in (1, 2, 3, 5):                                # fail the k-th allocation of the stream set-up
        c = Correlator(n_ant, 2, n_chan, 4, n_int)
        c.set_delays(tau, phi)
        c.set_option("inject_alloc_fail", k)
        with pytest.raises(CorrError) as e:
            c.push(x)
        assert e.value.code == CORR_ENOMEM
        c.push(x)                                          # the injection fired once; now it succeeds
        c.flush()
        assert np.array_equal(c.get_vis(), v_ref)
        c.close()


def test_full_result_queue_refuses_pushes_until_popped():
    from paper_2604_20640_gb300 import Correlator, CorrError, CORR_EAGAIN
    n_ant, n_chan, n_int = 2, 64, 20
    M = 2 * n_chan
    x = make_stream(StreamSpec(n_ant=n_ant, n_pol=2, n_samples=M * n_int * 4, seed=2))
    c = Correlator(n_ant, 2, n_chan, 4, n_int, max_pending=1)
    c.push(x[:, :M * n_int + M])                           # one integration completes
    assert c.pending() == 1
    with pytest.raises(CorrError) as e:
        c.push(x[:, M * n_int + M:])
    assert e.value.code == CORR_EAGAIN
    assert c.get_vis(max_int=1).shape[0] == 1
    c.push(x[:, M * n_int + M:])                           # accepted now
    c.flush()
    assert c.get_vis().shape[0] == 3
    c.close()
