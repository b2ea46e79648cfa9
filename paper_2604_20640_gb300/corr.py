"""ctypes binding of libcorr.so (the C ABI declared in include/corr.h).

Argument marshalling only: every step of the correlator runs in the CUDA
library.  Device buffers are torch CUDA tensors (PyTorch supplies device
memory and streams); host buffers are numpy arrays.  If the library has not
been built, every call raises :class:`CorrError` -- there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcorr.so")

CORR_OK = 0
CORR_EINVAL = -1
CORR_ENOMEM = -2
CORR_ECUDA = -3
CORR_EAGAIN = -4
CORR_ETIMEDOUT = -5
CORR_ESTATE = -6

CORR_FP32, CORR_INT8, CORR_FP8 = 0, 1, 2
CORR_INT8_BYTES = 3          # corr_gram_dev: int8 codes stored as bytes
CORR_INT8_WORDS = 4          # corr_gram_dev: int8 code words [K][n_pairs][n_chan] (the pipeline's form)
CORR_FP8_WORDS = 5           # corr_gram_dev: e4m3 code words, same layout

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTED = [
    "corr_create", "corr_destroy", "corr_last_error", "corr_set_option", "corr_set_delays",
    "corr_push", "corr_push_dev", "corr_flush", "corr_reset", "corr_get_vis", "corr_get_flags",
    "corr_pending", "corr_run_dev", "corr_fengine_dev", "corr_xengine_dev", "corr_flag_dev",
    "corr_shape", "corr_kernel_launches", "corr_stage_times", "corr_xengine_noalloc",
    "corr_gram_dev", "corr_device_status", "corr_group_create", "corr_group_run_dev", "corr_autotune",
    "corr_get_tuning", "corr_spectrogram_dev", "corr_flagnet_create", "corr_flagnet_destroy",
    "corr_flagnet_num_params", "corr_flagnet_set_params", "corr_flagnet_get_params", "corr_flagnet_prepare",
    "corr_flagnet_forward", "corr_flagnet_loss_grad", "corr_flagnet_train_step", "corr_flagnet_flag",
    "corr_flagnet_status", "corr_flagnet_kernel_launches", "corr_tile_mad_dev", "corr_calibrate_dev",
    "corr_peak_fp32", "corr_save_state", "corr_load_state",
]


class CorrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libcorr error %d: %s" % (code, msg))
        self.code = code


_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_ll = ctypes.c_longlong
_sz = ctypes.c_size_t
_d = ctypes.c_double


def load_library(path: str = LIB_PATH):
    """Load libcorr.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise CorrError(CORR_ESTATE, "libcorr.so not built at %s (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    sig = {
        "corr_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _i]),
        "corr_destroy": (_i, [_vp]),
        "corr_last_error": (ctypes.c_char_p, [_vp]),
        "corr_set_option": (_i, [_vp, ctypes.c_char_p, _d]),
        "corr_set_delays": (_i, [_vp, _vp, _vp]),
        "corr_push": (_i, [_vp, _vp, _sz, _sz]),
        "corr_push_dev": (_i, [_vp, _vp, _sz, _sz, _vp]),
        "corr_flush": (_i, [_vp]),
        "corr_reset": (_i, [_vp]),
        "corr_get_vis": (_i, [_vp, _vp, _i, ctypes.POINTER(_i)]),
        "corr_get_flags": (_i, [_vp, _vp, _i, ctypes.POINTER(_i)]),
        "corr_pending": (_i, [_vp, ctypes.POINTER(_i)]),
        "corr_run_dev": (_i, [_vp, _vp, _sz, _sz, _vp, _vp, _i, _i, ctypes.POINTER(_i), _vp]),
        "corr_fengine_dev": (_i, [_vp, _vp, _sz, _sz, _ll, _i, _vp, _vp]),
        "corr_xengine_dev": (_i, [_vp, _vp, _i, _vp, _vp]),
        "corr_flag_dev": (_i, [_vp, _vp, _i, _vp, _vp]),
        "corr_shape": (_i, [_vp] + [ctypes.POINTER(_i)] * 5),
        "corr_kernel_launches": (_ll, [_vp]),
        "corr_stage_times": (_i, [_vp, _vp, _vp, _i]),
        "corr_xengine_noalloc": (_i, [_vp, _i, _i, _i, _vp, _vp]),
        "corr_gram_dev": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _vp]),
        "corr_device_status": (_i, [_vp, ctypes.POINTER(_i)]),
        "corr_group_create": (_i, [ctypes.POINTER(_vp), _vp, _i]),
        "corr_group_run_dev": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "corr_autotune": (_i, [_vp, _vp, _sz, _sz, ctypes.c_char_p, _vp]),
        "corr_get_tuning": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
        "corr_spectrogram_dev": (_i, [_vp, _vp, _sz, _sz, _i, _vp, _vp]),
        "corr_flagnet_create": (_i, [ctypes.POINTER(_vp)]),
        "corr_flagnet_destroy": (_i, [_vp]),
        "corr_flagnet_num_params": (_i, [ctypes.POINTER(_sz)]),
        "corr_flagnet_set_params": (_i, [_vp, _vp, _sz]),
        "corr_flagnet_get_params": (_i, [_vp, _vp, _sz]),
        "corr_flagnet_prepare": (_i, [_vp, _vp, _i, _vp, _vp]),
        "corr_flagnet_forward": (_i, [_vp, _vp, _i, _vp, _vp]),
        "corr_flagnet_loss_grad": (_i, [_vp, _vp, _vp, _i, ctypes.POINTER(ctypes.c_float), _vp, _sz, _vp]),
        "corr_flagnet_train_step": (_i, [_vp, _vp, _vp, _i, ctypes.c_float, ctypes.POINTER(ctypes.c_float), _vp]),
        "corr_flagnet_flag": (_i, [_vp, _vp, _i, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp]),
        "corr_flagnet_status": (_i, [_vp, ctypes.POINTER(_i)]),
        "corr_flagnet_kernel_launches": (_ll, [_vp]),
        "corr_tile_mad_dev": (_i, [_vp, _i, ctypes.c_float, _i, _vp, _vp]),
        "corr_calibrate_dev": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _d, _vp, _vp, _vp]),
        "corr_peak_fp32": (_i, [_i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d), _vp]),
        "corr_save_state": (_i, [_vp, _vp, _sz, ctypes.POINTER(_sz)]),
        "corr_load_state": (_i, [_vp, _vp, _sz]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, dtype_name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise CorrError(CORR_EINVAL, "expected a CUDA tensor for a device buffer")
    if not t.is_contiguous() and dtype_name != "samples":
        raise CorrError(CORR_EINVAL, "device buffer must be contiguous")
    return t.data_ptr()


class Group:
    """Batched sub-array streams run as one captured CUDA graph."""

    def __init__(self, members):
        self._L = load_library()
        self.members = list(members)
        arr = (_vp * len(self.members))(*[m._h.value for m in self.members])
        h = _vp()
        rc = self._L.corr_group_create(ctypes.byref(h), arr, len(self.members))
        if rc != CORR_OK:
            raise CorrError(rc, self._L.corr_last_error(None).decode())
        self._h = h

    def run_dev(self, samples, vis, flags=None, stream=None):
        n = len(self.members)
        ptrs = (_vp * n)(*[_dev_ptr(x, "samples") for x in samples])
        ns = (_sz * n)(*[x.shape[1] for x in samples])
        st = (_sz * n)(*[x.stride(0) for x in samples])
        vp = (_vp * n)(*[_dev_ptr(v, "vis") for v in vis])
        fp = (_vp * n)(*[_dev_ptr(f, "flags") for f in flags]) if flags is not None else None
        mx = (_i * n)(*[v.numel() * v.element_size() // (8 * m.n_chan * m.n_in * m.n_in)
                        for v, m in zip(vis, self.members)])
        out = (_i * n)()
        rc = self._L.corr_group_run_dev(self._h, ptrs, ns, st, vp, fp, mx, out, _stream_ptr(stream))
        if rc != CORR_OK:
            raise CorrError(rc, self._L.corr_last_error(self._h).decode())
        return list(out)

    def set_option(self, key: str, value: float):
        """Options of the group's own tail kernel ("tc_wait_ms", "inject_stall")."""
        rc = self._L.corr_set_option(self._h, key.encode(), float(value))
        if rc != CORR_OK:
            raise CorrError(rc, self._L.corr_last_error(self._h).decode())

    def device_status(self) -> int:
        """The group's device status word (CORR_ETIMEDOUT from its tail kernel), cleared on read."""
        st = _i()
        rc = self._L.corr_device_status(self._h, ctypes.byref(st))
        if rc != CORR_OK:
            raise CorrError(rc, self._L.corr_last_error(self._h).decode())
        return st.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.corr_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def xengine_noalloc(V, n_spec: int, n_in: int, n_chan: int, vis_out, stream=None):
    """X-engine without any device allocation (corr_xengine_noalloc): for
    callers that cannot allocate device memory (real-time loops in which an
    allocator call could synchronise the device, hosts that plan the GPU's
    memory themselves).  Same layouts as :meth:`Correlator.xengine_dev`; no
    handle needed."""
    L = load_library()
    rc = L.corr_xengine_noalloc(_dev_ptr(V, "V"), int(n_spec), int(n_in), int(n_chan),
                                _dev_ptr(vis_out, "vis"), _stream_ptr(stream))
    if rc != CORR_OK:
        raise CorrError(rc, L.corr_last_error(None).decode())


class Correlator:
    """One correlator handle: ``corr_create(n_ant, n_pol, n_chan, taps, n_int)``."""

    def __init__(self, n_ant: int, n_pol: int, n_chan: int, taps: int, n_int: int, **options):
        self._L = load_library()
        h = _vp()
        rc = self._L.corr_create(ctypes.byref(h), n_ant, n_pol, n_chan, taps, n_int)
        if rc != CORR_OK:
            raise CorrError(rc, self._L.corr_last_error(None).decode())
        self._h = h
        self.n_ant, self.n_pol, self.n_chan, self.taps, self.n_int = n_ant, n_pol, n_chan, taps, n_int
        self.n_in = n_ant * n_pol
        self.n_in_pad = (self.n_in + 3) // 4 * 4
        self.M = 2 * n_chan
        self.sample_bits = 8
        self.iq = False
        for k, v in options.items():
            self.set_option(k, v)

    # -- helpers ----------------------------------------------------------
    def _check(self, rc: int, allow=(CORR_OK,)):
        if rc not in allow:
            raise CorrError(rc, self._L.corr_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.corr_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration ----------------------------------------------------
    def set_option(self, key: str, value: float):
        self._check(self._L.corr_set_option(self._h, key.encode(), float(value)))
        if key == "sample_bits":
            self.sample_bits = int(value)
        elif key == "sample_format":
            self.iq = bool(value)
            self.M = self.n_chan if self.iq else 2 * self.n_chan

    def _counts(self, n_elems: int, stride_elems: int):
        """(samples per input, input stride) in the library's sample units for
        rows of n_elems array elements: complex input takes (I, Q) int8 pairs,
        so two elements make one sample."""
        if not self.iq:
            return n_elems, stride_elems
        if n_elems % 2 or stride_elems % 2:
            raise CorrError(CORR_EINVAL, "complex input: rows of interleaved (I, Q) int8 pairs")
        return n_elems // 2, stride_elems // 2

    def _sample_types(self):
        import torch
        return (np.int16, torch.int16) if self.sample_bits == 16 else (np.int8, torch.int8)

    def set_delays(self, tau, phi=None):
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        if tau.shape != (self.n_in,):
            raise CorrError(CORR_EINVAL, "tau must have n_in entries")
        pp = None
        if phi is not None:
            phi = np.ascontiguousarray(phi, dtype=np.float64)
            if phi.shape != (self.n_in,):
                raise CorrError(CORR_EINVAL, "phi must have n_in entries")
            pp = phi.ctypes.data
        self._check(self._L.corr_set_delays(self._h, tau.ctypes.data, pp))

    # -- streaming --------------------------------------------------------
    def push(self, samples):
        """Append host samples ``[n_in][n]`` (numpy array or CPU tensor of the
        handle's sample type: int8, or int16 with sample_bits=16)."""
        np_t = np.int16 if self.sample_bits == 16 else np.int8
        try:
            import torch
            if isinstance(samples, torch.Tensor):
                if samples.is_cuda:
                    return self.push_dev(samples)
                if samples.dtype != self._sample_types()[1] or samples.dim() != 2 or samples.shape[0] != self.n_in:
                    raise CorrError(CORR_EINVAL, "samples must be %s [n_in][n]" % np.dtype(np_t).name)
                if samples.stride(1) != 1:
                    raise CorrError(CORR_EINVAL, "samples rows must be contiguous")
                self._check(self._L.corr_push(self._h, samples.data_ptr(),
                                              *self._counts(samples.shape[1], samples.stride(0))))
                return
        except ImportError:
            pass
        a = np.asarray(samples)
        if a.dtype != np_t or a.ndim != 2 or a.shape[0] != self.n_in:
            raise CorrError(CORR_EINVAL, "samples must be %s [n_in][n]" % np.dtype(np_t).name)
        if a.strides[1] != a.itemsize or a.strides[0] % a.itemsize:
            a = np.ascontiguousarray(a)
        self._check(self._L.corr_push(self._h, a.ctypes.data, *self._counts(a.shape[1], a.strides[0] // a.itemsize)))

    def push_dev(self, samples, stream=None):
        """Append device samples (CUDA tensor ``[n_in][n]`` of the handle's
        sample type, rows contiguous)."""
        if samples.dim() != 2 or samples.shape[0] != self.n_in or samples.stride(1) != 1 or \
                samples.dtype != self._sample_types()[1]:
            raise CorrError(CORR_EINVAL, "samples must be [n_in][n] of the sample type with contiguous rows")
        self._check(self._L.corr_push_dev(self._h, _dev_ptr(samples, "samples"),
                                          *self._counts(samples.shape[1], samples.stride(0)), _stream_ptr(stream)))

    def flush(self):
        self._check(self._L.corr_flush(self._h))

    def save_state(self) -> bytes:
        """The streaming state (corr_save_state) as bytes."""
        n = _sz()
        self._check(self._L.corr_save_state(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(max(1, n.value))
        self._check(self._L.corr_save_state(self._h, buf, n.value, ctypes.byref(n)))
        return buf.raw[:n.value]

    def load_state(self, state: bytes):
        """Restore a saved state into this new (or reset) handle (corr_load_state)."""
        buf = ctypes.create_string_buffer(state, len(state))
        self._check(self._L.corr_load_state(self._h, buf, len(state)))

    def reset(self):
        self._check(self._L.corr_reset(self._h))

    def pending(self) -> int:
        n = _i()
        self._check(self._L.corr_pending(self._h, ctypes.byref(n)))
        return n.value

    def _result_out(self, out, max_int, np_t):
        """Pointer and array view of a caller-provided result buffer
        ``[>= max_int][n_chan][n_in][n_in]`` (numpy array or CPU tensor,
        contiguous; a pinned tensor is filled by DMA)."""
        shape = (self.n_chan, self.n_in, self.n_in)
        if type(out).__module__.startswith("torch"):
            import torch
            torch_t = {np.complex64: torch.complex64, np.uint8: torch.uint8}[np_t]
            if out.is_cuda or out.dtype != torch_t or tuple(out.shape[1:]) != shape or \
                    not out.is_contiguous() or out.shape[0] < max_int:
                raise CorrError(CORR_EINVAL, "out must be a contiguous CPU %s [>=%d]%s" % (torch_t, max_int, shape))
            return out.data_ptr(), out
        if not isinstance(out, np.ndarray) or out.dtype != np_t or out.shape[1:] != shape or \
                not out.flags["C_CONTIGUOUS"] or out.shape[0] < max_int:
            raise CorrError(CORR_EINVAL, "out must be a contiguous %s array [>=%d]%s" % (np.dtype(np_t).name, max_int, shape))
        return out.ctypes.data, out

    def get_vis(self, max_int: Optional[int] = None, out=None):
        """Pop up to ``max_int`` (default: all pending) integrations' visibilities
        ``[n][n_chan][n_in][n_in]`` complex64, into ``out`` when given (numpy
        array or CPU tensor, returned sliced to the count)."""
        if max_int is None:
            max_int = self.pending() if out is None else min(self.pending(), out.shape[0])
        if out is None:
            out = np.empty((max_int, self.n_chan, self.n_in, self.n_in), dtype=np.complex64)
        ptr, out = self._result_out(out, max_int, np.complex64)
        got = _i()
        self._check(self._L.corr_get_vis(self._h, ptr, max_int, ctypes.byref(got)),
                    allow=(CORR_OK, CORR_EAGAIN))
        return out[: got.value]

    def get_flags(self, max_int: Optional[int] = None, out=None):
        """Pop up to ``max_int`` (default: all queued) integrations' flags
        ``[n][n_chan][n_in][n_in]`` uint8, into ``out`` when given."""
        if out is not None:
            n = out.shape[0] if max_int is None else max_int
            ptr, out = self._result_out(out, n, np.uint8)
            got = _i()
            self._check(self._L.corr_get_flags(self._h, ptr, n, ctypes.byref(got)), allow=(CORR_OK, CORR_EAGAIN))
            return out[: got.value]
        if max_int is None:
            max_int = 1 << 20
            # flags FIFO may be longer than the vis FIFO; pop what is there
        out_list = []
        got = _i()
        while max_int > 0:
            n = min(max_int, 64)
            out = np.empty((n, self.n_chan, self.n_in, self.n_in), dtype=np.uint8)
            rc = self._check(self._L.corr_get_flags(self._h, out.ctypes.data, n, ctypes.byref(got)),
                             allow=(CORR_OK, CORR_EAGAIN))
            out_list.append(out[: got.value])
            max_int -= got.value
            if rc == CORR_EAGAIN or got.value < n:
                break
        if not out_list:
            return np.empty((0, self.n_chan, self.n_in, self.n_in), dtype=np.uint8)
        return np.concatenate(out_list, axis=0)

    # -- device-resident entry points ----------------------------------------
    def n_integrations(self, n_samples: int, include_partial: bool = False) -> int:
        n_spec = n_samples // self.M
        return n_spec // self.n_int + (1 if include_partial and n_spec % self.n_int else 0)

    def run_dev(self, samples, vis_out, flags_out=None, include_partial=False, stream=None) -> int:
        """Whole stream on device: samples [n_in][S] int8 CUDA -> vis / flags."""
        if samples.dim() != 2 or samples.shape[0] != self.n_in or samples.stride(1) != 1:
            raise CorrError(CORR_EINVAL, "samples must be int8 [n_in][S] with contiguous rows")
        n_out = _i()
        max_int = vis_out.numel() * vis_out.element_size() // (8 * self.n_chan * self.n_in * self.n_in)
        fp = _dev_ptr(flags_out, "flags") if flags_out is not None else None
        self._check(self._L.corr_run_dev(self._h, _dev_ptr(samples, "samples"),
                                         *self._counts(samples.shape[1], samples.stride(0)),
                                         _dev_ptr(vis_out, "vis"), fp, int(max_int),
                                         1 if include_partial else 0, ctypes.byref(n_out),
                                         _stream_ptr(stream)))
        return n_out.value

    def fengine_dev(self, samples, s0: int, n_spec: int, V_out, stream=None):
        if samples.dim() != 2 or samples.shape[0] != self.n_in or samples.stride(1) != 1:
            raise CorrError(CORR_EINVAL, "samples must be int8 [n_in][S] with contiguous rows")
        self._check(self._L.corr_fengine_dev(self._h, _dev_ptr(samples, "samples"),
                                             *self._counts(samples.shape[1], samples.stride(0)),
                                             int(s0), int(n_spec), _dev_ptr(V_out, "V"),
                                             _stream_ptr(stream)))

    def xengine_dev(self, V, n_spec: int, vis_out, stream=None):
        self._check(self._L.corr_xengine_dev(self._h, _dev_ptr(V, "V"), int(n_spec), _dev_ptr(vis_out, "vis"),
                                             _stream_ptr(stream)))

    def flag_dev(self, vis, n_vis: int, flags_out, stream=None):
        self._check(self._L.corr_flag_dev(self._h, _dev_ptr(vis, "vis"), int(n_vis),
                                          _dev_ptr(flags_out, "flags"), _stream_ptr(stream)))

    def autotune(self, samples, cache_path: Optional[str] = None, stream=None):
        """Pick ring size and FIR run length by timing (corr_autotune)."""
        cp = cache_path.encode() if cache_path else None
        self._check(self._L.corr_autotune(self._h, _dev_ptr(samples, "samples"),
                                          *self._counts(samples.shape[1], samples.stride(0)), cp,
                                          _stream_ptr(stream)))

    def tuning(self):
        """(ring_mb, fir_spt, x_depth) as set by autotune or the options."""
        r, s, d = _i(), _i(), _i()
        self._check(self._L.corr_get_tuning(self._h, ctypes.byref(r), ctypes.byref(s), ctypes.byref(d)))
        return r.value, s.value, d.value

    def gram_dev(self, Q, n_chan: int, k_pitch: int, K: int, dtype: int, G_out, stream=None):
        """Tensor-core Gram matrices of Q (see corr_gram_dev in include/corr.h)."""
        self._check(self._L.corr_gram_dev(self._h, _dev_ptr(Q, "Q"), int(n_chan), int(k_pitch), int(K),
                                          int(dtype), _dev_ptr(G_out, "G"), _stream_ptr(stream)))

    def spectrogram_dev(self, samples, n_row: int, tiles_out, stream=None):
        """Autocorrelation-power tiles [n_in][rows/64][n_chan/256][64][256] (FP32)."""
        rc = self._L.corr_spectrogram_dev(self._h, _dev_ptr(samples, "samples"), samples.shape[1],
                                          samples.stride(0), n_row, _dev_ptr(tiles_out, "tiles"),
                                          _stream_ptr(stream))
        self._check(rc)

    def device_status(self) -> int:
        st = _i()
        self._check(self._L.corr_device_status(self._h, ctypes.byref(st)))
        return st.value

    def stage_times(self):
        """(ms, counts) per stage (FIR, FFT, X, finalise, flag, requantise, tensor-core
        Gram) since the last call."""
        ms = (ctypes.c_double * 7)()
        n = (ctypes.c_longlong * 7)()
        self._check(self._L.corr_stage_times(self._h, ms, n, 7))
        return list(ms), list(n)

    @property
    def launches(self) -> int:
        return int(self._L.corr_kernel_launches(self._h))


def peak_fp32(packed: bool = False, iters: int = 4096, stream=None):
    """(TFLOP/s, ms) of the FP32 FMA probe (corr_peak_fp32)."""
    L = load_library()
    t, ms = _d(), _d()
    rc = L.corr_peak_fp32(1 if packed else 0, int(iters), ctypes.byref(t), ctypes.byref(ms), _stream_ptr(stream))
    if rc != CORR_OK:
        raise CorrError(rc, L.corr_last_error(None).decode())
    return t.value, ms.value


def tile_mad(power, flags_out, axes: int = 1, sigma: float = 5.0, stream=None):
    """Eq. 2 on power tiles [B][64][256]: axes 1 along channels (per row,
    64-channel windows), 2 along time (per channel), 3 both (union)."""
    L = load_library()
    rc = L.corr_tile_mad_dev(_dev_ptr(power, "power"), power.shape[0], sigma, axes, _dev_ptr(flags_out, "flags"),
                             _stream_ptr(stream))
    if rc != CORR_OK:
        raise CorrError(rc, L.corr_last_error(None).decode())


def calibrate(vis, flags=None, ref: int = 0, k_lo: int = 0, k_hi: Optional[int] = None, max_delay: float = 64.0,
              stream=None):
    """(tau [n_in], phi [n_in]) from one integration's visibilities
    vis [n_chan][n_in][n_in] (complex64, CUDA) -- the delay-spectrum peak,
    the weighted fit to the unwrapped phase and the residual phase of Sec. 7,
    in the convention of Correlator.set_delays."""
    L = load_library()
    n_chan, n_in = vis.shape[0], vis.shape[1]
    tau = np.empty(n_in)
    phi = np.empty(n_in)
    rc = L.corr_calibrate_dev(_dev_ptr(vis, "vis"), _dev_ptr(flags, "flags") if flags is not None else None,
                              n_chan, n_in, ref, k_lo, n_chan if k_hi is None else k_hi, float(max_delay),
                              tau.ctypes.data, phi.ctypes.data, _stream_ptr(stream))
    if rc != CORR_OK:
        raise CorrError(rc, L.corr_last_error(None).decode())
    return tau, phi


class FlagNet:
    """Learned RFI flagger on (64 x 256) tiles of autocorrelation power, with
    the Eq. 2 MAD rule as the fallback on tiles of low confidence."""

    TILE = (64, 256)

    def __init__(self, params: Optional[np.ndarray] = None):
        self._L = load_library()
        h = _vp()
        rc = self._L.corr_flagnet_create(ctypes.byref(h))
        if rc != CORR_OK:
            raise CorrError(rc, self._L.corr_last_error(None).decode())
        self._h = h
        n = _sz()
        self._L.corr_flagnet_num_params(ctypes.byref(n))
        self.n_params = n.value
        if params is not None:
            self.set_params(params)

    def _check(self, rc: int):
        if rc != CORR_OK:
            raise CorrError(rc, self._L.corr_last_error(None).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.corr_flagnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, np.float32)
        self._check(self._L.corr_flagnet_set_params(self._h, p.ctypes.data, p.size))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, np.float32)
        self._check(self._L.corr_flagnet_get_params(self._h, p.ctypes.data, p.size))
        return p

    def prepare(self, power, x_out, stream=None):
        self._check(self._L.corr_flagnet_prepare(self._h, _dev_ptr(power, "power"), power.shape[0],
                                                 _dev_ptr(x_out, "x"), _stream_ptr(stream)))

    def forward(self, x, logits_out, stream=None):
        self._check(self._L.corr_flagnet_forward(self._h, _dev_ptr(x, "x"), x.shape[0],
                                                 _dev_ptr(logits_out, "logits"), _stream_ptr(stream)))

    def loss_grad(self, x, truth, stream=None):
        loss = ctypes.c_float()
        g = np.empty(self.n_params, np.float32)
        self._check(self._L.corr_flagnet_loss_grad(self._h, _dev_ptr(x, "x"), _dev_ptr(truth, "truth"), x.shape[0],
                                                   ctypes.byref(loss), g.ctypes.data, g.size, _stream_ptr(stream)))
        return loss.value, g

    def train_step(self, x, truth, lr: float, stream=None) -> float:
        loss = ctypes.c_float()
        self._check(self._L.corr_flagnet_train_step(self._h, _dev_ptr(x, "x"), _dev_ptr(truth, "truth"), x.shape[0],
                                                    lr, ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value

    def flag(self, power, flags_out, conf_out=None, c_min: float = 0.9, sigma: float = 5.0, stream=None):
        self._check(self._L.corr_flagnet_flag(self._h, _dev_ptr(power, "power"), power.shape[0], c_min, sigma,
                                              _dev_ptr(flags_out, "flags"),
                                              _dev_ptr(conf_out, "conf") if conf_out is not None else None,
                                              _stream_ptr(stream)))

    def status(self) -> int:
        st = _i()
        self._check(self._L.corr_flagnet_status(self._h, ctypes.byref(st)))
        return st.value

    @property
    def launches(self) -> int:
        return int(self._L.corr_flagnet_kernel_launches(self._h))
