"""Python binding of the GPU receiver library librx.so (include/rx.h).

Argument marshalling only: every step of the receiver runs in the library's
CUDA kernels.  The names follow the C ABI.  PyTorch is used only to hold device
memory and to hand over the current CUDA stream.  There is no fallback: if
librx.so is missing or cannot be loaded, every entry point raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librx.so")

RX_PAM2, RX_PAM4, RX_PAM8, RX_KK_QPSK, RX_KK_16QAM = range(5)
RX_FIR_ADAPTIVE, RX_FIR_FROZEN_F32, RX_FIR_BF16, RX_FIR_FP16, RX_FIR_FP8 = range(5)
RX_DBG_FIELD, RX_DBG_MF, RX_DBG_SOFT, RX_DBG_DEC, RX_DBG_WIN, RX_DBG_TAPS, RX_DBG_SCAL, RX_DBG_CODES, RX_DBG_RS, \
    RX_DBG_CLK = range(1, 11)
BITS_PER_SYMBOL = {0: 1, 1: 2, 2: 3, 3: 2, 4: 4}


class RxConfig(C.Structure):
    _fields_ = [
        ("pack_order", C.c_int32), ("ols_n", C.c_int32), ("ols_v", C.c_int32),
        ("ds_num", C.c_int32), ("ds_den", C.c_int32), ("rrc_beta", C.c_double),
        ("mf_span", C.c_int32), ("ntaps", C.c_int32), ("ntrain", C.c_int32),
        ("ncma", C.c_int32), ("eq_block", C.c_int32), ("win", C.c_int32),
        ("mu", C.c_double), ("mu_train", C.c_double), ("mu_cma", C.c_double),
        ("bps_b", C.c_int32), ("amb_syms", C.c_int32), ("prbs_seed", C.c_uint32),
        ("debug", C.c_int32), ("fir_prec", C.c_int32), ("kk_front", C.c_int32), ("eq_warps", C.c_int32),
        ("mf_mode", C.c_int32), ("fd_n", C.c_int32), ("fd_taps", C.c_int32),
        ("clk_track", C.c_int32), ("rs_step", C.c_int64), ("rs_phase0", C.c_int64),
        ("cnn_bf16", C.c_int32), ("diff_code", C.c_int32), ("deadline_ms", C.c_double), ("eq_mode", C.c_int32), ("pad_eq", C.c_int32),
    ]


class RxStats(C.Structure):
    _fields_ = [
        ("calls", C.c_int64), ("samples", C.c_int64), ("symbols", C.c_int64),
        ("bits", C.c_int64), ("bit_errors", C.c_int64), ("raw_bit_errors", C.c_int64),
        ("sym_errors", C.c_int64), ("slip_windows", C.c_int64), ("near_threshold", C.c_int64),
        ("ambiguous_windows", C.c_int64), ("windows", C.c_int64), ("amb_rot", C.c_int32),
        ("device_error", C.c_int32), ("ber", C.c_double), ("q_db", C.c_double),
        ("lat_calls", C.c_int64), ("deadline_misses", C.c_int64), ("deadline_ms", C.c_double),
        ("lat_p50_ms", C.c_double), ("lat_p99_ms", C.c_double), ("lat_max_ms", C.c_double),
    ]


class RxError(RuntimeError):
    pass


EXPORTED = sorted(["rx_selftest_wait_timeout", "rx_selftest_fma_rate", "rx_clock_estimate", "rx_default_config", "rx_create", "rx_process", "rx_process_host", "rx_max_bits",
                   "rx_stats", "rx_debug_copy", "rx_set_taps", "rx_destroy", "rx_strerror",
                   "rx_profile", "rx_profile_read", "rx_kk_field_noalloc", "rx_cnn_nparams", "rx_cnn_create",
                   "rx_cnn_set_params", "rx_cnn_get_params", "rx_cnn_forward", "rx_cnn_grad",
                   "rx_cnn_adam_step", "rx_cnn_destroy", "rx_set_cnn", "rx_process_batch",
                   "rx_process_host_batch", "rx_fir_block", "rx_group_create", "rx_group_process",
                   "rx_group_tuning", "rx_group_destroy", "rx_flush", "rx_resampler_from_clock",
                   "rx_set_fd_taps", "rx_fd_ls_taps",
                   "rx_clock_track", "rx_clock_retime", "rx_set_resampler"])
RX_GROUP_GRAPH, RX_GROUP_TUNE = 1, 2
RX_MF_TIME, RX_MF_FD = 0, 1
RX_EQ_WINDOW, RX_EQ_DD_SYMBOL = 0, 1
STAGES = ["unpack", "kk_fwd", "kk_rows", "kk_inv", "mf", "eq", "demap"]

_lib = None


def load(path: str = LIB_PATH):
    """Load librx.so (built by __graft_entry__.build()); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RxError(f"{path} is missing: build it with __graft_entry__.build() (no CPU fallback exists)")
    L = C.CDLL(path)
    vp, i64, P = C.c_void_p, C.c_int64, C.POINTER
    L.rx_default_config.argtypes = [C.c_int, P(RxConfig)]
    L.rx_selftest_wait_timeout.argtypes = [vp]
    L.rx_selftest_wait_timeout.restype = C.c_int
    L.rx_selftest_fma_rate.argtypes = [C.c_int, P(C.c_double), vp]
    L.rx_clock_estimate.argtypes = [vp, P(C.c_double), P(C.c_double), vp]
    L.rx_clock_track.argtypes = [vp, P(C.c_double), P(C.c_double), P(i64), vp]
    L.rx_clock_retime.argtypes = [vp, P(i64), P(i64), vp]
    L.rx_set_resampler.argtypes = [vp, i64, i64, vp]
    L.rx_create.argtypes = [C.c_int, C.c_double, C.c_double, i64, P(RxConfig), P(vp)]
    L.rx_process.argtypes = [vp, vp, vp, vp, P(i64)]
    L.rx_process_host.argtypes = [vp, vp, vp, vp, P(i64)]
    L.rx_flush.argtypes = [vp, vp, vp, P(i64)]
    L.rx_resampler_from_clock.argtypes = [C.c_double, C.c_double, P(i64), P(i64)]
    L.rx_set_fd_taps.argtypes = [vp, vp, vp, C.c_int]
    L.rx_fd_ls_taps.argtypes = [vp, vp, i64, i64, C.c_int, vp, vp, i64, C.c_int, C.c_double, vp, vp]
    L.rx_process_batch.argtypes = [vp, vp, vp, C.c_int, vp, vp]
    L.rx_process_host_batch.argtypes = [vp, vp, vp, C.c_int, vp, vp]
    L.rx_fir_block.argtypes = [vp, i64, vp, C.c_int, C.c_int, i64, C.c_int, vp, vp, vp]
    L.rx_group_create.argtypes = [vp, C.c_int, C.c_int, P(vp)]
    L.rx_group_process.argtypes = [vp, vp, vp, vp, vp]
    L.rx_group_tuning.argtypes = [vp, C.c_int, P(C.c_int32), P(C.c_int32)]
    L.rx_group_destroy.argtypes = [vp]
    L.rx_max_bits.argtypes = [vp]
    L.rx_max_bits.restype = i64
    L.rx_stats.argtypes = [vp, P(RxStats), vp]
    L.rx_debug_copy.argtypes = [vp, C.c_int, vp, i64, P(i64), P(i64), vp]
    L.rx_set_taps.argtypes = [vp, vp, vp, C.c_int]
    L.rx_destroy.argtypes = [vp]
    L.rx_destroy.restype = None
    L.rx_profile.argtypes = [vp, C.c_int]
    L.rx_profile_read.argtypes = [vp, P(C.c_double), C.c_int, P(i64)]
    L.rx_kk_field_noalloc.argtypes = [vp, i64, C.c_int32, C.c_int32, C.c_int32, vp, vp]
    L.rx_cnn_nparams.restype = C.c_int
    L.rx_cnn_create.argtypes = [C.c_int, P(vp)]
    L.rx_cnn_set_params.argtypes = [vp, vp, C.c_int]
    L.rx_cnn_get_params.argtypes = [vp, vp, C.c_int]
    L.rx_cnn_forward.argtypes = [vp, vp, vp, C.c_int, vp, vp]
    L.rx_cnn_grad.argtypes = [vp, vp, vp, vp, C.c_int, vp, vp, vp]
    L.rx_cnn_adam_step.argtypes = [vp, C.c_float, vp]
    L.rx_cnn_destroy.argtypes = [vp]
    L.rx_cnn_destroy.restype = None
    L.rx_set_cnn.argtypes = [vp, vp]
    L.rx_strerror.argtypes = [C.c_int]
    L.rx_strerror.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("rx_max_bits", "rx_destroy", "rx_strerror", "rx_cnn_nparams", "rx_cnn_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise RxError(f"rx status {status}: {rx_strerror(status)}")


# ------------------------------------------------------------- C ABI, 1:1
def rx_resampler_from_clock(ppm: float, delay: float):
    """(rs_step, rs_phase0) of the resampler for a measured ADC clock (see include/rx.h)."""
    st, ph = C.c_int64(), C.c_int64()
    _check(load().rx_resampler_from_clock(ppm, delay, C.byref(st), C.byref(ph)))
    return st.value, ph.value



def rx_set_fd_taps(h: int, taps):
    """Zero-phase taps of the static frequency-domain filter, h_{-L} first (real or complex)."""
    taps = np.asarray(taps)
    re = np.ascontiguousarray(taps.real, dtype=np.float64)
    im = np.ascontiguousarray(taps.imag, dtype=np.float64) if np.iscomplexobj(taps) else None
    _check(load().rx_set_fd_taps(h, re.ctypes.data, None if im is None else im.ctypes.data, len(re)))


def rx_fd_ls_taps(x, first: int, step: int, a, ntaps: int, ridge: float = 0.0):
    """Least-squares static filter taps (see include/rx.h); real in and real targets
    give real taps, otherwise complex."""
    x, a = np.asarray(x), np.asarray(a)
    cplx = np.iscomplexobj(x) or np.iscomplexobj(a)
    xr = np.ascontiguousarray(x.real, dtype=np.float64)
    xi = np.ascontiguousarray(x.imag, dtype=np.float64) if np.iscomplexobj(x) else None
    ar = np.ascontiguousarray(a.real, dtype=np.float64)
    ai = np.ascontiguousarray(a.imag, dtype=np.float64) if np.iscomplexobj(a) else None
    hr = np.zeros(ntaps, np.float64)
    hi = np.zeros(ntaps, np.float64) if cplx else None
    _check(load().rx_fd_ls_taps(xr.ctypes.data, None if xi is None else xi.ctypes.data, len(xr), int(first),
                                int(step), ar.ctypes.data, None if ai is None else ai.ctypes.data, len(ar),
                                int(ntaps), float(ridge), hr.ctypes.data, None if hi is None else hi.ctypes.data))
    return hr + 1j * hi if cplx else hr


def rx_flush(h: int, bits_out: int, stream: int = 0) -> int:
    """Emit the payload the stream still holds back (device pointer); returns the bit count."""
    n = C.c_int64()
    _check(load().rx_flush(h, bits_out, stream, C.byref(n)))
    return n.value


def rx_clock_estimate(h: int, stream: int = 0):
    """(ppm, delay in ADC samples) of the ADC clock from the last call (FD form, KK or PAM)."""
    ppm, dl = C.c_double(), C.c_double()
    _check(load().rx_clock_estimate(h, C.byref(ppm), C.byref(dl), stream))
    return ppm.value, dl.value


def rx_clock_track(h: int, stream: int = 0):
    """(ppm, delay, blocks) of the running clock estimate across calls (clk_track=1)."""
    ppm, dl, n = C.c_double(), C.c_double(), C.c_int64()
    _check(load().rx_clock_track(h, C.byref(ppm), C.byref(dl), C.byref(n), stream))
    return ppm.value, dl.value, n.value


def rx_clock_retime(h: int, stream: int = 0):
    """Closed clock loop between calls; returns the applied (step, nudge)."""
    st, nu = C.c_int64(), C.c_int64()
    _check(load().rx_clock_retime(h, C.byref(st), C.byref(nu), stream))
    return st.value, nu.value


def rx_set_resampler(h: int, step: int, nudge: int = 0, stream: int = 0):
    _check(load().rx_set_resampler(h, step, nudge, stream))


def rx_selftest_fma_rate(iters: int = 1 << 16, stream: int = 0) -> float:
    """Measured FP32 FMA rate of this GPU in TFLOP/s (see include/rx.h)."""
    t = C.c_double()
    _check(load().rx_selftest_fma_rate(int(iters), C.byref(t), stream))
    return t.value


def rx_selftest_wait_timeout(stream: int = 0) -> int:
    """Bounded-wait self-test; returns the status code (RX_ETIMEOUT = 5 expected)."""
    return load().rx_selftest_wait_timeout(stream)


def rx_strerror(status: int) -> str:
    return load().rx_strerror(status).decode()


def rx_default_config(fmt: int) -> RxConfig:
    c = RxConfig()
    _check(load().rx_default_config(fmt, C.byref(c)))
    return c


def rx_create(fmt: int, baud: float, fs: float, buf_len: int, cfg: RxConfig | None = None) -> int:
    h = C.c_void_p()
    _check(load().rx_create(fmt, baud, fs, buf_len, C.byref(cfg) if cfg is not None else None, C.byref(h)))
    return h.value


def rx_process(h: int, packed12_in: int, bits_out: int, stream: int = 0) -> int:
    n = C.c_int64()
    _check(load().rx_process(h, packed12_in, bits_out, stream, C.byref(n)))
    return n.value


def rx_process_batch(h: int, ins, outs, stream: int = 0):
    """ins, outs: sequences of device pointers; returns the bit count per buffer."""
    n = len(ins)
    ia = (C.c_void_p * n)(*ins)
    oa = (C.c_void_p * n)(*outs)
    nb = (C.c_int64 * n)()
    _check(load().rx_process_batch(h, ia, oa, n, stream, nb))
    return list(nb)


def rx_process_host_batch(h: int, host_ins, host_outs, stream: int = 0):
    """host_ins, host_outs: sequences of (page-locked) host pointers; bit count per buffer."""
    n = len(host_ins)
    ia = (C.c_void_p * n)(*host_ins)
    oa = (C.c_void_p * n)(*host_outs)
    nb = (C.c_int64 * n)()
    _check(load().rx_process_host_batch(h, ia, oa, n, stream, nb))
    return list(nb)


def rx_fir_block(y: int, ny: int, w: int, ntaps: int, prec: int, nsym: int, scale_block: int, z: int,
                 status: int, stream: int = 0):
    """Tensor-core block-Toeplitz FIR (device pointers; see include/rx.h)."""
    _check(load().rx_fir_block(y, ny, w, ntaps, prec, nsym, scale_block, z, status, stream))


def rx_group_create(handles, flags: int = 0) -> int:
    """A group over existing receiver handles (see include/rx.h)."""
    arr = (C.c_void_p * len(handles))(*handles)
    g = C.c_void_p()
    _check(load().rx_group_create(arr, len(handles), flags, C.byref(g)))
    return g.value


def rx_group_process(g: int, ins, outs, stream: int = 0):
    """One buffer per member (device pointers); returns the bit count per member."""
    n = len(ins)
    ia = (C.c_void_p * n)(*ins)
    oa = (C.c_void_p * n)(*outs)
    nb = (C.c_int64 * n)()
    _check(load().rx_group_process(g, ia, oa, stream, nb))
    return list(nb)


def rx_group_tuning(g: int, i: int):
    f, w = C.c_int32(), C.c_int32()
    _check(load().rx_group_tuning(g, i, C.byref(f), C.byref(w)))
    return f.value, w.value


def rx_group_destroy(g: int):
    _check(load().rx_group_destroy(g))


def rx_process_host(h: int, host_in: int, host_bits_out: int, stream: int = 0) -> int:
    n = C.c_int64()
    _check(load().rx_process_host(h, host_in, host_bits_out, stream, C.byref(n)))
    return n.value


def rx_max_bits(h: int) -> int:
    return load().rx_max_bits(h)


def rx_stats(h: int, stream: int = 0) -> dict:
    s = RxStats()
    _check(load().rx_stats(h, C.byref(s), stream))
    return {k: getattr(s, k) for k, _ in RxStats._fields_}


def rx_debug_copy(h: int, what: int, dst: int, cap: int, stream: int = 0):
    n, s = C.c_int64(), C.c_int64()
    _check(load().rx_debug_copy(h, what, dst, cap, C.byref(n), C.byref(s), stream))
    return n.value, s.value


def rx_set_taps(h: int, re, im=None):
    re = np.ascontiguousarray(re, dtype=np.float64)
    imv = None if im is None else np.ascontiguousarray(im, dtype=np.float64)
    _check(load().rx_set_taps(h, re.ctypes.data, None if imv is None else imv.ctypes.data, len(re)))


def rx_profile(h: int, every: int):
    """Record stage events on every `every`-th call (0 stops; True means every call)."""
    _check(load().rx_profile(h, int(every)))


def rx_profile_read(h: int) -> tuple[dict, int]:
    ms = (C.c_double * len(STAGES))()
    n = C.c_int64()
    _check(load().rx_profile_read(h, ms, len(STAGES), C.byref(n)))
    return {s: ms[i] for i, s in enumerate(STAGES)}, n.value


def rx_kk_field_noalloc(packed12_in: int, nsamp: int, pack_order: int, ols_n: int, ols_v: int,
                        field_out: int, stream: int = 0):
    """KK field of one buffer with no device allocation (scratch is a fixed array
    inside librx.so); see include/rx.h."""
    _check(load().rx_kk_field_noalloc(packed12_in, nsamp, pack_order, ols_n, ols_v, field_out, stream))


def rx_cnn_nparams() -> int:
    return load().rx_cnn_nparams()


def rx_cnn_create(max_seg: int) -> int:
    h = C.c_void_p()
    _check(load().rx_cnn_create(max_seg, C.byref(h)))
    return h.value


def rx_cnn_set_params(c: int, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().rx_cnn_set_params(c, p.ctypes.data, len(p)))


def rx_cnn_get_params(c: int) -> np.ndarray:
    p = np.zeros(rx_cnn_nparams(), dtype=np.float32)
    _check(load().rx_cnn_get_params(c, p.ctypes.data, len(p)))
    return p


def rx_cnn_forward(c: int, y: int, seg_start: int, nseg: int, out: int, stream: int = 0):
    _check(load().rx_cnn_forward(c, y, seg_start, nseg, out, stream))


def rx_cnn_grad(c: int, y: int, seg_start: int, tgt: int, nseg: int, grad_out: int | None, loss_out: int | None,
                stream: int = 0):
    _check(load().rx_cnn_grad(c, y, seg_start, tgt, nseg, grad_out, loss_out, stream))


def rx_cnn_adam_step(c: int, lr: float, stream: int = 0):
    _check(load().rx_cnn_adam_step(c, lr, stream))


def rx_cnn_destroy(c: int):
    if c:
        load().rx_cnn_destroy(c)


def rx_set_cnn(h: int, c: int | None):
    _check(load().rx_set_cnn(h, c))


def rx_destroy(h: int):
    if h:
        load().rx_destroy(h)


# ------------------------------------------------------------- convenience
class Receiver:
    """One stream of ADC buffers on the current CUDA device.

    ``process`` takes a uint8 CUDA tensor of buf_len*3/2 packed bytes and
    returns (bits tensor on the device, number of bits).  The work is enqueued
    on torch's current stream; nothing waits for the GPU.
    """

    def __init__(self, fmt: int, buf_len: int, baud: float | None = None, fs: float = 4e9, **cfg):
        import torch
        self.torch = torch
        load()
        self.fmt = fmt
        self.buf_len = buf_len
        baud = baud if baud is not None else (fs / 4 if fmt >= 3 else fs / 2)
        c = rx_default_config(fmt)
        names = {f for f, _ in RxConfig._fields_}
        for k, v in cfg.items():
            if k not in names:
                raise TypeError(f"unknown receiver option {k!r}")
            setattr(c, k, v)
        self.cfg = c
        self.h = rx_create(fmt, baud, fs, buf_len, c)
        self.max_bits = rx_max_bits(self.h)
        self.bits = torch.zeros((self.max_bits + 7) // 8 + 16, dtype=torch.uint8, device="cuda")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            rx_destroy(h)
            self.h = None

    def stream(self) -> int:
        return self.torch.cuda.current_stream().cuda_stream

    def process(self, packed):
        assert packed.is_cuda and packed.dtype == self.torch.uint8
        n = rx_process(self.h, packed.data_ptr(), self.bits.data_ptr(), self.stream())
        return self.bits[: (n + 7) // 8], n

    def process_batch(self, packed_list):
        """Consecutive buffers in one pipelined call; returns [(bits tensor, nbits)]."""
        t = self.torch
        if not hasattr(self, "_bbufs") or len(self._bbufs) < len(packed_list):
            self._bbufs = [t.zeros((self.max_bits + 7) // 8 + 16, dtype=t.uint8, device="cuda")
                           for _ in range(len(packed_list))]
        outs = self._bbufs[: len(packed_list)]
        n = rx_process_batch(self.h, [p.data_ptr() for p in packed_list], [o.data_ptr() for o in outs],
                             self.stream())
        return [(o[: (k + 7) // 8], k) for o, k in zip(outs, n)]

    def flush(self):
        """End of the stream: (bits tensor on the device, number of bits) of the held-back payload."""
        n = rx_flush(self.h, self.bits.data_ptr(), self.stream())
        return self.bits[: (n + 7) // 8], n

    def stats(self) -> dict:
        return rx_stats(self.h, self.stream())

    def set_taps(self, taps):
        taps = np.asarray(taps, dtype=np.complex128)
        rx_set_taps(self.h, taps.real, taps.imag)

    def set_fd_taps(self, taps):
        rx_set_fd_taps(self.h, taps)

    _DT = {RX_DBG_FIELD: (np.complex64, 1), RX_DBG_SOFT: (np.complex64, 1), RX_DBG_DEC: (np.uint8, 1),
           RX_DBG_WIN: (np.float32, 4), RX_DBG_TAPS: (np.complex64, 1), RX_DBG_SCAL: (np.float64, 1),
           RX_DBG_CODES: (np.uint16, 1), RX_DBG_RS: (np.complex64, 1), RX_DBG_CLK: (np.complex64, 1)}

    def debug(self, what: int):
        n, s = rx_debug_copy(self.h, what, None, 0, self.stream())
        if what == RX_DBG_MF:
            dt, w = (np.complex64, 1) if self.fmt >= 3 else (np.float32, 1)
        else:
            dt, w = self._DT[what]
        out = np.zeros(max(n, 0) * w, dtype=dt)
        if n > 0:
            rx_debug_copy(self.h, what, out.ctypes.data, n, self.stream())
        return (out.reshape(-1, w) if w > 1 else out), s
