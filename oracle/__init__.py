"""FP64 CPU oracle of the receiver -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``rx_oracle.c`` (plain C,
double precision) with ctypes.  The CUDA receiver shares no code with it.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborx.so")

ORX_E, ORX_Y, ORX_Z, ORX_V, ORX_AHAT, ORX_BERR, ORX_WIN, ORX_TAPS, ORX_SCAL, ORX_NEAR, ORX_DRAW, ORX_RS, ORX_CLK = \
    range(1, 14)


class OrxCfg(C.Structure):
    _fields_ = [
        ("format", C.c_int32), ("sps", C.c_int32), ("buf_len", C.c_int64),
        ("pack_order", C.c_int32), ("ols_n", C.c_int32), ("ols_v", C.c_int32),
        ("ds_num", C.c_int32), ("ds_den", C.c_int32), ("rrc_beta", C.c_double),
        ("mf_span", C.c_int32), ("ntaps", C.c_int32), ("ntrain", C.c_int32),
        ("ncma", C.c_int32), ("eq_block", C.c_int32), ("win", C.c_int32),
        ("mu", C.c_double), ("mu_train", C.c_double), ("mu_cma", C.c_double),
        ("bps_b", C.c_int32), ("amb_syms", C.c_int32), ("prbs_seed", C.c_uint32),
        ("eq_frozen", C.c_int32), ("mf_mode", C.c_int32), ("fd_n", C.c_int32), ("fd_taps", C.c_int32),
        ("clk_track", C.c_int32), ("rs_step", C.c_int64), ("rs_phase0", C.c_int64),
        ("diff_code", C.c_int32), ("eq_mode", C.c_int32),
    ]


class OrxStats(C.Structure):
    _fields_ = [
        ("calls", C.c_int64), ("samples", C.c_int64), ("symbols", C.c_int64),
        ("bits", C.c_int64), ("bit_errors", C.c_int64), ("sym_errors", C.c_int64),
        ("near_threshold", C.c_int64), ("ambiguous_windows", C.c_int64),
        ("windows", C.c_int64), ("raw_bit_errors", C.c_int64), ("slip_windows", C.c_int64),
        ("amb_rot", C.c_int32), ("ber", C.c_double),
        ("q_db", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile rx_oracle.c into liborx.so beside it (gcc, -O2, IEEE double)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rx_oracle.h"))):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.orx_unpack.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p]
        L.orx_fft.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int]
        L.orx_hilbert_circ.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
        L.orx_kk_circ.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.orx_rrc.argtypes = [C.c_double, C.c_int, C.c_int, C.c_void_p]
        L.orx_rrc_half.argtypes = [C.c_double, C.c_int, C.c_int, C.c_void_p]
        L.orx_fd_response.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        L.orx_fd_block.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]
        L.orx_rs_taps.argtypes = [C.c_double, C.c_void_p]
        L.orx_fd_clock.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                   C.c_void_p, C.c_void_p]
        L.orx_clock_fit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                    C.c_void_p]
        L.orx_clock_fit.restype = C.c_int
        L.orx_fd_block_full.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p]
        L.orx_prbs15.argtypes = [C.c_uint32, C.c_int64, C.c_void_p]
        L.orx_q_db.argtypes = [C.c_double]
        L.orx_q_db.restype = C.c_double
        L.orx_bps_metrics.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                      C.c_int, C.c_void_p]
        L.orx_cnn_nparams.restype = C.c_int
        L.orx_cnn_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                        C.c_void_p]
        L.orx_cnn_loss_grad.restype = C.c_double
        L.orx_create.argtypes = [P(OrxCfg)]
        L.orx_create.restype = C.c_void_p
        L.orx_process.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
        L.orx_process.restype = C.c_int64
        L.orx_flush.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        L.orx_flush.restype = C.c_int64
        L.orx_clock_track.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orx_clock_track.restype = C.c_int64
        L.orx_set_rs.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
        L.orx_set_rs.restype = C.c_int
        L.orx_clock_retime.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orx_clock_retime.restype = C.c_int
        L.orx_get.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, P(C.c_int64)]
        L.orx_get.restype = C.c_int64
        L.orx_set_taps.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.orx_set_fd_taps.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.orx_set_fd_taps.restype = C.c_int
        L.orx_stats.argtypes = [C.c_void_p, P(OrxStats)]
        L.orx_destroy.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------ building blocks
def unpack(packed: np.ndarray, nsamp: int, order: int = 0) -> np.ndarray:
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    out = np.zeros(nsamp, dtype=np.int32)
    lib().orx_unpack(_ptr(packed), nsamp, order, _ptr(out))
    return out


def fft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    re = np.ascontiguousarray(np.real(x), dtype=np.float64).copy()
    im = np.ascontiguousarray(np.imag(x), dtype=np.float64).copy()
    lib().orx_fft(_ptr(re), _ptr(im), len(re), int(inverse))
    return re + 1j * im


def hilbert_circ(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    phi = np.zeros_like(u)
    lib().orx_hilbert_circ(_ptr(u), _ptr(phi), len(u))
    return phi


def kk_circ(intensity: np.ndarray) -> np.ndarray:
    I = np.ascontiguousarray(intensity, dtype=np.float64)
    re, im = np.zeros_like(I), np.zeros_like(I)
    lib().orx_kk_circ(_ptr(I), _ptr(re), _ptr(im), len(I))
    return re + 1j * im


def rrc(beta: float, sps: int, span: int) -> np.ndarray:
    h = np.zeros(sps * span + 1)
    lib().orx_rrc(beta, sps, span, _ptr(h))
    return h


def rrc_half(beta: float, sps: int, half: int) -> np.ndarray:
    h = np.zeros(2 * half + 1)
    lib().orx_rrc_half(beta, sps, half, _ptr(h))
    return h


def fd_response(h: np.ndarray, n: int) -> np.ndarray:
    """H_k = sum_i h_i e^{-2 pi i k i / n}, taps i = -(L-1)/2 .. (L-1)/2."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    re, im = np.zeros(n), np.zeros(n)
    lib().orx_fd_response(_ptr(h), len(h), n, _ptr(re), _ptr(im))
    return re + 1j * im


def fd_block(x: np.ndarray, H: np.ndarray) -> np.ndarray:
    """One frequency-domain block with bin-truncation downsampling: N inputs -> N/4 outputs."""
    n = len(x)
    xr = np.ascontiguousarray(np.real(x), dtype=np.float64)
    xi = np.ascontiguousarray(np.imag(x), dtype=np.float64)
    Hr = np.ascontiguousarray(np.real(H), dtype=np.float64)
    Hi = np.ascontiguousarray(np.imag(H), dtype=np.float64)
    yr, yi = np.zeros(n // 4), np.zeros(n // 4)
    lib().orx_fd_block(_ptr(xr), _ptr(xi), n, _ptr(Hr), _ptr(Hi), _ptr(yr), _ptr(yi))
    return yr + 1j * yi


def fd_block_full(x: np.ndarray, H: np.ndarray) -> np.ndarray:
    """One frequency-domain block at the input rate: N inputs -> the N/2 central outputs."""
    n = len(x)
    xr = np.ascontiguousarray(np.real(x), dtype=np.float64)
    xi = np.ascontiguousarray(np.imag(x), dtype=np.float64)
    Hr = np.ascontiguousarray(np.real(H), dtype=np.float64)
    Hi = np.ascontiguousarray(np.imag(H), dtype=np.float64)
    yr, yi = np.zeros(n // 2), np.zeros(n // 2)
    lib().orx_fd_block_full(_ptr(xr), _ptr(xi), n, _ptr(Hr), _ptr(Hi), _ptr(yr), _ptr(yi))
    return yr + 1j * yi


def rs_taps(mu: float) -> np.ndarray:
    """The resampler's 16 interpolator taps (j = -7 .. 8) at fraction mu."""
    c = np.zeros(16)
    lib().orx_rs_taps(mu, _ptr(c))
    return c


def fd_clock(x: np.ndarray, H: np.ndarray, w: int, sps: int = 4) -> complex:
    """Band-edge clock correlation of one FD block (N inputs at sps samples/symbol)."""
    xr = np.ascontiguousarray(np.real(x), dtype=np.float64)
    xi = np.ascontiguousarray(np.imag(x), dtype=np.float64)
    Hr = np.ascontiguousarray(np.real(H), dtype=np.float64)
    Hi = np.ascontiguousarray(np.imag(H), dtype=np.float64)
    cr, ci = C.c_double(), C.c_double()
    lib().orx_fd_clock(_ptr(xr), _ptr(xi), len(xr), _ptr(Hr), _ptr(Hi), sps, w, C.byref(cr), C.byref(ci))
    return complex(cr.value, ci.value)


def clock_fit(c: np.ndarray, centers: np.ndarray, sps: int = 4):
    """(ppm, delay in ADC samples) from block correlations and block centres
    (symbol period sps ADC samples: 4 for KK, 2 for PAM)."""
    cr = np.ascontiguousarray(np.real(c), dtype=np.float64)
    ci = np.ascontiguousarray(np.imag(c), dtype=np.float64)
    ce = np.ascontiguousarray(centers, dtype=np.int64)
    ppm, dl = C.c_double(), C.c_double()
    if lib().orx_clock_fit(_ptr(cr), _ptr(ci), _ptr(ce), len(cr), sps, C.byref(ppm), C.byref(dl)) != 0:
        raise ValueError("too few blocks")
    return ppm.value, dl.value


def rs_params(clock_step: int, clock_phase0: int):
    """Resampler accumulator (rs_step, rs_phase0) that inverts an ADC clock whose
    sample n lies at transmitter time (clock_phase0 + n clock_step) / 2^32."""
    step = ((1 << 64) + clock_step // 2) // clock_step
    ph = -(((clock_phase0 << 32) + clock_step // 2) // clock_step)
    return int(step), int(ph)


def prbs15(seed: int, nbits: int) -> np.ndarray:
    out = np.zeros(nbits, dtype=np.uint8)
    lib().orx_prbs15(seed, nbits, _ptr(out))
    return out


def q_db(ber: float) -> float:
    return lib().orx_q_db(ber)


def bps_metrics(z: np.ndarray, mq: int, scale: float, B: int) -> np.ndarray:
    re = np.ascontiguousarray(np.real(z), dtype=np.float64)
    im = np.ascontiguousarray(np.imag(z), dtype=np.float64)
    out = np.zeros(B)
    lib().orx_bps_metrics(_ptr(re), _ptr(im), len(re), mq, scale, B, _ptr(out))
    return out


# ------------------------------------------------------------------ CNN
CNN_C, CNN_K, CNN_H = 32, 9, 64


def cnn_nparams() -> int:
    return lib().orx_cnn_nparams()


def cnn_loss_grad(prm: np.ndarray, x: np.ndarray, tgt: np.ndarray, grad: bool = True):
    """x: (nseg, 2S+24, 2) inputs, tgt: (nseg, S, 2) -> (loss, grad or None, out)."""
    prm = np.ascontiguousarray(prm, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    tgt = np.ascontiguousarray(tgt, dtype=np.float64)
    nseg, S = tgt.shape[0], tgt.shape[1]
    assert x.shape == (nseg, 2 * S + 24, 2)
    g = np.zeros(cnn_nparams()) if grad else None
    out = np.zeros((nseg, S, 2))
    loss = lib().orx_cnn_loss_grad(_ptr(prm), _ptr(x), _ptr(tgt), nseg, S, _ptr(g) if grad else None, _ptr(out))
    return loss, g, out


def cnn_param_slices():
    """name -> (offset, shape) of the parameter vector."""
    C, K, H = CNN_C, CNN_K, CNN_H
    shapes = [("W1", (C, K, 2)), ("b1", (C,)), ("W2", (C, K, C)), ("b2", (C,)), ("W3", (C, K, C)), ("b3", (C,)),
              ("M1", (H, C)), ("c1", (H,)), ("M2", (2, H)), ("c2", (2,))]
    out, off = {}, 0
    for n, sh in shapes:
        out[n] = (off, sh)
        off += int(np.prod(sh))
    assert off == cnn_nparams()
    return out


# ------------------------------------------------------------------ receiver
KK_DEFAULTS = dict(sps=4, pack_order=0, ols_n=65536, ols_v=4096, ds_num=11, ds_den=80,
                   rrc_beta=0.1, mf_span=16, ntaps=31, ntrain=16384, ncma=8192, eq_block=128,
                   win=64, mu=1e-3, mu_train=1e-3, mu_cma=1e-3, bps_b=32, amb_syms=1024,
                   prbs_seed=1, eq_frozen=0, mf_mode=0, fd_n=1024, fd_taps=203, clk_track=0, rs_step=0,
                   rs_phase0=0, diff_code=0, eq_mode=0)
PAM_DEFAULTS = dict(sps=2, pack_order=0, ols_n=0, ols_v=0, ds_num=0, ds_den=1, rrc_beta=0.1,
                    mf_span=16, ntaps=15, ntrain=4096, ncma=0, eq_block=256, win=64, mu=1e-3,
                    mu_train=1e-3, mu_cma=0.0, bps_b=1, amb_syms=0, prbs_seed=1, eq_frozen=0, mf_mode=0,
                    fd_n=1024, fd_taps=503, clk_track=0, rs_step=0, rs_phase0=0,
                    diff_code=0, eq_mode=0)


def default_cfg(fmt: int, buf_len: int, **kw) -> dict:
    d = dict(KK_DEFAULTS if fmt >= 3 else PAM_DEFAULTS)
    d.update(format=fmt, buf_len=buf_len)
    d.update(kw)
    return d


class Oracle:
    """Streaming FP64 receiver; ``process`` takes one packed buffer per call."""

    def __init__(self, **cfg):
        self.cfg = dict(cfg)
        c = OrxCfg(**{k: cfg[k] for k, _ in OrxCfg._fields_})
        self._h = lib().orx_create(C.byref(c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.kk = cfg["format"] >= 3
        self.bps = [1, 2, 3, 2, 4][cfg["format"]]

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orx_destroy(self._h)
            self._h = None

    def process(self, packed: np.ndarray) -> np.ndarray:
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        c = self.cfg   # a call can emit the symbols held back by the previous one: one block more
        cap = self.bps * (c["buf_len"] // c["sps"] + c["eq_block"] + c["ntrain"] + 64)
        out = np.zeros((cap + 7) // 8, dtype=np.uint8)
        nbits = lib().orx_process(self._h, _ptr(packed), _ptr(out), cap)
        return out[: (nbits + 7) // 8].copy(), int(nbits)

    def flush(self):
        """End of the stream: (bits, nbits) of the symbols still held back."""
        c = self.cfg
        cap = self.bps * (2 * c["buf_len"] + 4 * c["eq_block"] + c["ntrain"] + 2 * c.get("ols_n", 0) + 8192)
        out = np.zeros((cap + 7) // 8, dtype=np.uint8)
        nbits = lib().orx_flush(self._h, _ptr(out), cap)
        return out[: (nbits + 7) // 8].copy(), int(nbits)

    def clock_track(self):
        """(ppm, delay, blocks) of the clock tracker's running fit (clk_track=1), or None."""
        ppm, dl = C.c_double(), C.c_double()
        n = lib().orx_clock_track(self._h, C.byref(ppm), C.byref(dl))
        return None if n < 0 else (ppm.value, dl.value, int(n))

    def set_rs(self, step: int, nudge: int = 0):
        if lib().orx_set_rs(self._h, int(step), int(nudge)) != 0:
            raise ValueError("resampler step rejected")

    def clock_retime(self):
        """Closed loop: re-time the resampler from the tracker; returns (step, nudge)."""
        st, nu = C.c_int64(), C.c_int64()
        if lib().orx_clock_retime(self._h, C.byref(st), C.byref(nu)) != 0:
            raise ValueError("no retime (no resampler or too few blocks)")
        return int(st.value), int(nu.value)

    def get(self, what: int):
        start = C.c_int64(0)
        n = lib().orx_get(self._h, what, None, 0, C.byref(start))
        if what in (ORX_E, ORX_Y, ORX_Z, ORX_V, ORX_TAPS, ORX_RS, ORX_CLK):
            buf = np.zeros(2 * n, dtype=np.float64)
            lib().orx_get(self._h, what, _ptr(buf), n, C.byref(start))
            return buf[0::2] + 1j * buf[1::2], start.value
        if what in (ORX_AHAT, ORX_DRAW):
            buf = np.zeros(2 * n, dtype=np.int32)
            lib().orx_get(self._h, what, _ptr(buf), n, C.byref(start))
            return buf.reshape(-1, 2), start.value
        if what in (ORX_BERR, ORX_NEAR):
            buf = np.zeros(n, dtype=np.int32)
            lib().orx_get(self._h, what, _ptr(buf), n, C.byref(start))
            return buf, start.value
        if what == ORX_WIN:
            buf = np.zeros(4 * n, dtype=np.float64)
            lib().orx_get(self._h, what, _ptr(buf), n, C.byref(start))
            return buf.reshape(-1, 4), start.value
        if what == ORX_SCAL:
            buf = np.zeros(5, dtype=np.float64)
            lib().orx_get(self._h, what, _ptr(buf), 5, C.byref(start))
            return buf, 0
        raise ValueError(what)

    def set_taps(self, taps: np.ndarray):
        taps = np.asarray(taps, dtype=np.complex128)
        re = np.ascontiguousarray(taps.real)
        im = np.ascontiguousarray(taps.imag)
        lib().orx_set_taps(self._h, _ptr(re), _ptr(im), len(taps))

    def set_fd_taps(self, taps: np.ndarray):
        """Zero-phase taps of the static frequency-domain filter, h_{-L} first."""
        taps = np.asarray(taps)
        re = np.ascontiguousarray(taps.real, dtype=np.float64)
        im = np.ascontiguousarray(taps.imag, dtype=np.float64) if np.iscomplexobj(taps) else None
        if lib().orx_set_fd_taps(self._h, _ptr(re), None if im is None else _ptr(im), len(taps)) != 0:
            raise ValueError("static FD taps refused")

    def stats(self) -> dict:
        s = OrxStats()
        lib().orx_stats(self._h, C.byref(s))
        return {k: getattr(s, k) for k, _ in OrxStats._fields_}
