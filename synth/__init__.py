"""Seeded synthetic transmitter, channel and 12-bit ADC.

This module stands in for the optical hardware of the field trial (laser, IQ
modulator, fibre link, photodiode and the 4 GS/s 12-bit PCIe ADC of Sec. 2 and
Sec. 3).  It produces the packed ADC buffers that both the FP64 oracle and the
CUDA receiver consume, plus the transmitted truth.  It contains none of the
receiver's arithmetic: no unpacking, no Kramers-Kronig step, no matched filter,
no equaliser and no decisions.  It shares no code with either receiver.

Transmitter and channel readings (the paper gives the hardware, not a model):

* bits: PRBS-15 (x^15 + x^14 + 1), consumed MSB-first per symbol;
* symbols: binary-reflected Gray maps onto odd-integer levels; QAM is scaled
  to unit mean power;
* pulse: root-raised cosine, unit energy, span ``span`` symbols, zero phase
  (symbol k peaks at sample k*sps);
* PAM (direct detection, Sec. 2 PAM chain): intensity I = 1 + m*s/3 with a
  fixed symbol-spaced ISI FIR applied to the symbols, then real AWGN on the
  detected intensity with variance Var(I)/SNR;
* KK (Kramers-Kronig chain, Sec. 2): the RRC-shaped complex baseband is shifted
  up by ``fd`` so it occupies [0, 2*fd], Wiener phase noise of linewidth
  ``linewidth`` is applied relative to a real tone at 0 Hz whose power is CSPR
  times the signal power, complex AWGN of per-sample variance P_s*sps/SNR is
  added and the photodiode returns |E|^2;
* ADC: code = clamp(floor(I/I_fs*4095 + 0.5), 0, 4095) with
  I_fs = mean(I) + 4*std(I) per buffer, packed two samples per three bytes.
"""

from __future__ import annotations

import numpy as np

try:  # overlap-add convolution is much faster for long buffers
    from scipy.signal import oaconvolve as _conv
except Exception:  # pragma: no cover - scipy is present on both machines
    _conv = None

__all__ = [
    "FORMATS", "prbs15_bits", "gray_index", "tx_levels", "rrc_pulse",
    "pack12", "gen_pam_stream", "gen_kk_stream",
]

# format id -> (name, bits per symbol, kind)
FORMATS = {
    0: ("PAM2", 1, "pam"),
    1: ("PAM4", 2, "pam"),
    2: ("PAM8", 3, "pam"),
    3: ("KK_QPSK", 2, "qam"),
    4: ("KK_16QAM", 4, "qam"),
}


# ---------------------------------------------------------------- bits, maps
def prbs15_bits(seed: int, nbits: int) -> np.ndarray:
    """PRBS-15 bit stream (uint8 0/1), Fibonacci LFSR x^15 + x^14 + 1.

    Register r1..r15 is loaded with ((seed mod 32767) + 1), bit i-1 -> r_i.
    Each step outputs and shifts in r14 XOR r15.  One period (32767 bits) is
    generated and tiled.
    """
    reg = (int(seed) % 32767) + 1
    period = np.empty(32767, dtype=np.uint8)
    for i in range(32767):
        new = ((reg >> 13) ^ (reg >> 14)) & 1
        reg = ((reg << 1) | new) & 0x7FFF
        period[i] = new
    reps = nbits // 32767 + 1
    return np.tile(period, reps)[:nbits].copy()


def gray_index(bits: np.ndarray, nb: int) -> np.ndarray:
    """Level index L (0 = lowest level) of each nb-bit MSB-first Gray word."""
    bits = bits.reshape(-1, nb).astype(np.int64)
    g = np.zeros(bits.shape[0], dtype=np.int64)
    for i in range(nb):
        g = (g << 1) | bits[:, i]
    # inverse of binary-reflected Gray: L = g ^ (g>>1) ^ (g>>2) ...
    L = g.copy()
    shift = g >> 1
    while np.any(shift):
        L ^= shift
        shift >>= 1
    return L


def tx_levels(fmt: int, bits: np.ndarray) -> np.ndarray:
    """Transmitted symbols: real odd-integer PAM levels or unit-power QAM."""
    name, bps, kind = FORMATS[fmt]
    if kind == "pam":
        M = 1 << bps
        L = gray_index(bits, bps)
        return (2 * L - (M - 1)).astype(np.float64)
    if fmt == 3:  # QPSK: b0 -> I, b1 -> Q, 0 -> -1, 1 -> +1
        b = bits.reshape(-1, 2).astype(np.float64)
        return ((2 * b[:, 0] - 1) + 1j * (2 * b[:, 1] - 1)) / np.sqrt(2.0)
    b = bits.reshape(-1, 4)
    li = gray_index(b[:, :2].reshape(-1), 2)
    lq = gray_index(b[:, 2:].reshape(-1), 2)
    return ((2 * li - 3) + 1j * (2 * lq - 3)) / np.sqrt(10.0)


def rrc_pulse(beta: float, sps: int, span: int) -> np.ndarray:
    """Root-raised-cosine pulse, sps*span+1 taps, unit energy, zero phase."""
    half = sps * span // 2
    t = np.arange(-half, half + 1, dtype=np.float64) / sps
    p = np.empty_like(t)
    for i, ti in enumerate(t):
        if abs(ti) < 1e-12:
            p[i] = 1.0 - beta + 4.0 * beta / np.pi
        elif abs(abs(4.0 * beta * ti) - 1.0) < 1e-12:
            p[i] = beta / np.sqrt(2.0) * ((1 + 2 / np.pi) * np.sin(np.pi / (4 * beta))
                                          + (1 - 2 / np.pi) * np.cos(np.pi / (4 * beta)))
        else:
            num = np.sin(np.pi * ti * (1 - beta)) + 4 * beta * ti * np.cos(np.pi * ti * (1 + beta))
            p[i] = num / (np.pi * ti * (1 - (4 * beta * ti) ** 2))
    return p / np.sqrt(np.sum(p * p))


def pack12(codes: np.ndarray, order: int = 0) -> np.ndarray:
    """Pack 12-bit codes two per three bytes.

    order 0 (little-endian 24-bit word): b0 = s0[7:0], b1 = s0[11:8] | s1[3:0]<<4,
    b2 = s1[11:4].  order 1 (big-endian nibbles): b0 = s0[11:4],
    b1 = s0[3:0]<<4 | s1[11:8], b2 = s1[7:0].
    """
    c = np.asarray(codes, dtype=np.uint16).reshape(-1, 2)
    s0 = c[:, 0].astype(np.uint32)
    s1 = c[:, 1].astype(np.uint32)
    out = np.empty((c.shape[0], 3), dtype=np.uint8)
    if order == 0:
        out[:, 0] = s0 & 0xFF
        out[:, 1] = ((s0 >> 8) & 0x0F) | ((s1 & 0x0F) << 4)
        out[:, 2] = (s1 >> 4) & 0xFF
    else:
        out[:, 0] = (s0 >> 4) & 0xFF
        out[:, 1] = ((s0 & 0x0F) << 4) | ((s1 >> 8) & 0x0F)
        out[:, 2] = s1 & 0xFF
    return out.reshape(-1)


# ------------------------------------------------------------------- helpers
def _shape(sym: np.ndarray, pulse: np.ndarray, sps: int, n0: int, n1: int) -> np.ndarray:
    """Samples [n0, n1) of sum_k sym[k] * pulse[n - sps*k + half]."""
    half = (len(pulse) - 1) // 2
    k0 = max(0, -((-(n0 - half)) // sps))
    k1 = min(len(sym), (n1 - 1 + half) // sps + 1)
    out_len = n1 - n0
    if k1 <= k0:
        return np.zeros(out_len, dtype=sym.dtype)
    up = np.zeros((k1 - k0) * sps, dtype=sym.dtype)
    up[::sps] = sym[k0:k1]
    if _conv is not None and len(up) > 4096:
        full = _conv(up, pulse)
    else:
        full = np.convolve(up, pulse)
    # full[j] = sum_i up[i] pulse[j-i]; sample n = sps*k0 + j - half
    start = n0 - (sps * k0 - half)
    res = np.zeros(out_len, dtype=full.dtype)
    lo = max(0, -start)
    hi = min(out_len, len(full) - start)
    if hi > lo:
        res[lo:hi] = full[start + lo:start + hi]
    return res


def _quantise(I: np.ndarray):
    i_fs = float(np.mean(I) + 4.0 * np.std(I))
    q = np.floor(I / i_fs * 4095.0 + 0.5)
    clips = int(np.count_nonzero(q > 4095) + np.count_nonzero(q < 0))
    return np.clip(q, 0, 4095).astype(np.uint16), clips


# ------------------------------------------------------------------- streams
def gen_pam_stream(fmt: int, buf_len: int, nbufs: int, seed: int = 1, snr_db: float = 18.0,
                   isi=(0.1, 1.0, 0.2), beta: float = 0.1, span: int = 16, sps: int = 2,
                   mod_index: float = 0.5, noise: bool = True, prbs_seed: int = 1,
                   pack_order: int = 0):
    """Direct-detection PAM-M stream split into nbufs ADC buffers of buf_len samples.

    Returns dict with 'packed' (list of uint8 arrays), 'codes', 'bits',
    'symbols' (transmitted levels), 'intensity' (noiseless I_tx) and 'clips'.
    """
    name, bps, kind = FORMATS[fmt]
    assert kind == "pam"
    total = buf_len * nbufs
    nsym = total // sps + span + 8
    bits = prbs15_bits(prbs_seed, nsym * bps)
    a = tx_levels(fmt, bits)
    M = 1 << bps
    # symbol-spaced ISI: pre-cursor isi[0], main isi[1], post-cursor isi[2]
    a_isi = isi[1] * a.copy()
    a_isi[:-1] += isi[0] * a[1:]
    a_isi[1:] += isi[2] * a[:-1]
    pulse = rrc_pulse(beta, sps, span)
    packed, codes_all, itx_all, clips = [], [], [], 0
    for b in range(nbufs):
        n0, n1 = b * buf_len, (b + 1) * buf_len
        s = _shape(a_isi, pulse, sps, n0, n1)
        itx = 1.0 + mod_index * s / float(M - 1)
        clips += int(np.count_nonzero(itx < 0))
        itx = np.maximum(itx, 0.0)
        I = itx.copy()
        if noise:
            rng = np.random.default_rng([int(seed), b, 17])
            sig2 = float(np.var(itx)) / 10.0 ** (snr_db / 10.0)
            I = I + rng.standard_normal(len(I)) * np.sqrt(sig2)
        codes, c = _quantise(I)
        clips += c
        packed.append(pack12(codes, pack_order))
        codes_all.append(codes)
        itx_all.append(itx)
    return dict(packed=packed, codes=np.concatenate(codes_all), bits=bits, symbols=a,
                intensity=np.concatenate(itx_all), clips=clips, fmt=fmt, sps=sps,
                buf_len=buf_len)


def gen_kk_stream(fmt: int, buf_len: int, nbufs: int, seed: int = 1, snr_db: float = 20.0,
                  cspr_db: float = 10.0, linewidth: float = 100e3, fs: float = 4e9,
                  sps: int = 4, beta: float = 0.1, span: int = 16, fd_num: int = 11,
                  fd_den: int = 80, noise: bool = True, phase_noise: bool = True,
                  volterra=(0.0, 0.0), prbs_seed: int = 1, pack_order: int = 0,
                  symbols=None, phase_offset: float = 0.0, phase_steps=()):
    """Kramers-Kronig single-sideband QAM stream split into ADC buffers.

    The signal sits above a real tone at 0 Hz after an up-shift of fd_num/fd_den
    cycles per sample.  ``volterra`` = (c1, c2) adds c1*x|x|^2 + c2*x[n-sps]|x[n-sps]|^2
    to the shaped baseband before the shift.  ``symbols`` overrides the PRBS
    symbols (used for training data that must not follow an LFSR recurrence).
    Returns dict with 'packed', 'codes', 'bits', 'symbols', 'field' (noiseless
    complex baseband at sps, before the shift: what the receiver should recover)
    and 'clips'.
    """
    name, bps, kind = FORMATS[fmt]
    assert kind == "qam"
    total = buf_len * nbufs
    nsym = total // sps + span + 8
    if symbols is None:
        bits = prbs15_bits(prbs_seed, nsym * bps)
        a = tx_levels(fmt, bits)
    else:
        bits = None
        a = np.asarray(symbols, dtype=np.complex128)
        assert len(a) >= nsym
    pulse = rrc_pulse(beta, sps, span)
    Ps = float(np.mean(np.abs(a) ** 2)) / sps  # per-sample power of the shaped signal
    A = np.sqrt(10.0 ** (cspr_db / 10.0) * Ps)
    sig2 = Ps * sps / 10.0 ** (snr_db / 10.0)
    pn_std = np.sqrt(2.0 * np.pi * linewidth / fs)
    theta0 = float(phase_offset)
    packed, codes_all, field_all, clips = [], [], [], 0
    c1, c2 = volterra
    for b in range(nbufs):
        n0, n1 = b * buf_len, (b + 1) * buf_len
        s = _shape(a, pulse, sps, n0 - sps, n1)
        if c1 != 0.0 or c2 != 0.0:
            p = np.abs(s) ** 2
            nl = c1 * s * p
            nl[sps:] += c2 * s[:-sps] * p[:-sps]
            s = s + nl
        s = s[sps:]
        field_all.append(s.copy())
        n = np.arange(n0, n1, dtype=np.int64)
        up = np.exp(2j * np.pi * ((n * fd_num) % fd_den) / fd_den)
        rng = np.random.default_rng([int(seed), b, 29])
        if phase_noise and linewidth > 0:
            th = theta0 + np.cumsum(rng.standard_normal(len(s)) * pn_std)
            theta0 = float(th[-1])
        else:
            th = np.full(len(s), theta0)
        for (ns, dth) in phase_steps:
            if ns < n1:
                th[max(0, ns - n0):] += dth
        E = A + s * up * np.exp(1j * th)
        if noise:
            E = E + (rng.standard_normal(len(s)) + 1j * rng.standard_normal(len(s))) * np.sqrt(sig2 / 2.0)
        I = np.abs(E) ** 2
        codes, c = _quantise(I)
        clips += c
        packed.append(pack12(codes, pack_order))
        codes_all.append(codes)
    return dict(packed=packed, codes=np.concatenate(codes_all), bits=bits, symbols=a,
                field=np.concatenate(field_all), clips=clips, fmt=fmt, sps=sps,
                buf_len=buf_len, tone=A, Ps=Ps)
