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
    "pack12", "gen_pam_stream", "gen_kk_stream", "splitmix64_bits", "random_symbols",
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


def splitmix64_bits(seed: int, nbits: int) -> np.ndarray:
    """Bits from the counter-based splitmix64 generator (Steele, Lea, Flood 2014):
    word i = mix(seed + (i+1) * 0x9E3779B97F4A7C15), 64 bits per word, MSB first.
    Used for learned-equaliser data, which must not follow an LFSR recurrence."""
    nw = (nbits + 63) // 64
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.arange(1, nw + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    bits = np.unpackbits(z.astype(">u8").view(np.uint8))
    return bits[:nbits].copy()


def random_symbols(fmt: int, n: int, seed: int) -> np.ndarray:
    """n symbols of the format from splitmix64 bits (Gray mapped like the PRBS data)."""
    return tx_levels(fmt, splitmix64_bits(seed, n * FORMATS[fmt][1]))


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


def rrc_at(beta: float, sps: int, span: int, t: np.ndarray) -> np.ndarray:
    """The pulse of rrc_pulse(beta, sps, span) at arbitrary sample offsets t (zero
    beyond +-span/2 symbols), on the same scale as its integer-offset taps."""
    x = np.asarray(t, dtype=np.float64) / sps
    v = np.empty_like(x)
    z = np.abs(x) < 1e-12
    e = (~z) & (np.abs(np.abs(4.0 * beta * x) - 1.0) < 1e-9) if beta > 0 else np.zeros_like(z)
    g = ~(z | e)
    v[z] = 1.0 - beta + 4.0 * beta / np.pi
    if beta > 0:
        v[e] = beta / np.sqrt(2.0) * ((1 + 2 / np.pi) * np.sin(np.pi / (4 * beta))
                                      + (1 - 2 / np.pi) * np.cos(np.pi / (4 * beta)))
    xg = x[g]
    v[g] = (np.sin(np.pi * xg * (1 - beta)) + 4 * beta * xg * np.cos(np.pi * xg * (1 + beta))) / \
        (np.pi * xg * (1 - (4 * beta * xg) ** 2))
    v[np.abs(x) > span / 2] = 0.0
    ref = rrc_pulse(beta, sps, span)
    return v * (ref[len(ref) // 2] / (1.0 - beta + 4.0 * beta / np.pi))


def _shape_at(sym_seg: np.ndarray, k0: int, beta: float, sps: int, span: int, ti: np.ndarray,
              tf: np.ndarray) -> np.ndarray:
    """sum_k sym[k] p(t - sps k) at sample times t = ti + tf (integer and fractional
    parts, nominal samples) for the pulse of rrc_pulse; sym_seg[i] is symbol k0 + i.
    With u = ((ti mod sps) + tf) / sps and x = u - d (d the symbol offset), the two
    sines of the pulse follow from sin / cos of u by angle addition, so each sample
    costs four trigonometric evaluations whatever the span."""
    kc = ti // sps
    u = ((ti - sps * kc) + tf) / sps
    c1, c2 = np.pi * (1 - beta), np.pi * (1 + beta)
    S1, C1, S2, C2 = np.sin(c1 * u), np.cos(c1 * u), np.sin(c2 * u), np.cos(c2 * u)
    ref = rrc_pulse(beta, sps, span)
    scale = ref[len(ref) // 2] / (1.0 - beta + 4.0 * beta / np.pi)
    out = np.zeros(len(ti), dtype=np.complex128)
    for d in range(-(span // 2) - 1, span // 2 + 2):
        x = u - d
        num = (S1 * np.cos(c1 * d) - C1 * np.sin(c1 * d)) + 4 * beta * x * (C2 * np.cos(c2 * d) + S2 * np.sin(c2 * d))
        den = np.pi * x * (1 - (4 * beta * x) ** 2)
        special = (np.abs(x) < 1e-9) | (np.abs(np.abs(4 * beta * x) - 1.0) < 1e-6)
        v = np.where(special, 0.0, num / np.where(special, 1.0, den)) * scale
        if special.any():
            v[special] = rrc_at(beta, sps, span, sps * x[special])
        v[np.abs(x) > span / 2] = 0.0
        out += sym_seg[kc + d - k0] * v
    return out


def adc_times(n0: int, n1: int, clock_step: int, clock_phase0: int):
    """Transmitter time of ADC samples n0..n1-1 in nominal samples, from the integer
    phase accumulator phi_n = phase0 + n * step (2^32 per nominal sample):
    returns (integer part, fraction) of phi_n / 2^32."""
    assert 0 <= n0 and n1 < (1 << 30) and abs(clock_phase0) < (1 << 62) and 0 < clock_step < (1 << 33)
    phi = np.int64(clock_phase0) + np.arange(n0, n1, dtype=np.int64) * np.int64(clock_step)   # < 2^63
    ip = phi >> 32
    fr = (phi & 0xFFFFFFFF).astype(np.float64) / 4294967296.0
    return ip, fr


def clock_step(ppm: float) -> int:
    """Accumulator step of an ADC clock whose period is (1 + ppm 1e-6) nominal samples."""
    return int(round((1.0 + ppm * 1e-6) * 4294967296.0))


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
    """Samples [n0, n1) of sum_k sym[k] * pulse[n - sps*k + half] (polyphase: for
    n = sps*m + p, s[n] = sum_j sym[m - j] * pulse[sps*j + p + half])."""
    half = (len(pulse) - 1) // 2
    out_len = n1 - n0
    res = np.zeros(out_len, dtype=np.result_type(sym.dtype, pulse.dtype))
    m0 = n0 // sps - 1
    m1 = (n1 - 1) // sps + 1
    for p in range(sps):
        js = [j for j in range(-(half + p) // sps - 1, (half - p) // sps + 2)
              if 0 <= sps * j + p + half <= 2 * half]
        jlo, jhi = js[0], js[-1]
        taps = np.array([pulse[sps * j + p + half] for j in range(jlo, jhi + 1)])
        # symbols needed for outputs m in [m0, m1]: k = m - j in [m0 - jhi, m1 - jlo]
        k0, k1 = m0 - jhi, m1 - jlo
        seg = np.zeros(k1 - k0 + 1, dtype=sym.dtype)
        a, b = max(k0, 0), min(k1, len(sym) - 1)
        if b >= a:
            seg[a - k0:b - k0 + 1] = sym[a:b + 1]
        full = np.convolve(seg, taps)           # full[i] = sum_t seg[i - t] taps[t]
        # output m uses seg index (m - jlo) - k0 ... full index i = (m - jlo - k0) + 0
        ms = np.arange(m0, m1 + 1)
        vals = full[ms - jlo - k0 + 0]
        n = ms * sps + p
        sel = (n >= n0) & (n < n1)
        res[n[sel] - n0] = vals[sel]
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
                   pack_order: int = 0, clock_step: int = 1 << 32, clock_phase0: int = 0):
    """Direct-detection PAM-M stream split into nbufs ADC buffers of buf_len samples.

    Returns dict with 'packed' (list of uint8 arrays), 'codes', 'bits',
    'symbols' (transmitted levels), 'intensity' (noiseless I_tx) and 'clips'.
    ``clock_step`` / ``clock_phase0``: the ADC takes sample n at transmitter time
    (clock_phase0 + n clock_step) / 2^32 nominal samples, as in gen_kk_stream.
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
    offclock = clock_step != (1 << 32) or clock_phase0 != 0
    packed, codes_all, itx_all, clips = [], [], [], 0
    for b in range(nbufs):
        n0, n1 = b * buf_len, (b + 1) * buf_len
        if offclock:   # the ADC samples at transmitter times phi_n / 2^32 (nominal samples)
            ti, tf = adc_times(n0, n1, clock_step, clock_phase0)
            half = span // 2 + 2
            ka, kb = int(ti[0]) // sps - half - 2, int(ti[-1]) // sps + half + 3
            seg = np.zeros(kb - ka)
            lo, hi = max(ka, 0), min(kb, len(a_isi))
            if hi > lo:
                seg[lo - ka:hi - ka] = a_isi[lo:hi]
            s = _shape_at(seg, ka, beta, sps, span, ti, tf).real
        else:
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


def diff_qam_symbols(fmt: int, bits: np.ndarray, q0: int = 0):
    """Differentially quadrant-coded QAM (the optional coding of the KK chain): per
    symbol the first two bits, Gray-decoded, step the quadrant, Q_k = (Q_{k-1} + D_k)
    mod 4 (Q_{-1} = q0); 16QAM's last two bits pick the point of the first quadrant,
    (1 + 2 b2) + j (1 + 2 b3), which is then turned by Q_k quarter turns (so a pi/2
    rotation of the whole constellation changes the quadrants only).  Unit power.
    Returns (symbols, quadrant of the last symbol)."""
    name, bps, kind = FORMATS[fmt]
    b = bits.reshape(-1, bps).astype(np.int64)
    D = gray_index(b[:, :2].reshape(-1), 2)
    Q = (q0 + np.cumsum(D)) % 4
    base = (1 + 2 * b[:, 2] + 1j * (1 + 2 * b[:, 3])) if bps == 4 else np.full(len(b), 1 + 1j)
    sym = base * (1j ** Q) / (np.sqrt(10.0) if bps == 4 else np.sqrt(2.0))
    return sym, int(Q[-1]) if len(Q) else q0


def _tx_symbols(fmt: int, prbs_seed: int, k0: int, k1: int, period_cache={}, diff: bool = False) -> np.ndarray:
    """Transmitted symbols k in [k0, k1) of the PRBS-15 stream (k < 0 gives 0); with
    diff, the differentially quadrant-coded QAM symbols (diff_qam_symbols from
    stream symbol 0; the quadrant is a prefix sum, periodic up to a constant step per
    PRBS period of 32767 symbols)."""
    name, bps, kind = FORMATS[fmt]
    key = (prbs_seed,)
    if key not in period_cache:
        period_cache[key] = prbs15_bits(prbs_seed, 32767)
    per = period_cache[key]
    ks = np.arange(max(k0, 0), max(k1, 0), dtype=np.int64)
    out = np.zeros(k1 - k0, dtype=np.float64 if kind == "pam" else np.complex128)
    if len(ks):
        idx = (ks[:, None] * bps + np.arange(bps)[None, :]) % 32767
        if not diff:
            out[max(k0, 0) - k0:] = tx_levels(fmt, per[idx].reshape(-1))
        else:
            dkey = ("diff", prbs_seed, fmt)
            if dkey not in period_cache:   # quadrant prefix over one period, and its total step
                pidx = (np.arange(32767, dtype=np.int64)[:, None] * bps + np.arange(bps)[None, :]) % 32767
                pb = per[pidx].reshape(-1, bps)
                D = gray_index(pb[:, :2].reshape(-1), 2)
                P = np.cumsum(D) % 4
                period_cache[dkey] = (P, int(P[-1]))
            P, C = period_cache[dkey]
            Q = ((ks // 32767) * C + P[ks % 32767]) % 4
            b = per[idx].reshape(-1, bps).astype(np.int64)
            base = (1 + 2 * b[:, 2] + 1j * (1 + 2 * b[:, 3])) if bps == 4 else np.full(len(b), 1 + 1j)
            out[max(k0, 0) - k0:] = base * (1j ** Q) / (np.sqrt(10.0) if bps == 4 else np.sqrt(2.0))
    return out


def kk_phase_starts(buf_len: int, nbufs: int, seed: int, linewidth: float, fs: float,
                    phase_noise: bool = True, phase_offset: float = 0.0):
    """Wiener phase at the first sample of each buffer (the increments of buffer
    b come from their own generator, so buffers can be made independently)."""
    pn_std = np.sqrt(2.0 * np.pi * linewidth / fs)
    th, out = float(phase_offset), []
    for b in range(nbufs):
        out.append(th)
        if phase_noise and linewidth > 0:
            inc = np.random.default_rng([int(seed), b, 31]).standard_normal(buf_len) * pn_std
            th += float(np.sum(inc))
    return out


def kk_buffer(fmt: int, buf_len: int, b: int, theta0: float, seed: int = 1, snr_db: float = 20.0,
              cspr_db: float = 10.0, linewidth: float = 100e3, fs: float = 4e9, sps: int = 4,
              beta: float = 0.1, span: int = 16, fd_num: int = 11, fd_den: int = 80,
              noise: bool = True, phase_noise: bool = True, volterra=(0.0, 0.0),
              prbs_seed: int = 1, pack_order: int = 0, symbols=None, phase_steps=(),
              truth: bool = True, clock_step: int = 1 << 32, clock_phase0: int = 0,
              isi=None, sym_snr_db=None, diff: bool = False):
    """Buffer b of a Kramers-Kronig single-sideband QAM stream (see gen_kk_stream)."""
    name, bps, kind = FORMATS[fmt]
    assert kind == "qam"
    n0, n1 = b * buf_len, (b + 1) * buf_len
    pulse = rrc_pulse(beta, sps, span)
    half = span // 2 + 2
    ka, kb = (n0 - sps) // sps - half, n1 // sps + half + 1
    offclock = clock_step != (1 << 32) or clock_phase0 != 0
    if offclock:   # the ADC samples at transmitter times phi_n / 2^32 (nominal samples)
        ti, tf = adc_times(n0, n1, clock_step, clock_phase0)
        ka, kb = int(ti[0]) // sps - half - 2, int(ti[-1]) // sps + half + 3
    if symbols is None:
        a_seg = _tx_symbols(fmt, prbs_seed, ka, kb, diff=diff)
        Es = 1.0   # unit-power constellation
    else:
        sy = np.asarray(symbols, dtype=np.complex128)
        a_seg = np.zeros(kb - ka, dtype=np.complex128)
        lo, hi = max(ka, 0), min(kb, len(sy))
        if hi > lo:
            a_seg[lo - ka:hi - ka] = sy[lo:hi]
        Es = float(np.mean(np.abs(sy) ** 2))
    if isi is not None:
        # symbol-spaced ISI: a'_k = isi[0] a_{k+1} + isi[1] a_k + isi[2] a_{k-1}
        ext = np.concatenate(([0j], a_seg, [0j]))
        if symbols is None:
            ext[0] = _tx_symbols(fmt, prbs_seed, ka - 1, ka, diff=diff)[0]
            ext[-1] = _tx_symbols(fmt, prbs_seed, kb, kb + 1, diff=diff)[0]
        a_seg = isi[0] * ext[2:] + isi[1] * ext[1:-1] + isi[2] * ext[:-2]
    if sym_snr_db is not None:
        a_seg = a_seg + _symbol_noise(seed, ka, kb, Es / 10.0 ** (sym_snr_db / 10.0))
    Ps = Es / sps                      # per-sample power of the shaped signal
    A = np.sqrt(10.0 ** (cspr_db / 10.0) * Ps)
    sig2 = Ps * sps / 10.0 ** (snr_db / 10.0)
    pn_std = np.sqrt(2.0 * np.pi * linewidth / fs)
    # shaped baseband for samples [n0 - sps, n1): symbols re-indexed from ka
    if offclock:
        assert volterra == (0.0, 0.0), "clock offset with the Volterra channel is not generated"
        s = _shape_at(a_seg, ka, beta, sps, span, ti, tf)
        n = ti                           # integer part of the transmitter time
        frac_up = np.exp(2j * np.pi * (fd_num / fd_den) * tf)
    else:
        s = _shape(a_seg, pulse, sps, n0 - sps - ka * sps, n1 - ka * sps)
        c1, c2 = volterra
        if c1 != 0.0 or c2 != 0.0:
            p = np.abs(s) ** 2
            nl = c1 * s * p
            nl[sps:] += c2 * s[:-sps] * p[:-sps]
            s = s + nl
        s = s[sps:]
        n = np.arange(n0, n1, dtype=np.int64)
        frac_up = 1.0
    up = np.exp(2j * np.pi * np.arange(fd_den) / fd_den)[(n * fd_num) % fd_den] * frac_up
    if phase_noise and linewidth > 0:
        inc = np.random.default_rng([int(seed), b, 31]).standard_normal(buf_len) * pn_std
        th = theta0 + np.cumsum(inc)
    else:
        th = np.full(buf_len, theta0)
    for (ns, dth) in phase_steps:
        if ns < n1:
            th[max(0, ns - n0):] += dth
    E = A + s * up * np.exp(1j * th)
    if noise:
        rng = np.random.default_rng([int(seed), b, 29])
        E = E + (rng.standard_normal(buf_len) + 1j * rng.standard_normal(buf_len)) * np.sqrt(sig2 / 2.0)
    codes, clips = _quantise(np.abs(E) ** 2)
    out = dict(packed=pack12(codes, pack_order), clips=clips, tone=A, Ps=Ps)
    if truth:
        out.update(codes=codes, field=s)
    return out


def _symbol_noise(seed: int, ka: int, kb: int, var: float) -> np.ndarray:
    """Complex Gaussian noise of variance var for symbols [ka, kb) (zero for k < 0),
    drawn in blocks of 4096 symbols keyed by the block index, so a symbol gets the
    same value in every buffer whose span holds it."""
    out = np.zeros(kb - ka, dtype=np.complex128)
    for blk in range(max(ka, 0) // 4096, max(kb - 1, 0) // 4096 + 1):
        lo, hi = blk * 4096, blk * 4096 + 4096
        a, b = max(lo, ka, 0), min(hi, kb)
        if b <= a:
            continue
        r = np.random.default_rng([int(seed), blk, 41]).standard_normal((4096, 2))
        v = (r[:, 0] + 1j * r[:, 1]) * np.sqrt(var / 2.0)
        out[a - ka:b - ka] = v[a - lo:b - lo]
    return out


def _kk_worker(args):
    kw, b, th0 = args
    return kk_buffer(b=b, theta0=th0, **kw)


def gen_kk_stream(fmt: int, buf_len: int, nbufs: int, seed: int = 1, snr_db: float = 20.0,
                  cspr_db: float = 10.0, linewidth: float = 100e3, fs: float = 4e9,
                  sps: int = 4, beta: float = 0.1, span: int = 16, fd_num: int = 11,
                  fd_den: int = 80, noise: bool = True, phase_noise: bool = True,
                  volterra=(0.0, 0.0), prbs_seed: int = 1, pack_order: int = 0,
                  symbols=None, phase_offset: float = 0.0, phase_steps=(), workers: int = 1,
                  truth: bool = True, clock_step: int = 1 << 32, clock_phase0: int = 0,
                  isi=None, sym_snr_db=None, diff: bool = False):
    """Kramers-Kronig single-sideband QAM stream split into ADC buffers.

    The signal sits above a real tone at 0 Hz after an up-shift of fd_num/fd_den
    cycles per sample.  ``volterra`` = (c1, c2) adds c1*x|x|^2 + c2*x[n-sps]|x[n-sps]|^2
    to the shaped baseband before the shift.  ``symbols`` overrides the PRBS
    symbols (used for training data that must not follow an LFSR recurrence).
    ``phase_steps`` = [(sample, dtheta), ...] adds instantaneous phase jumps.
    ``workers`` > 1 makes the buffers in a spawn-started process pool.
    ``clock_step`` / ``clock_phase0``: the ADC takes sample n at transmitter time
    (clock_phase0 + n clock_step) / 2^32 nominal samples (integer accumulator; see
    clock_step()); the default is the nominal grid.
    ``isi`` = (pre, main, post): symbol-spaced ISI on the symbols before shaping, as
    in gen_pam_stream.  ``sym_snr_db``: complex AWGN of that Es/N0 added to the
    symbols before shaping, i.e. noise confined to the signal band (after the unit-
    energy matched filter the symbol samples carry exactly that noise); usually
    with noise=False.  ``diff``: differentially quadrant-coded symbols of the PRBS bits
    (diff_qam_symbols); the receiver needs rx_config.diff_code = 1.
    Returns dict with 'packed' (per buffer), 'codes', 'symbols' (the transmitted
    symbols of the stream), 'field' (noiseless complex baseband at sps, before the
    shift: what the receiver should recover; with truth=True) and 'clips'.
    """
    name, bps, kind = FORMATS[fmt]
    assert kind == "qam"
    nsym = buf_len * nbufs // sps + span + 8
    kw = dict(fmt=fmt, buf_len=buf_len, seed=seed, snr_db=snr_db, cspr_db=cspr_db,
              linewidth=linewidth, fs=fs, sps=sps, beta=beta, span=span, fd_num=fd_num,
              fd_den=fd_den, noise=noise, phase_noise=phase_noise, volterra=volterra,
              prbs_seed=prbs_seed, pack_order=pack_order, symbols=symbols,
              phase_steps=tuple(phase_steps), truth=truth, clock_step=int(clock_step),
              clock_phase0=int(clock_phase0), isi=None if isi is None else tuple(isi),
              sym_snr_db=sym_snr_db, diff=bool(diff))
    th0 = kk_phase_starts(buf_len, nbufs, seed, linewidth, fs, phase_noise, phase_offset)
    jobs = [(kw, b, th0[b]) for b in range(nbufs)]
    if workers > 1 and nbufs > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_kk_worker, jobs))
    else:
        parts = [_kk_worker(j) for j in jobs]
    if symbols is None:
        a = _tx_symbols(fmt, prbs_seed, 0, nsym, diff=diff)
        bits = prbs15_bits(prbs_seed, nsym * bps)
    else:
        a, bits = np.asarray(symbols, dtype=np.complex128), None
    out = dict(packed=[p["packed"] for p in parts], symbols=a, bits=bits,
               clips=sum(p["clips"] for p in parts), fmt=fmt, sps=sps, buf_len=buf_len,
               tone=parts[0]["tone"], Ps=parts[0]["Ps"])
    if truth:
        out["codes"] = np.concatenate([p["codes"] for p in parts])
        out["field"] = np.concatenate([p["field"] for p in parts])
    return out
