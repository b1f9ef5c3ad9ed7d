"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against a closed form, a brute-force computation,
an independent library routine, a mathematical property or a textbook
statistic, chosen so that a plausible slip (a dropped term, a wrong sign, a
wrong index or block offset) fails at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest
from scipy.special import erfc
from scipy.stats import norm

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- FFT
@pytest.mark.parametrize("n", [2, 4, 8, 64, 256, 1024])
def test_fft_matches_brute_force_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(k, k) / n)   # DFT matrix written out
    ref = F @ x
    got = oracle.fft(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * n * np.max(np.abs(ref))
    back = oracle.fft(got, inverse=True)
    assert np.max(np.abs(back - x)) <= 1e-13 * n


def test_fft_matches_pocketfft_large():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(65536) + 1j * rng.standard_normal(65536)
    got = oracle.fft(x)
    ref = np.fft.fft(x)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-13


# -------------------------------------------------------------- Hilbert
@pytest.mark.parametrize("k0", [1, 5, 37, 511])
def test_hilbert_of_cos_is_sin(k0):
    n = 1024
    t = np.arange(n)
    u = np.cos(2 * np.pi * k0 * t / n + 0.3)
    phi = oracle.hilbert_circ(u)
    assert np.max(np.abs(phi - np.sin(2 * np.pi * k0 * t / n + 0.3))) < 1e-12


def test_hilbert_kills_dc_and_nyquist():
    n = 256
    t = np.arange(n)
    u = 3.5 + 0.7 * np.cos(np.pi * t)   # DC and the Nyquist bin only
    assert np.max(np.abs(oracle.hilbert_circ(u))) < 1e-13


def _min_phase_field(n, rng, sign=+1):
    t = np.arange(n)
    ks = rng.choice(np.arange(1, 40), size=6, replace=False)
    c = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    c *= 0.3 / np.sum(np.abs(c))
    return 1.0 + sum(ci * np.exp(sign * 2j * np.pi * ki * t / n) for ci, ki in zip(c, ks))


def test_kk_reconstructs_minimum_phase_field():
    # strong carrier (1 > sum|c_k| = 0.3), tones on one side: ln E is analytic,
    # so sqrt(I) exp(j H{ln I / 2}) returns E up to the aliasing of ln's
    # harmonics, which decays as 0.3^m
    rng = np.random.default_rng(3)
    E = _min_phase_field(4096, rng)
    got = oracle.kk_circ(np.abs(E) ** 2)
    assert np.max(np.abs(got - E)) < 1e-12


def test_kk_mirror_sideband_gives_conjugate():
    rng = np.random.default_rng(4)
    E = _min_phase_field(4096, rng, sign=-1)
    got = oracle.kk_circ(np.abs(E) ** 2)
    assert np.max(np.abs(got - np.conj(E))) < 1e-12
    assert np.max(np.abs(got - E)) > 1e-2


# -------------------------------------------------------------------- RRC
@pytest.mark.parametrize("sps", [2, 4])
def test_rrc_is_unit_energy_symmetric_nyquist(sps):
    h = oracle.rrc(0.1, sps, 16)
    assert len(h) == 16 * sps + 1
    assert abs(np.sum(h * h) - 1.0) < 1e-14
    assert np.max(np.abs(h - h[::-1])) < 1e-15
    rc = np.convolve(h, h)          # raised cosine
    mid = len(rc) // 2
    at_symbols = rc[mid % sps::sps]
    k = (np.arange(len(at_symbols)) * sps + mid % sps) - mid
    assert abs(at_symbols[k == 0][0] - 1.0) < 2e-3
    assert np.max(np.abs(at_symbols[k != 0])) < 2e-2   # zero ISI up to truncation
    # spectrum: flat in-band, small beyond the roll-off edge
    f = np.array([0.0, 0.2, 0.35]) / sps
    H = np.abs([np.sum(h * np.exp(-2j * np.pi * fi * np.arange(len(h)))) for fi in f])
    assert np.max(np.abs(H / H[0] - 1.0)) < 0.02   # truncation ripple of a 16-symbol span
    Hs = np.abs(np.sum(h * np.exp(-2j * np.pi * (0.7 / sps) * np.arange(len(h)))))
    assert Hs / H[0] < 0.03


def test_rrc_beta_zero_is_sinc():
    h = oracle.rrc(0.0, 4, 16)
    t = (np.arange(len(h)) - 32) / 4
    s = np.sinc(t)
    assert np.max(np.abs(h - s / np.sqrt(np.sum(s * s)))) < 1e-14


# ------------------------------------------------------------------- PRBS
def test_prbs15_period_balance_recurrence():
    b = oracle.prbs15(1, 3 * 32767).astype(np.int64)
    assert np.array_equal(b[:32767], b[32767:65534])
    for p in (3, 7, 31, 127, 151, 217, 1057, 4681):   # divisors of 32767 are not periods
        assert not np.array_equal(b[:2000], b[p:p + 2000])
    assert int(b[:32767].sum()) == 16384
    n = np.arange(15, 5000)
    assert np.array_equal(b[n], b[n - 14] ^ b[n - 15])


def test_prbs15_matches_generator():
    assert np.array_equal(oracle.prbs15(5, 40000), synth.prbs15_bits(5, 40000))


# ----------------------------------------------------------------- unpack
@pytest.mark.parametrize("order", [0, 1])
def test_unpack_round_trip_every_code_pair(order):
    a = np.repeat(np.arange(4096, dtype=np.uint16), 4096)
    b = np.tile(np.arange(4096, dtype=np.uint16), 4096)
    codes = np.empty(2 * a.size, dtype=np.uint16)
    codes[0::2] = a
    codes[1::2] = b
    packed = synth.pack12(codes, order)
    got = oracle.unpack(packed, codes.size, order)
    assert np.array_equal(got, codes.astype(np.int32))


def test_unpack_bit_layout():
    # 0xABC, 0x123 little-endian 24-bit word: 0x123ABC -> bytes BC 3A 12
    got = oracle.unpack(np.array([0xBC, 0x3A, 0x12], np.uint8), 2, 0)
    assert list(got) == [0xABC, 0x123]
    got = oracle.unpack(np.array([0xAB, 0xC1, 0x23], np.uint8), 2, 1)
    assert list(got) == [0xABC, 0x123]


# --------------------------------------------------------------- Q factor
def test_q_from_ber_closed_form():
    for q_lin in (2.0, 3.0, 4.5, 6.0):
        ber = 0.5 * erfc(q_lin / math.sqrt(2.0))
        assert abs(oracle.q_db(ber) - 20 * math.log10(q_lin)) < 1e-9


def test_paper_numbers():
    """Real-time budget and HD-FEC Q threshold as printed in the paper."""
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))
    assert g["buffer_samples"] == 2 ** 22
    budget_ms = g["streams"] * g["buffer_samples"] / g["adc_rate_sps"] * 1e3
    assert abs(budget_ms - g["budget_ms"]) < 5e-4
    # Q of 8.4 dB corresponds to the 6.7 % HD-FEC limit (pre-FEC BER 3.8e-3)
    assert abs(oracle.q_db(g["hd_fec_6p7_ber"]) - g["hd_fec_6p7_q_db"]) < 0.15


# ------------------------------------------------------------- streaming KK
def _periodic_codes(P, total, rng):
    """Integer intensities of a P-periodic minimum-phase field."""
    t = np.arange(P)
    E = 40.0 + sum((rng.standard_normal() + 1j * rng.standard_normal()) * 1.5 *
                   np.exp(2j * np.pi * k * t / P) for k in (1, 3, 7, 12))
    I = np.round(np.abs(E) ** 2).astype(np.int64)
    assert I.min() > 0 and I.max() < 4096
    return np.tile(I, total // P + 1)[:total]


@pytest.mark.parametrize("buf_len", [1536, 2000, 4096, 9000])
def test_ols_hilbert_exact_on_periodic_input(buf_len):
    """A P-periodic input with P | N is reproduced exactly by every OLS block
    that lies inside the stream, whatever the call boundaries and block
    alignment; only blocks that read the pre-stream fill may differ."""
    N, V, P, calls = 1024, 256, 256, 4
    rng = np.random.default_rng(11)
    codes = _periodic_codes(P, buf_len * calls, rng)
    exact = oracle.kk_circ(codes[:P].astype(np.float64))
    cfg = oracle.default_cfg(4, buf_len, ols_n=N, ols_v=V, ntrain=64, ncma=0, eq_block=64)
    o = oracle.Oracle(**cfg)
    got = {}
    for c in range(calls):
        o.process(synth.pack12(codes[c * buf_len:(c + 1) * buf_len]))
        E, e0 = o.get(oracle.ORX_E)
        for i, v in enumerate(E):
            got[e0 + i] = v
    n = np.array(sorted(got))
    assert n[0] == 0 and np.array_equal(n, np.arange(len(n)))
    assert n[-1] == buf_len * calls - V // 2 - 1
    E = np.array([got[i] for i in n])
    sel = n >= N - V // 2
    assert np.max(np.abs(E[sel] - exact[n[sel] % P])) < 1e-10


def _noiseless_kk(fmt, nbufs=1, buf_len=1 << 20, **kw):
    g = synth.gen_kk_stream(fmt, buf_len, nbufs, seed=2, noise=False, phase_noise=False, **kw)
    o = oracle.Oracle(**oracle.default_cfg(fmt, buf_len, ols_n=8192, ols_v=1024))
    return g, o


def test_front_end_recovers_symbols():
    """Noiseless KK: after field reconstruction, carrier removal, downshift,
    matched filter and gain, the 2-sps samples at even indices are the
    transmitted unit-power symbols (up to the KK/OLS method error), with unit
    scale and zero phase, on both sides of a buffer boundary."""
    g, o = _noiseless_kk(4, nbufs=2)
    ys = {}
    for b in range(2):
        o.process(g["packed"][b])
        y, y0 = o.get(oracle.ORX_Y)
        for i in range(0, len(y)):
            ys[y0 + i] = y[i]
    m = np.array(sorted(ys))
    m = m[(m % 2 == 0) & (m > 64)]
    k = m // 2
    y = np.array([ys[i] for i in m])
    a = g["symbols"][k]
    scale = np.vdot(a, y) / np.vdot(a, a)
    assert abs(abs(scale) - 1.0) < 0.05 and abs(np.angle(scale)) < 0.02
    err = np.abs(y - a) ** 2
    assert np.sqrt(err.mean()) < 0.06
    boundary = np.abs(m - (1 << 20) // 2) < 2000      # symbols around the buffer edge
    assert np.sqrt(err[boundary].mean()) < 0.06


@pytest.mark.parametrize("fmt", [3, 4])
def test_noiseless_qam_zero_errors(fmt):
    g, o = _noiseless_kk(fmt)
    o.process(g["packed"][0])
    s = o.stats()
    assert s["bits"] > 400_000 and s["bit_errors"] == 0 and s["raw_bit_errors"] == 0


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_noiseless_pam_with_isi_zero_errors(fmt):
    N = 1 << 19
    g = synth.gen_pam_stream(fmt, N, 2, seed=3, noise=False)
    o = oracle.Oracle(**oracle.default_cfg(fmt, N))
    for b in range(2):
        o.process(g["packed"][b])
    s = o.stats()
    assert s["bits"] > 400_000 and s["bit_errors"] == 0


@pytest.mark.parametrize("theta0", [0.3, -0.5, 1.2, 2.9])
def test_bps_recovers_constant_rotation(theta0):
    g, o = _noiseless_kk(4, buf_len=1 << 19, phase_offset=theta0)
    o.process(g["packed"][0])
    s = o.stats()
    assert s["bit_errors"] == 0 and s["raw_bit_errors"] == 0
    w, _ = o.get(oracle.ORX_WIN)
    est = w[:, 0] / 32 * (np.pi / 2) - np.pi / 4 + (w[:, 1] + s["amb_rot"]) * np.pi / 2
    d = np.angle(np.exp(1j * (est - theta0)))
    assert np.max(np.abs(d)) <= np.pi / 64 + 1e-9


def test_injected_slip_is_counted():
    # an instantaneous pi/2 phase jump cannot be followed by the unwrap
    g, o = _noiseless_kk(4, buf_len=1 << 20, phase_steps=[(3 << 18, np.pi / 2)])
    o.process(g["packed"][0])
    s = o.stats()
    assert s["bit_errors"] <= 16          # only the filter transient around the jump
    assert s["slip_windows"] > 0 and s["raw_bit_errors"] > 1000


def _pam_gray_ber(M, d):
    """Exact BER of Gray PAM-M, equiprobable odd-integer levels, AWGN with
    half level spacing / sigma = d, midpoint thresholds."""
    levels = np.arange(M)
    gray = levels ^ (levels >> 1)
    nb = int(np.log2(M))
    edges = np.concatenate(([-np.inf], np.arange(1, M) * 2.0 - M, [np.inf]))   # in units of half spacing
    total = 0.0
    for L in levels:
        x = 2.0 * L - (M - 1)
        for R in levels:
            p = norm.cdf((edges[R + 1] - x) * d) - norm.cdf((edges[R] - x) * d)
            total += p * bin(int(gray[L] ^ gray[R])).count("1")
    return total / (M * nb)


@pytest.mark.parametrize("snr_db", [11.0, 13.0])
def test_awgn_pam4_ber_matches_textbook(snr_db):
    """PAM-4, no ISI, AWGN only, ideal frozen taps: the BER lies in the 99 %
    binomial interval of the textbook Gray PAM-4 BER at the decision SNR
    implied by the generator (d = sqrt(2 SNR/5) after the unit-energy MF)."""
    N = 1 << 20
    g = synth.gen_pam_stream(1, N, 1, seed=9, snr_db=snr_db, isi=(0.0, 1.0, 0.0))
    snr = 10 ** (snr_db / 10)
    # ideal gain mapping the normalised MF output onto the levels +-1, +-3
    G = math.sqrt(2.5 * (1.0 + 1.0 / snr))
    cfg = oracle.default_cfg(1, N, mu=0.0, mu_train=0.0)
    o = oracle.Oracle(**cfg)
    taps = np.zeros(cfg["ntaps"])
    taps[cfg["ntaps"] // 2] = G
    o.set_taps(taps)
    o.process(g["packed"][0])
    s = o.stats()
    p = _pam_gray_ber(4, math.sqrt(2 * snr / 5))
    n = s["bits"]
    tol = 2.576 * math.sqrt(n * p * (1 - p)) + 0.03 * n * p
    assert abs(s["bit_errors"] - n * p) <= tol, (s["bit_errors"], n * p, tol)


def test_ols_each_output_has_v_over_2_margin():
    """Perturbing one input sample changes the phase of exactly the outputs
    whose block window holds it at an odd distance (the circular Hilbert
    kernel of an even-length block vanishes at even distances).  Reading each
    output's window off those dependencies, every kept output must lie at
    least V/2 samples inside an N-sample window (the overlap-save rule).  V/2
    is odd here so that a window misplaced by one sample is visible."""
    N, V, buf_len, calls = 256, 66, 1000, 2
    rng = np.random.default_rng(5)
    codes = rng.integers(800, 3000, size=buf_len * calls)
    cfg = oracle.default_cfg(4, buf_len, ols_n=N, ols_v=V, ntrain=64, ncma=0, eq_block=64)

    def run(c):
        o = oracle.Oracle(**cfg)
        out = []
        for k in range(calls):
            o.process(synth.pack12(c[k * buf_len:(k + 1) * buf_len]))
            out.append(o.get(oracle.ORX_E)[0])
        return np.concatenate(out)

    base = run(codes)
    total = len(base)
    dep = np.zeros((total, len(codes)), dtype=bool)
    for p in range(len(codes)):
        c2 = codes.copy()
        c2[p] += 97
        dep[:, p] = np.abs(np.angle(run(c2) / base)) > 1e-13
    h = V // 2
    for n in range(N, total):          # windows clear of the pre-stream fill
        ps = np.flatnonzero(dep[n])
        ps = ps[(ps - n) % 2 == 1]
        lo, hi = ps.min(), ps.max()
        assert hi - lo == N - 2 and len(ps) == N // 2
        assert n - lo >= h - 1 and hi - n >= h - 1, (n, lo, hi)


@pytest.mark.parametrize("mq,scale", [(2, math.sqrt(2.0)), (4, math.sqrt(10.0))])
def test_bps_metric_brute_force(mq, scale):
    """Window metric against a brute force over every constellation point."""
    rng = np.random.default_rng(mq)
    B, W = 32, 64
    lv = np.arange(-(mq - 1), mq, 2, dtype=np.float64)
    pts = (lv[:, None] + 1j * lv[None, :]).reshape(-1)
    z = (rng.choice(pts, W) * np.exp(0.37j) + 0.2 * (rng.standard_normal(W) + 1j * rng.standard_normal(W))) / scale
    got = oracle.bps_metrics(z, mq, scale, B)
    for b in range(B):
        th = b / B * np.pi / 2 - np.pi / 4
        v = scale * z * np.exp(-1j * th)
        ref = np.sum(np.min(np.abs(v[:, None] - pts[None, :]) ** 2, axis=1))
        assert abs(got[b] - ref) <= 1e-12 * ref
    assert abs((np.argmin(got) / B * np.pi / 2 - np.pi / 4) - 0.37) <= np.pi / 64


@pytest.mark.parametrize("fmt,snr_db", [(4, 14.0), (4, 16.0), (3, 8.0), (3, 10.0)])
def test_awgn_kk_qam_ber_matches_textbook(fmt, snr_db):
    """KK-16QAM / KK-QPSK with AWGN confined to the signal band (added to the
    symbols before shaping, Es/N0 = snr), no phase noise, CSPR 20 dB (the field
    is minimum phase everywhere, so KK reconstructs it), ideal frozen taps that
    undo the chain's power normalisation and a phase search on {-pi/4, 0}: the BER
    lies in the 99 % binomial interval of the exact Gray-QAM BER (two independent
    Gray PAM-sqrt(M) dimensions, half level spacing / sigma = d).  The chain's own
    deterministic distortion (filter truncation, KK residual) is measured on the
    same stream without noise and added as an independent Gaussian term; it must be
    small (> 30 dB below the symbols)."""
    N = 1 << 21
    snr = 10 ** (snr_db / 10)
    scale2 = 10.0 if fmt == 4 else 2.0        # unnormalised level units: z * sqrt(10) or sqrt(2)
    cfg = oracle.default_cfg(fmt, N, mu=0.0, mu_cma=0.0, ntrain=4096, ncma=2048, bps_b=2)

    def run(noisy):
        g = synth.gen_kk_stream(fmt, N, 1, seed=11, noise=False, phase_noise=False, cspr_db=20.0,
                                sym_snr_db=snr_db if noisy else None, truth=False)
        o = oracle.Oracle(**cfg)
        taps = np.zeros(cfg["ntaps"], complex)
        # the chain divides by sqrt(sps * signal power), which includes the symbol noise
        taps[cfg["ntaps"] // 2] = math.sqrt(1 + 1 / snr) if noisy else 1.0
        o.set_taps(taps)
        o.process(g["packed"][0])
        return o, g

    o0, g0 = run(False)
    v, s0 = o0.get(oracle.ORX_V)
    a = g0["symbols"][s0:s0 + len(v)] * math.sqrt(scale2)
    floor = float(np.mean(np.abs(v[5000:-100] - a[5000:-100]) ** 2) / 2)   # per dimension
    assert o0.stats()["bit_errors"] == 0 and floor < 1e-3 * scale2 / 2
    o, _ = run(True)
    s = o.stats()
    M = 4 if fmt == 4 else 2
    p = _pam_gray_ber(M, 1.0 / math.sqrt(scale2 / (2 * snr) + floor))
    n = s["bits"]
    tol = 2.576 * math.sqrt(n * p * (1 - p))
    assert abs(s["bit_errors"] - n * p) <= tol, (s["bit_errors"], n * p, tol)


@pytest.mark.parametrize("fmt", [3, 4])
@pytest.mark.parametrize("isi,closed", [((0.1, 1.0, 0.2), False), ((0.3 + 0.2j, 1.0, -0.45 + 0.25j), True)])
def test_kk_isi_channel_equalised_to_zero_errors(fmt, isi, closed):
    """Noiseless KK stream through a symbol-spaced ISI channel (mild and real; strong
    and complex, which closes the eye of both formats): CMA then DD-LMS from
    identity taps converge, and every payload bit is right.  On the strong channel
    the same stream with the taps frozen at identity has errors, so the equaliser is
    what removes the ISI."""
    N = 1 << 20
    g = synth.gen_kk_stream(fmt, N, 2, seed=3, noise=False, phase_noise=False, cspr_db=14.0, isi=isi,
                            truth=False)
    o = oracle.Oracle(**oracle.default_cfg(fmt, N))
    for b in range(2):
        o.process(g["packed"][b])
    s = o.stats()
    assert s["bits"] > 900_000 and s["bit_errors"] == 0 and s["raw_bit_errors"] == 0
    if closed:
        of = oracle.Oracle(**oracle.default_cfg(fmt, N, mu=0.0, mu_cma=0.0))
        for b in range(2):
            of.process(g["packed"][b])
        assert of.stats()["bit_errors"] > 10000
