"""Pins of the oracle's frequency-domain filter forms (the paper's static FD
equalisers on overlap-save blocks of an N-point FFT, Sec. 2: in the KK chain an
N/2-point IFFT of the kept bins is the downsampler to 2 samples/symbol; the PAM
chain stays at its input rate), against what the mathematics fixes
independently of the oracle's FFT: closed-form filter responses, pure tones
through the block (the response at the tone's bin, or nothing outside the kept
band), brute-force double sums on a tiny block, the block grid of a stream, and
noiseless streams decoded without errors."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_fd_response_closed_forms():
    n = 64
    k = np.arange(n)
    assert np.allclose(oracle.fd_response(np.array([1.0]), n), 1.0, atol=1e-15)
    a, b, c = 0.3, -1.1, 0.7        # taps at i = -1, 0, +1
    want = a * np.exp(2j * np.pi * k / n) + b + c * np.exp(-2j * np.pi * k / n)
    assert np.abs(oracle.fd_response(np.array([a, b, c]), n) - want).max() < 1e-14
    h = oracle.rrc_half(0.1, 4, 101)   # zero-phase symmetric taps: real response
    H = oracle.fd_response(h, 1024)
    assert np.abs(H.imag).max() < 1e-12
    assert abs(H[0] - h.sum()) < 1e-12


def test_rrc_half_matches_span_form():
    assert np.array_equal(oracle.rrc_half(0.1, 4, 32), oracle.rrc(0.1, 4, 16))


@pytest.mark.parametrize("n", [64, 1024])
def test_fd_block_in_band_tones(n):
    """Tones on the block's bin grid with |k| < N/4 come out as the tone times
    H at that bin, sampled at the even indices of the kept half."""
    rng = np.random.default_rng(5)
    ks = [0, 1, 3, n // 8, n // 4 - 1, -1, -5, -(n // 4)]
    amps = rng.standard_normal(len(ks)) + 1j * rng.standard_normal(len(ks))
    t = np.arange(n)
    x = sum(A * np.exp(2j * np.pi * k * t / n) for A, k in zip(amps, ks))
    h = rng.standard_normal(n // 2 + 1)
    H = oracle.fd_response(h, n)
    y = oracle.fd_block(x, H)
    m = np.arange(n // 8, 3 * n // 8)
    want = sum(A * H[k % n] * np.exp(2j * np.pi * k * 2 * m / n) for A, k in zip(amps, ks))
    assert np.abs(y - want).max() < 1e-11 * max(1.0, np.abs(want).max())


def test_fd_block_drops_out_of_band_tones():
    n = 256
    t = np.arange(n)
    H = oracle.fd_response(np.ones(65), n)
    for k in (n // 4, n // 4 + 7, n // 2, 3 * n // 4 - 1):
        y = oracle.fd_block(np.exp(2j * np.pi * k * t / n), H)
        assert np.abs(y).max() < 1e-12, k


def test_fd_block_brute_force_tiny():
    """N = 16: the definition as explicit double sums over samples and bins."""
    n = 16
    rng = np.random.default_rng(11)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    H = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = oracle.fd_block(x, H)
    want = []
    for m in range(n // 8, 3 * n // 8):
        acc = 0j
        for k in range(-n // 4, n // 4):
            Xk = 0j
            for t in range(n):
                Xk += x[t] * np.exp(-2j * np.pi * t * k / n)
            acc += Xk * H[k % n] * np.exp(2j * np.pi * (k % (n // 2)) * m / (n // 2))
        want.append(acc / n)
    assert np.abs(y - np.array(want)).max() < 1e-12


def _fd_stream(nbufs, nb, **gen):
    g = synth.gen_kk_stream(4, nb, nbufs, seed=2, **gen)
    cfg = oracle.default_cfg(4, nb, ols_n=8192, ols_v=1024, mf_mode=1)
    return g, oracle.Oracle(**cfg), cfg


def test_fd_stream_block_grid():
    """The stream output of call 2 equals the pinned block applied on the stream
    grid (block b from index N/2 b - N/4) to the carrier-removed, downshifted field
    of calls 1 and 2, including the history carried across the buffer edge."""
    nb = 1 << 16
    g, o, cfg = _fd_stream(2, nb, noise=False, phase_noise=False)
    N, hop = cfg["fd_n"], cfg["fd_n"] // 2
    E = {}
    for b in range(2):
        o.process(g["packed"][b])
        e, e0 = o.get(oracle.ORX_E)
        for i, v in enumerate(e):
            E[e0 + i] = v
    y, y0 = o.get(oracle.ORX_Y)
    scal, _ = o.get(oracle.ORX_SCAL)
    carrier, gain = scal[0] + 1j * scal[1], scal[2]
    assert len(y) > 0 and y0 % (hop // 2) == 0 and len(y) % (hop // 2) == 0
    h = oracle.rrc_half(cfg["rrc_beta"], 4, (cfg["fd_taps"] - 1) // 2)
    H = oracle.fd_response(h, N)
    for b in range(y0 // (hop // 2), (y0 + len(y)) // (hop // 2)):
        n = hop * b - N // 4 + np.arange(N)
        p = (n % cfg["ds_den"]) * cfg["ds_num"] % cfg["ds_den"]
        x = np.array([E.get(int(i), 0.0) for i in n]) - carrier
        x = np.where(n >= 0, x * np.exp(-2j * np.pi * p / cfg["ds_den"]), 0.0)
        want = gain * oracle.fd_block(x, H)
        got = y[(hop // 2) * b - y0 + np.arange(N // 4)]
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), b


def test_fd_stream_noiseless_zero_errors():
    g, o, _ = _fd_stream(1, 1 << 20, noise=False, phase_noise=False)
    o.process(g["packed"][0])
    s = o.stats()
    assert s["bits"] > 400_000 and s["bit_errors"] == 0 and s["raw_bit_errors"] == 0


def test_fd_close_to_time_domain_filter():
    """With the same 201-tap filter, the FD form differs from the time-domain
    matched filter only by the truncated out-of-band bins: a small relative
    difference on a noisy stream."""
    nb = 1 << 18
    g = synth.gen_kk_stream(4, nb, 1, seed=4)
    ys = []
    for mode in (0, 1):
        o = oracle.Oracle(**oracle.default_cfg(4, nb, ols_n=8192, ols_v=1024, mf_mode=mode, mf_span=50,
                                               fd_taps=201))
        o.process(g["packed"][0])
        ys.append(o.get(oracle.ORX_Y))
    (yt, t0), (yf, f0) = ys
    lo, hi = max(t0, f0) + 200, min(t0 + len(yt), f0 + len(yf)) - 200
    a, b = yt[lo - t0:hi - t0], yf[lo - f0:hi - f0]
    rel = np.linalg.norm(a - b) / np.linalg.norm(a)
    assert rel < 2e-2, rel


def test_fd_rejects_bad_configurations():
    for fmt in (4, 1):
        for kw in (dict(fd_n=1000), dict(fd_taps=202), dict(fd_taps=1024 // 2 + 3), dict(fd_n=8)):
            with pytest.raises(ValueError):
                oracle.Oracle(**oracle.default_cfg(fmt, 1 << 16, mf_mode=1, **kw))


@pytest.mark.parametrize("n", [64, 1024])
def test_fd_block_full_tones(n):
    """Without downsampling every bin passes: tones anywhere on the bin grid leave
    as the tone times H at the bin, on the central half of the block."""
    rng = np.random.default_rng(6)
    ks = [0, 1, n // 4, n // 2, n // 2 + 3, n - 1, -(n // 8)]
    amps = rng.standard_normal(len(ks)) + 1j * rng.standard_normal(len(ks))
    t = np.arange(n)
    x = sum(A * np.exp(2j * np.pi * k * t / n) for A, k in zip(amps, ks))
    H = oracle.fd_response(rng.standard_normal(n // 2 + 1), n)
    y = oracle.fd_block_full(x, H)
    m = np.arange(n // 4, 3 * n // 4)
    want = sum(A * H[k % n] * np.exp(2j * np.pi * k * m / n) for A, k in zip(amps, ks))
    assert np.abs(y - want).max() < 1e-11 * max(1.0, np.abs(want).max())


def test_fd_block_full_brute_force_tiny():
    n = 16
    rng = np.random.default_rng(12)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    H = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    want = []
    for m in range(n // 4, 3 * n // 4):
        acc = 0j
        for k in range(n):
            Xk = sum(x[t] * np.exp(-2j * np.pi * t * k / n) for t in range(n))
            acc += Xk * H[k] * np.exp(2j * np.pi * k * m / n)
        want.append(acc / n)
    assert np.abs(oracle.fd_block_full(x, H) - np.array(want)).max() < 1e-12


def test_fd_pam_stream_block_grid():
    """PAM-4 in the frequency-domain form: the stream output of call 2 is the pinned
    full-rate block on the stream grid over the normalised codes of calls 1 and 2."""
    nb = 1 << 16
    g = synth.gen_pam_stream(1, nb, 2, seed=3)
    cfg = oracle.default_cfg(1, nb, mf_mode=1)
    o = oracle.Oracle(**cfg)
    N, hop = cfg["fd_n"], cfg["fd_n"] // 2
    codes = np.concatenate([oracle.unpack(g["packed"][b], nb) for b in range(2)]).astype(np.float64)
    for b in range(2):
        o.process(g["packed"][b])
    y, y0 = o.get(oracle.ORX_Y)
    scal, _ = o.get(oracle.ORX_SCAL)
    mu, sd = scal[3], scal[4]
    assert len(y) > 0 and y0 % hop == 0 and len(y) % hop == 0
    H = oracle.fd_response(oracle.rrc_half(cfg["rrc_beta"], 2, (cfg["fd_taps"] - 1) // 2), N)
    for b in range(y0 // hop, (y0 + len(y)) // hop):
        n = hop * b - N // 4 + np.arange(N)
        x = np.where(n >= 0, (codes[np.clip(n, 0, None)] - mu) / sd, 0.0)
        want = oracle.fd_block_full(x, H).real
        got = np.real(y[hop * b - y0 + np.arange(N // 2)])
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), b


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_fd_pam_noiseless_with_isi_zero_errors(fmt):
    N = 1 << 19
    g = synth.gen_pam_stream(fmt, N, 2, seed=3, noise=False)
    o = oracle.Oracle(**oracle.default_cfg(fmt, N, mf_mode=1))
    for b in range(2):
        o.process(g["packed"][b])
    s = o.stats()
    assert s["bits"] > 400_000 and s["bit_errors"] == 0
