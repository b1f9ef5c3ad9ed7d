"""Pins of the oracle's resampler to the transmitter's sample grid (the ADC runs on
its own clock; the paper recovers the clock phase in the DSP, Sec. 2), against
what the mathematics fixes: the interpolator is the identity at zero fraction and
mirror-symmetric, band-limited tones land at the exact fractional position, an
identity accumulator changes nothing, and an off-clock stream resampled with the
matching accumulator gives the on-clock stream's filter output and no errors."""

import numpy as np
import pytest

import oracle
import synth

SMALL = dict(ols_n=8192, ols_v=1024, ntrain=4096, ncma=2048)


def test_taps_identity_and_mirror():
    c0 = oracle.rs_taps(0.0)
    assert abs(c0[7] - 1.0) < 1e-15 and np.abs(np.delete(c0, 7)).max() < 1e-15
    for mu in (0.125, 0.3, 0.5, 0.71):
        c, m = oracle.rs_taps(mu), oracle.rs_taps(1.0 - mu)
        # c_j(mu) = c_{1-j}(1-mu): j = -7..8 -> index j+7, 1-j -> index 8-j
        assert np.abs(c - m[::-1]).max() < 1e-15


@pytest.mark.parametrize("f", [0.02, 0.1, 0.2, -0.15])
def test_taps_interpolate_band_limited_tone(f):
    """e^{2 pi i f n} sampled at integers, interpolated at n0 + mu, against the exact
    value; a wrong sign of mu or an index off by one misses by O(1)."""
    n0 = 100
    n = np.arange(200)
    x = np.exp(2j * np.pi * f * n)
    for mu in (0.0, 0.25, 0.5, 0.8):
        c = oracle.rs_taps(mu)
        got = np.dot(c, x[n0 - 7:n0 + 9])
        want = np.exp(2j * np.pi * f * (n0 + mu))
        assert abs(got - want) < 3e-3, (f, mu, abs(got - want))


def _run(g, nb, nbufs, **kw):
    o = oracle.Oracle(**oracle.default_cfg(4, nb, **SMALL, **kw))
    ys = {}
    for b in range(nbufs):
        o.process(g["packed"][b])
        y, y0 = o.get(oracle.ORX_Y)
        for i, v in enumerate(y):
            ys[y0 + i] = v
    return o, ys


def test_identity_accumulator_changes_nothing():
    nb = 1 << 16
    g = synth.gen_kk_stream(4, nb, 2, seed=5)
    _, ya = _run(g, nb, 2)
    o, yb = _run(g, nb, 2, rs_step=1 << 32, rs_phase0=0)
    r, r0 = o.get(oracle.ORX_RS)
    e, e0 = o.get(oracle.ORX_E)
    common = sorted(set(ya) & set(yb))
    assert len(common) > 40000
    a, b = np.array([ya[i] for i in common]), np.array([yb[i] for i in common])
    # identical except the few outputs at each call edge that the 8-sample look-ahead
    # moves into the next call (which applies its own carrier and gain estimate)
    moved = np.abs(a - b) > 1e-12 * np.abs(a).max()
    assert moved.sum() <= 4 * 2, moved.sum()
    # the resampled field is the ADC field, emitted 8 samples behind it
    assert r0 + len(r) == e0 + len(e) - 8
    lo = max(r0, e0)
    assert np.abs(r[lo - r0:] - e[lo - e0:r0 + len(r) - e0]).max() < 1e-12 * np.abs(e).max()


@pytest.mark.parametrize("ppm,delay", [(20.0, 0.37), (-35.0, -0.6)])
def test_off_clock_stream_matches_on_clock_stream(ppm, delay):
    """The same symbols through an ADC clock ppm fast (delay in samples) and through
    the nominal clock: with the matching accumulator the filter outputs agree up to
    the interpolation and KK errors, and the noiseless stream decodes error-free."""
    nb = 1 << 17
    st, ph = synth.clock_step(ppm), int(round(delay * (1 << 32)))
    g0 = synth.gen_kk_stream(4, nb, 3, seed=2, noise=False, phase_noise=False)
    g1 = synth.gen_kk_stream(4, nb, 3, seed=2, noise=False, phase_noise=False, clock_step=st, clock_phase0=ph)
    rs_step, rs_phase0 = oracle.rs_params(st, ph)
    _, y0 = _run(g0, nb, 3)
    o1, y1 = _run(g1, nb, 3, rs_step=rs_step, rs_phase0=rs_phase0)
    common = sorted(set(y0) & set(y1))
    common = [i for i in common if i > 200]
    a, b = np.array([y0[i] for i in common]), np.array([y1[i] for i in common])
    assert len(common) > 100000
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 2e-2
    s = o1.stats()
    assert s["bits"] > 100000 and s["bit_errors"] == 0
    o2, _ = _run(g1, nb, 3)                 # without the resampler the clock drift breaks it
    assert o2.stats()["ber"] > 0.1


def test_rejects_bad_accumulators():
    for kw in (dict(rs_step=1 << 31), dict(rs_step=(1 << 32) * 2)):
        with pytest.raises(ValueError):
            oracle.Oracle(**oracle.default_cfg(4, 1 << 16, **kw))
    with pytest.raises(ValueError):   # the PAM resampler feeds the time-domain filter only
        oracle.Oracle(**oracle.default_cfg(1, 1 << 16, rs_step=1 << 32, mf_mode=1))


def test_binding_resampler_params_match_the_oracle():
    """librx's rx_resampler_from_clock (C ABI; host integer arithmetic, no GPU)
    turns a clock estimate into the accumulator exactly as the oracle does, which
    the pins above check against exact positions; out-of-range clocks are refused."""
    import paper_2010_14333_gb300 as rx
    for ppm, delay in ((-35.0, 0.4), (20.0, -0.7), (80.0, 1.1), (0.0, 0.0), (-0.3, -1.9),
                       (1234.5, -100.25), (-8999.0, 1e6), (7.25, 3.5)):
        want = oracle.rs_params(synth.clock_step(ppm), int(round(delay * (1 << 32))))
        assert rx.rx_resampler_from_clock(ppm, delay) == want, (ppm, delay)
    for ppm, delay in ((9000.0, 0.0), (-1e5, 0.0), (0.0, 2.0 ** 31), (float("nan"), 0.0)):
        with pytest.raises(rx.RxError):
            rx.rx_resampler_from_clock(ppm, delay)


@pytest.mark.parametrize("ppm,delay", [(-35.0, 0.4), (20.0, -0.7)])
def test_pam_resampler_recovers_an_off_clock_stream(ppm, delay):
    """PAM-4 sampled by an ADC clock off the transmitter's: the resampler with the
    matching accumulator interpolates the normalised codes back to the transmitter's
    grid, and every bit is right (about half are wrong without it); an identity
    accumulator leaves the on-clock stream's decisions unchanged."""
    nb = 1 << 18
    step = synth.clock_step(ppm)
    g = synth.gen_pam_stream(1, nb, 4, seed=6, snr_db=25.0, clock_step=step,
                             clock_phase0=int(round(delay * 2 ** 32)))
    st, ph = oracle.rs_params(step, int(round(delay * 2 ** 32)))
    res = []
    for kw in (dict(), dict(rs_step=st, rs_phase0=ph)):
        o = oracle.Oracle(**oracle.default_cfg(1, nb, **kw))
        for p in g["packed"]:
            o.process(p)
        res.append(o.stats())
    assert res[1]["bits"] > 1_000_000 and res[1]["bit_errors"] == 0
    assert res[0]["bit_errors"] > 0.3 * res[0]["bits"]
    g0 = synth.gen_pam_stream(1, nb, 2, seed=6, snr_db=18.0)
    outs = []
    for kw in (dict(), dict(rs_step=1 << 32, rs_phase0=0)):
        o = oracle.Oracle(**oracle.default_cfg(1, nb, **kw))
        outs.append([o.process(p)[0] for p in g0["packed"]])
    assert all(np.array_equal(a, b) for a, b in zip(outs[0], outs[1]))
