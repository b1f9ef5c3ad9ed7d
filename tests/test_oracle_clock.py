"""Pins of the oracle's frequency-domain clock estimate (the paper recovers the
clock phase in the frequency domain block by block and unwraps it across blocks
and buffers, Sec. 2): the line fit over exact band-edge phases, whole-sample delays
on the nominal clock, off-clock streams, and the estimate driving the resampler."""

import numpy as np
import pytest

import oracle
import synth

SMALL = dict(ols_n=8192, ols_v=1024)


def test_fit_recovers_exact_phases_across_wraps():
    """C_b = exp(-i pi d_b / 2) with d_b = -tau0 - eps c_b, through many wraps of the
    4-sample period: the unwrap and the line give eps and tau0 back."""
    for ppm, tau0 in ((-35.0, 0.4), (120.0, -1.3), (0.5, 1.9)):
        centers = 512 * np.arange(3000, 9000) + 256
        d = -tau0 - ppm * 1e-6 * centers
        c = 7.0 * np.exp(-0.5j * np.pi * d)
        p, t = oracle.clock_fit(c, centers)
        assert abs(p - ppm) < 1e-9 and abs(t - tau0) < 1e-9, (p, t)


def _estimate(g, nb, nbufs):
    o = oracle.Oracle(**oracle.default_cfg(4, nb, mf_mode=1, **SMALL))
    for b in range(nbufs):
        o.process(g["packed"][b])
    c, c0 = o.get(oracle.ORX_CLK)
    return oracle.clock_fit(c, 512 * (c0 + np.arange(len(c))) + 256)


@pytest.mark.parametrize("d", [0, 1, -1, 2])
def test_whole_sample_delays_on_the_nominal_clock(d):
    nb = 1 << 18
    g = synth.gen_kk_stream(4, nb, 2, seed=4, noise=False, phase_noise=False, clock_phase0=d << 32)
    ppm, delay = _estimate(g, nb, 2)
    err = (delay - d + 2.0) % 4.0 - 2.0    # the delay is known modulo one symbol (4 samples)
    assert abs(ppm) < 0.2 and abs(err) < 0.02, (ppm, delay)


@pytest.mark.parametrize("ppm,delay", [(-35.0, 0.4), (20.0, -0.7), (80.0, 1.1)])
def test_off_clock_streams(ppm, delay):
    nb = 1 << 19
    g = synth.gen_kk_stream(4, nb, 2, seed=2, clock_step=synth.clock_step(ppm),
                            clock_phase0=int(round(delay * (1 << 32))))
    p, t = _estimate(g, nb, 2)
    assert abs(p - ppm) < 0.5 and abs(t - delay) < 0.05, (p, t)


def test_estimate_drives_the_resampler():
    """Estimate the clock on the first two buffers without the resampler, configure
    the resampler with the estimate, and decode the noiseless stream error-free."""
    nb = 1 << 18
    st, ph = synth.clock_step(-35.0), int(round(0.4 * (1 << 32)))
    g = synth.gen_kk_stream(4, nb, 4, seed=6, noise=False, phase_noise=False, clock_step=st, clock_phase0=ph)
    p, t = _estimate(g, nb, 2)
    rs_step, rs_phase0 = oracle.rs_params(synth.clock_step(p), int(round(t * (1 << 32))))
    o = oracle.Oracle(**oracle.default_cfg(4, nb, rs_step=rs_step, rs_phase0=rs_phase0, ntrain=4096, ncma=2048,
                                           **SMALL))
    for b in range(4):
        o.process(g["packed"][b])
    s = o.stats()
    assert s["bits"] > 200000 and s["bit_errors"] == 0


# ---- PAM: the band-edge correlation on the FD form's blocks at 2 samples/symbol
def test_fit_recovers_exact_phases_across_wraps_pam():
    """C_b = exp(-2 pi i d_b / 2) with d_b = -tau0 - eps c_b through many wraps of the
    2-sample period."""
    for ppm, tau0 in ((-35.0, 0.4), (120.0, -0.7), (0.5, 0.95)):
        centers = 512 * np.arange(3000, 9000) + 256
        d = -tau0 - ppm * 1e-6 * centers
        c = 3.0 * np.exp(-1j * np.pi * d)
        p, t = oracle.clock_fit(c, centers, sps=2)
        assert abs(p - ppm) < 1e-9 and abs(t - tau0) < 1e-9, (p, t)


def test_pam_generator_whole_sample_offset_is_a_shift():
    """The off-clock path of the PAM generator at a whole-sample phase is the nominal
    stream shifted by that many samples."""
    a = synth.gen_pam_stream(1, 1 << 14, 2, noise=False)
    b = synth.gen_pam_stream(1, 1 << 14, 2, noise=False, clock_phase0=3 << 32)
    assert np.max(np.abs(a["intensity"][3:] - b["intensity"][:-3])) < 1e-12


def _estimate_pam(g, fmt, nb, nbufs):
    o = oracle.Oracle(**oracle.default_cfg(fmt, nb, mf_mode=1))
    for b in range(nbufs):
        o.process(g["packed"][b])
    c, c0 = o.get(oracle.ORX_CLK)   # the blocks of the last call
    assert len(c) == nb // 512, (len(c), c0)
    return oracle.clock_fit(c, 512 * (c0 + np.arange(len(c))) + 256, sps=2)


@pytest.mark.parametrize("fmt,d", [(1, 0), (1, 1), (0, 1), (2, 0)])
def test_pam_whole_sample_delays_on_the_nominal_clock(fmt, d):
    nb = 1 << 17
    g = synth.gen_pam_stream(fmt, nb, 2, seed=4, noise=False, isi=(0.0, 1.0, 0.0), clock_phase0=d << 32)
    ppm, delay = _estimate_pam(g, fmt, nb, 2)
    err = (delay - d + 1.0) % 2.0 - 1.0    # the delay is known modulo one symbol (2 samples)
    assert abs(ppm) < 0.2 and abs(err) < 0.01, (ppm, delay)


@pytest.mark.parametrize("ppm,delay", [(-35.0, 0.4), (20.0, -0.3), (80.0, 0.85)])
def test_pam_off_clock_streams(ppm, delay):
    nb = 1 << 18
    g = synth.gen_pam_stream(1, nb, 2, seed=2, isi=(0.0, 1.0, 0.0), clock_step=synth.clock_step(ppm),
                             clock_phase0=int(round(delay * (1 << 32))))
    p, t = _estimate_pam(g, 1, nb, 2)
    err = (t - delay + 1.0) % 2.0 - 1.0
    assert abs(p - ppm) < 0.5 and abs(err) < 0.05, (p, t)


def test_pam_off_clock_with_isi():
    """With the default asymmetric ISI the symbol-rate line moves by a constant: the
    clock offset (the slope) stays."""
    nb = 1 << 18
    g = synth.gen_pam_stream(1, nb, 2, seed=3, clock_step=synth.clock_step(-35.0), clock_phase0=0)
    p, _ = _estimate_pam(g, 1, nb, 2)
    assert abs(p + 35.0) < 0.5, p


# ------------------------------------------------------------ tracking across calls
TRK = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024, mf_mode=1, clk_track=1)


def _ramp_stream(nb, ppms, seed=9, **gen):
    """Buffer b sampled by an ADC clock of ppms[b], the accumulator continuous at the
    buffer edges (a staircase approximation of a drifting clock)."""
    steps = [synth.clock_step(p) for p in ppms]
    bufs, ph = [], 0
    for b in range(len(ppms)):
        if b > 0:
            ph += b * nb * (steps[b - 1] - steps[b])
        bufs.append(synth.kk_buffer(4, nb, b, 0.0, seed=seed, truth=False, clock_step=steps[b],
                                    clock_phase0=ph, **gen)["packed"])
    return bufs, steps


def test_tracker_equals_one_fit_over_all_calls():
    """The running estimate after several calls equals the line fit of the same
    blocks concatenated (orx_clock_fit, which unwraps block to block): the unwrap
    carries from the last block of a call to the first of the next."""
    nb = 1 << 17
    g = synth.gen_kk_stream(4, nb, 4, seed=4, clock_step=synth.clock_step(-35.0), clock_phase0=int(0.3 * 2 ** 32),
                            truth=False, noise=False, phase_noise=False)
    o = oracle.Oracle(**oracle.default_cfg(4, nb, **TRK))
    cs, cents = [], []
    for p in g["packed"]:
        o.process(p)
        c, b0 = o.get(oracle.ORX_CLK)
        cs.append(c)
        cents.append(512 * (b0 + np.arange(len(c))) + 256)
    ppm, dl, n = o.clock_track()
    ppm_f, dl_f = oracle.clock_fit(np.concatenate(cs), np.concatenate(cents), 4)
    assert n == sum(len(c) for c in cs) > 500
    assert abs(ppm - ppm_f) < 1e-9 and abs(dl - dl_f) < 1e-9
    assert abs(ppm + 35.0) < 0.1 and abs(dl - 0.3) < 0.02


def test_retime_with_unchanged_accumulator_changes_nothing():
    """A re-timing to the same step with no nudge continues the accumulator exactly:
    every later output equals that of the stream left alone."""
    nb = 1 << 16
    step = synth.clock_step(20.0)
    g = synth.gen_kk_stream(4, nb, 3, seed=6, clock_step=step, truth=False)
    st, ph = oracle.rs_params(step, 0)
    outs = []
    for retime in (False, True):
        o = oracle.Oracle(**oracle.default_cfg(4, nb, rs_step=st, rs_phase0=ph, **TRK))
        bits = []
        for b, p in enumerate(g["packed"]):
            bits.append(o.process(p)[0])
            if retime:
                o.set_rs(st, 0)
        outs.append((np.concatenate(bits), o.get(oracle.ORX_RS)[0]))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_closed_loop_follows_a_drifting_clock():
    """A noiseless KK-16QAM stream whose ADC clock drifts by 1 ppm per 2^18-sample
    buffer (-35 to -22 ppm): with the resampler fixed at the starting clock the
    timing runs off by whole symbols and the decisions fall apart; re-timed after
    every buffer from the tracker (frequency and phase) every payload bit is right."""
    nb, nbufs = 1 << 18, 14
    bufs, steps = _ramp_stream(nb, [-35.0 + b for b in range(nbufs)], noise=False, phase_noise=False)
    st, ph = oracle.rs_params(steps[0], 0)
    res = {}
    for loop in (False, True):
        o = oracle.Oracle(**oracle.default_cfg(4, nb, rs_step=st, rs_phase0=ph, **TRK))
        for p in bufs:
            o.process(p)
            if loop:
                o.clock_retime()
        res[loop] = o.stats()
    assert res[True]["bits"] > 3_000_000 and res[True]["bit_errors"] == 0
    assert res[False]["bit_errors"] > 0.1 * res[False]["bits"]
