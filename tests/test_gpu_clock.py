"""Parity of the frequency-domain clock estimate (Sec. 2: the clock recovered in the
frequency domain block by block) with the FP64 oracle: the band-edge correlation of
every block within 1e-4 relative, the fitted clock offset and delay equal to the
oracle's and to the generator's clock, and the estimate driving the GPU resampler."""

import numpy as np
import pytest
import torch

from parity_util import Pair, make_stream
import oracle
import paper_2010_14333_gb300 as rx
import synth

pytestmark = pytest.mark.gpu

SMALL_KK = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)


def gen(ppm, delay, nb, nbufs, **kw):
    return make_stream(4, nb, nbufs, clock_step=synth.clock_step(ppm), clock_phase0=int(round(delay * (1 << 32))),
                       **kw)


@pytest.mark.parametrize("fd_n", [1024, 256])
def test_block_correlations_match_oracle(fd_n):
    nb = 1 << 17
    g = gen(2.0, 0.3, nb, 3)
    p = Pair(4, nb, mf_mode=1, fd_n=fd_n, fd_taps=fd_n // 4 + 1, **SMALL_KK)
    for b in range(3):
        p.feed(g["packed"][b])
        c, c0 = p.g.debug(rx.RX_DBG_CLK)
        co, co0 = p.o.get(oracle.ORX_CLK)
        assert (c0, len(c)) == (co0, len(co)) and len(c) > 0
        assert np.linalg.norm(c - co) / np.linalg.norm(co) < 1e-4
    p.compare_stats()


@pytest.mark.parametrize("ppm,delay", [(-35.0, 0.4), (20.0, -0.7)])
def test_estimate_matches_oracle_and_clock(ppm, delay):
    nb = 1 << 19
    g = gen(ppm, delay, nb, 2)
    r = rx.Receiver(4, nb, mf_mode=1, **SMALL_KK)
    o = oracle.Oracle(**oracle.default_cfg(4, nb, mf_mode=1, **SMALL_KK))
    for b in range(2):
        r.process(torch.from_numpy(g["packed"][b]).cuda())
        o.process(g["packed"][b])
    gp, gd = rx.rx_clock_estimate(r.h, torch.cuda.current_stream().cuda_stream)
    c, c0 = o.get(oracle.ORX_CLK)
    op, od = oracle.clock_fit(c, 512 * (c0 + np.arange(len(c))) + 256)
    assert abs(gp - op) < 0.01 and abs(gd - od) < 1e-3, (gp, op, gd, od)
    assert abs(gp - ppm) < 0.5 and abs(gd - delay) < 0.05, (gp, gd)


def test_estimate_drives_the_gpu_resampler():
    nb = 1 << 18
    g = gen(-35.0, 0.4, nb, 5, seed=6)
    est = rx.Receiver(4, nb, mf_mode=1, **SMALL_KK)
    for b in range(2):
        est.process(torch.from_numpy(g["packed"][b]).cuda())
    ppm, delay = rx.rx_clock_estimate(est.h, torch.cuda.current_stream().cuda_stream)
    rs_step, rs_phase0 = oracle.rs_params(synth.clock_step(ppm), int(round(delay * (1 << 32))))
    r = rx.Receiver(4, nb, rs_step=rs_step, rs_phase0=rs_phase0, **SMALL_KK)
    plain = rx.Receiver(4, nb, **SMALL_KK)
    for p in g["packed"]:
        d = torch.from_numpy(p).cuda()
        r.process(d)
        plain.process(d)
    s, sp = r.stats(), plain.stats()
    assert s["bits"] > 0 and s["ber"] < 0.02 and sp["ber"] > 0.1, (s["ber"], sp["ber"])


# ---- PAM: the band-edge correlation in the PAM FD kernel (2 samples/symbol)
def pam_clock(ppm, delay):
    return dict(clock_step=synth.clock_step(ppm), clock_phase0=int(round(delay * (1 << 32))))


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_pam_block_correlations_match_oracle(fmt):
    nb = 1 << 17
    g = make_stream(fmt, nb, 3, seed=5, **pam_clock(15.0, 0.3))
    p = Pair(fmt, nb, mf_mode=1)
    for b in range(3):
        p.feed(g["packed"][b], check=False)
        c, c0 = p.g.debug(rx.RX_DBG_CLK)
        co, co0 = p.o.get(oracle.ORX_CLK)
        assert (c0, len(c)) == (co0, len(co)) and len(c) > 0
        assert np.linalg.norm(c - co) / np.linalg.norm(co) < 1e-4


@pytest.mark.parametrize("ppm,delay", [(-35.0, 0.4), (20.0, -0.3)])
def test_pam_estimate_matches_oracle_and_clock(ppm, delay):
    nb = 1 << 18
    g = make_stream(1, nb, 2, seed=7, isi=(0.0, 1.0, 0.0), **pam_clock(ppm, delay))
    r = rx.Receiver(1, nb, mf_mode=1)
    o = oracle.Oracle(**oracle.default_cfg(1, nb, mf_mode=1))
    for b in range(2):
        r.process(torch.from_numpy(g["packed"][b]).cuda())
        o.process(g["packed"][b])
    gp, gd = rx.rx_clock_estimate(r.h, torch.cuda.current_stream().cuda_stream)
    c, c0 = o.get(oracle.ORX_CLK)
    op, od = oracle.clock_fit(c, 512 * (c0 + np.arange(len(c))) + 256, sps=2)
    assert abs(gp - op) < 0.01 and abs(gd - od) < 1e-3, (gp, op, gd, od)
    err = (gd - delay + 1.0) % 2.0 - 1.0
    assert abs(gp - ppm) < 0.5 and abs(err) < 0.05, (gp, gd)


# ------------------------------------------------------------ tracking across calls
def _ramp(nb, ppms, seed=9, **kw):
    steps = [synth.clock_step(p) for p in ppms]
    bufs, ph = [], 0
    for b in range(len(ppms)):
        if b > 0:
            ph += b * nb * (steps[b - 1] - steps[b])
        bufs.append(synth.kk_buffer(4, nb, b, 0.0, seed=seed, truth=False, clock_step=steps[b], clock_phase0=ph,
                                    **kw)["packed"])
    return bufs, steps


def test_running_estimate_matches_oracle_tracker():
    """KK with the resampler and PAM-4: after every call the GPU's running estimate
    (blocks unwrapped across calls, one line fit) equals the oracle tracker's within
    0.01 ppm and 1e-3 samples, over the same number of blocks."""
    sid = torch.cuda.current_stream().cuda_stream
    nb = 1 << 17
    step = synth.clock_step(-35.0)
    st, ph = oracle.rs_params(synth.clock_step(-30.0), 0)   # a resampler 5 ppm off the clock
    g = gen(-35.0, 0.4, nb, 4)
    p = Pair(4, nb, mf_mode=1, clk_track=1, rs_step=st, rs_phase0=ph, **SMALL_KK)
    for b in range(4):
        p.feed(g["packed"][b])
        gp, gd, gn = rx.rx_clock_track(p.g.h, sid)
        op, od, on = p.o.clock_track()
        assert gn == on and abs(gp - op) < 0.01 and abs(gd - od) < 1e-3, (b, gp, op, gd, od)
    assert abs(gp + 5.0) < 0.2   # the residual of a -35 ppm clock against a -30 ppm resampler
    gpam = make_stream(1, 1 << 18, 3, clock_step=synth.clock_step(20.0))
    p = Pair(1, 1 << 18, mf_mode=1, clk_track=1)
    for b in range(3):
        p.feed(gpam["packed"][b])
        gp, gd, gn = rx.rx_clock_track(p.g.h, sid)
        op, od, on = p.o.clock_track()
        assert gn == on and abs(gp - op) < 0.01 and abs(gd - od) < 1e-3, (b, gp, op, gd, od)


def test_retime_parity_with_oracle():
    """The GPU closes the loop between calls (rx_clock_retime); the oracle is re-timed
    with the same integers, and every later call stays at parity (fields, filter
    output, decisions, counts)."""
    sid = torch.cuda.current_stream().cuda_stream
    nb = 1 << 17
    bufs, steps = _ramp(nb, [-35.0 + 2.0 * b for b in range(6)])
    st, ph = oracle.rs_params(steps[0], 0)
    p = Pair(4, nb, mf_mode=1, clk_track=1, rs_step=st, rs_phase0=ph, **SMALL_KK)
    applied = []
    for b, buf in enumerate(bufs):
        p.feed(buf)
        step, nudge = rx.rx_clock_retime(p.g.h, sid)
        p.o.set_rs(step, nudge)
        applied.append((step, nudge))
    p.compare_stats()
    assert len({a for a, _ in applied}) > 3   # the step followed the drift


def test_closed_loop_follows_a_drifting_clock_on_gpu():
    """As the oracle pin: 1 ppm per 2^18-sample buffer of drift, re-timed after every
    buffer by the GPU's own loop: every payload bit right; open loop falls apart."""
    sid = torch.cuda.current_stream().cuda_stream
    nb, nbufs = 1 << 18, 14
    bufs, steps = _ramp(nb, [-35.0 + b for b in range(nbufs)], noise=False, phase_noise=False)
    st, ph = oracle.rs_params(steps[0], 0)
    res = {}
    for loop in (False, True):
        r = rx.Receiver(4, nb, mf_mode=1, clk_track=1, rs_step=st, rs_phase0=ph, **SMALL_KK)
        for buf in bufs:
            r.process(torch.from_numpy(buf).cuda())
            if loop:
                rx.rx_clock_retime(r.h, sid)
        res[loop] = r.stats()
    assert res[True]["bits"] > 3_000_000 and res[True]["bit_errors"] == 0
    assert res[False]["bit_errors"] > 0.1 * res[False]["bits"]


def test_tracker_argument_errors():
    nb = 1 << 16
    r = rx.Receiver(4, nb, **SMALL_KK)
    with pytest.raises(rx.RxError):
        rx.rx_clock_track(r.h)
    with pytest.raises(rx.RxError):
        rx.rx_clock_retime(r.h)
    with pytest.raises(rx.RxError):
        rx.Receiver(4, nb, clk_track=1, **SMALL_KK)   # needs the frequency-domain form
    r = rx.Receiver(1, nb, mf_mode=1, clk_track=1)
    with pytest.raises(rx.RxError):
        rx.rx_clock_retime(r.h)                        # the PAM chain has no resampler
