"""Parity of the resampler to the transmitter's grid (an ADC clocked off the
transmitter's clock, Sec. 2) with the FP64 oracle: the resampled field within
1e-5 relative RMS, then the whole chain under the usual rules; off-clock streams
at +20 and -35 ppm with fractional delays, ragged buffers, QPSK, the
frequency-domain filter, the full 2^22-sample buffer, and batch = sequential."""

import numpy as np
import pytest
import torch

from parity_util import FIELD_TOL, Pair, make_stream, rel_rms
import oracle
import paper_2010_14333_gb300 as rx
import synth

pytestmark = pytest.mark.gpu

SMALL_KK = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)


def clock(ppm, delay):
    st, ph = synth.clock_step(ppm), int(round(delay * (1 << 32)))
    rs_step, rs_phase0 = oracle.rs_params(st, ph)
    return dict(clock_step=st, clock_phase0=ph), dict(rs_step=rs_step, rs_phase0=rs_phase0)


def run(fmt, nb, nbufs, gen, **cfg):
    g = make_stream(fmt, nb, nbufs, **gen)
    p = Pair(fmt, nb, **cfg)
    for b in range(nbufs):
        p.feed(g["packed"][b])
        r, r0 = p.g.debug(rx.RX_DBG_RS)
        ro, ro0 = p.o.get(oracle.ORX_RS)
        assert (r0, len(r)) == (ro0, len(ro))
        if len(r):
            assert rel_rms(r, ro) <= FIELD_TOL, ("resampled field", rel_rms(r, ro))
    return p.compare_stats()


@pytest.mark.parametrize("nb,ppm,delay", [(1 << 17, 20.0, 0.37), (98304 + 32 * 7, -35.0, -0.6),
                                          (65536 * 3 - 160, 80.0, 0.0)])
def test_rs_off_clock_streams(nb, ppm, delay):
    gen, cfg = clock(ppm, delay)
    s, so = run(4, nb, 3, gen, **cfg, **SMALL_KK)
    assert s["bits"] > 0 and so["ber"] < 0.05


def test_rs_qpsk_and_frequency_domain_filter():
    gen, cfg = clock(-12.0, 0.25)
    run(3, 1 << 17, 2, gen, **cfg, **SMALL_KK)
    run(4, 1 << 17, 2, gen, mf_mode=1, **cfg, **SMALL_KK)


def test_rs_full_size_buffer():
    gen, cfg = clock(-35.0, 0.4)
    s, so = run(4, 1 << 22, 2, dict(gen, workers=2), **cfg)
    assert s["bits"] == so["bits"] > 8_000_000
    assert so["ber"] < 2e-2


def test_rs_batch_equals_sequential():
    nb, nbufs = 1 << 18, 5
    gen, cfg = clock(25.0, 0.5)
    g = make_stream(4, nb, nbufs, seed=8, **gen)
    dev = [torch.from_numpy(p).cuda() for p in g["packed"]]
    a = rx.Receiver(4, nb, **cfg, **SMALL_KK)
    seq = []
    for d in dev:
        bits, n = a.process(d)
        seq.append(bits[: (n + 7) // 8].cpu().numpy().copy())
    b = rx.Receiver(4, nb, **cfg, **SMALL_KK)
    for (bits, n), ref in zip(b.process_batch(dev), seq):
        assert np.array_equal(bits[: (n + 7) // 8].cpu().numpy(), ref)
    assert a.stats()["bit_errors"] == b.stats()["bit_errors"]


@pytest.mark.parametrize("fmt,ppm,delay", [(1, -35.0, 0.4), (0, 20.0, -0.7), (2, 80.0, 0.2)])
def test_pam_resampler_parity(fmt, ppm, delay):
    """PAM-2/4/8 through an ADC clock off the transmitter's: the GPU resampler (the
    call's normalised codes interpolated to the nominal grid, then the matched filter)
    at parity with the oracle's: the resampled series within 1e-5, then the chain's
    parity rules call by call; ragged buffer length."""
    nb = (1 << 18) + 96
    step = synth.clock_step(ppm)
    g = make_stream(fmt, nb, 3, clock_step=step, clock_phase0=int(round(delay * 2 ** 32)), snr_db=22.0)
    st, ph = oracle.rs_params(step, int(round(delay * 2 ** 32)))
    p = Pair(fmt, nb, rs_step=st, rs_phase0=ph)
    for b in range(3):
        p.feed(g["packed"][b])
        R, r0 = p.g.debug(rx.RX_DBG_RS)
        Ro, ro0 = p.o.get(oracle.ORX_RS)
        assert (r0, len(R)) == (ro0, len(Ro)) and len(R) > 0
        assert rel_rms(R, Ro) <= 1e-5, rel_rms(R, Ro)
    s, so = p.compare_stats()
    assert s["ber"] < 1e-2   # about 0.5 without the resampler
