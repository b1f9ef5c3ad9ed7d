"""Pins of the oracle's end of stream (orx_flush).

Every stage of the chain emits only what its full support allows, so the last
few thousand samples of a stream stay undecided after its last buffer.  The
flush continues the stream with its last sample repeated and decides every
symbol whose centre lies inside the stream.  What the mathematics fixes: on a
noiseless stream the bits of process + flush are exactly the transmitted PRBS
bits of every payload symbol of the stream (the last few, whose filter supports
reach into the pad, excepted from scoring), the count is bps (S - ntrain), the
pad buffers keep the last real buffer's normalisation, and nothing is emitted
twice.
"""

import numpy as np
import pytest

import oracle
import synth

BPS = {0: 1, 1: 2, 2: 3, 3: 2, 4: 4}
KK_SMALL = dict(ntrain=1024, ncma=512, amb_syms=256, ols_n=4096, ols_v=512)


def _stream(fmt, nb, nbufs, seed=5, **gen):
    if fmt >= 3:
        return synth.gen_kk_stream(fmt, nb, nbufs, seed=seed, **gen)
    return synth.gen_pam_stream(fmt, nb, nbufs, seed=seed, **gen)


def _run(fmt, nb, nbufs, gen, **kw):
    g = _stream(fmt, nb, nbufs, **gen)
    o = oracle.Oracle(**oracle.default_cfg(fmt, nb, **kw))
    bits, tot = [], 0
    for b in range(nbufs):
        ob, n = o.process(g["packed"][b])
        bits.append(np.unpackbits(ob)[:n])
        tot += n
    fb, fn = o.flush()
    bits.append(np.unpackbits(fb)[:fn])
    return o, np.concatenate(bits), tot, fn


@pytest.mark.parametrize("fmt", [0, 1, 2, 3, 4])
def test_noiseless_stream_is_decoded_to_its_last_symbol(fmt):
    nb = 1 << 15 if fmt < 3 else 1 << 16
    nbufs = 3
    kw = dict(KK_SMALL) if fmt >= 3 else dict(ntrain=4096)
    gen = dict(noise=False, phase_noise=False) if fmt >= 3 else dict(snr_db=80)
    o, allbits, tot, fn = _run(fmt, nb, nbufs, gen, **kw)
    bps, sps = BPS[fmt], (4 if fmt >= 3 else 2)
    S = nbufs * nb // sps
    assert fn > 0 and tot + fn == bps * (S - kw["ntrain"])
    ref = oracle.prbs15(1, 32767)[np.arange(bps * kw["ntrain"], bps * S) % 32767]
    bad = np.nonzero((allbits != ref).reshape(-1, bps).any(1))[0] + kw["ntrain"]
    guard = (16 + (31 if fmt >= 3 else 15) + 1) // 2
    assert np.all(bad >= S - guard), bad[:8]
    st = o.stats()
    assert st["bit_errors"] == 0 and st["calls"] == nbufs and st["samples"] == nbufs * nb
    # scored: whole windows ending at or before S - guard, after training (and the
    # ambiguity-resolution symbols of the KK chain)
    k_lo = kw["ntrain"] + kw.get("amb_syms", 0)
    n_scored = (S - guard - k_lo) // 64
    assert st["bits"] == bps * 64 * n_scored


def test_second_flush_and_later_buffers():
    nb = 1 << 14
    g = _stream(1, nb, 2, snr_db=30)
    o = oracle.Oracle(**oracle.default_cfg(1, nb, ntrain=1024))
    for b in range(2):
        o.process(g["packed"][b])
    _, n1 = o.flush()
    _, n2 = o.flush()
    assert n1 > 0 and n2 == 0
    assert oracle.lib().orx_process(o._h, oracle._ptr(g["packed"][0]), None, 0) == -1


@pytest.mark.parametrize("nb", [2048, 4096 + 64])
def test_short_buffers_take_several_pad_buffers(nb):
    """Buffers shorter than the chain's lag: the flush needs more than one pad buffer,
    and the count still ends exactly at the stream's last symbol."""
    nbufs = 12
    o, allbits, tot, fn = _run(1, nb, nbufs, dict(snr_db=80), ntrain=1024)
    S = nbufs * nb // 2
    assert tot + fn == 2 * (S - 1024)
    ref = oracle.prbs15(1, 32767)[np.arange(2 * 1024, 2 * S) % 32767]
    bad = np.nonzero((allbits != ref).reshape(-1, 2).any(1))[0] + 1024
    assert np.all(bad >= S - 16)


def test_pad_keeps_the_last_buffers_normalisation_and_carrier():
    nb = 1 << 15
    g = _stream(1, nb, 2, snr_db=25)
    o = oracle.Oracle(**oracle.default_cfg(1, nb, ntrain=1024))
    for b in range(2):
        o.process(g["packed"][b])
    before, _ = o.get(oracle.ORX_SCAL)
    o.flush()
    after, _ = o.get(oracle.ORX_SCAL)
    assert after[3] == before[3] and after[4] == before[4]
    nb = 1 << 16
    g = _stream(4, nb, 2, snr_db=25)
    o = oracle.Oracle(**oracle.default_cfg(4, nb, **KK_SMALL))
    for b in range(2):
        o.process(g["packed"][b])
    before, _ = o.get(oracle.ORX_SCAL)
    o.flush()
    after, _ = o.get(oracle.ORX_SCAL)
    assert np.array_equal(after[:3], before[:3])


def test_resampled_stream_ends_at_its_last_nominal_symbol():
    """With the ADC off the transmitter's clock the stream's symbols are counted on
    the nominal grid: S = ceil(r_end / 4) with r_end the nominal samples whose ADC
    position lies inside the stream."""
    nb, nbufs, ppm = 1 << 16, 3, -35.0
    step = synth.clock_step(ppm)
    rs_step, rs_phase0 = oracle.rs_params(step, 0)
    g = _stream(4, nb, nbufs, noise=False, phase_noise=False, clock_step=step)
    o = oracle.Oracle(**oracle.default_cfg(4, nb, rs_step=rs_step, rs_phase0=rs_phase0, **KK_SMALL))
    tot = 0
    for b in range(nbufs):
        tot += o.process(g["packed"][b])[1]
    fn = o.flush()[1]
    total = nbufs * nb
    r_end = -(-((total << 32) - rs_phase0) // rs_step)
    S = (r_end - 1) // 4 + 1
    assert tot + fn == 4 * (S - KK_SMALL["ntrain"])
    assert o.stats()["bit_errors"] == 0
