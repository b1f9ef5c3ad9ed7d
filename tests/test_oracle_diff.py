"""Pins of the optional differential quadrant coding (KK chain).

The transmitter steps the quadrant by the Gray-decoded first two bits of each
symbol and places the rest as a rotation-invariant point of the quadrant; the
receiver decodes quadrant differences.  What the construction fixes: the decoded
output of a noiseless stream is exactly the PRBS, whatever constant rotation the
stream carries; a pi/2 cycle slip costs a symbol or two instead of every later bit
(the plain Gray mapping loses a third of the stream); the generator's quadrant
sequence equals the recurrence run symbol by symbol."""

import numpy as np
import pytest

import oracle
import synth


def _run(fmt, diff, nb=1 << 20, nbufs=2, **gen):
    g = synth.gen_kk_stream(fmt, nb, nbufs, seed=3, noise=False, phase_noise=False, diff=bool(diff), truth=False,
                            **gen)
    o = oracle.Oracle(**oracle.default_cfg(fmt, nb, diff_code=diff))
    bits = []
    for p in g["packed"]:
        b, n = o.process(p)
        bits.append(np.unpackbits(b)[:n])
    return o.stats(), np.concatenate(bits)


@pytest.mark.parametrize("fmt", [3, 4])
@pytest.mark.parametrize("rot", [0.0, np.pi / 2, np.pi])
def test_decoded_bits_are_the_prbs_under_any_rotation(fmt, rot):
    s, bits = _run(fmt, 1, phase_offset=rot)
    bps = 4 if fmt == 4 else 2
    k0 = 16384
    ref = oracle.prbs15(1, 32767)[np.arange(bps * k0, bps * k0 + len(bits)) % 32767]
    bad = np.nonzero((bits != ref).reshape(-1, bps).any(1))[0]
    assert len(bad) <= 1 and (len(bad) == 0 or bad[0] == 0)   # only the first payload symbol has no predecessor
    assert s["bit_errors"] == 0 and s["raw_bit_errors"] == 0 and s["bits"] > 900_000


@pytest.mark.parametrize("fmt", [3, 4])
def test_slip_costs_one_symbol_with_differential_coding(fmt):
    slip = ((3 << 18, np.pi / 2),)
    plain, _ = _run(fmt, 0, phase_steps=slip)
    diff, _ = _run(fmt, 1, phase_steps=slip)
    bps = 4 if fmt == 4 else 2
    assert plain["raw_bit_errors"] > 0.2 * plain["bits"]
    assert diff["raw_bit_errors"] <= 2 * bps and diff["bit_errors"] == diff["raw_bit_errors"]


@pytest.mark.parametrize("fmt", [3, 4])
def test_generator_quadrants_follow_the_recurrence(fmt):
    bps = 4 if fmt == 4 else 2
    n = 70000
    bits = synth.prbs15_bits(1, 32767)
    idx = (np.arange(n)[:, None] * bps + np.arange(bps)[None, :]) % 32767
    b = bits[idx]
    q, out = 0, np.zeros(n, complex)
    for k in range(n):   # the recurrence, one symbol at a time
        d = [0, 1, 3, 2][2 * b[k, 0] + b[k, 1]]     # Gray-decoded step: 00 0, 01 1, 11 2, 10 3
        q = (q + d) % 4
        base = (1 + 2 * b[k, 2]) + 1j * (1 + 2 * b[k, 3]) if bps == 4 else 1 + 1j
        out[k] = base * 1j ** q / (np.sqrt(10) if bps == 4 else np.sqrt(2))
    assert np.max(np.abs(out - synth._tx_symbols(fmt, 1, 0, n, diff=True))) < 1e-12
