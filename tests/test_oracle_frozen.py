"""Pins of the oracle's frozen-tap equaliser form (every payload block filters
with the taps its call started from; the block-Toeplitz reading of the
precision sweep), against things other than the oracle itself: a library
convolution, the adaptive form at zero step, noiseless data, and the direction
of the tap step on a known gain error."""

import numpy as np
import pytest

import oracle
import synth

NB = 1 << 19
CFG = dict(ols_n=8192, ols_v=1024, ntrain=4096, ncma=2048, amb_syms=1024, eq_block=1024)


def _stream(nbufs=3, **gen):
    return synth.gen_kk_stream(4, NB, nbufs, seed=31, **gen)


def _run(g, nbufs, set_taps=None, **cfg):
    o = oracle.Oracle(**oracle.default_cfg(4, NB, **{**CFG, **cfg}))
    ys, calls = {}, []
    for b in range(nbufs):
        if b == 1 and set_taps is not None:
            o.set_taps(set_taps(o.get(oracle.ORX_TAPS)[0]))
        w0 = o.get(oracle.ORX_TAPS)[0].copy()
        bits, n = o.process(g["packed"][b])
        y, y0 = o.get(oracle.ORX_Y)
        for i, v in enumerate(y):
            ys[y0 + i] = v
        z, z0 = o.get(oracle.ORX_Z)
        calls.append(dict(w0=w0, w1=o.get(oracle.ORX_TAPS)[0].copy(), z=z.copy(), z0=z0, bits=bits, n=n))
    return o, ys, calls


def test_frozen_call_is_one_fir():
    """With frozen taps, the soft symbols of a trained call are the fixed FIR of
    the 2-sps samples with the call's start taps: numpy's convolution."""
    g = _stream()
    o, ys, calls = _run(g, 3, eq_frozen=1)
    th = 15
    lo, hi = min(ys), max(ys) + 1
    yarr = np.array([ys.get(m, 0) for m in range(lo, hi)])
    for c in calls[1:]:
        full = np.convolve(yarr, np.conj(c["w0"]))
        k = c["z0"] + np.arange(len(c["z"]))
        ref = full[2 * k + th - lo]
        assert np.max(np.abs(c["z"] - ref)) < 1e-12 * np.max(np.abs(ref)) * 100
        assert not np.allclose(c["w1"], c["w0"])          # the call does move the taps


def test_frozen_equals_adaptive_at_zero_step():
    g = _stream()
    _, _, fa = _run(g, 3, eq_frozen=1, mu=0.0)
    _, _, ad = _run(g, 3, eq_frozen=0, mu=0.0)
    for a, b in zip(fa, ad):
        assert a["n"] == b["n"] and np.array_equal(a["bits"], b["bits"])
        assert np.array_equal(a["z"], b["z"]) and np.array_equal(a["w1"], b["w1"])


def test_frozen_noiseless_zero_errors():
    g = _stream(2, noise=False, phase_noise=False)
    o, _, _ = _run(g, 2, eq_frozen=1)
    s = o.stats()
    assert s["bits"] > 400_000 and s["bit_errors"] == 0 and s["raw_bit_errors"] == 0


def test_frozen_step_reduces_a_gain_error():
    """Noiseless data, taps scaled by 1.1 after training: every decision is
    right, the error is -0.1 z, and the step must shrink the scale back."""
    g = _stream(2, noise=False, phase_noise=False)
    _, _, calls = _run(g, 2, set_taps=lambda w: 1.1 * w, eq_frozen=1)
    w0, w1 = calls[1]["w0"], calls[1]["w1"]
    r = np.vdot(w0, w1) / np.vdot(w0, w0)        # projection of the new taps on the old ones
    assert 0.98 < abs(r) < 0.999 and abs(np.angle(r)) < 1e-2   # one averaged step, not sixteen
