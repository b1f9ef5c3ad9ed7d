"""The paper's short KK equaliser (Sec. 2, KK chain: a 4-tap decision-directed LMS
that recovers the clock phase and the symbol phase, 8192 blocks per buffer), the
oracle's eq_mode = 1: the taps are updated after every symbol and no phase search
runs.  Pins:
- with the steps at zero the filter is its definition, z_k = sum_j conj(w_j)
  y[2k + th - j] (th = (ntaps - 1) / 2), checked against the oracle's own 2-sps
  samples for the start taps and for taps set by hand;
- noiseless KK-16QAM and KK-QPSK streams without relative phase noise (the paper's
  self-coherent link) decode with no error, also through a 0.35-sample clock delay;
- at 20 dB the BER is that of the 31-tap window equaliser with its phase search
  within a factor of 1.25."""

import numpy as np
import pytest

import oracle
import synth

SMALL = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)
NB = 1 << 17


def stream(fmt=4, nbufs=3, seed=3, **kw):
    kw.setdefault("linewidth", 0.0)
    kw.setdefault("phase_noise", False)
    return synth.gen_kk_stream(fmt, NB, nbufs, seed=seed, **kw)


def run(g, fmt=4, **cfg):
    o = oracle.Oracle(**oracle.default_cfg(fmt, NB, eq_mode=1, ntaps=4, **SMALL, **cfg))
    for p in g["packed"]:
        o.process(p)
    return o


@pytest.mark.parametrize("taps", [None, np.array([0.1 - 0.05j, 0.9 + 0.2j, -0.2 + 0.1j, 0.05j])])
def test_dd_filter_definition(taps):
    """mu = mu_cma = 0: the taps never move, so z_k is the plain filter of the
    2-sps samples (start taps: a unit tap at th)."""
    g = stream(nbufs=2, noise=False)
    o = oracle.Oracle(**oracle.default_cfg(4, NB, eq_mode=1, ntaps=4, mu=0.0, mu_cma=0.0, **SMALL))
    if taps is not None:
        o.set_taps(taps)
    w = np.zeros(4, complex) if taps is None else taps
    if taps is None:
        w[1] = 1.0
    for p in g["packed"]:
        o.process(p)
        y, y0 = o.get(oracle.ORX_Y)
        z, z0 = o.get(oracle.ORX_Z)
        if not len(z):
            continue
        k = np.arange(z0, z0 + len(z))
        # symbols whose four samples lie in this call's view of the 2-sps samples
        sel = (2 * k - 2 >= y0) & (2 * k + 1 < y0 + len(y))
        assert sel.sum() > 30000
        k = k[sel]
        ref = sum(np.conj(w[j]) * y[2 * k + 1 - j - y0] for j in range(4))
        got = z[k - z0]
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("nt", [2, 3, 4, 6, 8])
def test_dd_filter_definition_across_calls(nt):
    """The same definition for every symbol of a stream, the first symbols of each
    call included: they reach back into the previous call's 2-sps samples (ntaps - 1 -
    th of them, one more than th for an even tap count).  The calls' views of the
    samples are consecutive, so their concatenation is the whole 2-sps stream."""
    g = stream(nbufs=3, noise=False)
    o = oracle.Oracle(**oracle.default_cfg(4, NB, eq_mode=1, ntaps=nt, mu=0.0, mu_cma=0.0, **SMALL))
    w = np.exp(1j * np.arange(nt)) * np.linspace(0.2, 1.0, nt)   # every tap non-zero
    o.set_taps(w)
    ys, zs = [], []
    for p in g["packed"]:
        o.process(p)
        ys.append(o.get(oracle.ORX_Y))
        zs.append(o.get(oracle.ORX_Z))
    for (y_a, a0), (y_b, b0) in zip(ys, ys[1:]):
        assert b0 == a0 + len(y_a)
    assert ys[0][1] == 0
    Y = np.concatenate([y for y, _ in ys])
    th = (nt - 1) // 2
    checked = 0
    for z, z0 in zs[1:]:   # calls after the first: their first symbols read the previous call's samples
        k = np.arange(z0, z0 + len(z))
        k = k[2 * k + th < len(Y)]
        ref = sum(np.conj(w[j]) * np.where(2 * k + th - j >= 0, Y[np.maximum(2 * k + th - j, 0)], 0) for j in range(nt))
        assert np.max(np.abs(z[: len(k)] - ref)) < 1e-12 * np.max(np.abs(ref)), nt
        checked += len(k)
    assert checked > 60000


@pytest.mark.parametrize("fmt,delay", [(4, 0.0), (4, 0.35), (3, 0.0), (3, 0.35)])
def test_dd_noiseless_zero_errors(fmt, delay):
    g = stream(fmt, noise=False, clock_phase0=int(delay * (1 << 32)))
    s = run(g, fmt).stats()
    assert s["bits"] > (300_000 if fmt == 4 else 150_000)
    assert s["bit_errors"] == 0 and s["raw_bit_errors"] == 0 and s["slip_windows"] == 0
    assert s["ambiguous_windows"] == 0


def test_dd_ber_close_to_the_window_equaliser():
    g = stream(snr_db=20.0)
    s_dd = run(g).stats()
    o = oracle.Oracle(**oracle.default_cfg(4, NB, **SMALL))
    for p in g["packed"]:
        o.process(p)
    s_w = o.stats()
    assert s_dd["bits"] == s_w["bits"] > 300_000
    assert 0 < s_dd["ber"] < 1.25 * s_w["ber"], (s_dd["ber"], s_w["ber"])
    assert s_dd["slip_windows"] == 0


def test_dd_mode_rejected_where_undefined():
    for bad in (dict(format=1), dict(ntaps=1), dict(ntaps=33), dict(eq_frozen=1), dict(eq_mode=2)):
        cfg = oracle.default_cfg(bad.get("format", 4), NB, eq_mode=1, ntaps=4, **SMALL)
        cfg.update(bad)
        if cfg["format"] < 3:
            cfg.update(oracle.default_cfg(1, NB, eq_mode=1, ntaps=4))
        with pytest.raises(Exception):
            oracle.Oracle(**cfg)
