"""End of stream (rx_flush) and the per-buffer latency record, through the C ABI.

The flush of the CUDA receiver is compared with the FP64 oracle's (orx_flush):
the same number of bits, the same bits except symbols the parity rules exempt
(oracle soft value within 1e-4 of a threshold, or after one in the same block),
and the same counters.  The latency record is checked against budgets that every
call must miss or must meet, with no device fault involved."""

import numpy as np
import pytest
import torch

from parity_util import Pair, make_stream
import oracle
import paper_2010_14333_gb300 as rx

pytestmark = pytest.mark.gpu

SMALL_KK = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)


def _flush_pair(fmt, nb, nbufs, gen=None, **cfg):
    g = make_stream(fmt, nb, nbufs, **(gen or {}))
    p = Pair(fmt, nb, **cfg)
    for b in range(nbufs):
        p.feed(g["packed"][b])
    ob, on = p.o.flush()
    gb, gn = p.g.flush()
    gb = gb.cpu().numpy()
    assert gn == on and on > 0, (gn, on)
    bps = rx.BITS_PER_SYMBOL[fmt]
    obits = np.unpackbits(ob)[:on].reshape(-1, bps)
    gbits = np.unpackbits(gb)[:gn].reshape(-1, bps)
    bad = np.nonzero(np.any(obits != gbits, axis=1))[0]
    near, s0 = p.o.get(oracle.ORX_NEAR)
    s, so = p.g.stats(), p.o.stats()
    # a differing symbol needs an exempt symbol at or before it in the flush output
    if len(bad):
        assert np.any(near) or p.report["exempt"], f"flushed symbols differ with no exemption: {bad[:8]}"
    for k in ("bits", "symbols", "windows", "calls", "samples"):
        assert s[k] == so[k], (k, s[k], so[k])
    if not p.report["exempt"] and not np.any(near):
        assert len(bad) == 0
        for k in ("bit_errors", "raw_bit_errors", "sym_errors", "slip_windows"):
            assert s[k] == so[k], (k, s[k], so[k])
    assert s["device_error"] == 0
    return p, gn


@pytest.mark.parametrize("fmt", [3, 4])
def test_kk_flush_matches_oracle(fmt):
    _flush_pair(fmt, 1 << 17, 3, **SMALL_KK)


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_pam_flush_matches_oracle(fmt):
    _flush_pair(fmt, 1 << 18, 2)


def test_flush_fd_forms_and_resampler():
    _flush_pair(1, 1 << 18, 2, mf_mode=1)
    _flush_pair(4, 1 << 17, 3, mf_mode=1, **SMALL_KK)
    import synth
    step = synth.clock_step(-35.0)
    rs_step, rs_phase0 = rx.rx_resampler_from_clock(-35.0, 0.0)
    _flush_pair(4, 1 << 17, 3, gen=dict(clock_step=step), rs_step=rs_step, rs_phase0=rs_phase0, **SMALL_KK)


def test_flush_short_buffers_several_pad_calls():
    _flush_pair(1, 4096, 12, ntrain=1024)
    _flush_pair(4, 8192, 12, ols_n=4096, ols_v=512, ntrain=1024, ncma=512, amb_syms=256)


def test_flush_full_size_kk16():
    p, n = _flush_pair(4, 1 << 22, 2)
    assert n > 0


def test_after_flush():
    nb = 1 << 16
    g = make_stream(1, nb, 2)
    r = rx.Receiver(1, nb, ntrain=1024)
    for b in range(2):
        r.process(torch.from_numpy(g["packed"][b]).cuda())
    _, n1 = r.flush()
    _, n2 = r.flush()
    assert n1 > 0 and n2 == 0
    with pytest.raises(rx.RxError):
        r.process(torch.from_numpy(g["packed"][0]).cuda())


def _lat_run(nb, nbufs, batch=False, **cfg):
    g = make_stream(4, nb, nbufs)
    r = rx.Receiver(4, nb, **SMALL_KK, **cfg)
    bufs = [torch.from_numpy(g["packed"][b]).cuda() for b in range(nbufs)]
    if batch:
        r.process_batch(bufs)
    else:
        for b in bufs:
            r.process(b)
    return r.stats()


def test_latency_budget_missed_by_every_call():
    """A budget of 1 ns: every recorded call misses it; no device fault, no timeout."""
    s = _lat_run(1 << 17, 6, deadline_ms=1e-6)
    assert s["lat_calls"] >= 4 and s["deadline_misses"] == s["lat_calls"]
    assert 0 < s["lat_p50_ms"] <= s["lat_p99_ms"] <= s["lat_max_ms"] + 0.0005
    assert s["device_error"] == 0


def test_latency_budget_met_and_batch_recorded():
    s = _lat_run(1 << 17, 6, deadline_ms=10000.0)
    assert s["lat_calls"] >= 4 and s["deadline_misses"] == 0 and s["deadline_ms"] == 10000.0
    s = _lat_run(1 << 17, 8, batch=True, deadline_ms=10000.0)
    assert s["lat_calls"] >= 6 and s["deadline_misses"] == 0 and s["lat_p50_ms"] > 0


def test_latency_default_budget_and_off():
    s = _lat_run(1 << 17, 4)
    assert abs(s["deadline_ms"] - 5 * (1 << 17) / 4e9 * 1e3) < 1e-12
    s = _lat_run(1 << 17, 4, deadline_ms=-1.0)
    assert s["lat_calls"] == 0 and s["deadline_ms"] == 0.0


def test_latency_record_outlives_its_slot_ring():
    """More recorded calls than the record's 64 device slots, in one pipelined batch:
    every call is closed once, and no latency exceeds the batch's wall time."""
    import time
    g = make_stream(4, 1 << 17, 4)
    r = rx.Receiver(4, 1 << 17, **SMALL_KK, deadline_ms=10000.0)
    bufs = [torch.from_numpy(g["packed"][b]).cuda() for b in range(4)]
    r.process_batch(bufs)
    s0 = r.stats()
    torch.cuda.synchronize()
    t = time.perf_counter()
    r.process_batch([bufs[i % 4] for i in range(150)])
    r.stats()
    wall_ms = (time.perf_counter() - t) * 1e3
    s = r.stats()
    assert s["lat_calls"] - s0["lat_calls"] == 150
    assert s["deadline_misses"] == 0 and s["device_error"] == 0
    assert 0 < s["lat_p50_ms"] <= s["lat_p99_ms"] <= s["lat_max_ms"] < wall_ms
