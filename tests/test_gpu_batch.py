"""The pipelined batch entry points against one call per buffer: the same bits,
bit counts and counters, whatever the split of the stream into batches."""

import numpy as np
import pytest
import torch

from parity_util import make_stream
import paper_2010_14333_gb300 as rx
from paper_2010_14333_gb300 import cnn

pytestmark = pytest.mark.gpu

COUNTERS = ("calls", "samples", "symbols", "bits", "bit_errors", "raw_bit_errors", "sym_errors", "slip_windows",
            "near_threshold", "ambiguous_windows", "windows", "amb_rot", "device_error")


def sequential(fmt, nb, packed, cnn_h=None, **cfg):
    r = rx.Receiver(fmt, nb, **cfg)
    if cnn_h:
        rx.rx_set_cnn(r.h, cnn_h)
    out = []
    for p in packed:
        bits, n = r.process(torch.from_numpy(p).cuda())
        out.append((bits.cpu().numpy().copy(), n))
    return out, r.stats()


def batched(fmt, nb, packed, splits, cnn_h=None, **cfg):
    r = rx.Receiver(fmt, nb, **cfg)
    if cnn_h:
        rx.rx_set_cnn(r.h, cnn_h)
    dev = [torch.from_numpy(p).cuda() for p in packed]
    out, i = [], 0
    for k in splits:
        if k == 1:                                   # a plain call between batches
            bits, n = r.process(dev[i])
            out.append((bits.cpu().numpy().copy(), n))
        else:
            for bits, n in r.process_batch(dev[i:i + k]):
                out.append((bits.cpu().numpy().copy(), n))
        i += k
    assert i == len(packed)
    return out, r.stats()


def same(a, b):
    (oa, sa), (ob, sb) = a, b
    assert len(oa) == len(ob)
    for i, ((ba, na), (bb, nb)) in enumerate(zip(oa, ob)):
        assert na == nb, (i, na, nb)
        assert np.array_equal(ba, bb), i
    for k in COUNTERS:
        assert sa[k] == sb[k], (k, sa[k], sb[k])


@pytest.mark.parametrize("splits", [[10], [1, 3, 6], [4, 1, 5]])
def test_kk16_batch_equals_sequential(splits):
    nb = 1 << 19
    g = make_stream(4, nb, 10, seed=11, workers=4)
    ref = sequential(4, nb, g["packed"])
    assert ref[1]["bits"] > 0
    same(batched(4, nb, g["packed"], splits), ref)


@pytest.mark.parametrize("splits", [[7], [2, 1, 4]])
def test_kk_cluster_front_batch_equals_sequential(splits):
    """The fused cluster front end in the pipeline: the field of consecutive buffers
    alternates over two streams, each launch ordered after the previous buffer's
    history copy and field."""
    nb = 1 << 19
    g = make_stream(4, nb, 7, seed=16, workers=4)
    ref = sequential(4, nb, g["packed"], kk_front=1)
    assert ref[1]["bits"] > 0
    same(batched(4, nb, g["packed"], splits, kk_front=1), ref)


def test_kk_small_fft_batch_equals_sequential():
    """Many overlap-save blocks per buffer and a ragged buffer length."""
    nb = 65536 * 3 - 160
    cfg = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)
    g = make_stream(4, nb, 7, seed=12)
    same(batched(4, nb, g["packed"], [7], **cfg), sequential(4, nb, g["packed"], **cfg))


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_pam_batch_equals_sequential(fmt):
    nb = 1 << 18
    g = make_stream(fmt, nb, 6, seed=13)
    same(batched(fmt, nb, g["packed"], [2, 4]), sequential(fmt, nb, g["packed"]))


def test_tiny_buffers_batch_equals_sequential():
    """Calls that emit nothing (training not complete) inside a batch."""
    nb = 2048
    cfg = dict(ols_n=4096, ols_v=512, ntrain=1024, ncma=512, amb_syms=512, eq_block=512)
    g = make_stream(4, nb, 40, seed=5)
    same(batched(4, nb, g["packed"], [25, 15], **cfg), sequential(4, nb, g["packed"], **cfg))


def test_cnn_receiver_batch_equals_sequential():
    nb = 1 << 19
    tr = cnn.CnnTrainer(batch=8, seed=3)
    g = make_stream(4, nb, 5, seed=14, workers=4)
    same(batched(4, nb, g["packed"], [5], cnn_h=tr.h), sequential(4, nb, g["packed"], cnn_h=tr.h))


def test_host_batch_equals_sequential():
    nb = 1 << 19
    g = make_stream(4, nb, 8, seed=15, workers=4)
    ref, sref = sequential(4, nb, g["packed"])
    h = rx.rx_create(4, 1e9, 4e9, nb, rx.rx_default_config(4))
    try:
        cap = rx.rx_max_bits(h) // 8 + 16
        hin = [torch.from_numpy(p).pin_memory() for p in g["packed"]]
        hout = [torch.zeros(cap, dtype=torch.uint8).pin_memory() for _ in hin]
        got = []
        for lo, hi in ((0, 3), (3, 8)):
            ns = rx.rx_process_host_batch(h, [t.data_ptr() for t in hin[lo:hi]],
                                          [t.data_ptr() for t in hout[lo:hi]], 0)
            torch.cuda.synchronize()
            got += [(hout[lo + i][: (n + 7) // 8].numpy().copy(), n) for i, n in enumerate(ns)]
        same((got, rx.rx_stats(h)), (ref, sref))
    finally:
        rx.rx_destroy(h)


def test_sampled_stage_profile():
    """rx_profile(h, 4) times calls 0, 4, 8 of ten, on both pipeline streams."""
    nb = 1 << 19
    g = make_stream(4, nb, 10, seed=16, workers=4)
    r = rx.Receiver(4, nb)
    rx.rx_profile(r.h, 4)
    r.process_batch([torch.from_numpy(p).cuda() for p in g["packed"]])
    ms, calls = rx.rx_profile_read(r.h)
    rx.rx_profile(r.h, 0)
    assert calls == 3
    for s in ("kk_fwd", "mf", "eq", "demap"):    # 2^16-point blocks: the fused front is kk_fwd
        assert ms[s] > 0, s
    assert ms["unpack"] == 0                      # the KK chain reads the packed input itself


@pytest.mark.parametrize("warps", [2, 8])
def test_eq_warps_do_not_change_results(warps):
    """Equaliser blocks per CTA are a launch shape only: bit-identical output."""
    nb = 1 << 19
    g = make_stream(4, nb, 4, seed=17, workers=4)
    same(batched(4, nb, g["packed"], [4], eq_warps=warps), sequential(4, nb, g["packed"]))


def test_handles_with_different_cta_shapes_coexist():
    """A kernel's shared-memory limit belongs to the function: creating a handle
    with small equaliser CTAs after one with large CTAs must not break the latter."""
    nb = 1 << 19
    g = make_stream(4, nb, 3, seed=18, workers=4)
    r8 = rx.Receiver(4, nb, eq_warps=8)
    r2 = rx.Receiver(4, nb, eq_warps=2)
    for p in g["packed"]:
        d = torch.from_numpy(p).cuda()
        r8.process(d)
        r2.process(d)
    s8, s2 = r8.stats(), r2.stats()
    assert s8["bits"] == s2["bits"] > 0 and s8["bit_errors"] == s2["bit_errors"]
    assert s8["device_error"] == 0 and s2["device_error"] == 0


def test_full_size_batch_equals_sequential():
    """The bench's launch configuration: 2^22-sample KK-16QAM buffers through the
    two-stream pipeline, against one call per buffer."""
    nb = 1 << 22
    g = make_stream(4, nb, 4, seed=19, workers=8)
    same(batched(4, nb, g["packed"], [4]), sequential(4, nb, g["packed"]))


def test_bounded_wait_reports_timeout_and_context_stays_usable():
    """A wait on an mbarrier phase that nothing completes gives up after its poll
    bound and reports RX_ETIMEOUT (no fault, no hang); the receiver then still runs
    and its streams report no device error."""
    assert rx.rx_selftest_wait_timeout(torch.cuda.current_stream().cuda_stream) == 5   # RX_ETIMEOUT
    nb = 1 << 17
    g = make_stream(4, nb, 2, seed=3)
    r = rx.Receiver(4, nb, ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)
    for p in g["packed"]:
        r.process(torch.from_numpy(p).cuda())
    s = r.stats()
    assert s["device_error"] == 0 and s["bits"] > 0


def test_fma_rate_selftest():
    """The FMA-rate self-test reports a rate between a tenth of and a little above the
    peak derived from the SM count and the maximum SM clock, and rejects bad sizes."""
    props = torch.cuda.get_device_properties(0)
    derived = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    sid = torch.cuda.current_stream().cuda_stream
    t = rx.rx_selftest_fma_rate(1 << 14, sid)
    assert 0.1 * derived < t < 1.1 * derived, (t, derived)
    for bad in (0, (1 << 24) + 1):
        with pytest.raises(rx.RxError):
            rx.rx_selftest_fma_rate(bad, sid)
