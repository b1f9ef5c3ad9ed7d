"""Parity of the CUDA receiver (through the C ABI) with the FP64 oracle."""

import numpy as np
import pytest
import torch

from parity_util import Pair, make_stream, rel_rms
import oracle
import paper_2010_14333_gb300 as rx

pytestmark = pytest.mark.gpu

SMALL_KK = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)


def run(fmt, nb, nbufs, gen=None, **cfg):
    g = make_stream(fmt, nb, nbufs, **(gen or {}))
    p = Pair(fmt, nb, **cfg)
    for b in range(nbufs):
        p.feed(g["packed"][b])
    s, so = p.compare_stats()
    return p, s, so


@pytest.mark.parametrize("nb", [1 << 17, 98304 + 32 * 7, 65536 * 3 - 160])
def test_kk16_small_blocks_ragged_buffers(nb):
    p, s, so = run(4, nb, 3, **SMALL_KK)
    assert s["bits"] > 0 and so["ber"] < 0.05


@pytest.mark.parametrize("pack_order", [0, 1])
def test_kk_qpsk_pack_orders(pack_order):
    p, s, so = run(3, 1 << 17, 2, gen=dict(pack_order=pack_order), pack_order=pack_order, **SMALL_KK)
    assert s["bits"] > 0


def test_kk_small_overlap_many_blocks():
    run(4, 1 << 16, 2, ols_n=4096, ols_v=64, ntrain=2048, ncma=1024, amb_syms=1024)


def test_kk16_full_size_buffer():
    """The 2^22-sample KK-16QAM buffer with the 2^16-point overlap-save FFT,
    two consecutive buffers (the second one carries every history)."""
    p, s, so = run(4, 1 << 22, 2)
    assert s["bits"] == so["bits"] > 8_000_000
    assert 1e-4 < so["ber"] < 2e-2


def test_kk16_full_size_cluster_front():
    """The same two 2^22-sample buffers through the one-kernel cluster front end."""
    p, s, so = run(4, 1 << 22, 2, kk_front=1)
    assert s["bits"] == so["bits"] > 8_000_000


@pytest.mark.parametrize("fmt", [0, 1, 2])
def test_pam_chain(fmt):
    p, s, so = run(fmt, 1 << 20 if fmt == 1 else 1 << 18, 2)
    assert s["bits"] > 0


def test_noiseless_zero_errors_gpu():
    p, s, so = run(4, 1 << 17, 2, gen=dict(noise=False, phase_noise=False), **SMALL_KK)
    assert s["bit_errors"] == 0 and so["bit_errors"] == 0


def test_tiny_buffers_many_calls():
    """Buffers shorter than one FFT block: many calls pass before training
    completes and the first payload is emitted."""
    nb = 2048
    g = make_stream(4, nb, 40, seed=5)
    p = Pair(4, nb, ols_n=4096, ols_v=512, ntrain=1024, ncma=512, amb_syms=512, eq_block=512)
    emitted = 0
    for b in range(40):
        emitted += p.feed(g["packed"][b])
    assert emitted > 0
    p.compare_stats()


def test_host_buffers_match_device_path():
    nb = 1 << 17
    g = make_stream(4, nb, 2, seed=7)
    a = rx.Receiver(4, nb, **SMALL_KK)
    h = rx.rx_create(4, 1e9, 4e9, nb, a.cfg)
    try:
        out = np.zeros(rx.rx_max_bits(h) // 8 + 16, np.uint8)
        for b in range(2):
            bits, n = a.process(torch.from_numpy(g["packed"][b]).cuda())
            inp = np.ascontiguousarray(g["packed"][b])
            n2 = rx.rx_process_host(h, inp.ctypes.data, out.ctypes.data, 0)
            torch.cuda.synchronize()
            assert n2 == n
            assert np.array_equal(out[: (n + 7) // 8], bits.cpu().numpy())
        assert rx.rx_stats(h)["bit_errors"] == a.stats()["bit_errors"]
    finally:
        rx.rx_destroy(h)


@pytest.mark.parametrize("fmt", [3, 4])
def test_differential_coding_parity(fmt):
    """Differentially quadrant-coded KK streams (noise and laser phase noise): GPU at
    parity with the oracle, bits and counts; the decoded output's raw BER equals the
    BER-tester view."""
    p, s, so = run(fmt, 1 << 17, 3, gen=dict(diff=True), diff_code=1, **SMALL_KK)
    assert s["bits"] > 0 and s["raw_bit_errors"] == s["bit_errors"] and s["slip_windows"] == 0


def test_differential_coding_survives_a_slip_on_gpu():
    import synth
    nb = 1 << 20
    res = {}
    for diff in (0, 1):
        g = synth.gen_kk_stream(4, nb, 2, seed=3, noise=False, phase_noise=False, diff=bool(diff), truth=False,
                                phase_steps=((3 << 18, np.pi / 2),))
        r = rx.Receiver(4, nb, diff_code=diff)
        for pk in g["packed"]:
            r.process(torch.from_numpy(pk).cuda())
        res[diff] = r.stats()
    assert res[0]["raw_bit_errors"] > 0.2 * res[0]["bits"]
    assert res[1]["raw_bit_errors"] <= 8
