"""Parity of the frequency-domain filter forms (the paper's static FD filters on
overlap-save blocks, Sec. 2: KK with a bin-truncation inverse as the downsampler
to 2 samples/symbol, PAM at its input rate) with the FP64 oracle: the 2-sps
samples within 1e-5 relative RMS, decisions and bits exact up to the exemptions
of the parity rules; KK block sizes from 64 to 1024, ragged buffers, the full
2^22-sample buffer, PAM-2/4/8 with the 503-tap filter, and batched calls equal
to sequential ones."""

import numpy as np
import pytest
import torch

from parity_util import Pair, make_stream
import paper_2010_14333_gb300 as rx

pytestmark = pytest.mark.gpu

SMALL_KK = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)


def run(fmt, nb, nbufs, **cfg):
    g = make_stream(fmt, nb, nbufs)
    p = Pair(fmt, nb, **cfg)
    for b in range(nbufs):
        p.feed(g["packed"][b])
    return p.compare_stats()


@pytest.mark.parametrize("nb", [1 << 17, 98304 + 32 * 7, 65536 * 3 - 160])
def test_fd_ragged_buffers(nb):
    s, so = run(4, nb, 3, mf_mode=1, **SMALL_KK)
    assert s["bits"] > 0 and so["ber"] < 0.05


@pytest.mark.parametrize("fd_n,fd_taps", [(64, 33), (128, 1), (256, 101), (512, 257), (1024, 513)])
def test_fd_block_lengths(fd_n, fd_taps):
    s, so = run(4, 1 << 16, 3, mf_mode=1, fd_n=fd_n, fd_taps=fd_taps, **SMALL_KK)
    assert s["bits"] > 0


def test_fd_qpsk():
    s, so = run(3, 1 << 17, 2, mf_mode=1, **SMALL_KK)
    assert s["bits"] > 0


def test_fd_full_size_buffer():
    s, so = run(4, 1 << 22, 2, mf_mode=1)
    assert s["bits"] == so["bits"] > 8_000_000
    assert 1e-4 < so["ber"] < 2e-2


def test_fd_batch_equals_sequential():
    nb, nbufs = 1 << 18, 6
    g = make_stream(4, nb, nbufs, seed=8)
    dev = [torch.from_numpy(p).cuda() for p in g["packed"]]
    a = rx.Receiver(4, nb, mf_mode=1, **SMALL_KK)
    seq = []
    for d in dev:
        bits, n = a.process(d)
        seq.append(bits[: (n + 7) // 8].cpu().numpy().copy())
    b = rx.Receiver(4, nb, mf_mode=1, **SMALL_KK)
    outs = b.process_batch(dev)
    assert len(outs) == nbufs
    for (bits, n), ref in zip(outs, seq):
        assert np.array_equal(bits[: (n + 7) // 8].cpu().numpy(), ref)
    sa, sb = a.stats(), b.stats()
    for k in ("bits", "bit_errors", "raw_bit_errors", "sym_errors", "windows"):
        assert sa[k] == sb[k], k


@pytest.mark.parametrize("fmt,nb", [(0, 1 << 18), (1, 1 << 20), (2, 1 << 18), (1, 98304 + 32 * 5)])
def test_fd_pam(fmt, nb):
    s, so = run(fmt, nb, 3, mf_mode=1)
    assert s["bits"] > 0


def test_fd_pam_batch_equals_sequential():
    nb, nbufs = 1 << 18, 5
    g = make_stream(1, nb, nbufs, seed=9)
    dev = [torch.from_numpy(p).cuda() for p in g["packed"]]
    a = rx.Receiver(1, nb, mf_mode=1)
    seq = []
    for d in dev:
        bits, n = a.process(d)
        seq.append(bits[: (n + 7) // 8].cpu().numpy().copy())
    b = rx.Receiver(1, nb, mf_mode=1)
    for (bits, n), ref in zip(b.process_batch(dev), seq):
        assert np.array_equal(bits[: (n + 7) // 8].cpu().numpy(), ref)
    assert a.stats()["bit_errors"] == b.stats()["bit_errors"]


def _pair_with_taps(fmt, nb, nbufs, taps, gen, **cfg):
    g = make_stream(fmt, nb, nbufs, **gen)
    p = Pair(fmt, nb, mf_mode=1, **cfg)
    t = taps(g) if callable(taps) else taps
    p.o.set_fd_taps(t)
    p.g.set_fd_taps(t)
    for b in range(nbufs):
        p.feed(g["packed"][b])
    return p.compare_stats()


def test_fd_pam_least_squares_taps():
    """PAM-4 through the ISI channel (0.1, 1, 0.2) with the 503 static taps fitted
    by least squares on the first buffer (numpy, oracle side), set on both receivers."""
    from test_fd_ls import pam_ls_taps
    nb = 1 << 17
    s, so = _pair_with_taps(1, nb, 3, lambda g: pam_ls_taps(g, nb), dict(seed=5, snr_db=14.0))
    assert s["bits"] > 0 and so["ber"] < 5e-3


def test_fd_kk_complex_taps():
    """KK-16QAM with complex, asymmetric static taps (207): the RRC taps plus an echo
    of 0.1 of them two input samples later, turned by e^{0.3j}."""
    import oracle
    rrc = oracle.rrc_half(0.1, 4, 101)
    taps = (np.concatenate([np.zeros(2), rrc, np.zeros(2)]) +
            0.1 * np.concatenate([np.zeros(4), rrc])) * np.exp(0.3j)
    s, so = _pair_with_taps(4, 1 << 17, 3, taps, {}, **SMALL_KK)
    assert s["bits"] > 0 and so["ber"] < 0.05


def test_fd_taps_rejected():
    r = rx.Receiver(1, 1 << 16, mf_mode=1)
    for bad in (np.ones(4), np.ones(5) * (1 + 0.5j), np.ones(515), np.array([1.0, np.nan, 1.0])):
        with pytest.raises(rx.RxError):
            r.set_fd_taps(bad)
    t = rx.Receiver(1, 1 << 16)   # time-domain form
    with pytest.raises(rx.RxError):
        t.set_fd_taps(np.ones(5))
