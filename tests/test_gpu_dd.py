"""The paper's short KK equaliser on the GPU (rx_config.eq_mode = RX_EQ_DD_SYMBOL:
a decision-directed LMS updated symbol by symbol, one thread per block) against
the FP64 oracle's eq_mode 1, through the C ABI: decisions, bits and counters under
the parity rules of the window equaliser (a symbol within 1e-4 of a threshold
exempts the rest of its adaptive block), on streams without relative laser phase
noise (the self-coherent link the form is meant for)."""

import numpy as np
import pytest
import torch

from parity_util import Pair, make_stream
import paper_2010_14333_gb300 as rx

pytestmark = pytest.mark.gpu

SMALL_KK = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024)
DD = dict(eq_mode=rx.RX_EQ_DD_SYMBOL, ntaps=4)


def run(fmt, nb, nbufs, gen, **cfg):
    g = make_stream(fmt, nb, nbufs, linewidth=0.0, phase_noise=False, **gen)
    p = Pair(fmt, nb, **DD, **cfg)
    for b in range(nbufs):
        p.feed(g["packed"][b])
    return p.compare_stats()


@pytest.mark.parametrize("fmt", [4, 3])
@pytest.mark.parametrize("delay", [0.0, 0.35])
def test_dd_parity(fmt, delay):
    s, so = run(fmt, 1 << 17, 3, dict(seed=3, snr_db=20.0 if fmt == 4 else 12.0,
                                      clock_phase0=int(delay * (1 << 32))), **SMALL_KK)
    assert s["bits"] > 0 and 0 < so["ber"] < 0.01


def test_dd_noiseless_zero_errors():
    s, so = run(4, 1 << 17, 3, dict(seed=4, noise=False), **SMALL_KK)
    assert s["bit_errors"] == so["bit_errors"] == 0 and s["bits"] > 300_000


def test_dd_full_size_buffer():
    s, so = run(4, 1 << 22, 2, dict(seed=5, snr_db=20.0, workers=4))
    assert s["bits"] == so["bits"] > 8_000_000 and so["ber"] < 5e-3


def test_dd_batch_equals_sequential():
    nb, nbufs = 1 << 18, 6
    g = make_stream(4, nb, nbufs, seed=8, linewidth=0.0, phase_noise=False)
    dev = [torch.from_numpy(p).cuda() for p in g["packed"]]
    a = rx.Receiver(4, nb, **DD, **SMALL_KK)
    seq = []
    for d in dev:
        bits, n = a.process(d)
        seq.append(bits[: (n + 7) // 8].cpu().numpy().copy())
    b = rx.Receiver(4, nb, **DD, **SMALL_KK)
    outs = b.process_batch(dev)
    for (bits, n), ref in zip(outs, seq):
        assert np.array_equal(bits[: (n + 7) // 8].cpu().numpy(), ref)
    assert a.stats()["bit_errors"] == b.stats()["bit_errors"]


def test_dd_rejected_where_undefined():
    for bad in (dict(fmt=1), dict(ntaps=9), dict(ntaps=1), dict(fir_prec=rx.RX_FIR_BF16, eq_block=1024),
                dict(eq_mode=2)):
        kw = dict(DD)
        fmt = bad.pop("fmt", 4)
        kw.update(bad)
        with pytest.raises(rx.RxError):
            rx.Receiver(fmt, 1 << 17, **kw)
