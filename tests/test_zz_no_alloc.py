"""The allocation-free KK field entry point against the regular receiver.

rx_kk_field_noalloc serves callers that may not allocate device memory while
running (its scratch is a fixed array inside librx.so).  Its output must equal
the field the regular entry point rx_process emits for the first buffer of a
stream, within the field tolerance of the parity tests, on two calls in a row
with different sizes and FFT lengths (the second call reuses the array the first
one left behind).  This file is collected last so that a run that stops at the
first failure has already run every other test.
"""

import numpy as np
import pytest
import torch

import paper_2010_14333_gb300 as rx
from parity_util import FIELD_TOL, make_stream, rel_rms

pytestmark = pytest.mark.gpu


def regular_field(packed, nb, ols_n, ols_v):
    r = rx.Receiver(rx.RX_KK_16QAM, nb, ols_n=ols_n, ols_v=ols_v, ntrain=4096, ncma=2048, amb_syms=1024)
    r.process(torch.from_numpy(packed).cuda())
    E, e0 = r.debug(rx.RX_DBG_FIELD)
    assert e0 == 0
    return E


def test_noalloc_field_matches_regular_entry_point_twice():
    cases = [(1 << 19, 65536, 4096, 11), ((1 << 17) + 96, 4096, 512, 12)]
    stream = torch.cuda.current_stream().cuda_stream
    for nb, n, v, seed in cases:
        g = make_stream(rx.RX_KK_16QAM, nb, 1, seed=seed, truth=False)
        packed = g["packed"][0]
        dev_in = torch.from_numpy(packed).cuda()
        count = nb - v // 2
        out = torch.full((2 * count,), float("nan"), dtype=torch.float32, device="cuda")
        rx.rx_kk_field_noalloc(dev_in.data_ptr(), nb, 0, n, v, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.complex64)
        ref = regular_field(packed, nb, n, v)
        assert len(ref) == count and np.all(np.isfinite(got))
        assert rel_rms(got, ref) <= FIELD_TOL, rel_rms(got, ref)


def test_noalloc_rejects_oversize_and_bad_arguments():
    lib = rx.load()
    buf = torch.zeros(3 * (1 << 19) // 2 + 64, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2 << 20, dtype=torch.float32, device="cuda")
    assert lib.rx_kk_field_noalloc(buf.data_ptr(), (1 << 19) + 32, 0, 65536, 4096, out.data_ptr(), None) == 1
    assert lib.rx_kk_field_noalloc(buf.data_ptr(), 1000, 0, 4096, 512, out.data_ptr(), None) == 1
    assert lib.rx_kk_field_noalloc(buf.data_ptr(), 4096, 0, 8192, 512, out.data_ptr(), None) == 1
    # legal sizes whose overlap-save blocks need more FFT rows than the array holds
    assert lib.rx_kk_field_noalloc(buf.data_ptr(), 1 << 19, 0, 65536, 61440, out.data_ptr(), None) == 1
