"""Learned equaliser on the GPU: gradients against the FP64 oracle, and the
trained network against the adaptive FIR it stands in for."""

import math

import numpy as np
import pytest
import torch
from scipy.special import erf

import oracle
import paper_2010_14333_gb300 as rx
import synth
from paper_2010_14333_gb300 import cnn

pytestmark = pytest.mark.gpu
S, L0 = 64, 152


def gpu_grad(params, y, seg, tgt):
    c = rx.rx_cnn_create(len(seg))
    try:
        rx.rx_cnn_set_params(c, params)
        yd = torch.view_as_real(torch.from_numpy(y.astype(np.complex64)).cuda()).contiguous()
        sd = torch.from_numpy(np.asarray(seg, dtype=np.int64)).cuda()
        td = torch.from_numpy(tgt.astype(np.float32)).cuda()
        g = torch.zeros(rx.rx_cnn_nparams(), dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        out = torch.zeros(len(seg) * S * 2, dtype=torch.float32, device="cuda")
        rx.rx_cnn_grad(c, yd.data_ptr(), sd.data_ptr(), td.data_ptr(), len(seg), g.data_ptr(), loss.data_ptr())
        rx.rx_cnn_forward(c, yd.data_ptr(), sd.data_ptr(), len(seg), out.data_ptr())
        torch.cuda.synchronize()
        return g.cpu().numpy().astype(np.float64), float(loss.item()), out.cpu().numpy().reshape(len(seg), S, 2)
    finally:
        rx.rx_cnn_destroy(c)


def test_cnn_gradients_match_oracle():
    rng = np.random.default_rng(5)
    params = cnn.init_params(3).astype(np.float64)
    params += rng.standard_normal(len(params)) * 0.01           # non-zero biases
    y = (rng.standard_normal(4000) + 1j * rng.standard_normal(4000)) * 0.7
    nseg = 24
    seg = rng.integers(0, len(y) - L0, size=nseg)
    tgt = rng.standard_normal((nseg, S, 2)) * 0.7
    x = np.stack([np.stack([y[s:s + L0].real, y[s:s + L0].imag], axis=1) for s in seg])
    lo, go, oo = oracle.cnn_loss_grad(params, x, tgt)
    g, lg, og = gpu_grad(params.astype(np.float32), y, seg, tgt)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(og, oo) < 2e-2, rel(og, oo)
    assert abs(lg - lo) < 2e-2 * lo
    cos = float(np.dot(g, go) / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos > 0.999 and rel(g, go) < 2e-2, (cos, rel(g, go))
    for name, (off, shape) in oracle.cnn_param_slices().items():   # every tensor on its own
        n = int(np.prod(shape))
        a, b = g[off:off + n], go[off:off + n]
        assert rel(a, b) < 5e-2, (name, rel(a, b))


def test_cnn_pass_through_on_gpu():
    p = np.zeros(rx.rx_cnn_nparams(), dtype=np.float32)
    sl = oracle.cnn_param_slices()
    for name, cin in (("W1", 2), ("W2", 32), ("W3", 32)):
        W = p[sl[name][0]:sl[name][0] + 32 * 9 * cin].reshape(32, 9, cin)
        W[0, 4, 0] = W[1, 4, 1] = 1.0
    p[sl["M1"][0] + 0 * 32 + 0] = p[sl["M1"][0] + 1 * 32 + 1] = 1.0
    p[sl["M2"][0] + 0 * 64 + 0] = p[sl["M2"][0] + 1 * 64 + 1] = 1.0
    rng = np.random.default_rng(6)
    y = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    _, _, out = gpu_grad(p, y, [10, 200], np.zeros((2, S, 2)))
    g = lambda u: 0.5 * u * (1 + erf(u / math.sqrt(2)))
    for si, s in enumerate([10, 200]):
        ref = g(g(g(g(np.stack([y[s + 12:s + 140:2].real, y[s + 12:s + 140:2].imag], axis=1)))))
        assert np.max(np.abs(out[si] - ref)) < 2e-2


VOLT = dict(volterra=(0.05, 0.02), cspr_db=6.0, snr_db=19.0, linewidth=0.0, phase_noise=False)


def test_trained_cnn_beats_the_adaptive_fir():
    """Train on counter-based random symbols through the Volterra + SSBI channel
    (CSPR 6 dB); judge on a fresh PRBS stream: the CNN must reach a lower BER
    than the 31-tap CMA/DD-LMS FIR with blind phase search on the same buffers."""
    nb = 1 << 20
    ntr = 6
    sym_tr = synth.random_symbols(4, ntr * nb // 4 + 64, seed=99)
    gtr = synth.gen_kk_stream(4, nb, ntr, seed=21, symbols=sym_tr, truth=False, **VOLT)
    y = cnn.mf_output(gtr["packed"], nb)
    tr = cnn.CnnTrainer(batch=64, seed=1)
    tr.set_data(y, sym_tr, k_lo=64)
    losses = tr.train(3000, lr=1e-3, report=500)
    tr.train(1000, lr=3e-4)
    assert losses[-1] < losses[0]
    gev = synth.gen_kk_stream(4, nb, 3, seed=22, truth=False, **VOLT)
    lms = rx.Receiver(4, nb)
    net = rx.Receiver(4, nb)
    rx.rx_set_cnn(net.h, tr.h)
    for p in gev["packed"]:
        d = torch.from_numpy(p).cuda()
        lms.process(d)
        net.process(d)
    sl, sn = lms.stats(), net.stats()
    print("BER lms", sl["ber"], "cnn", sn["ber"], "losses", losses)
    assert sl["bits"] == sn["bits"] > 0
    assert sn["ber"] < sl["ber"], (sn["ber"], sl["ber"])
