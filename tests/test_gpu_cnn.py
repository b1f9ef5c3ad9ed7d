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
    (CSPR 6 dB); evaluate on a fresh PRBS stream: the CNN must reach a lower BER
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
    netb = rx.Receiver(4, nb, cnn_bf16=0)   # the same network with FP16 operands
    rx.rx_set_cnn(net.h, tr.h)
    rx.rx_set_cnn(netb.h, tr.h)
    for p in gev["packed"]:
        d = torch.from_numpy(p).cuda()
        lms.process(d)
        net.process(d)
        netb.process(d)
    sl, sn, sb = lms.stats(), net.stats(), netb.stats()
    print("BER lms", sl["ber"], "cnn", sn["ber"], "cnn fp16", sb["ber"], "losses", losses)
    assert sl["bits"] == sn["bits"] == sb["bits"] > 0
    assert sn["ber"] < sl["ber"], (sn["ber"], sl["ber"])
    assert sb["ber"] < sl["ber"], (sb["ber"], sl["ber"])


@pytest.mark.parametrize("bf16,tol", [(0, 1e-2), (1, 2e-2)])
def test_cnn_receiver_soft_matches_training_forward(bf16, tol):
    """The receiver's tensor-core inference (tcgen05, row-shifted activation
    planes, 128-symbol tiles; FP16 or BF16 operands) against the training forward
    (mma.sync, 64-symbol segments) on the same 2-sps samples, with random weights."""
    nb = 1 << 19
    g = synth.gen_kk_stream(4, nb, 2, seed=23, truth=False, **VOLT)
    p = cnn.init_params(11).astype(np.float32)
    p += np.random.default_rng(12).standard_normal(len(p)).astype(np.float32) * 0.02
    c = rx.rx_cnn_create(64)
    try:
        rx.rx_cnn_set_params(c, p)
        r = rx.Receiver(4, nb, debug=1, cnn_bf16=bf16)
        rx.rx_set_cnn(r.h, c)
        for b in range(2):
            r.process(torch.from_numpy(g["packed"][b]).cuda())
        soft, s0 = r.debug(rx.RX_DBG_SOFT)
        y, y0 = r.debug(rx.RX_DBG_MF)
        assert len(soft) > 0
        # windows well inside the call, whose inputs lie in the MF view
        ks = [k for k in range(s0 + 64 * 20, s0 + len(soft) - 64 * 20, 64 * 37)][:24]
        seg = [2 * k - 12 - y0 for k in ks]
        assert min(seg) >= 0 and max(seg) + L0 <= len(y)
        yd = torch.view_as_real(torch.from_numpy(y.astype(np.complex64)).cuda()).contiguous()
        sd = torch.from_numpy(np.asarray(seg, dtype=np.int64)).cuda()
        out = torch.zeros(len(seg) * S * 2, dtype=torch.float32, device="cuda")
        rx.rx_cnn_forward(c, yd.data_ptr(), sd.data_ptr(), len(seg), out.data_ptr())
        torch.cuda.synchronize()
        ref = out.cpu().numpy().reshape(len(seg), S, 2)
        ref = ref[..., 0] + 1j * ref[..., 1]
        got = np.stack([soft[k - s0: k - s0 + S] for k in ks])
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < tol, rel
    finally:
        rx.rx_cnn_destroy(c)


@pytest.mark.parametrize("bf16,tol", [(0, 2e-2), (1, 4e-2)])
def test_cnn_receiver_pass_through_closed_form(bf16, tol):
    """Identity-like weights: the receiver's soft symbol is GELU^4 of the 2-sps
    sample at the symbol position (channel-wise), computed here from its MF view;
    FP16 or BF16 activations (8 or 11 significant bits per layer)."""
    nb = 1 << 19
    g = synth.gen_kk_stream(4, nb, 2, seed=24, truth=False)
    p = np.zeros(rx.rx_cnn_nparams(), dtype=np.float32)
    sl = oracle.cnn_param_slices()
    for name, cin in (("W1", 2), ("W2", 32), ("W3", 32)):
        W = p[sl[name][0]:sl[name][0] + 32 * 9 * cin].reshape(32, 9, cin)
        W[0, 4, 0] = W[1, 4, 1] = 1.0
    p[sl["M1"][0] + 0 * 32 + 0] = p[sl["M1"][0] + 1 * 32 + 1] = 1.0
    p[sl["M2"][0] + 0 * 64 + 0] = p[sl["M2"][0] + 1 * 64 + 1] = 1.0
    c = rx.rx_cnn_create(8)
    try:
        rx.rx_cnn_set_params(c, p)
        r = rx.Receiver(4, nb, debug=1, cnn_bf16=bf16)
        rx.rx_set_cnn(r.h, c)
        for b in range(2):
            r.process(torch.from_numpy(g["packed"][b]).cuda())
        soft, s0 = r.debug(rx.RX_DBG_SOFT)
        y, y0 = r.debug(rx.RX_DBG_MF)
        k = np.arange(s0 + 64, s0 + len(soft) - 64)
        k = k[(2 * k - y0 >= 0) & (2 * k - y0 < len(y))]
        gl = lambda u: 0.5 * u * (1 + erf(u / math.sqrt(2)))
        v = y[2 * k - y0]
        ref = gl(gl(gl(gl(v.real)))) + 1j * gl(gl(gl(gl(v.imag))))
        got = soft[k - s0]
        assert np.max(np.abs(got - ref)) < tol * max(1.0, np.max(np.abs(ref)))
    finally:
        rx.rx_cnn_destroy(c)


@pytest.mark.parametrize("bf16,tol", [(0, 1.5e-2), (1, 3e-2)])
def test_cnn_receiver_soft_matches_oracle_forward(bf16, tol):
    """The receiver's tensor-core inference against the FP64 oracle's forward pass
    (orx_cnn_loss_grad's outputs) on the same 2-sps samples, random weights: FP16
    or BF16 activations between layers, FP32 accumulation."""
    nb = 1 << 19
    g = synth.gen_kk_stream(4, nb, 2, seed=25, truth=False, **VOLT)
    p = cnn.init_params(13).astype(np.float32)
    p += np.random.default_rng(14).standard_normal(len(p)).astype(np.float32) * 0.02
    c = rx.rx_cnn_create(64)
    try:
        rx.rx_cnn_set_params(c, p)
        r = rx.Receiver(4, nb, debug=1, cnn_bf16=bf16)
        rx.rx_set_cnn(r.h, c)
        for b in range(2):
            r.process(torch.from_numpy(g["packed"][b]).cuda())
        soft, s0 = r.debug(rx.RX_DBG_SOFT)
        y, y0 = r.debug(rx.RX_DBG_MF)
        ks = [k for k in range(s0 + 64 * 20, s0 + len(soft) - 64 * 20, 64 * 41)][:24]
        seg = [2 * k - 12 - y0 for k in ks]
        assert min(seg) >= 0 and max(seg) + L0 <= len(y)
        yv = y.astype(np.complex128)
        x = np.stack([np.stack([yv[s:s + L0].real, yv[s:s + L0].imag], axis=1) for s in seg])
        _, _, out = oracle.cnn_loss_grad(p.astype(np.float64), x, np.zeros((len(seg), S, 2)), grad=False)
        ref = out[..., 0] + 1j * out[..., 1]
        got = np.stack([soft[k - s0: k - s0 + S] for k in ks])
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < tol, rel
    finally:
        rx.rx_cnn_destroy(c)


def test_cnn_receiver_small_calls_and_ragged_tiles():
    """Calls of 32512 samples (127 windows of 64 symbols: far fewer 128-symbol tiles per
    call than the receiver kernel has tile groups, so most groups get none, and an odd
    window count leaves a half-filled last tile; 64-symbol equaliser blocks keep every
    window in the payload): every call's soft outputs
    against the FP64 oracle's forward pass on segments across the call, and the bits of
    one batch call equal to those of the calls made one at a time."""
    nb, ncall = 127 * 256, 6
    small = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024, eq_block=64)
    g = synth.gen_kk_stream(4, nb, ncall, seed=26, truth=False, **VOLT)
    p = cnn.init_params(15).astype(np.float32)
    p += np.random.default_rng(16).standard_normal(len(p)).astype(np.float32) * 0.02
    c = rx.rx_cnn_create(64)
    try:
        rx.rx_cnn_set_params(c, p)
        dev = [torch.from_numpy(b).cuda() for b in g["packed"]]
        r = rx.Receiver(4, nb, debug=1, **small)
        rx.rx_set_cnn(r.h, c)
        seq, checked, ragged = [], 0, 0
        for d in dev:
            bits, n = r.process(d)
            seq.append(bits.cpu().numpy().copy())
            soft, s0 = r.debug(rx.RX_DBG_SOFT)
            y, y0 = r.debug(rx.RX_DBG_MF)
            if len(soft) < 3 * S:
                continue
            ragged += (len(soft) // S) % 2
            # payload symbols only: the first call's view starts with the training
            # symbols, which the adaptive filter decides before the network takes over
            ks = [k for k in range(max(s0, small["ntrain"]), s0 + len(soft) - S + 1, 5 * S)
                  if 2 * k - 12 - y0 >= 0 and 2 * k - 12 - y0 + L0 <= len(y)]
            if not ks:
                continue
            seg = [2 * k - 12 - y0 for k in ks]
            yv = y.astype(np.complex128)
            x = np.stack([np.stack([yv[s:s + L0].real, yv[s:s + L0].imag], axis=1) for s in seg])
            _, _, out = oracle.cnn_loss_grad(p.astype(np.float64), x, np.zeros((len(seg), S, 2)), grad=False)
            ref = out[..., 0] + 1j * out[..., 1]
            got = np.stack([soft[k - s0: k - s0 + S] for k in ks])
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 3e-2
            checked += len(ks)
        assert checked >= 20 and ragged >= 1, (checked, ragged)
        b = rx.Receiver(4, nb, **small)
        rx.rx_set_cnn(b.h, c)
        for (bits, n), ref in zip(b.process_batch(dev), seq):
            assert np.array_equal(bits.cpu().numpy(), ref)
    finally:
        rx.rx_cnn_destroy(c)
