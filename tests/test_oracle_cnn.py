"""Pins of the FP64 CNN equaliser oracle (forward and hand-written backward)."""

import math

import numpy as np
import pytest
from scipy.special import erf

import oracle


def gelu(u):
    return 0.5 * u * (1.0 + erf(u / math.sqrt(2.0)))


def random_params(rng, scale=1.0):
    p = np.zeros(oracle.cnn_nparams())
    for name, (off, shape) in oracle.cnn_param_slices().items():
        n = int(np.prod(shape))
        fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else 1
        if name.startswith(("W", "M")):
            p[off:off + n] = rng.standard_normal(n) * scale / math.sqrt(fan_in)
        else:
            p[off:off + n] = rng.standard_normal(n) * 0.1
    return p


def test_cnn_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    S, nseg = 3, 2
    p = random_params(rng)
    x = rng.standard_normal((nseg, 2 * S + 24, 2))
    t = rng.standard_normal((nseg, S, 2))
    loss, g, _ = oracle.cnn_loss_grad(p, x, t)
    sl = oracle.cnn_param_slices()
    idx = []
    for name, (off, shape) in sl.items():   # a few entries of every tensor
        n = int(np.prod(shape))
        idx += list(off + rng.choice(n, size=min(n, 12), replace=False))
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.cnn_loss_grad(pp, x, t, grad=False)[0] - oracle.cnn_loss_grad(pm, x, t, grad=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), abs(g[i]), 1e-3), (i, fd, g[i])


def test_cnn_pass_through_is_four_gelus_of_the_centre_sample():
    """Centre-tap pass-through weights: output = GELU^4 of the symbol's own
    2-sps sample (three conv layers and the MLP hidden layer), which fixes the
    layer alignment (symbol j reads input 2j + 12) and the exact GELU."""
    S, nseg = 5, 1
    p = np.zeros(oracle.cnn_nparams())
    sl = oracle.cnn_param_slices()
    for name, cin in (("W1", 2), ("W2", 32), ("W3", 32)):
        off = sl[name][0]
        W = p[off:off + 32 * 9 * cin].reshape(32, 9, cin)
        W[0, 4, 0] = 1.0
        W[1, 4, 1] = 1.0
    M1 = p[sl["M1"][0]:sl["M1"][0] + 64 * 32].reshape(64, 32)
    M1[0, 0] = M1[1, 1] = 1.0
    M2 = p[sl["M2"][0]:sl["M2"][0] + 2 * 64].reshape(2, 64)
    M2[0, 0] = M2[1, 1] = 1.0
    rng = np.random.default_rng(2)
    x = rng.standard_normal((nseg, 2 * S + 24, 2))
    t = np.zeros((nseg, S, 2))
    _, _, out = oracle.cnn_loss_grad(p, x, t, grad=False)
    for j in range(S):
        ref = gelu(gelu(gelu(gelu(x[0, 2 * j + 12]))))
        assert np.max(np.abs(out[0, j] - ref)) < 1e-14


def test_cnn_loss_is_mean_squared_error():
    rng = np.random.default_rng(3)
    p = random_params(rng)
    x = rng.standard_normal((3, 2 * 4 + 24, 2))
    t = rng.standard_normal((3, 4, 2))
    loss, _, out = oracle.cnn_loss_grad(p, x, t)
    assert abs(loss - np.mean(np.sum((out - t) ** 2, axis=2))) < 1e-12


def test_linear_network_reaches_the_least_squares_equaliser():
    """A network made linear: biases of +20 put every GELU where it is the identity
    to double precision (Phi(17) = 1 - 1e-64), layer 1 copies the 9 input samples
    of its window into channels 0..17 and layers 2, 3 and the first MLP layer pass
    them on (centre tap / identity).  The output layer then sees, per symbol, the 9
    2-sps samples around the symbol centre plus 20 and fits them linearly: the
    oracle's MSE at the least-squares solution of that linear model (numpy lstsq,
    the Wiener equaliser of the channel) equals the LS residual, its gradient there
    vanishes, and one Newton step from zero built from the oracle's gradient lands
    on the LS solution.  Symbols pass through a known T/2-spaced ISI channel with
    a little noise."""
    rng = np.random.default_rng(7)
    S, nseg, C, K, H = 16, 12, oracle.CNN_C, oracle.CNN_K, oracle.CNN_H
    L0 = 2 * S + 24
    ch = np.array([0.15, 0.45, 1.0, 0.35, -0.1])   # T/2-spaced channel, peak at offset 2
    x = np.zeros((nseg, L0, 2))
    tgt = np.zeros((nseg, S, 2))
    for s in range(nseg):
        nsym = L0 // 2 + 4
        a = (rng.choice([-1.0, 1.0], nsym) + 1j * rng.choice([-1.0, 1.0], nsym)) / math.sqrt(2)
        up = np.zeros(2 * nsym, complex)
        up[::2] = a
        sig = np.convolve(up, ch)[2:2 + 2 * nsym]            # symbol k centred at sample 2k
        sig = sig + 0.05 * (rng.standard_normal(len(sig)) + 1j * rng.standard_normal(len(sig)))
        seg = sig[:L0]
        x[s, :, 0], x[s, :, 1] = seg.real, seg.imag
        # symbol j of the segment sits at input position 2j + 12 (symbol index j + 6)
        tgt[s, :, 0], tgt[s, :, 1] = a[6:6 + S].real, a[6:6 + S].imag
    sl = oracle.cnn_param_slices()
    p = np.zeros(oracle.cnn_nparams())

    def view(name):
        off, shape = sl[name]
        return p[off:off + int(np.prod(shape))].reshape(shape)

    W1, b1, W2, b2, W3, b3, M1, c1 = (view(n) for n in ("W1", "b1", "W2", "b2", "W3", "b3", "M1", "c1"))
    for t in range(K):
        for ri in range(2):
            W1[2 * t + ri, t, ri] = 1.0
    b1[:18] = 20.0
    for c in range(18):
        W2[c, K // 2, c] = 1.0
        W3[c, K // 2, c] = 1.0
        M1[c, c] = 1.0
    # features of symbol j: x[2j + 8 + t] + 20 (t = 0..8) in channel 2t + ri, and 1 for c2
    F = np.zeros((nseg * S, 19))
    for s in range(nseg):
        for j in range(S):
            F[s * S + j, :18] = x[s, 2 * j + 8:2 * j + 17, :].reshape(-1) + 20.0
    F[:, 18] = 1.0
    T = tgt.reshape(-1, 2)
    sol, res, rank, _ = np.linalg.lstsq(F, T, rcond=None)
    assert rank == 19

    def set_out(M):
        off, _ = sl["M2"]
        m2 = np.zeros((2, H))
        m2[:, :18] = M[:18].T
        p[off:off + 2 * H] = m2.reshape(-1)
        p[sl["c2"][0]:sl["c2"][0] + 2] = M[18]

    def grad_out(g):
        m2 = g[sl["M2"][0]:sl["M2"][0] + 2 * H].reshape(2, H)
        assert np.all(m2[:, 18:] == 0.0)
        return np.vstack([m2[:, :18].T, g[sl["c2"][0]:sl["c2"][0] + 2][None, :]])

    set_out(sol)
    loss, g, _ = oracle.cnn_loss_grad(p, x, tgt)
    n = nseg * S
    assert abs(loss - res.sum() / n) <= 1e-9 * max(res.sum() / n, 1e-12)
    assert np.max(np.abs(grad_out(g))) <= 1e-9
    # Newton from zero: the MSE is quadratic in the output layer, Hessian 2/n F^T F
    set_out(np.zeros((19, 2)))
    _, g0, _ = oracle.cnn_loss_grad(p, x, tgt)
    step = np.linalg.solve(2.0 / n * F.T @ F, grad_out(g0))
    assert np.max(np.abs(-step - sol)) <= 1e-7 * np.max(np.abs(sol))
    # the Wiener equaliser beats no equaliser on this channel
    raw = ((x[:, 12:12 + 2 * S:2, 0] + 1j * x[:, 12:12 + 2 * S:2, 1]) / 1.0).reshape(-1)
    assert res.sum() / n < 0.5 * np.mean(np.abs(raw - (T[:, 0] + 1j * T[:, 1])) ** 2)
