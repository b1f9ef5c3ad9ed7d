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
