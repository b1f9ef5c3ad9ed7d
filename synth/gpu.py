"""Seeded Kramers-Kronig QAM stream generated on the GPU (torch), for long runs.

The recipe is that of ``synth.kk_buffer`` (see the module docstring of
``synth``): PRBS-15 bits, Gray QAM at unit power, root-raised-cosine pulse at
``sps`` samples/symbol, up-shift by fd_num/fd_den cycles per sample, Wiener
phase noise of the given linewidth relative to a real tone at CSPR times the
signal power, complex AWGN of per-sample variance P_s sps / SNR, photodiode
|E|^2 and the 12-bit ADC (full scale mean + 4 std per buffer), packed two
samples per three bytes (little-endian 24-bit word).  Only the random numbers
differ (torch's generator instead of numpy's), so a stream of thousands of
buffers (the 6-second Q time series, 5720 buffers of 2^22 samples) takes seconds
instead of the CPU generator's minutes.  Like ``synth`` it holds none of the
receiver's arithmetic.
"""

from __future__ import annotations

import math

import numpy as np

from . import FORMATS, prbs15_bits, rrc_pulse, tx_levels


class KKStreamGPU:
    """Consecutive buffers of one continuous KK stream: ``next()`` returns the packed
    uint8 CUDA tensor of the next buffer (buf_len * 3 / 2 bytes)."""

    def __init__(self, fmt: int = 4, buf_len: int = 1 << 22, seed: int = 1, snr_db: float = 20.0,
                 cspr_db: float = 10.0, linewidth: float = 100e3, fs: float = 4e9, sps: int = 4,
                 beta: float = 0.1, span: int = 16, fd_num: int = 11, fd_den: int = 80, prbs_seed: int = 1,
                 device: str = "cuda"):
        import torch
        name, bps, kind = FORMATS[fmt]
        assert kind == "qam" and buf_len % 2 == 0
        self.t = torch
        self.dev = torch.device(device)
        self.buf_len, self.sps, self.half = buf_len, sps, sps * span // 2
        # the symbol sequence repeats with the PRBS period (gcd(bps, 32767) = 1)
        per = prbs15_bits(prbs_seed, 32767)
        idx = (np.arange(32767, dtype=np.int64)[:, None] * bps + np.arange(bps)[None, :]) % 32767
        a = tx_levels(fmt, per[idx].reshape(-1))
        self.sym = torch.tensor(np.stack([a.real, a.imag], 1), dtype=torch.float32, device=self.dev)
        p = rrc_pulse(beta, sps, span)
        self.pulse = torch.tensor(p[::-1].copy(), dtype=torch.float32, device=self.dev).view(1, 1, -1)
        ps = 1.0 / sps                                   # per-sample power of the unit-power shaped signal
        self.A = math.sqrt(10.0 ** (cspr_db / 10.0) * ps)
        self.sig = math.sqrt(ps * sps / 10.0 ** (snr_db / 10.0) / 2.0)
        self.pn = math.sqrt(2.0 * math.pi * linewidth / fs)
        ang = 2.0 * math.pi * np.arange(fd_den) / fd_den
        self.up = torch.tensor(np.stack([np.cos(ang), np.sin(ang)], 1), dtype=torch.float32, device=self.dev)
        self.fd_num, self.fd_den = fd_num, fd_den
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(int(seed))
        self.theta = 0.0
        self.b = 0

    def next(self):
        t = self.t
        n0, n1 = self.b * self.buf_len, (self.b + 1) * self.buf_len
        sps, half = self.sps, self.half
        ka = (n0 - half) // sps - 1
        kb = (n1 + half) // sps + 2
        k = t.arange(ka, kb, device=self.dev, dtype=t.int64)
        a = self.sym[k.remainder(32767)]
        a[k < 0] = 0.0
        up = t.zeros((2, 1, sps * (kb - ka)), dtype=t.float32, device=self.dev)
        up[:, 0, ::sps] = a.t()
        # s[n] = sum_k a_k p[n - sps k]: output i of the correlation sits at n = sps ka + i + half
        s = t.nn.functional.conv1d(up, self.pulse).view(2, -1)
        off = n0 - sps * ka - half
        sr, si = s[0, off:off + self.buf_len], s[1, off:off + self.buf_len]
        n = t.arange(n0, n1, device=self.dev, dtype=t.int64)
        u = self.up[(n * self.fd_num).remainder(self.fd_den)]
        th = self.theta + t.cumsum(t.randn(self.buf_len, generator=self.gen, device=self.dev,
                                           dtype=t.float64) * self.pn, 0)
        self.theta = float(th[-1])
        c, sn = t.cos(th).float(), t.sin(th).float()
        # rotate the shaped signal by the up-shift, then by the phase noise
        xr = sr * u[:, 0] - si * u[:, 1]
        xi = sr * u[:, 1] + si * u[:, 0]
        er = self.A + xr * c - xi * sn
        ei = xr * sn + xi * c
        nz = t.randn((2, self.buf_len), generator=self.gen, device=self.dev, dtype=t.float32) * self.sig
        er, ei = er + nz[0], ei + nz[1]
        I = (er * er + ei * ei).double()
        i_fs = float(I.mean() + 4.0 * I.std(unbiased=False))
        q = t.floor(I / i_fs * 4095.0 + 0.5).clamp_(0, 4095).to(t.int32).view(-1, 2)
        s0, s1 = q[:, 0], q[:, 1]
        out = t.empty((q.shape[0], 3), dtype=t.uint8, device=self.dev)
        out[:, 0] = (s0 & 0xFF).to(t.uint8)
        out[:, 1] = (((s0 >> 8) & 0x0F) | ((s1 & 0x0F) << 4)).to(t.uint8)
        out[:, 2] = ((s1 >> 4) & 0xFF).to(t.uint8)
        self.b += 1
        return out.view(-1)
