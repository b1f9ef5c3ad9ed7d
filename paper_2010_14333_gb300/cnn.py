"""Training loop of the learned equaliser (argument marshalling only).

The gradient, the loss and the Adam update run in librx.so's kernels
(rx_cnn_grad, rx_cnn_adam_step); this module picks training segments and hands
device pointers over.  Training inputs are the receiver's own 2-sps
matched-filter output (RX_DBG_MF) of a stream whose transmitted symbols are
known; targets are those symbols in unit-power units.
"""

from __future__ import annotations

import math

import numpy as np

from . import (RX_DBG_MF, Receiver, rx_cnn_adam_step, rx_cnn_create, rx_cnn_destroy, rx_cnn_get_params,
               rx_cnn_grad, rx_cnn_nparams, rx_cnn_set_params)

SEG = 64          # symbols per segment
CTX = 12          # 2-sps samples of context on each side


def init_params(seed: int = 0) -> np.ndarray:
    """Fan-in scaled normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    C, K, H = 32, 9, 64
    parts = [rng.standard_normal(C * K * 2) * math.sqrt(2.0 / (K * 2)), np.zeros(C),
             rng.standard_normal(C * K * C) * math.sqrt(2.0 / (K * C)), np.zeros(C),
             rng.standard_normal(C * K * C) * math.sqrt(2.0 / (K * C)), np.zeros(C),
             rng.standard_normal(H * C) * math.sqrt(2.0 / C), np.zeros(H),
             rng.standard_normal(2 * H) * math.sqrt(1.0 / H), np.zeros(2)]
    p = np.concatenate(parts).astype(np.float32)
    assert len(p) == rx_cnn_nparams()
    return p


def mf_output(packed_buffers, buf_len: int, fmt: int = 4, **cfg):
    """Run the receiver over the buffers and return its whole 2-sps MF output
    (complex64, index = 2-sps stream index) on the host."""
    r = Receiver(fmt, buf_len, debug=1, **cfg)
    import torch
    parts = []
    for p in packed_buffers:
        r.process(torch.from_numpy(np.ascontiguousarray(p)).cuda())
        y, y0 = r.debug(RX_DBG_MF)
        parts.append((y0, y))
    n = parts[-1][0] + len(parts[-1][1])
    out = np.zeros(n, dtype=np.complex64)
    for y0, y in parts:
        out[y0:y0 + len(y)] = y
    return out


class CnnTrainer:
    """FP32 master weights and Adam on the GPU; batches of `batch` segments."""

    def __init__(self, batch: int = 64, seed: int = 0, params: np.ndarray | None = None):
        import torch
        self.torch = torch
        self.batch = batch
        self.h = rx_cnn_create(batch)
        rx_cnn_set_params(self.h, init_params(seed) if params is None else params)
        self.rng = np.random.default_rng(seed + 1)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            rx_cnn_destroy(h)
            self.h = None

    def set_data(self, y: np.ndarray, symbols: np.ndarray, k_lo: int = 0):
        """y: 2-sps MF output (complex); symbols: transmitted symbols (unit power)."""
        t = self.torch
        self.y = t.from_numpy(np.ascontiguousarray(y, dtype=np.complex64)).cuda()
        n_sym = min(len(symbols), (len(y) - CTX - 2 * SEG) // 2)
        self.sym = t.from_numpy(np.ascontiguousarray(symbols[:n_sym], dtype=np.complex64)).cuda()
        self.k_lo = max(k_lo, (CTX + 1) // 2)
        self.k_hi = n_sym - SEG

    def step(self, lr: float = 1e-3) -> None:
        t = self.torch
        k0 = self.rng.integers(self.k_lo, self.k_hi, size=self.batch)
        seg = t.from_numpy(2 * k0 - CTX).cuda()
        idx = t.from_numpy(k0[:, None] + np.arange(SEG)[None, :]).cuda()
        tgt = t.view_as_real(self.sym[idx]).contiguous()
        st = t.cuda.current_stream().cuda_stream
        yv = t.view_as_real(self.y)
        rx_cnn_grad(self.h, yv.data_ptr(), seg.data_ptr(), tgt.data_ptr(), self.batch, None,
                    self.loss.data_ptr(), st)
        rx_cnn_adam_step(self.h, lr, st)
        self._keep = (seg, tgt)

    def train(self, steps: int, lr: float = 1e-3, report: int = 0):
        hist = []
        for i in range(steps):
            self.step(lr)
            if report and (i + 1) % report == 0:
                hist.append(float(self.loss.item()))
        return hist

    def params(self) -> np.ndarray:
        return rx_cnn_get_params(self.h)
