"""Equaliser forms against the FP64 oracle.

- The tensor-core block-Toeplitz FIR (tcgen05, BF16 / FP16 / FP8-E4M3 operands,
  FP32 accumulation) equals the FP64 convolution of the operands rounded to its
  precision, up to FP32 accumulation: this pins the operand layouts, the
  descriptors and the FP8 scaling exactly, and bounds each precision's error.
- The frozen-tap receiver in FP32 matches the oracle's frozen form under the
  parity rules of the adaptive form.
- The tensor-core receivers stay within each precision's soft-symbol error of
  the oracle and reach its BER."""

import numpy as np
import pytest
import torch

from parity_util import Pair, make_stream, rel_rms
import oracle
import paper_2010_14333_gb300 as rx

pytestmark = pytest.mark.gpu

PRECS = {"bf16": rx.RX_FIR_BF16, "fp16": rx.RX_FIR_FP16, "fp8": rx.RX_FIR_FP8}


def round_bf16(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_e4m3(x):
    """Round to nearest even on the E4M3 grid (3 mantissa bits, minimum normal
    2^-6, subnormal step 2^-9), saturating at 448."""
    v = np.clip(np.asarray(x, np.float64), -448.0, 448.0)
    a = np.abs(v)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -6)))
    step = 2.0 ** (e - 3)
    return np.clip(np.round(v / step) * step, -448.0, 448.0)


def fp8_exp(m):
    if not m > 0:
        return 0
    _, e = np.frexp(np.float32(448.0) / np.float32(m))
    return int(min(max(e - 1, -60), 60))


def emulate(y, w, prec, nsym, sblk):
    """FP64 convolution of the operands the tensor core sees (y, w already FP32)."""
    nt = len(w)
    k = np.arange(nsym)
    if prec == rx.RX_FIR_FP8:
        q8 = lambda v, e: (round_e4m3(v.real * 2.0 ** e) + 1j * round_e4m3(v.imag * 2.0 ** e)) / 2.0 ** e
        eB = fp8_exp(max(np.abs(w.real).max(), np.abs(w.imag).max()))
        wq = q8(w, eB)
        ns = 30 + nt
        z = np.zeros(nsym, complex)
        for b in range(nsym // sblk):
            # a block's rows read [2 sblk b, 2 sblk (b+1) - 32 + ns); each block rounds
            # its inputs with its own scale (halo samples included)
            lo, hi = 2 * sblk * b, 2 * sblk * (b + 1) - 32 + ns
            seg = y[lo:hi]
            yq = np.zeros(len(y), complex)
            yq[lo:hi] = q8(seg, fp8_exp(max(np.abs(seg.real).max(), np.abs(seg.imag).max())))
            kb = k[b * sblk:(b + 1) * sblk]
            for i in range(nt):
                z[kb] += np.conj(wq[i]) * yq[2 * kb + nt - 1 - i]
        return z
    r = round_bf16 if prec == rx.RX_FIR_BF16 else (lambda v: np.asarray(v, np.float32).astype(np.float16).astype(np.float64))
    wq = r(w.real) + 1j * r(w.imag)
    yq = r(y.real) + 1j * r(y.imag)
    z = np.zeros(nsym, complex)
    for i in range(nt):
        z += np.conj(wq[i]) * yq[2 * k + nt - 1 - i]
    return z


def gpu_fir(y, w, prec, nsym, sblk):
    yd = torch.from_numpy(np.stack([y.real, y.imag], 1).astype(np.float32).ravel()).cuda()
    wd = torch.from_numpy(np.stack([w.real, w.imag], 1).astype(np.float32).ravel()).cuda()
    zd = torch.zeros(2 * nsym, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rx.rx_fir_block(yd.data_ptr(), len(y), wd.data_ptr(), len(w), prec, nsym, sblk, zd.data_ptr(), st.data_ptr(),
                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    z = zd.cpu().numpy().astype(np.float64)
    return z[0::2] + 1j * z[1::2]


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("nt,nsym,sblk", [(31, 16 * 130, 16), (31, 1 << 14, 1024), (7, 2048 + 256, 256),
                                          (31, 1 << 16, 256), (31, 1 << 15, 2048)])
def test_fir_block_equals_rounded_operands(prec, nt, nsym, sblk):
    """Ragged last tile (130 rows), short filters, scale blocks 16..2048 symbols."""
    rng = np.random.default_rng(nt + nsym)
    ny = 2 * nsym + nt + 1
    y = (rng.standard_normal(ny) + 1j * rng.standard_normal(ny)) * 0.7
    y[ny // 3: ny // 3 + 500] *= 20.0                  # a loud stretch: per-block FP8 scales differ
    w = (rng.standard_normal(nt) + 1j * rng.standard_normal(nt)) * 0.05
    w[nt // 2] += 1.0
    y = y.astype(np.complex64).astype(complex)         # what the device holds
    w = w.astype(np.complex64).astype(complex)
    z = gpu_fir(y, w, PRECS[prec], nsym, sblk)
    ze = emulate(y, w, PRECS[prec], nsym, sblk)
    # exact operands, FP32 accumulation of <= 62 products
    assert np.max(np.abs(z - ze)) <= 2e-5 * np.max(np.abs(ze)), np.max(np.abs(z - ze))
    k = np.arange(nsym)
    zt = sum(np.conj(w[i]) * y[2 * k + nt - 1 - i] for i in range(nt))
    bound = {"bf16": 8e-3, "fp16": 1e-3, "fp8": 8e-2}[prec]
    assert rel_rms(z, zt) < bound, rel_rms(z, zt)


SMALL = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024, eq_block=1024)


def test_frozen_fp32_parity():
    nb = 1 << 18
    g = make_stream(4, nb, 4, seed=41)
    p = Pair(4, nb, fir_prec=rx.RX_FIR_FROZEN_F32, **SMALL)
    for b in range(4):
        p.feed(g["packed"][b])
    s, so = p.compare_stats()
    assert s["bits"] > 0


@pytest.mark.parametrize("prec", list(PRECS))
def test_tensor_forms_against_oracle(prec):
    nb = 1 << 20
    g = make_stream(4, nb, 3, seed=42, workers=4)
    o = oracle.Oracle(**oracle.default_cfg(4, nb, eq_frozen=1, eq_block=1024))
    r = rx.Receiver(4, nb, fir_prec=PRECS[prec], eq_block=1024, debug=1)
    errs = []
    for b in range(3):
        o.process(g["packed"][b])
        r.process(torch.from_numpy(g["packed"][b]).cuda())
        z, z0 = r.debug(rx.RX_DBG_SOFT)
        zo, zo0 = o.get(oracle.ORX_Z)
        if len(z):
            zo = zo[z0 - zo0: z0 - zo0 + len(z)]
            errs.append(rel_rms(z, zo))
    s, so = r.stats(), o.stats()
    assert s["bits"] == so["bits"] > 0 and s["device_error"] == 0
    bound = {"bf16": 1e-2, "fp16": 2e-3, "fp8": 8e-2}[prec]
    assert max(errs) < bound, errs
    ber_bound = {"bf16": 1.1, "fp16": 1.05, "fp8": 2.0}[prec]
    assert s["ber"] <= so["ber"] * ber_bound + 2e-4, (s["ber"], so["ber"])
