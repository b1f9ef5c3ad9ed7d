"""C ABI checks that need no GPU: the library loads, exports every function
include/rx.h declares, and rejects bad arguments before touching the device."""

import ctypes as C
import os
import re

import pytest

import paper_2010_14333_gb300 as rx

HDR = os.path.join(os.path.dirname(__file__), "..", "include", "rx.h")


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rx_[a-z_]+)\s*\(", src)))


def test_header_functions_are_exported():
    lib = rx.load()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(rx.EXPORTED) == names


def test_binding_raises_without_library(tmp_path):
    saved = rx._lib
    rx._lib = None
    try:
        with pytest.raises(rx.RxError):
            rx.load(str(tmp_path / "missing.so"))
    finally:
        rx._lib = saved


def test_default_config_and_strerror():
    c = rx.rx_default_config(rx.RX_KK_16QAM)
    assert (c.ols_n, c.ols_v, c.ntaps, c.bps_b, c.win) == (65536, 4096, 31, 32, 64)
    assert (c.ds_num, c.ds_den) == (11, 80)
    p = rx.rx_default_config(rx.RX_PAM4)
    assert (p.ntaps, p.ntrain, p.mu) == (15, 4096, 1e-3)
    assert rx.rx_strerror(1).startswith("invalid")


@pytest.mark.parametrize("args", [
    (rx.RX_KK_16QAM, 1e9, 4e9, 1000),          # buf_len not a multiple of 32
    (rx.RX_KK_16QAM, 2e9, 4e9, 1 << 20),       # KK needs 4 samples/symbol
    (rx.RX_PAM4, 1e9, 4e9, 1 << 20),           # PAM needs 2 samples/symbol
    (7, 1e9, 4e9, 1 << 20),                    # unknown format
    (rx.RX_PAM4, 2e9, 4e9, (1 << 30) + 32),    # above 2^30 samples
])
def test_create_rejects_bad_arguments(args):
    lib = rx.load()
    h = C.c_void_p()
    st = lib.rx_create(args[0], args[1], args[2], args[3], None, C.byref(h))
    assert st == 1 and not h.value


@pytest.mark.parametrize("field,value", [("ntaps", 33), ("ntaps", 14), ("ols_n", 8192), ("ols_n", 256),
                                         ("ols_v", 96), ("win", 32),
                                         ("eq_block", 100), ("bps_b", 0), ("amb_syms", 100),
                                         ("ncma", 20000)])
def test_create_rejects_bad_config(field, value):
    lib = rx.load()
    c = rx.rx_default_config(rx.RX_KK_16QAM)
    setattr(c, field, value)
    h = C.c_void_p()
    assert lib.rx_create(rx.RX_KK_16QAM, 1e9, 4e9, 1 << 22, C.byref(c), C.byref(h)) == 1


@pytest.mark.parametrize("kw", [dict(mf_mode=2), dict(mf_mode=1, fd_n=2048), dict(mf_mode=1, fd_n=1000),
                                dict(mf_mode=1, fd_n=8), dict(mf_mode=1, fd_taps=202),
                                dict(mf_mode=1, fd_n=256, fd_taps=131)])
def test_create_rejects_bad_fd_config(kw):
    lib = rx.load()
    c = rx.rx_default_config(rx.RX_KK_16QAM)
    for k, v in kw.items():
        setattr(c, k, v)
    h = C.c_void_p()
    assert lib.rx_create(rx.RX_KK_16QAM, 1e9, 4e9, 1 << 22, C.byref(c), C.byref(h)) == 1
    p = rx.rx_default_config(rx.RX_PAM4)   # the PAM form runs 1024-point blocks only
    p.mf_mode, p.fd_n, p.fd_taps = 1, 512, 101
    assert lib.rx_create(rx.RX_PAM4, 2e9, 4e9, 1 << 20, C.byref(p), C.byref(h)) == 1
    p.fd_n, p.fd_taps = 1024, 515
    assert lib.rx_create(rx.RX_PAM4, 2e9, 4e9, 1 << 20, C.byref(p), C.byref(h)) == 1


def test_create_rejects_too_many_overlap_save_blocks():
    """A buffer of more overlap-save blocks than the forward pass's grid holds."""
    lib = rx.load()
    h = C.c_void_p()
    c = rx.rx_default_config(rx.RX_KK_16QAM)
    c.ols_n, c.ols_v = 4096, 4032            # hop of 64 samples: 2^24 / 64 blocks
    assert lib.rx_create(rx.RX_KK_16QAM, 1e9, 4e9, 1 << 24, C.byref(c), C.byref(h)) == 1


def test_create_rejects_bad_resampler():
    lib = rx.load()
    h = C.c_void_p()
    for step in (1 << 31, 2 << 32):
        c = rx.rx_default_config(rx.RX_KK_16QAM)
        c.rs_step = step
        assert lib.rx_create(rx.RX_KK_16QAM, 1e9, 4e9, 1 << 22, C.byref(c), C.byref(h)) == 1
    p = rx.rx_default_config(rx.RX_PAM4)   # the PAM resampler feeds the time-domain filter only
    p.rs_step = 1 << 32
    p.mf_mode = rx.RX_MF_FD
    assert lib.rx_create(rx.RX_PAM4, 2e9, 4e9, 1 << 20, C.byref(p), C.byref(h)) == 1


def test_fd_default_taps():
    assert rx.rx_default_config(rx.RX_KK_16QAM).fd_taps == 203
    assert rx.rx_default_config(rx.RX_PAM4).fd_taps == 503


def test_null_handle_calls_are_rejected():
    lib = rx.load()
    n = (C.c_int64 * 2)()
    ptrs = (C.c_void_p * 2)(16, 32)
    assert lib.rx_process(None, ptrs[0], ptrs[1], None, n) == 1
    assert lib.rx_process_batch(None, ptrs, ptrs, 2, None, n) == 1
    assert lib.rx_process_host_batch(None, ptrs, ptrs, 2, None, n) == 1
    assert lib.rx_process_host(None, ptrs[0], ptrs[1], None, n) == 1


@pytest.mark.parametrize("args", [
    (0, 1000, 16, 31, 2, 256, 256, 16, 16),         # null input
    (16, 1000, 16, 31, 1, 256, 256, 16, 16),        # FP32 is not a tensor-core precision
    (16, 1000, 16, 31, 2, 250, 256, 16, 16),        # nsym not a multiple of 16
    (16, 1000, 16, 30, 2, 256, 256, 16, 16),        # even tap count
    (16, 500, 16, 31, 2, 256, 256, 16, 16),         # input shorter than 2 nsym + ntaps + 1
    (16, 1000, 16, 31, 4, 256, 96, 16, 16),         # FP8 scale block must divide 2048
    (8, 1000, 16, 31, 2, 256, 256, 16, 16),         # input not 16-byte aligned
])
def test_fir_block_rejects_bad_arguments(args):
    y, ny, w, nt, prec, nsym, sblk, z, st = args
    assert rx.load().rx_fir_block(y, ny, w, nt, prec, nsym, sblk, z, st, None) == 1


def test_receiver_rejects_unknown_option_and_bad_precision():
    with pytest.raises(TypeError):
        rx.Receiver(4, 1 << 20, eq_frozen=1)
    lib = rx.load()
    h = C.c_void_p()
    c = rx.rx_default_config(rx.RX_PAM4)
    c.fir_prec = rx.RX_FIR_BF16                       # the tensor-core forms are KK only
    assert lib.rx_create(rx.RX_PAM4, 2e9, 4e9, 1 << 20, C.byref(c), C.byref(h)) == 1
    c = rx.rx_default_config(rx.RX_KK_16QAM)
    c.fir_prec = rx.RX_FIR_FP8
    c.eq_block = 192 * 16                             # 2048 % eq_block != 0
    assert lib.rx_create(rx.RX_KK_16QAM, 1e9, 4e9, 1 << 22, C.byref(c), C.byref(h)) == 1
    c.fir_prec = 5
    c.eq_block = 1024
    assert lib.rx_create(rx.RX_KK_16QAM, 1e9, 4e9, 1 << 22, C.byref(c), C.byref(h)) == 1


def test_group_rejects_bad_arguments():
    lib = rx.load()
    g = C.c_void_p()
    arr = (C.c_void_p * 2)(None, None)
    assert lib.rx_group_create(arr, 2, 0, C.byref(g)) == 1          # null members
    assert lib.rx_group_create(arr, 0, 0, C.byref(g)) == 1          # empty group
    assert lib.rx_group_create(None, 2, 0, C.byref(g)) == 1
    assert lib.rx_group_process(None, None, None, None, None) == 1
    f, w = C.c_int32(), C.c_int32()
    assert lib.rx_group_tuning(None, 0, C.byref(f), C.byref(w)) == 1
    assert lib.rx_group_destroy(None) == 1


@pytest.mark.parametrize("fmt,kw", [(rx.RX_KK_16QAM, dict(eq_mode=2)), (rx.RX_KK_16QAM, dict(eq_mode=-1)),
                                    (rx.RX_KK_16QAM, dict(eq_mode=1, ntaps=9)),
                                    (rx.RX_KK_16QAM, dict(eq_mode=1, ntaps=1)),
                                    (rx.RX_KK_16QAM, dict(eq_mode=1, ntaps=4, fir_prec=2, eq_block=1024)),
                                    (rx.RX_KK_16QAM, dict(eq_mode=0, ntaps=4)),
                                    (rx.RX_PAM4, dict(eq_mode=1, ntaps=4))])
def test_create_rejects_bad_equaliser_form(fmt, kw):
    """The symbol-by-symbol form: KK only, 2..8 taps, adaptive; even tap counts in it only."""
    lib = rx.load()
    c = rx.rx_default_config(fmt)
    for k, v in kw.items():
        setattr(c, k, v)
    h = C.c_void_p()
    baud, nb = (1e9, 1 << 22) if fmt >= 3 else (2e9, 1 << 20)
    assert lib.rx_create(fmt, baud, 4e9, nb, C.byref(c), C.byref(h)) == 1
