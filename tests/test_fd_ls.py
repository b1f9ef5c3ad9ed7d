"""Static frequency-domain filter taps from a least-squares fit (Sec. 2: the static
FD equalisers' taps come from the link; the paper does not publish its lab taps).

- rx_fd_ls_taps (host code of the library, no device) recovers a filter exactly
  when the targets are that filter's output, for real and complex data and one,
  two or four input samples per target; it equals numpy's least-squares solution
  on noisy targets, and its ridge term is the stated one.
- The oracle's orx_set_fd_taps with the RRC taps reproduces its default filter
  bit for bit, and an LS fit on a PAM-4 capture through the ISI channel of the
  PAM workload equalises the filter output better than the RRC taps do."""

import numpy as np
import pytest

import oracle
import synth
import paper_2010_14333_gb300 as rx


def data_matrix(x, first, step, na, n):
    L = (n - 1) // 2
    k = np.arange(na)[:, None]
    c = np.arange(n)[None, :]
    return x[first + step * k - c + L]


@pytest.mark.parametrize("step", [1, 2, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_ls_recovers_a_known_filter(step, cplx):
    rng = np.random.default_rng(10 * step + cplx)
    n, na = 21, 3000
    L = (n - 1) // 2
    nx = step * na + 2 * n + 8
    x = rng.standard_normal(nx) + (1j * rng.standard_normal(nx) if cplx else 0.0)
    g = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0.0)
    first = L + 3
    # a_k = sum_i g_i x[first + step k - i], taps i = -L .. L at index i + L
    a = sum(g[i + L] * x[first + step * np.arange(na) - i] for i in range(-L, L + 1))
    h = rx.rx_fd_ls_taps(x, first, step, a, n)
    assert np.iscomplexobj(h) == cplx
    assert np.max(np.abs(h - g)) < 1e-9 * np.max(np.abs(g))


@pytest.mark.parametrize("cplx", [False, True])
def test_ls_equals_numpy_lstsq(cplx):
    rng = np.random.default_rng(7 + cplx)
    n, na, step, first = 31, 4000, 2, 40
    nx = first + step * na + n
    x = rng.standard_normal(nx) + (1j * rng.standard_normal(nx) if cplx else 0.0)
    a = rng.standard_normal(na) + (1j * rng.standard_normal(na) if cplx else 0.0)
    h = rx.rx_fd_ls_taps(x, first, step, a, n)
    X = data_matrix(x, first, step, na, n)
    ref = np.linalg.lstsq(X, a, rcond=None)[0]
    assert np.max(np.abs(h - ref)) < 1e-9 * np.max(np.abs(ref))


def test_ls_ridge_term():
    rng = np.random.default_rng(3)
    n, na, step, first = 15, 500, 4, 20
    nx = first + step * na + n
    x = rng.standard_normal(nx) + 1j * rng.standard_normal(nx)
    a = rng.standard_normal(na) + 1j * rng.standard_normal(na)
    ridge = 0.05
    h = rx.rx_fd_ls_taps(x, first, step, a, n, ridge=ridge)
    X = data_matrix(x, first, step, na, n)
    R = X.conj().T @ X
    R += ridge * np.trace(R).real / n * np.eye(n)
    ref = np.linalg.solve(R, X.conj().T @ a)
    assert np.max(np.abs(h - ref)) < 1e-10 * np.max(np.abs(ref))
    assert np.linalg.norm(h) < np.linalg.norm(rx.rx_fd_ls_taps(x, first, step, a, n))


def test_ls_rejects_bad_arguments():
    x = np.random.default_rng(1).standard_normal(1000)
    a = np.ones(100)
    for args in [(x, 10, 2, a, 20),            # even tap count
                 (x, 5, 2, a, 21),             # first < L
                 (x, 850, 2, a, 21),           # last input past the end
                 (x, 10, 0, a, 21),            # step 0
                 (x, 10, 2, a[:10], 21),       # fewer targets than taps
                 (np.zeros(1000), 10, 2, a, 21)]:   # singular normal matrix
        with pytest.raises(rx.RxError):
            rx.rx_fd_ls_taps(*args)


@pytest.mark.parametrize("fmt", [1, 4])
def test_oracle_fd_taps_reproduce_the_default(fmt):
    """Setting the RRC taps the FD form starts with changes nothing (bit for bit)."""
    nb = 1 << 16 if fmt < 3 else 1 << 17
    kw = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024) if fmt >= 3 else {}
    g = synth.gen_pam_stream(fmt, nb, 2) if fmt < 3 else synth.gen_kk_stream(fmt, nb, 2)
    cfg = oracle.default_cfg(fmt, nb, mf_mode=1, **kw)
    a, b = oracle.Oracle(**cfg), oracle.Oracle(**cfg)
    taps = oracle.rrc_half(cfg["rrc_beta"], cfg["sps"], (cfg["fd_taps"] - 1) // 2)
    b.set_fd_taps(taps)
    for p in g["packed"]:
        ba, na = a.process(p)
        bb, nbb = b.process(p)
        assert na == nbb and np.array_equal(ba, bb)
        ya, _ = a.get(oracle.ORX_Y)
        yb, _ = b.get(oracle.ORX_Y)
        assert np.array_equal(ya, yb)


def test_oracle_fd_taps_rejected():
    o = oracle.Oracle(**oracle.default_cfg(1, 1 << 16, mf_mode=1))
    with pytest.raises(ValueError):
        o.set_fd_taps(np.ones(4))                        # even count
    with pytest.raises(ValueError):
        o.set_fd_taps(np.ones(5) * (1 + 0.5j))           # complex taps for PAM
    with pytest.raises(ValueError):
        o.set_fd_taps(np.ones(515))                      # longer than N/2 + 1
    t = oracle.Oracle(**oracle.default_cfg(1, 1 << 16))  # time-domain form
    with pytest.raises(ValueError):
        t.set_fd_taps(np.ones(5))


def pam_ls_taps(g, nb, ntaps=503, na=30000):
    """LS fit of the FD filter on the first buffer (numpy's least squares, so that the
    oracle's taps do not come from the library): normalised codes (the filter's
    input) against the transmitted levels at the symbol centres y[2k]."""
    codes = g["codes"][:nb].astype(np.float64)
    x = (codes - codes.mean()) / codes.std()
    L = (ntaps - 1) // 2
    k0 = L // 2 + 1
    na = min(na, (nb - 1 - L - 2 * k0) // 2 + 1)
    X = data_matrix(x, 2 * k0, 2, na, ntaps)
    return np.linalg.lstsq(X, g["symbols"][k0:k0 + na], rcond=None)[0]


@pytest.mark.parametrize("snr", [18.0, 14.0])
def test_oracle_pam_ls_taps_equalise_the_isi_channel(snr):
    """PAM-4 through ISI (0.1, 1, 0.2): on a held-out buffer the LS filter's output at
    the symbol centres is within a quarter of the RRC output's error of the
    transmitted levels (the RRC output scaled by its best gain) at 18 dB, and within
    a half at 14 dB.  The 15-tap LMS after the filter equalises the RRC chain's ISI
    too, so the two chains' BER agree: within 15 % (plus three standard deviations)."""
    nb, fmt = 1 << 17, 1
    g = synth.gen_pam_stream(fmt, nb, 3, seed=5, snr_db=snr)
    h = pam_ls_taps(g, nb)
    cfg = oracle.default_cfg(fmt, nb, mf_mode=1)
    o_rrc, o_ls = oracle.Oracle(**cfg), oracle.Oracle(**cfg)
    o_ls.set_fd_taps(h)
    mse = {}
    for name, o in (("rrc", o_rrc), ("ls", o_ls)):
        for p in g["packed"]:
            o.process(p)
        y, y0 = o.get(oracle.ORX_Y)
        y = y.real
        m = np.arange(y0 + (y0 & 1), y0 + len(y) - 1, 2)
        m = m[(m >= 2 * nb) & (m < 3 * nb - 600)]            # symbol centres of the third buffer
        ys, a = y[m - y0], g["symbols"][m // 2]
        gain = (ys @ a) / (ys @ ys)
        mse[name] = np.mean((a - gain * ys) ** 2) / np.mean(a ** 2)
        mse[name + "_nogain"] = np.mean((a - ys) ** 2) / np.mean(a ** 2)
        mse[name + "_errors"] = o.stats()["bit_errors"]
    assert mse["ls_nogain"] < (0.25 if snr >= 18 else 0.5) * mse["rrc"], mse
    assert mse["ls_errors"] <= 1.15 * mse["rrc_errors"] + 3 * np.sqrt(mse["rrc_errors"] + 1), mse


def test_oracle_fd_taps_complex_rotation_and_delay():
    """KK form: taps multiplied by e^{j phi} turn the 2-sps output by e^{j phi} (not
    e^{-j phi}: no conjugate), and taps delayed by two input samples delay it by one
    output sample (index order of the taps)."""
    fmt, nb = 4, 1 << 16
    kw = dict(ols_n=4096, ols_v=512, ntrain=4096, ncma=2048, amb_syms=1024, mf_mode=1)
    g = synth.gen_kk_stream(fmt, nb, 1)
    cfg = oracle.default_cfg(fmt, nb, **kw)
    rrc = oracle.rrc_half(cfg["rrc_beta"], cfg["sps"], (cfg["fd_taps"] - 1) // 2)
    phi = 0.7
    outs = {}
    for name, taps in (("def", None), ("rot", rrc * np.exp(1j * phi)),
                       ("del", np.concatenate([np.zeros(4), rrc]).astype(complex))):
        o = oracle.Oracle(**cfg)
        if taps is not None:
            o.set_fd_taps(taps)
        o.process(g["packed"][0])
        outs[name] = o.get(oracle.ORX_Y)
    (yd, d0), (yr, r0), (yl, l0) = outs["def"], outs["rot"], outs["del"]
    assert d0 == r0 == l0
    assert np.max(np.abs(yr - yd * np.exp(1j * phi))) < 1e-12 * np.max(np.abs(yd))
    # the 207 delayed taps h_i = rrc_{i-2}: y_del[m] = y[m - 1] away from the stream
    # start, within each block's 256 outputs (the first output of a block and the last
    # of the one before come from different blocks, whose bin truncation differs)
    m = np.arange(d0 + 200, d0 + len(yd))
    m = m[m % 256 != 0]
    assert np.max(np.abs(yl[m - l0] - yd[m - 1 - d0])) < 1e-9 * np.max(np.abs(yd))
