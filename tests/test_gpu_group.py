"""Groups of independent streams (mixed formats and buffer lengths) processed
per round on worker streams, directly or as an updated CUDA graph: the same bits,
bit counts and counters as each stream on its own; the autotuner's choices are
valid and reproduce with the same configuration on a single handle."""

import numpy as np
import pytest
import torch

from parity_util import make_stream
import paper_2010_14333_gb300 as rx

pytestmark = pytest.mark.gpu

# (format, buffer length, seed): KK-16QAM, KK-QPSK, PAM-2/4/8, two lengths
MEMBERS = [(4, 1 << 18, 51), (3, 1 << 19, 52), (1, 1 << 18, 53), (0, 1 << 19, 54), (2, 1 << 18, 55),
           (4, 1 << 19, 56)]
ROUNDS = 4
COUNTERS = ("calls", "samples", "symbols", "bits", "bit_errors", "raw_bit_errors", "sym_errors", "slip_windows",
            "near_threshold", "ambiguous_windows", "windows", "amb_rot", "device_error")


@pytest.fixture(scope="module")
def streams():
    return [make_stream(f, nb, ROUNDS, seed=s)["packed"] for f, nb, s in MEMBERS]


def individual(streams, cfgs=None):
    out, stats = [], []
    for m, (f, nb, _) in enumerate(MEMBERS):
        r = rx.Receiver(f, nb, **(cfgs[m] if cfgs else {}))
        bits = []
        for p in streams[m]:
            b, n = r.process(torch.from_numpy(p).cuda())
            bits.append((b.cpu().numpy().copy(), n))
        out.append(bits)
        stats.append(r.stats())
    return out, stats


def grouped(streams, flags):
    recv = [rx.Receiver(f, nb) for f, nb, _ in MEMBERS]
    g = rx.rx_group_create([r.h for r in recv], flags)
    try:
        st = torch.cuda.Stream()
        dev = [[torch.from_numpy(p).cuda() for p in s] for s in streams]
        outs = [torch.zeros(r.max_bits // 8 + 16, dtype=torch.uint8, device="cuda") for r in recv]
        res = [[] for _ in MEMBERS]
        torch.cuda.synchronize()
        for k in range(ROUNDS):
            with torch.cuda.stream(st):
                ns = rx.rx_group_process(g, [dev[m][k].data_ptr() for m in range(len(MEMBERS))],
                                         [o.data_ptr() for o in outs], st.cuda_stream)
            st.synchronize()
            for m, n in enumerate(ns):
                res[m].append((outs[m][: (n + 7) // 8].cpu().numpy().copy(), n))
        tuning = [rx.rx_group_tuning(g, m) for m in range(len(MEMBERS))]
    finally:
        rx.rx_group_destroy(g)
    stats = [r.stats() for r in recv]
    return res, stats, tuning


def same(a, sa, b, sb):
    for m in range(len(MEMBERS)):
        for k in range(ROUNDS):
            assert a[m][k][1] == b[m][k][1], (m, k)
            assert np.array_equal(a[m][k][0], b[m][k][0]), (m, k)
        for c in COUNTERS:
            assert sa[m][c] == sb[m][c], (m, c)


@pytest.mark.parametrize("flags", [0, rx.RX_GROUP_GRAPH])
def test_group_equals_individual_streams(streams, flags):
    ref, sref = individual(streams)
    assert all(s["bits"] > 0 for s in sref)
    got, sgot, _ = grouped(streams, flags)
    same(got, sgot, ref, sref)


def test_group_tuning_is_valid_and_reproducible(streams):
    got, sgot, tuning = grouped(streams, rx.RX_GROUP_GRAPH | rx.RX_GROUP_TUNE)
    for (f, nb, _), (front, warps) in zip(MEMBERS, tuning):
        assert front in (0, 1) and warps in (2, 4, 8)
        if f < 3:
            assert front == 0                      # no KK front end to choose
    ref, sref = individual(streams, [dict(kk_front=fr, eq_warps=w) for fr, w in tuning])
    same(got, sgot, ref, sref)
