"""bench.py's roofline arithmetic on the host (no GPU): algorithmic flops of
the dominant family per launch (Theorem 4's count for the asymmetric
assembly) and the DRAM-traffic entry, which stands only for the sources it
was captured from."""
from types import SimpleNamespace

import numpy as np
import pytest

import bench


def _side(lengths):
    indptr = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=indptr[1:])
    return SimpleNamespace(indptr=indptr)


P = SimpleNamespace(train_rows=_side([10, 40, 100, 2000]), train_cols=_side([33, 1024, 1025, 5]))


def _flops(lengths, lo, hi, f, r):
    tot = 0.0
    for n in lengths:
        if lo < n <= hi:
            s = np.floor(n * r)
            tot += 2 * s * f * f + 2 * s * f
    return tot


def test_cta_rows_flops_per_launch():
    f, r, launches = 32, 0.25, 12
    roof = bench.roofline("cta_rows", 1e-4, P, f, r, launches)
    # Resident rows are 32 < n <= 1024 on both sides: 40, 100 | 33, 1024.
    want = (_flops([10, 40, 100, 2000], 32, 1024, f, r) + _flops([33, 1024, 1025, 5], 32, 1024, f, r)) / launches
    assert roof["algorithmic_flops_per_launch"] == pytest.approx(want)
    assert roof["achieved"] == pytest.approx(want / 1e-4 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / bench.FP32_ALU_PEAK_TFLOPS)
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"


def test_split_family_counts_only_split_rows():
    f, r = 32, 0.25
    roof = bench.roofline("split_gram", 1e-3, P, f, r, 2)
    want = (_flops([2000], 1024, 1 << 40, f, r) + _flops([1025], 1024, 1 << 40, f, r)) / 2
    assert roof["algorithmic_flops_per_launch"] == pytest.approx(want)


def test_traffic_only_for_matching_sources(monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC", {"kernel": "cta_rows", "bytes_per_sweep": 1200.0,
                                           "sources_sha256_16": bench.kernel_sources_hash()})
    assert bench.roofline("cta_rows", 1e-4, P, 32, 0.25, 12)["traffic"] == pytest.approx(100.0)
    monkeypatch.setattr(bench, "TRAFFIC", {"kernel": "cta_rows", "bytes_per_sweep": 1200.0,
                                           "sources_sha256_16": "0000000000000000"})
    assert bench.roofline("cta_rows", 1e-4, P, 32, 0.25, 12)["traffic"] is None

