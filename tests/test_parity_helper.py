"""The parity comparison enforces the contract (CPU only): a fast-path or wedge value
that differs by a single ulp fails; a value through log (a tail) may differ by up
to 4 ulp; a stream may stop at a flip only where the oracle's margin is tiny."""

import numpy as np
import pytest

import oracle as O
from paper_2405_19493_gb300 import workloads as W
from tests.parity import compare_streams, offsets_of

SEEDS = W.seeds(8)
L = 20000


def _case():
    o, m, _, vl = O.generate("splitmix64", "zig128", SEEDS, uniform_len=L, with_margins=True,
                             with_via_log=True)
    Ls = np.full(len(SEEDS), L, dtype=np.uint64)
    return o, m, vl, offsets_of(Ls), Ls


def _bump(x, k, ulps):
    y = x.copy()
    y.view(np.int64)[k] += ulps
    return y


def test_identical_passes():
    o, m, vl, off, Ls = _case()
    rep = compare_streams(o.copy(), o, m, off, Ls, via_log=vl)
    assert rep.flips == 0 and rep.max_ulp == 0


def test_wedge_value_off_by_one_ulp_fails():
    o, m, vl, off, Ls = _case()
    # a wedge-accepted value: an exp test was taken (finite margin), not through log
    k = int(np.nonzero(np.isfinite(m) & (vl == 0) & (m > 1e-9))[0][0])
    with pytest.raises(AssertionError):
        compare_streams(_bump(o, k, 1), o, m, off, Ls, via_log=vl)


def test_fast_value_off_by_one_ulp_fails():
    o, m, vl, off, Ls = _case()
    k = int(np.nonzero(~np.isfinite(m) & (vl == 0))[0][5])
    with pytest.raises(AssertionError):
        compare_streams(_bump(o, k, 1), o, m, off, Ls, via_log=vl)


def test_tail_value_within_four_ulp_passes_and_five_fails():
    o, m, vl, off, Ls = _case()
    k = int(np.nonzero(vl)[0][0])
    rep = compare_streams(_bump(o, k, 3), o, m, off, Ls, via_log=vl)
    assert rep.inexact == 1 and rep.max_ulp == 3
    with pytest.raises(AssertionError):
        compare_streams(_bump(o, k, 5), o, m, off, Ls, via_log=vl)


def test_binary64_needs_the_flags():
    o, m, vl, off, Ls = _case()
    with pytest.raises(ValueError):
        compare_streams(o.copy(), o, m, off, Ls)
