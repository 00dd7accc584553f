"""Helpers for comparing the CUDA path with the oracle (imported by the tests).

Tolerances (applied per stream, in stream order):
  * binary64: values equal bit for bit -- fast-path values, wedge and overhang
    values (the same exact arithmetic on both sides) -- except a value the
    oracle computed through log (a tail value; its via_log flag), which may
    differ by at most 4 ulp (CUDA's and the C library's log may round
    differently);
  * an accept/reject flip is allowed only where the oracle's exp-test margin for
    that variate is below 1e-12 (relative); a flip desynchronises the rest of the
    stream, so the comparison of that stream stops there, and flips are capped
    at one per 1e9 variates (rounded up to at least one per test);
  * binary32 / bfloat16 outputs: within 1 ulp (of the narrow type) of the
    oracle's binary64 value rounded to nearest even in that type.
"""

from __future__ import annotations

import math

import numpy as np

import oracle as O


def ulp_diff64(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """|ulps| between binary64 arrays; +0.0 and -0.0 are one step apart."""
    ia = a.view(np.int64)
    ib = b.view(np.int64)

    def ordered(i):
        return np.where(i < 0, np.int64(-0x8000000000000000) - i - 1, i)

    return np.abs(ordered(ia) - ordered(ib)).astype(np.uint64)


def ulp_diff32(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    ia = a.astype(np.float32).view(np.int32).astype(np.int64)
    ib = b.astype(np.float32).view(np.int32).astype(np.int64)

    def ordered(i):
        return np.where(i < 0, -0x80000000 - i - 1, i)

    return np.abs(ordered(ia) - ordered(ib))


def ulp_diff_bf16(a_bits: np.ndarray, b_bits: np.ndarray) -> np.ndarray:
    ia = a_bits.astype(np.uint16).view(np.int16).astype(np.int64)
    ib = b_bits.astype(np.uint16).view(np.int16).astype(np.int64)

    def ordered(i):
        return np.where(i < 0, -0x8000 - i - 1, i)

    return np.abs(ordered(ia) - ordered(ib))


class Report:
    def __init__(self):
        self.n = 0
        self.flips = 0
        self.max_ulp = 0
        self.inexact = 0

    def flip_cap(self) -> int:
        return max(1, math.ceil(self.n / 1e9))

    def __repr__(self):
        return (f"Report(n={self.n}, flips={self.flips}, max_ulp={self.max_ulp}, "
                f"inexact={self.inexact})")


def compare_streams(gpu: np.ndarray, orc: np.ndarray, margins: np.ndarray, offsets, lengths,
                    kind: str = "f64", tail_ulp: int = 4, all_inexact: bool = False,
                    via_log: np.ndarray = None) -> Report:
    """Compare packed stream-major outputs.  gpu is f64 / f32 / uint16 (bf16 bits).

    via_log: the oracle's per-output flag (O.generate(..., with_via_log=True)):
    binary64 values without it must be bit-exact, those with it within tail_ulp.
    Required for binary64 unless all_inexact.
    all_inexact: every value goes through log/sqrt (the polar method), so any
    value may differ by up to tail_ulp, and no decision may flip.
    """
    if kind == "f64" and not all_inexact and via_log is None:
        raise ValueError("binary64 comparisons need the oracle's via_log flags")
    rep = Report()
    if kind == "f64":
        d = ulp_diff64(np.ascontiguousarray(gpu, dtype=np.float64), orc)
        bad_thr = tail_ulp
    elif kind == "f32":
        d = ulp_diff32(gpu, O.round_f32(orc))
        bad_thr = 1
    else:
        d = ulp_diff_bf16(gpu, O.round_bf16_bits(orc))
        bad_thr = 1
    rep.n = int(len(orc))
    for s, (off, L) in enumerate(zip(offsets, lengths)):
        off, L = int(off), int(L)
        if L == 0:
            continue
        ds = d[off:off + L]
        if kind == "f64" and not all_inexact:
            thr = np.where(via_log[off:off + L] != 0, tail_ulp, 0)
        else:
            thr = bad_thr
        over = np.nonzero(ds > thr)[0]
        upto = L
        if len(over):
            k = int(over[0])
            m = margins[off + k] if not all_inexact else np.inf
            # the first mismatch must be a decision within the margin
            assert np.isfinite(m) and m < 1e-12, (
                f"stream {s} index {k}: gpu {gpu[off + k]!r} oracle {orc[off + k]!r} "
                f"ulp {ds[k]} margin {m}")
            rep.flips += 1
            upto = k
        if upto:
            part = ds[:upto]
            rep.max_ulp = max(rep.max_ulp, int(part.max()))
            if kind == "f64" and not all_inexact:
                rep.inexact += int(np.count_nonzero(part))   # only values through log get here
    assert rep.flips <= rep.flip_cap(), rep
    return rep


def offsets_of(lengths: np.ndarray) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(lengths.astype(np.int64))[:-1]]).astype(np.int64)
