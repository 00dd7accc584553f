"""Pins for the oracle's stored ziggurat tables (CPU only).

The checks re-derive each geometric identity with double-precision libm/scipy
functions from the stored doubles alone, so a wrong sign, a dropped term or an
off-by-one layer index in ``oracle/tables.py`` breaks one of them:
  * zig128: equal layer areas, the top closure x_1 (1 - f(x_1)) = v, the base
    R f(R) + f(R)/R = v, y[i] = f(x_i), k[i] = floor(2^24 x_i / x_{i+1}), and R
    against the right-most step of the GSL form (3.44428647676);
  * zig256: equal rectangle areas sqrt(pi/2)/256, the overhang/tail partition of
    the remaining mass, the alias table's region probabilities against areas
    computed with scipy's erf/erfc, and the quick-accept margins.
"""

import math
import os

import numpy as np
import pytest
from scipy import special

import oracle as O

T128 = O.read_zig128()
T256 = O.read_zig256()
TWO24 = float(1 << 24)
TWO53 = float(1 << 53)


def f(x):
    return math.exp(-x * x / 2)


def test_stored_tables_match_generator():
    pytest.importorskip("mpmath")
    from oracle import gen_tables, tables
    with open(os.path.join(O.TABLE_DIR, "zig128.txt")) as fh:
        assert fh.read() == gen_tables.render_zig128(tables.zig128_tables())
    with open(os.path.join(O.TABLE_DIR, "zig256.txt")) as fh:
        assert fh.read() == gen_tables.render_zig256(tables.zig256_tables())


def test_zig128_geometry():
    k, w, y, R, v = T128["k"], T128["w"], T128["y"], T128["R"], T128["v"]
    x = [0.0] + [w[i] * TWO24 for i in range(127)]      # x_0 .. x_127
    assert x[127] == R
    assert abs(R - 3.44428647676) < 1e-10               # right-most step of the GSL form
    # base layer: rectangle R f(R) plus the exponential envelope's tail f(R)/R
    assert math.isclose(R * f(R) + f(R) / R, v, rel_tol=1e-14)
    assert math.isclose(w[127] * TWO24 * f(R), v, rel_tol=1e-14)
    # top closure and the 127 strips
    assert math.isclose(x[1] * (1 - f(x[1])), v, rel_tol=1e-13)
    for i in range(127):
        area = x[i + 1] * (f(x[i]) - f(x[i + 1]))
        assert math.isclose(area, v, rel_tol=1e-12), i
    for i in range(128):
        # y[i] rounds f at the exact x_i; x[i] here is itself rounded (|dx/x| <= 2^-53)
        tol = (1 + x[i] * x[i]) * 2.0 ** -52
        assert math.isclose(y[i], f(x[i]), rel_tol=tol, abs_tol=0), i
    assert y[0] == 1.0 and k[0] == 0
    for i in range(1, 127):
        ratio = TWO24 * x[i] / x[i + 1]
        assert k[i] <= ratio + 1e-6 and ratio < k[i] + 1, i
    ratio = TWO24 * R * f(R) / v
    assert k[127] <= ratio + 1e-6 and ratio < k[127] + 1
    assert all(y[i] > y[i + 1] for i in range(127))
    assert all(w[i] < w[i + 1] for i in range(127))
    # the ziggurat covers the half density: 128 v > sqrt(pi/2)
    assert 128 * v > math.sqrt(math.pi / 2)


def test_zig256_rectangles():
    n_r, xs, x0 = T256["n_r"], T256["xs"], T256["x0"]
    a = math.sqrt(math.pi / 2) / 256
    X = [xs[j] * TWO53 for j in range(n_r)]
    assert n_r == 253 and X[0] == x0
    assert math.isclose(X[0] * f(X[0]), a, rel_tol=1e-13) and X[0] > 1
    for j in range(1, n_r):
        assert X[j] < X[j - 1]
        assert math.isclose(X[j] * (f(X[j]) - f(X[j - 1])), a, rel_tol=1e-11), j
    # no further rectangle of area a fits above the last one
    grid = np.linspace(0, X[-1], 20001)
    assert np.max(grid * (np.exp(-grid ** 2 / 2) - f(X[-1]))) < a


def test_zig256_overhangs_and_alias():
    n_r, xs, x0 = T256["n_r"], T256["xs"], T256["x0"]
    X = [xs[j] * TWO53 for j in range(n_r)] + [0.0]
    a = math.sqrt(math.pi / 2) / 256
    s2 = math.sqrt(2.0)
    half = math.sqrt(math.pi / 2)
    areas = [half * special.erfc(x0 / s2)]
    for r in range(1, n_r + 1):
        lo, hi = X[r], X[r - 1]
        assert T256["ox"][r] == lo
        # X_r are themselves rounded: the double difference carries ~ulp(hi)
        assert math.isclose(T256["odx"][r], hi - lo, rel_tol=0, abs_tol=hi * 2.0 ** -51)
        assert math.isclose(T256["oy"][r], f(hi), rel_tol=(1 + hi * hi) * 2.0 ** -52)
        assert math.isclose(T256["ody"][r], f(lo) - f(hi), rel_tol=1e-13)
        kind = 1 if lo >= 1 else (-1 if hi <= 1 else 0)
        assert T256["kind"][r] == kind
        areas.append(half * (special.erf(hi / s2) - special.erf(lo / s2)) - (hi - lo) * f(hi))
    areas = np.array(areas)
    # rectangles + overhangs + tail partition the half area
    assert math.isclose(areas.sum(), (256 - n_r) * a, rel_tol=1e-10)
    # the alias table reproduces the region probabilities
    thr = np.array(T256["thr"], dtype=np.float64) / 2.0 ** 56
    alias = np.array(T256["alias"])
    p = np.zeros(256)
    for b in range(256):
        p[b] += thr[b] / 256
        p[alias[b]] += (1 - thr[b]) / 256
    want = np.zeros(256)
    want[: n_r + 1] = areas / areas.sum()
    assert np.allclose(p, want, rtol=0, atol=1e-12)


def test_zig256_quick_accept_margins():
    n_r = T256["n_r"]
    u = np.linspace(0, 1, 4001)
    for r in range(1, n_r + 1):
        if T256["kind"][r] != 1:
            continue
        lo, dx = T256["ox"][r], T256["odx"][r]
        dy = T256["ody"][r]
        curve = (np.exp(-(lo + dx * u) ** 2 / 2) - T256["oy"][r]) / dy
        gap = np.max((1 - u) - curve)
        assert gap >= -1e-12
        qa = T256["qa"][r] / TWO53
        assert gap <= qa and qa <= 1.02 * gap + 2.0 ** -39, r
