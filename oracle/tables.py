"""Oracle table construction for the two ziggurat samplers (mpmath, 50 digits).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (the CUDA library and its binding) never does.

The paper (Sec. 1 and Sec. 2, "Ziggurat" bullet) uses the original ziggurat of
Marsaglia & Tsang (2000) in the form of the GNU Scientific Library port, and
compares it with McFarland's modified ziggurat (Sec. 2, "Java 17" bullet;
Sec. 3).  It prints no tables, so both table sets are defined here from their
geometric equations and computed at 50 significant digits, then rounded once
(round-to-nearest-even) to IEEE binary64.

Original ziggurat, 128 levels (``zig128_tables``)
------------------------------------------------
Unnormalised half density f(x) = exp(-x^2/2), x >= 0.  Abscissae
0 = x_0 < x_1 < ... < x_127 = R.  Layer i < 127 is the strip
[0, x_{i+1}) x [f(x_{i+1}), f(x_i)); layer 127 is the base: the rectangle
[0, R) x [0, f(R)) plus the region under the exponential envelope
f(R) exp(-R (x - R)) for x >= R.  Every layer has the same area v:

    x_{i+1} (f(x_i) - f(x_{i+1})) = v              (i = 0 .. 126)
    R f(R) + f(R) / R             = v              (base)

The base counts the *envelope* tail f(R)/R, not the exact normal tail: the
sampler restarts from a fresh draw when a tail proposal is rejected, and it is
an exact sampler only when the tail proposal's whole envelope is part of the
base layer.  This reading gives R = 3.44428647676..., the right-most step used
by the GSL form.  R is found by bisection on the top closure residual
x_1 (1 - f(x_1)) - v after walking the recursion down from x_127 = R.

    w[i] = RN(x_{i+1} / 2^24)  (i < 127),   w[127] = RN(v / f(R) / 2^24)
    k[i] = floor(2^24 x_i / x_{i+1}) (i < 127, so k[0] = 0),
    k[127] = floor(2^24 R f(R) / v)
    y[i] = RN(f(x_i))  (y[0] = 1, y[127] = RN(f(R)))

Modified ziggurat, 256 slots (``zig256_tables``)
-----------------------------------------------
Written from the published description of McFarland's method (rectangles
that lie wholly under the curve are sampled with no test; the overhangs and
the tail are picked with Walker's alias method and sampled by rejection).  With
A = sqrt(pi/2) the half area and a = A/256:

    X_0 f(X_0) = a, X_0 > 1                         (base rectangle)
    X_r (f(X_r) - f(X_{r-1})) = a, X_r < X_{r-1}    (r = 1 .. n_r - 1)

stacking until no rectangle of area a fits (n_r = 253).  Rectangle r is
[0, X_r) x [f(X_{r-1}), f(X_r)) (f(X_{-1}) := 0).  Each has probability exactly
1/256, so a uniform byte j < n_r selects one.  The remaining mass
(256 - n_r) a is the tail (region 0: x > X_0) and the overhangs r = 1 .. n_r,
overhang r = {X_r <= x <= X_{r-1}, f(X_{r-1}) <= y < f(x)} with X_{n_r} := 0.
The alias table over those n_r + 1 regions uses 256 bins and Vose's pairing in
a fixed order (``_vose``); thresholds are integers out of 2^56.
"""

from __future__ import annotations

import math

import mpmath as mp

DPS = 50

ZIG128_LEVELS = 128
ZIG256_SLOTS = 256


def _f(x):
    return mp.exp(-x * x / 2)


def rn_double(x) -> float:
    """Round an mpf to the nearest binary64 (ties to even), by integer arithmetic."""
    x = mp.mpf(x)
    if x == 0:
        return 0.0
    sign, man, exp, bc = x._mpf_
    man = int(man)
    # value = man * 2^exp with bc significant bits; keep 53
    shift = bc - 53
    if shift > 0:
        q, r = divmod(man, 1 << shift)
        half = 1 << (shift - 1)
        if r > half or (r == half and (q & 1)):
            q += 1
        man, exp = q, exp + shift
    val = math.ldexp(man, exp)
    return -val if sign else val


def _zig128_walk(R):
    """Return (v, [x_0 .. x_127]) for a trial R, or (v, None) if the walk overshoots y=1."""
    fR = _f(R)
    v = R * fR + fR / R
    xs = [None] * ZIG128_LEVELS
    xs[127] = R
    x = R
    for i in range(126, 0, -1):
        y = _f(x) + v / x          # f(x_i) = f(x_{i+1}) + v / x_{i+1}
        if y >= 1:
            return v, None
        x = mp.sqrt(-2 * mp.log(y))
        xs[i] = x
    xs[0] = mp.mpf(0)
    return v, xs


def zig128_solve():
    """Solve the 128-level geometry.  Returns dict with R, v, xs (all mpf)."""
    with mp.workdps(DPS + 10):
        lo, hi = mp.mpf("3.3"), mp.mpf("3.6")
        for _ in range(190):
            mid = (lo + hi) / 2
            v, xs = _zig128_walk(mid)
            if xs is None:
                lo = mid                       # R too small: the walk passes the top
            else:
                resid = xs[1] * (1 - _f(xs[1])) - v
                if resid > 0:
                    hi = mid
                else:
                    lo = mid
        R = (lo + hi) / 2
        v, xs = _zig128_walk(R)
        return {"R": R, "v": v, "xs": xs}


def zig128_tables():
    """The oracle's 128-level tables: dict of R (float), v, k (list int), w, y (list float)."""
    g = zig128_solve()
    with mp.workdps(DPS + 10):
        R, v, xs = g["R"], g["v"], g["xs"]
        two24 = mp.mpf(2) ** 24
        k, w, y = [], [], []
        for i in range(ZIG128_LEVELS):
            if i < 127:
                kk = mp.floor(two24 * xs[i] / xs[i + 1])
                ww = xs[i + 1] / two24
            else:
                kk = mp.floor(two24 * R * _f(R) / v)
                ww = v / _f(R) / two24
            k.append(int(kk))
            w.append(rn_double(ww))
            y.append(rn_double(_f(xs[i])))
        return {"R": rn_double(R), "v": rn_double(v), "k": k, "w": w, "y": y,
                "R_mp": R, "v_mp": v, "xs_mp": xs}


# --------------------------------------------------------------------------
# 256-slot modified ziggurat
# --------------------------------------------------------------------------

def _bisect(g, lo, hi, n=200):
    """Root of g on [lo, hi] where g(lo) and g(hi) have opposite signs."""
    glo = g(lo)
    for _ in range(n):
        mid = (lo + hi) / 2
        gm = g(mid)
        if (gm > 0) == (glo > 0):
            lo, glo = mid, gm
        else:
            hi = mid
    return (lo + hi) / 2


def _argmax_unimodal(g, lo, hi, n=220):
    for _ in range(n):
        m1 = lo + (hi - lo) / 3
        m2 = hi - (hi - lo) / 3
        if g(m1) < g(m2):
            lo = m1
        else:
            hi = m2
    return (lo + hi) / 2


def _normal_area(a, b):
    """Integral of exp(-x^2/2) over [a, b] (b may be +inf)."""
    s2 = mp.sqrt(2)
    if b == mp.inf:
        return mp.sqrt(mp.pi / 2) * mp.erfc(a / s2)
    return mp.sqrt(mp.pi / 2) * (mp.erf(b / s2) - mp.erf(a / s2))


def _vose(q):
    """Walker alias table by Vose's pairing, in a fixed order.

    q: list of 256 mpf, sum 256.  Small and large bins are kept as FIFO lists in
    ascending bin order; the head small bin is paired with the head large bin.
    Returns (thr, alias) with thr an mpf in [0, 1] (1 = never alias).
    """
    n = len(q)
    q = list(q)
    thr = [mp.mpf(1)] * n
    alias = list(range(n))
    small = [r for r in range(n) if q[r] < 1]
    large = [r for r in range(n) if q[r] >= 1]
    while small and large:
        s = small.pop(0)
        l = large[0]
        thr[s] = q[s]
        alias[s] = l
        q[l] = q[l] - (1 - q[s])
        if q[l] < 1:
            large.pop(0)
            small.append(l)
    return thr, alias


def zig256_solve():
    """Solve the modified-ziggurat geometry at DPS digits (mpf values)."""
    with mp.workdps(DPS + 10):
        A = mp.sqrt(mp.pi / 2)
        a = A / ZIG256_SLOTS
        # base rectangle on the right branch of x f(x) (maximum at x = 1)
        X = [_bisect(lambda x: x * _f(x) - a, mp.mpf(1), mp.mpf(8))]
        while True:
            fp = _f(X[-1])
            g = lambda x, fp=fp: x * (_f(x) - fp)
            xm = _argmax_unimodal(g, mp.mpf(0), X[-1])
            if g(xm) < a:
                break
            X.append(_bisect(lambda x, g=g: g(x) - a, xm, X[-1]))
        n_r = len(X)
        # regions: 0 = tail, r = 1..n_r overhangs (X_{n_r} := 0)
        Xe = X + [mp.mpf(0)]
        areas = [_normal_area(X[0], mp.inf)]
        for r in range(1, n_r + 1):
            lo, hi = Xe[r], Xe[r - 1]
            areas.append(_normal_area(lo, hi) - (hi - lo) * _f(hi))
        rest = (ZIG256_SLOTS - n_r) * a
        q = [ZIG256_SLOTS * ar / rest for ar in areas]
        q += [mp.mpf(0)] * (ZIG256_SLOTS - len(q))
        thr, alias = _vose(q)
        return {"A": A, "a": a, "X": X, "n_r": n_r, "areas": areas, "rest": rest,
                "q": q, "thr": thr, "alias": alias}


def zig256_tables():
    """The oracle's modified-ziggurat tables (plain Python floats / ints).

    Keys:
      n_r                 number of rectangles (fast slots)
      xs[j]               RN(X_j / 2^53), j < n_r: fast value = RN(xs[j] * m), m < 2^53
      x0                  RN(X_0), tail start
      ox[r], odx[r]       overhang r (1..n_r): RN(X_r), RN(X_{r-1} - X_r)
      oy[r], ody[r]       RN(f(X_{r-1})), RN(f(X_r) - f(X_{r-1}))
      kind[r]             +1 convex (X_r >= 1), -1 concave (X_{r-1} <= 1), 0 mixed
      qa[r]               integer: convex -> quick accept if m1 + m2 <= 2^53 - qa[r];
                          concave -> quick accept if m1 + m2 < 2^53 (qa unused, 0)
      thr[b], alias[b]    alias bins: region b if (U >> 8) < thr[b], else alias[b]
    Index 0 of the ox/odx/oy/ody/kind/qa lists is unused (region 0 is the tail).
    """
    g = zig256_solve()
    with mp.workdps(DPS + 10):
        X, n_r = g["X"], g["n_r"]
        Xe = X + [mp.mpf(0)]
        two53 = mp.mpf(2) ** 53
        xs = [rn_double(X[j] / two53) for j in range(n_r)]
        ox, odx, oy, ody, kind, qa = [0.0], [0.0], [0.0], [0.0], [0], [0]
        for r in range(1, n_r + 1):
            lo, hi = Xe[r], Xe[r - 1]
            ox.append(rn_double(lo))
            odx.append(rn_double(hi - lo))
            oy.append(rn_double(_f(hi)))
            ody.append(rn_double(_f(lo) - _f(hi)))
            if lo >= 1:
                kd = 1
            elif hi <= 1:
                kd = -1
            else:
                kd = 0
            kind.append(kd)
            if kd == 1:
                # largest normalised gap between the chord v = 1 - u and the curve
                dx, dy = hi - lo, _f(lo) - _f(hi)
                curve = lambda u: (_f(lo + dx * u) - _f(hi)) / dy
                um = _argmax_unimodal(lambda u: (1 - u) - curve(u), mp.mpf(0), mp.mpf(1))
                delta = (1 - um) - curve(um)
                # safety: 2^-40 absolute plus 1% relative on the gap
                qa.append(int(mp.ceil((delta * mp.mpf("1.01") + mp.mpf(2) ** -40) * two53)))
            else:
                qa.append(0)
        two56 = mp.mpf(2) ** 56
        thr = [int(mp.floor(t * two56)) for t in g["thr"]]
        return {"n_r": n_r, "xs": xs, "x0": rn_double(X[0]), "ox": ox, "odx": odx,
                "oy": oy, "ody": ody, "kind": kind, "qa": qa, "thr": thr,
                "alias": list(g["alias"]), "_solve": g}
