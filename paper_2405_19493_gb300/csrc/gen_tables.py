"""Generate ``zig_tables.inc``: the library's ziggurat tables, as C++ constants.

Run:  python paper_2405_19493_gb300/csrc/gen_tables.py   (rewrites zig_tables.inc)

Uses only the standard library's ``decimal`` module at 80 significant digits.
Each table is computed from its defining geometry and rounded once to binary64
(or binary32) with ties to even.

128-level original ziggurat (GSL form; Sec. 1 and Sec. 2 "Ziggurat" bullet):
    f(x) = exp(-x^2/2); 0 = x_0 < x_1 < ... < x_127 = R
    x_{i+1} (f(x_i) - f(x_{i+1})) = v      for i = 0..126
    R f(R) + f(R)/R = v                    (base: rectangle + exponential-envelope tail,
                                            which makes restart-on-tail-rejection exact)
    K[i] = floor(2^24 x_i / x_{i+1}),  K[127] = floor(2^24 R f(R) / v)
    W[i] = RN(x_{i+1} 2^-24),          W[127] = RN(v / f(R) 2^-24)
    Y[i] = RN(f(x_i))
R is found with the Illinois variant of regula falsi on the top-closure residual.

256-slot modified ziggurat (after McFarland; Sec. 2 "Java 17" bullet, Sec. 3):
    a = sqrt(pi/2)/256; X_0 f(X_0) = a (X_0 > 1); X_r (f(X_r) - f(X_{r-1})) = a,
    stacked while a rectangle of area a still fits (253 rectangles).
    Overhang r = {X_r <= x <= X_{r-1}, f(X_{r-1}) <= y < f(x)} (X_253 := 0);
    region 0 = tail x > X_0.  Region probabilities feed a 256-bin Walker alias
    table, built by Vose's pairing with small and large bins kept as first-in
    first-out lists in ascending bin order (the pairing order is part of the
    table's definition).  Thresholds are integers out of 2^56.
    Convex overhangs (X_r >= 1) carry a quick-accept margin: the largest
    normalised gap between the chord and the curve, times 1.01, plus 2^-40,
    in units of 2^-53, rounded up.
"""

from __future__ import annotations

import os
import sys
from decimal import ROUND_FLOOR, ROUND_CEILING, Decimal, getcontext

getcontext().prec = 80
D = Decimal
ONE, TWO = D(1), D(2)
HERE = os.path.dirname(os.path.abspath(__file__))


# ---- elementary functions -----------------------------------------------------

def _arctan_inv(n: int) -> Decimal:
    """arctan(1/n) by its Taylor series."""
    x = ONE / n
    x2 = x * x
    term, total, k = x, x, 1
    eps = D(10) ** -(getcontext().prec + 2)
    while abs(term) > eps:
        term *= -x2
        total += term / (2 * k + 1)
        k += 1
    return total


PI = 16 * _arctan_inv(5) - 4 * _arctan_inv(239)      # Machin's formula


def f(x: Decimal) -> Decimal:
    return (-(x * x) / 2).exp()


def erf(z: Decimal) -> Decimal:
    """erf by its Maclaurin series (|z| < 3 here, so 80 digits leave >70 good ones)."""
    z2 = z * z
    term = z            # (-1)^n z^(2n+1) / n!
    total = z
    n = 0
    eps = D(10) ** -(getcontext().prec + 2)
    while True:
        n += 1
        term = -term * z2 / n
        add = term / (2 * n + 1)
        total += add
        if abs(add) < eps:
            break
    return 2 / PI.sqrt() * total


def area(lo: Decimal, hi) -> Decimal:
    """Integral of f over [lo, hi]; hi = None means +infinity."""
    s2 = TWO.sqrt()
    c = (PI / 2).sqrt()
    if hi is None:
        return c * (1 - erf(lo / s2))
    return c * (erf(hi / s2) - erf(lo / s2))


# ---- rounding -----------------------------------------------------------------

def _round_binary(x: Decimal, mant_bits: int) -> tuple[int, int]:
    """x > 0 -> (m, e) with m * 2^e = RN-even(x) to mant_bits significant bits."""
    assert x > 0
    e = int(x.ln() / D(2).ln()) - mant_bits + 1
    # fix e so that 2^(mant_bits-1) <= x / 2^e < 2^mant_bits
    while x / (TWO ** e) >= TWO ** mant_bits:
        e += 1
    while x / (TWO ** e) < TWO ** (mant_bits - 1):
        e -= 1
    scaled = x / (TWO ** e)
    m = int(scaled.to_integral_value(rounding=ROUND_FLOOR))
    frac = scaled - m
    if frac > D("0.5") or (frac == D("0.5") and (m & 1)):
        m += 1
    if m == 1 << mant_bits:
        m >>= 1
        e += 1
    return m, e


def rn64(x: Decimal) -> float:
    if x == 0:
        return 0.0
    neg = x < 0
    m, e = _round_binary(abs(x), 53)
    import math
    v = math.ldexp(m, e)
    return -v if neg else v


def rn32_hex(x: Decimal) -> str:
    """RN-even to binary32, as a C hex-float literal with an f suffix."""
    m, e = _round_binary(x, 24)
    import math
    v = math.ldexp(m, e)           # exact in binary64
    return v.hex() + "f"


def floor_int(x: Decimal) -> int:
    return int(x.to_integral_value(rounding=ROUND_FLOOR))


def ceil_int(x: Decimal) -> int:
    return int(x.to_integral_value(rounding=ROUND_CEILING))


# ---- 128-level geometry ---------------------------------------------------------

def _walk128(R: Decimal):
    """Residual x_1 (1 - f(x_1)) - v and the abscissae for a trial R.

    Returns (residual, v, xs); residual = +1 marker when the walk passes y = 1.
    """
    fR = f(R)
    v = R * fR + fR / R
    xs = [None] * 128
    xs[127] = R
    x = R
    for i in range(126, 0, -1):
        yv = f(x) + v / x
        if yv >= 1:
            return None, v, None
        x = (-2 * yv.ln()).sqrt()
        xs[i] = x
    xs[0] = D(0)
    return xs[1] * (1 - f(xs[1])) - v, v, xs


def solve128():
    # bracket: small R overshoots the top (no residual), large R leaves a positive residual
    lo, hi = D("3.44"), D("3.45")
    rlo, _, _ = _walk128(lo)
    while rlo is None:
        lo += D("0.0005")
        rlo, _, _ = _walk128(lo)
    rhi, _, _ = _walk128(hi)
    assert rlo < 0 < rhi
    side = 0
    for _ in range(400):
        m = (lo * rhi - hi * rlo) / (rhi - rlo)
        rm, _, _ = _walk128(m)
        if rm is None:           # outside the domain: fall back to bisection
            m = (lo + hi) / 2
            rm, _, _ = _walk128(m)
            if rm is None:
                lo = m
                continue
        if rm < 0:
            lo, rlo = m, rm
            if side == -1:
                rhi /= 2
            side = -1
        else:
            hi, rhi = m, rm
            if side == 1:
                rlo /= 2
            side = 1
        if hi - lo < D(10) ** -70 or rm == 0:
            break
    R = m
    _, v, xs = _walk128(R)
    return R, v, xs


def tables128():
    R, v, xs = solve128()
    two24 = TWO ** 24
    K, W, Y, W32 = [], [], [], []
    for i in range(128):
        if i < 127:
            K.append(floor_int(two24 * xs[i] / xs[i + 1]))
            wx = xs[i + 1] / two24
        else:
            K.append(floor_int(two24 * R * f(R) / v))
            wx = v / f(R) / two24
        W.append(rn64(wx))
        W32.append(rn32_hex(wx))
        Y.append(rn64(f(xs[i])))
    return {"R": rn64(R), "v": rn64(v), "K": K, "W": W, "Y": Y, "W32": W32}


# ---- 256-slot geometry ------------------------------------------------------------

def _newton_bisect(g, dg, lo: Decimal, hi: Decimal, x0: Decimal) -> Decimal:
    """Root of g in [lo, hi] (sign change), Newton steps guarded by bisection."""
    glo = g(lo)
    x = x0
    for _ in range(300):
        gx = g(x)
        if gx == 0:
            return x
        if (gx > 0) == (glo > 0):
            lo, glo = x, gx
        else:
            hi = x
        d = dg(x)
        nx = x - gx / d if d != 0 else (lo + hi) / 2
        if not (min(lo, hi) < nx < max(lo, hi)):
            nx = (lo + hi) / 2
        if abs(nx - x) < D(10) ** -72:
            return nx
        x = nx
    return x


def _bisect(g, lo: Decimal, hi: Decimal, n: int = 260) -> Decimal:
    glo = g(lo)
    for _ in range(n):
        mid = (lo + hi) / 2
        gm = g(mid)
        if (gm > 0) == (glo > 0):
            lo, glo = mid, gm
        else:
            hi = mid
    return (lo + hi) / 2


def solve256():
    A = (PI / 2).sqrt()
    a = A / 256
    # base: x f(x) = a on x > 1
    X = [_newton_bisect(lambda x: x * f(x) - a, lambda x: f(x) * (1 - x * x),
                        D(1), D(8), D("3.6"))]
    while True:
        c = f(X[-1])
        g = lambda x, c=c: x * (f(x) - c)
        dg = lambda x, c=c: f(x) * (1 - x * x) - c
        # g' is decreasing on [0, X]: its zero is the maximiser of g
        xm = _bisect(dg, D(0), X[-1])
        if g(xm) < a:
            break
        X.append(_newton_bisect(lambda x, g=g: g(x) - a, dg, xm, X[-1], X[-1]))
    n_r = len(X)
    Xe = X + [D(0)]
    areas = [area(X[0], None)]
    for r in range(1, n_r + 1):
        lo, hi = Xe[r], Xe[r - 1]
        areas.append(area(lo, hi) - (hi - lo) * f(hi))
    rest = (256 - n_r) * a
    q = [256 * ar / rest for ar in areas] + [D(0)] * (256 - n_r - 1)
    # Vose's pairing, FIFO lists in ascending bin order
    thr = [ONE] * 256
    alias = list(range(256))
    small = [b for b in range(256) if q[b] < 1]
    large = [b for b in range(256) if q[b] >= 1]
    si = li = 0
    while si < len(small) and li < len(large):
        s, l = small[si], large[li]
        si += 1
        thr[s], alias[s] = q[s], l
        q[l] -= 1 - q[s]
        if q[l] < 1:
            li += 1
            small.append(l)
    return X, n_r, thr, alias


def tables256():
    X, n_r, thr, alias = solve256()
    Xe = X + [D(0)]
    two53 = TWO ** 53
    XS = [rn64(X[j] / two53) for j in range(n_r)]
    OX, ODX, OY, ODY, KIND, QA = [], [], [], [], [], []
    for r in range(1, n_r + 1):
        lo, hi = Xe[r], Xe[r - 1]
        dx, dy = hi - lo, f(lo) - f(hi)
        OX.append(rn64(lo))
        ODX.append(rn64(dx))
        OY.append(rn64(f(hi)))
        ODY.append(rn64(dy))
        kind = 1 if lo >= 1 else (-1 if hi <= 1 else 0)
        KIND.append(kind)
        if kind == 1:
            # the gap (1 - u) - (f(lo + dx u) - f(hi))/dy peaks where x f(x) = dy/dx
            s = dy / dx
            xstar = _bisect(lambda x: x * f(x) - s, lo, hi)
            u = (xstar - lo) / dx
            gap = (1 - u) - (f(xstar) - f(hi)) / dy
            QA.append(ceil_int((gap * D("1.01") + TWO ** -40) * two53))
        else:
            QA.append(0)
    two56 = TWO ** 56
    THR = [floor_int(t * two56) for t in thr]
    return {"n_r": n_r, "x0": rn64(X[0]), "XS": XS, "OX": OX, "ODX": ODX, "OY": OY,
            "ODY": ODY, "KIND": KIND, "QA": QA, "THR": THR, "ALIAS": alias}


# ---- natural logarithm tables (P. T. P. Tang's table-driven method, 1990) -------------
# ln x = e ln2 + ln F_k + ln(1 + r) for x = 2^e m, F_k = 1 + k/128 the table point
# nearest m (k = 0..128) and r = (m - F_k)/F_k.  Stored: G_k = RN(1/F_k), and
# ln F_k and ln 2 split as hi + lo with hi on the grid 2^-40, so that e * LN2_HI +
# LOG_THI[k] is exact in binary64 for |e| < 2^10 (at most 50 significant bits).

def _ln(x: Decimal) -> Decimal:
    return x.ln()


def _grid(x: Decimal, step_log2: int) -> Decimal:
    """x rounded to the nearest multiple of 2^-step_log2 (ties to even multiple)."""
    q = x * (TWO ** step_log2)
    n = int(q.to_integral_value(rounding=ROUND_FLOOR))
    frac = q - n
    if frac > D("0.5") or (frac == D("0.5") and (n & 1)):
        n += 1
    return D(n) / (TWO ** step_log2)


def tables_log():
    ln2 = _ln(TWO)
    ln2_hi = _grid(ln2, 40)
    out = {"LN2_HI": rn64(ln2_hi), "LN2_LO": rn64(ln2 - ln2_hi), "G": [], "THI": [], "TLO": []}
    for k in range(129):
        F = ONE + D(k) / 128
        T = _ln(F)
        t_hi = ln2_hi if k == 128 else _grid(T, 40)   # k = 128: exactly LN2_HI + LN2_LO
        out["G"].append(rn64(ONE / F))
        out["THI"].append(rn64(t_hi))
        out["TLO"].append(rn64(T - t_hi) if k < 128 else out["LN2_LO"])
    return out


# ---- output -------------------------------------------------------------------------

def _arr(ctype, name, vals, fmt, per_line=4):
    lines = [f"static const {ctype} {name}[{len(vals)}] = {{"]
    for k in range(0, len(vals), per_line):
        lines.append("    " + ", ".join(fmt(v) for v in vals[k:k + per_line]) + ",")
    lines.append("};")
    return "\n".join(lines)


def render() -> str:
    t = tables128()
    m = tables256()
    lg = tables_log()
    hx = lambda v: v.hex()
    out = [
        "// Ziggurat tables for the CUDA library.  GENERATED by gen_tables.py "
        "(decimal, 80 digits); do not edit.",
        "// 128-level original ziggurat: K (u32), W (f64), Y (f64), W32 (f32); "
        "base layer = R f(R) + f(R)/R.",
        "// 256-slot modified ziggurat: rectangle widths, overhang boxes, alias table.",
        "// Natural-logarithm tables for the tail step's binary64 log.",
        "#pragma once",
        "#include <stdint.h>",
        "namespace zigtab {",
        f"static const double ZIG128_R = {hx(t['R'])};",
        f"static const double ZIG128_V = {hx(t['v'])};",
        _arr("uint32_t", "ZIG128_K", t["K"], lambda v: f"{v}u"),
        _arr("double", "ZIG128_W", t["W"], hx, 3),
        _arr("double", "ZIG128_Y", t["Y"], hx, 3),
        _arr("float", "ZIG128_W32", t["W32"], lambda v: v, 3),
        f"static const int ZIG256_NR = {m['n_r']};",
        f"static const double ZIG256_X0 = {hx(m['x0'])};",
        _arr("double", "ZIG256_XS", m["XS"], hx, 3),
        "// overhang r = 1..n_r stored at index r - 1",
        _arr("double", "ZIG256_OX", m["OX"], hx, 3),
        _arr("double", "ZIG256_ODX", m["ODX"], hx, 3),
        _arr("double", "ZIG256_OY", m["OY"], hx, 3),
        _arr("double", "ZIG256_ODY", m["ODY"], hx, 3),
        _arr("int", "ZIG256_KIND", m["KIND"], str, 16),
        _arr("uint64_t", "ZIG256_QA", m["QA"], lambda v: f"{v}ull"),
        _arr("uint64_t", "ZIG256_THR", m["THR"], lambda v: f"{v}ull"),
        _arr("int", "ZIG256_ALIAS", m["ALIAS"], str, 16),
        "// natural logarithm (Tang's table-driven method): F_k = 1 + k/128",
        f"static const double LN2_HI = {hx(lg['LN2_HI'])};",
        f"static const double LN2_LO = {hx(lg['LN2_LO'])};",
        _arr("double", "LOG_G", lg["G"], hx, 3),
        _arr("double", "LOG_THI", lg["THI"], hx, 3),
        _arr("double", "LOG_TLO", lg["TLO"], hx, 3),
        "}  // namespace zigtab",
        "",
    ]
    return "\n".join(out)


def main() -> int:
    with open(os.path.join(HERE, "zig_tables.inc"), "w") as fh:
        fh.write(render())
    return 0


if __name__ == "__main__":
    sys.exit(main())
