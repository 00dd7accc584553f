"""Pins for the oracle's uniform PRNGs (CPU only).

What pins what:
  * known answers of java.util.Random and SplitMix64 (tests/golden/known_answers.txt)
    pin the 48-bit LCG, Random.nextInt / nextDouble, the polar method and mix64;
  * the LCG's bit periods (bit b of the state has period 2^(b+1)) pin the modulus
    and the full-period conditions on a and c;
  * Berlekamp-Massey + a primitivity test pin xoroshiro128's shifts and rotations
    (the LXM engine has period 2^128 - 1 only for a primitive characteristic polynomial);
  * closed-form jump-ahead equals stepping, and jumps compose additively;
  * byte-level chi-square pins the mixers' uniformity (mix32 and mixLea64 have no
    known answer here: their JDK parity is unpinned).
"""

import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "known_answers.txt")


def _golden():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                p = line.split()
                rows.append((p[0], p[1], int(p[2]), p[3:]))
    return rows


def test_known_answers():
    rows = _golden()
    assert len(rows) == 5
    for prng, call, seed, vals in rows:
        g = O.Generator(prng, seed)
        if call == "nextInt":
            assert g.next_int() == int(vals[0])
        elif call == "nextLong":
            for v in vals:
                assert g.next_u64() == int(v, 16)
        elif call == "nextGaussian":
            got = np.float64(g.next_gaussian_polar())
            want = np.float64(vals[0])
            # StrictMath (fdlibm) log/sqrt vs the C library's: the polar tolerance is 4 ulp
            assert abs(int(got.view(np.int64)) - int(want.view(np.int64))) <= 4
        else:
            raise AssertionError(call)


def test_lcg_bit_periods():
    # nextInt = state bits 16..47; state bit b has period exactly 2^(b+1)
    x = O.prng_fill("lcg48", [12345], 1 << 19, kind="u32")[0]
    for out_bit, period in ((0, 1 << 17), (1, 1 << 18)):
        b = (x >> np.uint64(out_bit)) & np.uint64(1)
        assert np.array_equal(b[:period], b[period:2 * period])
        half = period // 2
        assert not np.array_equal(b[:half], b[half:2 * half])


def test_lcg_nextlong_and_nextdouble_composition():
    # nextLong = (nextInt << 32) + sign-extended nextInt; nextDouble uses 26 + 27 bits
    a = O.Generator("lcg48", 7)
    b = O.Generator("lcg48", 7)
    for _ in range(100):
        hi, lo = a.next_int(), a.next_int()
        assert b.next_u64() == ((hi << 32) + lo) % (1 << 64)
    a = O.Generator("lcg48", 9)
    b = O.Generator("lcg48", 9)
    for _ in range(100):
        hi, lo = a.next_u32() >> 6, a.next_u32() >> 5
        assert b.next_m53() == (hi << 27) + lo


def _steps(g, prng, n):
    for _ in range(n):
        g.next_u32()  # one raw step for every generator


@pytest.mark.parametrize("prng", list(O.PRNGS))
def test_jump_equals_stepping(prng):
    seed = 0x5EED + 3
    for n in (0, 1, 2, 3, 1000, 12345):
        g1 = O.Generator(prng, seed)
        _steps(g1, prng, n)
        g2 = O.Generator(prng, seed)
        g2.jump(n)
        assert g1.state() == g2.state(), (prng, n)
    # long jump vs stepping, via the C fill loop
    n = 1 << 20
    stepped = O.prng_fill(prng, [seed], n + 4, kind="u32")[0][n:]
    jumped = O.prng_fill(prng, [seed], 4, kind="u32", skip=n)[0]
    assert np.array_equal(stepped, jumped)


@pytest.mark.parametrize("prng", list(O.PRNGS))
def test_jump_composes(prng):
    a, b = 1 << 32, (1 << 40) + 7
    g1 = O.Generator(prng, 99)
    g1.jump(a)
    g1.jump(b)
    g2 = O.Generator(prng, 99)
    g2.jump(a + b)
    assert g1.state() == g2.state()


def test_splitmix_gamma_additivity():
    gamma = 0x9E3779B97F4A7C15
    g = O.Generator("splitmix64", 5)
    for _ in range(10):
        g.next_u64()
    h = O.Generator("splitmix64", (5 + 10 * gamma) % (1 << 64))
    assert g.next_u64() == h.next_u64()


# ---- xoroshiro128 primitivity ---------------------------------------------

def _berlekamp_massey(bits):
    """Shortest LFSR over GF(2) for a bit sequence; returns (L, C as int, bit i = c_i)."""
    n = len(bits)
    c, b = 1, 1
    L, m = 0, 1
    for i in range(n):
        d = bits[i]
        for j in range(1, L + 1):
            d ^= ((c >> j) & 1) & bits[i - j]
        if d == 0:
            m += 1
        elif 2 * L <= i:
            t = c
            c ^= b << m
            L, b, m = i + 1 - L, t, 1
        else:
            c ^= b << m
            m += 1
    return L, c


def _pmod_mul(a, b, p, deg):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if (a >> deg) & 1:
            a ^= p
    return r


def _pmod_pow_x(e, p, deg):
    result, base = 1, 2  # polynomials: 1 and x
    while e:
        if e & 1:
            result = _pmod_mul(result, base, p, deg)
        base = _pmod_mul(base, base, p, deg)
        e >>= 1
    return result


def _is_prime(n):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def test_xoroshiro128_primitive():
    g = O.Generator("l64x128mix", 2024)
    seq = []
    for _ in range(400):
        g.next_u64()
        seq.append(g.state()[2] & 1)  # bit 0 of x0
    L, c = _berlekamp_massey(seq)
    assert L == 128
    # characteristic polynomial = reciprocal of the connection polynomial
    p = 0
    for i in range(L + 1):
        if (c >> i) & 1:
            p |= 1 << (L - i)
    assert (p >> 128) & 1 and p & 1
    order = (1 << 128) - 1
    factors = [3, 5, 17, 257, 641, 65537, 274177, 6700417, 67280421310721]
    assert math.prod(factors) == order and all(_is_prime(f) for f in factors)
    assert _pmod_pow_x(order, p, 128) == 1
    for q in factors:
        assert _pmod_pow_x(order // q, p, 128) != 1


def test_xoroshiro128pp_engine_primitive():
    # the (49, 21, 28) engine has a primitive degree-128 characteristic
    # polynomial (full period 2^128 - 1); a wrong rotation or shift constant
    # almost surely breaks this
    g = O.Generator("xoroshiro128pp", 2024)
    seq = []
    for _ in range(400):
        g.next_u64()
        seq.append(g.state()[2] & 1)  # bit 0 of x0
    L, c = _berlekamp_massey(seq)
    assert L == 128
    p = 0
    for i in range(L + 1):
        if (c >> i) & 1:
            p |= 1 << (L - i)
    order = (1 << 128) - 1
    factors = [3, 5, 17, 257, 641, 65537, 274177, 6700417, 67280421310721]
    assert _pmod_pow_x(order, p, 128) == 1
    for q in factors:
        assert _pmod_pow_x(order // q, p, 128) != 1


def test_xoroshiro128pp_output_is_a_function_of_the_state_before_the_step():
    # nextLong's ++ scrambler reads (x0, x1) before the linear step: two
    # generators with equal states give equal outputs, and the output is not
    # a linear function of the state (its lowest bit is x0 + x1 + x0 with carries)
    g = O.Generator("xoroshiro128pp", 5)
    st = g.state()
    a = g.next_u64()
    h = O.Generator("xoroshiro128pp", 5)
    assert h.state() == st and h.next_u64() == a
    # bit 0 of rotl(x0 + x1, 17) + x0 is bit 47 of (x0 + x1) xor bit 0 of x0
    bits = []
    for _ in range(2000):
        x0, x1 = g.state()[2], g.state()[3]
        out = g.next_u64()
        bits.append(((((x0 + x1) % (1 << 64)) >> 47) ^ x0) & 1 == out & 1)
    assert all(bits)


def test_lxm_lcg_low_bit_periods():
    # LXM's LCG s <- M s + a (mod 2^64), a odd: state bit b has period 2^(b+1)
    g = O.Generator("l64x128mix", 77)
    s = []
    for _ in range(1 << 11):
        s.append(g.state()[0])
        g.next_u64()
    s = np.array(s, dtype=np.uint64)
    for b in range(0, 9):
        per = 1 << (b + 1)
        bits = (s >> np.uint64(b)) & np.uint64(1)
        assert np.array_equal(bits[:per], bits[per:2 * per])
        assert not np.array_equal(bits[:per // 2], bits[per // 2:per])


# ---- uniformity -------------------------------------------------------------

@pytest.mark.parametrize("prng", list(O.PRNGS))
@pytest.mark.parametrize("kind", ["u32", "u64", "m53"])
def test_byte_uniformity(prng, kind):
    x = O.prng_fill(prng, 0x5EED + np.arange(64, dtype=np.uint64), 4096, kind=kind).ravel()
    width = {"u32": 32, "u64": 64, "m53": 53}[kind]
    for shift in range(0, width - 7, 8):
        byte = ((x >> np.uint64(shift)) & np.uint64(0xFF)).astype(np.int64)
        counts = np.bincount(byte, minlength=256)
        p = stats.chisquare(counts).pvalue
        assert p > 1e-6, (prng, kind, shift, p)
    if kind == "m53":
        assert int(x.max()) < (1 << 53)
