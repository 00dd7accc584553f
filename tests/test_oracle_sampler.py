"""Pins for the oracle's samplers (CPU only).

  * hand-built draw words through the 128-level sampler and the 256-slot sampler:
    branch selection (fast / wedge / tail; rectangle / overhang / tail), the sign
    bit, the layer index, j * w[i], +-0.0, the restart after a wedge rejection;
  * per-iteration branch rates and iterations per variate against closed forms
    from the tables (128 v / sqrt(pi/2) for the exact rejection sampler);
  * the distribution against scipy's Phi: moments, Kolmogorov-Smirnov, 1000-bin
    chi-square, the tail mass beyond 3 and beyond R, and the conditional tail shape;
  * polar: acceptance pi/4; modified ziggurat: rectangle share n_r/256;
  * the chunked-substream driver and the narrow-type rounding helpers.
"""

import math

import numpy as np
import pytest
from scipy import stats

import oracle as O

T128 = O.read_zig128()
T256 = O.read_zig256()
SEEDS64 = 0x5EED + np.arange(64, dtype=np.uint64)


def w32(i, j, positive):
    """A 32-bit ziggurat draw: low byte = layer i (bit 7 = sign, set = +), upper 24 = j."""
    return (j << 8) | (0x80 if positive else 0) | i


def dbl(m):
    """A scripted word whose nextDouble is m * 2^-53."""
    return m << 11


# ---- hand cases --------------------------------------------------------------

def test_zig128_hand_cases():
    k, w, y, R = T128["k"], T128["w"], T128["y"], T128["R"]
    # (a, b) j = 0 gives +0.0 / -0.0 on the fast path
    v, used, st = O.zig128_scripted([w32(5, 0, True)], 1)
    assert used == 1 and v[0] == 0.0 and not math.copysign(1, v[0]) < 0 and st["fast"] == 1
    v, used, st = O.zig128_scripted([w32(5, 0, False)], 1)
    assert math.copysign(1, v[0]) < 0
    # (c) largest fast j in layer 5: value = j * w[5], one rounding
    j = k[5] - 1
    v, used, st = O.zig128_scripted([w32(5, j, True)], 1)
    assert v[0] == j * w[5] and st["fast"] == 1
    v, used, st = O.zig128_scripted([w32(5, j, False)], 1)
    assert v[0] == -(j * w[5])
    # (d) j = k[5] goes to the wedge; U = 0 puts y at the strip's bottom -> accepted
    j = k[5]
    v, used, st = O.zig128_scripted([w32(5, j, True), dbl(0)], 1)
    assert used == 2 and st["wedge"] == 1 and st["wedge_acc"] == 1 and v[0] == j * w[5]
    # (e) x near x_6 with y near the strip's top -> rejected, restart on the next word
    j = (1 << 24) - 1
    v, used, st = O.zig128_scripted([w32(5, j, True), dbl((1 << 53) - 1), w32(3, 7, False)], 1)
    assert used == 3 and st["wedge"] == 1 and st["wedge_acc"] == 0 and st["fast"] == 1
    assert v[0] == -(7 * w[3])
    # (f) base layer, j >= k[127]: tail with U1 = 1 - 0 -> x = R, U2 = 0 -> y = 0 -> accept
    v, used, st = O.zig128_scripted([w32(127, (1 << 24) - 1, True), dbl(0), dbl(0)], 1)
    assert used == 3 and st["tail"] == 1 and st["tail_acc"] == 1 and v[0] == R
    # base layer fast path just below k[127]
    v, used, st = O.zig128_scripted([w32(127, k[127] - 1, False)], 1)
    assert v[0] == -((k[127] - 1) * w[127]) and st["fast"] == 1
    # (g) layer 0 never accepts fast (k[0] = 0): j = 0 goes to the wedge, U = 1/2 accepts
    v, used, st = O.zig128_scripted([w32(0, 0, True), dbl(1 << 52)], 1)
    assert st["fast"] == 0 and st["wedge"] == 1 and st["wedge_acc"] == 1 and v[0] == 0.0
    # ... and y rounding to exactly f(0) = 1 is rejected by the strict test
    v, used, st = O.zig128_scripted([w32(0, 0, True), dbl((1 << 53) - 1), w32(2, 3, True)], 1)
    assert used == 3 and st["wedge_acc"] == 0 and v[0] == 3 * w[2]
    # wedge y formula: y = y1 + (y0 - y1) * U tested against exp(-x^2/2) -> decide by hand
    j = (k[60] + (1 << 24)) // 2
    x = j * w[60]
    for m in (1 << 20, 1 << 52, (1 << 53) - (1 << 30)):
        U = m * 2.0 ** -53
        yy = y[61] + (y[60] - y[61]) * U
        accept = yy < math.exp(-0.5 * x * x)
        v, used, st = O.zig128_scripted([w32(60, j, True), dbl(m), w32(1, 1, True)], 1)
        assert (used == 2) == accept
        assert v[0] == (x if accept else 1 * w[1])


def test_zig256_hand_cases():
    n_r, xs = T256["n_r"], T256["xs"]
    m = (1 << 53) - 12345
    # rectangle slot j < n_r: value = xs[j] * m, sign from bit 8 (set = negative)
    for j in (0, 17, n_r - 1):
        U = (m << 11) | (0 << 8) | j
        v, used, st = O.zig256_scripted([U], 1)
        assert used == 1 and v[0] == xs[j] * float(m)
        v, used, st = O.zig256_scripted([U | (1 << 8)], 1)
        assert v[0] == -(xs[j] * float(m))
    # slow slot -> alias bin; pick a bin whose own region is a convex overhang
    thr, alias, kind = T256["thr"], T256["alias"], T256["kind"]
    b = next(b for b in range(1, n_r + 1) if thr[b] > 0 and kind[b] == 1)
    V = (0 << 8) | b                       # (V >> 8) = 0 < thr[b] -> region b
    m1, m2 = 1 << 40, 1 << 40              # deep inside the lower triangle -> quick accept
    v, used, st = O.zig256_scripted([n_r, V, dbl(m1), dbl(m2)], 1)
    assert used == 4 and st["overhang_quick"] == 1
    assert v[0] == T256["ox"][b] + T256["odx"][b] * (m1 * 2.0 ** -53)
    # the same bin with (V >> 8) at the top of its range takes the alias
    Vt = (((1 << 56) - 1) << 8) | b
    ra = alias[b]
    v, used, st = O.zig256_scripted([n_r, Vt] + [dbl(1 << 40)] * 8, 1)
    if ra == 0:
        assert st["tail"] == 1
    else:
        assert st["overhang"] == 1 and v[0] >= T256["ox"][ra]
    # upper triangle of a convex overhang is reflected: (m1, m2) -> (2^53 - m1, 2^53 - m2)
    m1, m2 = (1 << 53) - (1 << 40), (1 << 53) - (1 << 41)
    v, used, st = O.zig256_scripted([n_r, V, dbl(m1), dbl(m2)], 1)
    assert v[0] == T256["ox"][b] + T256["odx"][b] * (((1 << 53) - m1) * 2.0 ** -53)


# ---- rates -----------------------------------------------------------------

def test_zig128_branch_rates_and_iterations():
    k = np.array(T128["k"], dtype=np.float64) / 2 ** 24
    p_fast = k.sum() / 128
    p_wedge = (1 - k[:127]).sum() / 128
    p_tail = (1 - k[127]) / 128
    mu = 128 * T128["v"] / math.sqrt(math.pi / 2)
    seeds = 0x5EED + np.arange(256, dtype=np.uint64)
    out, _, st = O.generate("splitmix64", "zig128", seeds, uniform_len=1 << 15)
    n_it, n_var = st["iters"], len(out)
    for p, c in ((p_fast, st["fast"]), (p_wedge, st["wedge"]), (p_tail, st["tail"])):
        sd = math.sqrt(p * (1 - p) / n_it)
        assert abs(c / n_it - p) < 5 * sd, (p, c / n_it)
    sd = math.sqrt(mu * (mu - 1) / n_var)
    assert abs(n_it / n_var - mu) < 5 * sd
    # tail acceptance = exact tail area / envelope tail area f(R)/R
    R = T128["R"]
    p_acc = math.sqrt(math.pi / 2) * math.erfc(R / math.sqrt(2)) / (math.exp(-R * R / 2) / R)
    sd = math.sqrt(p_acc * (1 - p_acc) / st["tail"])
    assert abs(st["tail_acc"] / st["tail"] - p_acc) < 5 * sd


def test_polar_acceptance():
    out, _, st = O.generate("splitmix64", "polar", SEEDS64, uniform_len=1 << 14)
    p = math.pi / 4
    n = st["polar_tries"]
    sd = math.sqrt(p * (1 - p) / n)
    assert abs(st["polar_pairs"] / n - p) < 5 * sd
    assert st["polar_pairs"] * 2 == len(out)


def test_zig256_slot_rates():
    out, _, st = O.generate("splitmix64", "zig256", SEEDS64, uniform_len=1 << 15)
    p = T256["n_r"] / 256
    n = st["iters"]
    assert n == len(out)
    assert abs(st["fast"] / n - p) < 5 * math.sqrt(p * (1 - p) / n)
    # tail share of the slow path from the alias table (region 0)
    thr = np.array(T256["thr"], dtype=np.float64) / 2.0 ** 56
    p0 = (thr[0] + sum(1 - thr[b] for b in range(256) if T256["alias"][b] == 0)) / 256
    ns = st["slow"]
    assert abs(st["tail"] / ns - p0) < 5 * math.sqrt(p0 * (1 - p0) / ns) + 1e-9


# ---- distribution ----------------------------------------------------------

COMBOS = [(p, a) for p in O.PRNGS for a in O.ALGS]


@pytest.mark.parametrize("prng,alg", COMBOS)
def test_distribution_config1_shape(prng, alg):
    """64 streams x 16,384 variates, seeds 0x5EED + s (the small correctness workload)."""
    z, _, _ = O.generate(prng, alg, SEEDS64, uniform_len=16384)
    n = len(z)
    assert n == 1 << 20
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(stats.skew(z)) < 5 * math.sqrt(6 / n)
    assert abs(stats.kurtosis(z)) < 5 * math.sqrt(24 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    edges = stats.norm.ppf(np.linspace(0, 1, 1001)[1:-1])
    counts = np.bincount(np.searchsorted(edges, z), minlength=1000)
    assert stats.chisquare(counts).pvalue > 1e-4


@pytest.mark.parametrize("prng,alg", [("splitmix64", "zig128"), ("lcg48", "zig128"),
                                      ("l64x128mix", "zig256")])
def test_tail_mass(prng, alg):
    """2^26 variates: mass beyond |x| > 3 and > R, and the shape of the tail beyond R."""
    R = T128["R"]
    n_tot, c3, cR, tail = 0, 0, 0, []
    for part in range(4):
        seeds = 0x5EED + (part << 14) + np.arange(1 << 14, dtype=np.uint64)
        z, _, _ = O.generate(prng, alg, seeds, uniform_len=1 << 10)
        a = np.abs(z)
        n_tot += len(z)
        c3 += int((a > 3).sum())
        cR += int((a > R).sum())
        tail.append(a[a > R])
    for thr, c in ((3.0, c3), (R, cR)):
        p = math.erfc(thr / math.sqrt(2))
        sd = math.sqrt(p * (1 - p) / n_tot)
        assert abs(c / n_tot - p) < 5 * sd, (thr, c / n_tot, p)
    tail = np.concatenate(tail)
    sfR = stats.norm.sf(R)
    cdf = lambda x: 1 - stats.norm.sf(x) / sfR
    assert stats.kstest(tail, cdf).pvalue > 1e-4


# ---- driver ----------------------------------------------------------------

def test_chunked_driver():
    seeds = 0x5EED + np.arange(8, dtype=np.uint64)
    lengths = np.array([1, 5, 1024, 3000, 0, 2049, 17, 1023], dtype=np.uint64)
    for prng in O.PRNGS:
        seq, _, _ = O.generate(prng, "zig128", seeds, lengths=lengths)
        ch, _, _ = O.generate(prng, "zig128", seeds, lengths=lengths, chunk_log2=10)
        off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
        for s, L in enumerate(lengths.astype(np.int64)):
            a, b = seq[off[s]:off[s + 1]], ch[off[s]:off[s + 1]]
            n0 = min(L, 1024)
            assert np.array_equal(a[:n0], b[:n0])           # chunk 0 is the plain stream
            if L > 1024:
                assert not np.array_equal(a[1024:], b[1024:])
        # a prefix of a chunked stream does not depend on its length
        short = lengths.copy()
        short[3] = 2048
        ch2, _, _ = O.generate(prng, "zig128", seeds, lengths=short, chunk_log2=10)
        off2 = np.concatenate([[0], np.cumsum(short)]).astype(np.int64)
        assert np.array_equal(ch2[off2[3]:off2[4]], ch[off[3]:off[3] + 2048])


def test_chunk_starts_at_jump_2_pow_32():
    """Chunk q begins at the seeded state advanced by exactly q * 2^32 raw steps."""
    k, w = T128["k"], T128["w"]
    seeds = 0x5EED + np.arange(32, dtype=np.uint64)
    lengths = np.full(32, 3 * 1024, dtype=np.uint64)
    checked = 0
    for prng in O.PRNGS:
        ch, _, _ = O.generate(prng, "zig128", seeds, lengths=lengths, chunk_log2=10)
        for q in (1, 2):
            u = O.prng_fill(prng, seeds, 1, kind="u32", skip=q << 32)[:, 0]
            for s in range(32):
                word = int(u[s])
                i, j = word & 0x7F, (word >> 8) & 0xFFFFFF
                if j < k[i]:                                   # first draw lands on the fast path
                    want = j * w[i] * (1.0 if word & 0x80 else -1.0)
                    assert ch[s * 3072 + q * 1024] == want
                    checked += 1
    assert checked > 150


def test_margins_reported():
    z, m, st = O.generate("lcg48", "zig128", SEEDS64[:4], uniform_len=4096, with_margins=True)
    assert np.isinf(m).sum() > 0.97 * len(z)
    # a variate has a finite margin iff at least one exp test was taken for it
    n_fin = int(np.isfinite(m).sum())
    assert st["wedge_acc"] + st["tail_acc"] <= n_fin <= st["wedge"] + st["tail"]
    assert np.min(m) == st["min_margin"]


def test_round_helpers():
    one = np.float64(1.0)
    assert O.round_bf16_bits(np.array([1.0]))[0] == 0x3F80
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1.0
    assert O.round_bf16_bits(np.array([1 + 2.0 ** -8]))[0] == 0x3F80
    assert O.round_bf16_bits(np.array([1 + 3 * 2.0 ** -8]))[0] == 0x3F82
    assert O.round_bf16_bits(np.array([-2.5]))[0] == 0xC020
    # above a tie by one binary64 ulp rounds up (no double rounding through binary32)
    x = 1 + 2.0 ** -8 + 2.0 ** -52
    assert O.round_bf16_bits(np.array([x]))[0] == 0x3F81
    assert np.float32(x) == np.float32(1 + 2.0 ** -8)       # the binary32 detour would tie
    z = np.array([0.0, -0.0])
    assert list(O.round_bf16_bits(z)) == [0x0000, 0x8000]
    r = np.random.default_rng(1).standard_normal(10000)
    back = O.bf16_bits_to_f64(O.round_bf16_bits(r))
    assert np.all(np.abs(back - r) <= np.abs(r) * 2.0 ** -8)
    del one
