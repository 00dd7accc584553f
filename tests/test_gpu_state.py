"""Streams that continue across calls (stream records on the device).

The paper's call draws each variate from a generator object the caller keeps
(Sec. 2, Listing 2).  With records, L1 outputs and then L2 outputs of a stream
must be exactly the first L1 + L2 outputs of that stream taken in one call, for
every transform, generator and dtype, including the polar method's pending
second variate and the binary64 kernel's rewinding of draws it took ahead.
"""

import numpy as np
import pytest

import oracle as O
from paper_2405_19493_gb300 import workloads as W
from tests.parity import compare_streams, offsets_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRNGS = ["lcg48", "splitmix64", "l64x128mix", "xoroshiro128pp"]
INT_VIEW = {"f64": torch.int64, "f32": torch.int32, "bf16": torch.int16}
TDT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    return Z


def dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def stateless(Z, prng, alg, seeds, lengths, dtype):
    out = torch.empty(int(lengths.sum()), dtype=TDT[dtype], device="cuda")
    Z.zig_generate(prng, alg, dev_u64(seeds), out, lengths=dev_u64(lengths), dtype=dtype)
    return out


def split_then_join(Z, prng, alg, seeds, parts, dtype):
    """Generate parts[0], parts[1], ... (arrays of per-stream lengths) with records; return
    the per-stream concatenation in stream-major packed order."""
    n = len(seeds)
    st = Z.zig_state_new(n)
    Z.zig_state_init(prng, dev_u64(seeds), st)
    outs = []
    for L in parts:
        o = torch.empty(max(int(L.sum()), 1), dtype=TDT[dtype], device="cuda")
        Z.zig_generate_state(prng, alg, st, o, n, lengths=dev_u64(L), dtype=dtype)
        outs.append((o, offsets_of(L), L))
    torch.cuda.synchronize()
    host = [(o.view(INT_VIEW[dtype]).cpu().numpy(), off, L) for o, off, L in outs]
    joined = []
    for s in range(n):
        for h, off, L in host:
            joined.append(h[int(off[s]):int(off[s] + L[s])])
    return np.concatenate(joined), st


@pytest.mark.parametrize("prng", PRNGS)
@pytest.mark.parametrize("alg", ["zig128", "polar", "zig256"])
def test_n_then_m_equals_n_plus_m_f64(Z, prng, alg):
    rng = np.random.default_rng(11 + PRNGS.index(prng))
    n = 700   # several warps of streams, a ragged last group
    seeds = W.seeds(n, base=0xC0 + 97 * PRNGS.index(prng))
    L1 = rng.integers(0, 700, n).astype(np.uint64)
    L2 = rng.integers(0, 700, n).astype(np.uint64)
    L3 = rng.integers(0, 40, n).astype(np.uint64)
    L1[:5] = [0, 1, 31, 32, 33]             # empty, single, around a batch's width
    L2[:5] = [5, 0, 1, 2, 63]
    got, st = split_then_join(Z, prng, alg, seeds, [L1, L2, L3], "f64")
    ref = stateless(Z, prng, alg, seeds, L1 + L2 + L3, "f64").view(torch.int64).cpu().numpy()
    assert np.array_equal(got, ref)
    rec = Z.zig_state_read(st, n)
    assert all(r["prng"] == Z._binding.PRNG[prng] for r in rec)
    if alg != "polar":
        assert not any(r["polar_have"] for r in rec)


@pytest.mark.parametrize("alg", ["zig128", "polar", "zig256"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_n_then_m_equals_n_plus_m_narrow(Z, alg, dtype):
    for k, prng in enumerate(PRNGS):
        rng = np.random.default_rng(50 + k)
        n = 300
        seeds = W.seeds(n, base=0xD0 + k)
        L1 = rng.integers(0, 3000, n).astype(np.uint64)
        L2 = rng.integers(0, 3000, n).astype(np.uint64)
        got, _ = split_then_join(Z, prng, alg, seeds, [L1, L2], dtype)
        ref = stateless(Z, prng, alg, seeds, L1 + L2, dtype).view(INT_VIEW[dtype]).cpu().numpy()
        assert np.array_equal(got, ref), prng


@pytest.mark.parametrize("prng", PRNGS)
def test_continued_streams_equal_the_oracle(Z, prng):
    # many short calls on uniform lengths; the joined streams against the oracle
    n, calls, L = 96, 7, 45
    seeds = W.seeds(n, base=0xE0 + PRNGS.index(prng))
    st = Z.zig_state_new(n)
    Z.zig_state_init(prng, dev_u64(seeds), st)
    outs = []
    for _ in range(calls):
        o = torch.empty(n * L, dtype=torch.float64, device="cuda")
        Z.zig_generate_state(prng, "zig128", st, o, n, uniform_len=L)
        outs.append(o.view(n, L))
    got = torch.cat(outs, dim=1).reshape(-1).cpu().numpy()
    o, m, _, vl = O.generate(prng, "zig128", seeds, uniform_len=calls * L, with_margins=True,
                             with_via_log=True)
    compare_streams(got, o, m, np.arange(n) * calls * L, np.full(n, calls * L), via_log=vl)


def test_polar_pending_variate_is_kept(Z):
    n = 64
    seeds = W.seeds(n, base=0xF0)
    st = Z.zig_state_new(n)
    Z.zig_state_init("splitmix64", dev_u64(seeds), st)
    o = torch.empty(n * 3, dtype=torch.float64, device="cuda")
    Z.zig_generate_state("splitmix64", "polar", st, o, n, uniform_len=3)   # odd: one pending
    rec = Z.zig_state_read(st, n)
    assert all(r["polar_have"] == 1 for r in rec)
    ref = stateless(Z, "splitmix64", "polar", seeds, np.full(n, 4, dtype=np.uint64), "f64").cpu().numpy()
    assert np.array_equal(np.array([r["polar_cached"] for r in rec]), ref.reshape(n, 4)[:, 3])
    # a call of another transform discards the pending variate
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    Z.zig_generate_state("splitmix64", "zig128", st, z, n, uniform_len=1)
    assert not any(r["polar_have"] for r in Z.zig_state_read(st, n))


def test_record_of_another_generator_is_refused(Z):
    n = 40
    seeds = W.seeds(n, base=0x123)
    st = Z.zig_state_new(n)
    Z.zig_state_init("lcg48", dev_u64(seeds), st)
    before = st.clone()
    out = torch.full((n * 10,), float("nan"), dtype=torch.float64, device="cuda")
    word = torch.zeros(1, dtype=torch.int32, device="cuda")
    Z.zig_generate_state("splitmix64", "zig128", st, out, n, uniform_len=10, status=word)
    torch.cuda.synchronize()
    assert Z.zig_status_decode(int(word.item())) == 1
    assert torch.equal(st, before)                       # no record advanced
    assert torch.isnan(out).all()                        # nothing written


def fmaf_ref(x, sigma, z):
    """RN_binary32(x + sigma z) with one rounding, as fmaf computes it on the device.

    sigma z is exact in binary64 (24 + 24 significant bits) and x + sigma z = s + e
    exactly (TwoSum); rounding s to binary32 is the single rounding except when s is
    exactly halfway between two binary32 values and e != 0, which e's sign decides.
    """
    x64 = x.astype(np.float64)
    p = np.float64(np.float32(sigma)) * z.astype(np.float64)
    s = x64 + p
    bb = s - x64
    e = (x64 - (s - bb)) + (p - bb)
    f = s.astype(np.float32)
    f64 = f.astype(np.float64)
    up = f64 < s
    other = np.where(up, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf)))
    mid = (f64 + other.astype(np.float64)) / 2
    tie = (f64 != s) & (s == mid) & (e != 0)
    toward = np.where((e > 0) == (other.astype(np.float64) > f64), other, f)
    return np.where(tie, toward, f)


@pytest.mark.parametrize("prng", ["splitmix64", "l64x128mix"])
def test_mutate_state_twice_is_one_stream_of_2L(Z, prng):
    P, L, sigma = 37, 1500, 0.3   # rows longer than the stateless mutation's 1024-output chunks
    seeds = np.array([99 + p for p in range(P)], dtype=np.uint64)
    st = Z.zig_state_new(P)
    Z.zig_state_init(prng, dev_u64(seeds), st)
    x0 = torch.randn(P, L, generator=torch.Generator().manual_seed(3)).float().cuda()
    x = x0.clone()
    Z.zig_mutate_state(x, sigma, P, L, st, prng=prng)
    Z.zig_mutate_state(x, sigma, P, L, st, prng=prng)
    z = stateless(Z, prng, "zig128", seeds, np.full(P, 2 * L, dtype=np.uint64), "f32").view(P, 2 * L)
    zc = z.cpu().numpy()
    ref = fmaf_ref(fmaf_ref(x0.cpu().numpy(), sigma, zc[:, :L]), sigma, zc[:, L:])
    assert np.array_equal(x.cpu().numpy().view(np.int32), ref.view(np.int32))
    # the batched form with records continues the same streams
    st2 = Z.zig_state_new(P)
    Z.zig_state_init(prng, dev_u64(seeds), st2)
    xb = x0.clone()
    Z.zig_mutate_batch([(xb, sigma, 0, "mutate", st2)], prng=prng)
    Z.zig_mutate_batch([(xb, sigma, 0, "mutate", st2)], prng=prng)
    assert torch.equal(xb, x)
    # and generation requests with records return the stream itself
    st3 = Z.zig_state_new(P)
    Z.zig_state_init(prng, dev_u64(seeds), st3)
    g = torch.empty(P, L, device="cuda")
    Z.zig_mutate_batch([(g, 0.0, 0, "generate", st3)], prng=prng)
    assert torch.equal(g, z[:, :L])
    Z.zig_mutate_batch([(g, 0.0, 0, "generate", st3)], prng=prng)
    assert torch.equal(g, z[:, L:])


def test_server_population_continues_its_streams(Z):
    from paper_2405_19493_gb300.serving import MutationServer
    P, L, sigma, seed = 64, 700, 0.25, 4242
    seeds = np.array([seed + p for p in range(P)], dtype=np.uint64)
    z = stateless(Z, "splitmix64", "zig128", seeds, np.full(P, 3 * L, dtype=np.uint64), "f32").view(P, 3 * L)
    x0 = torch.randn(P, L, generator=torch.Generator().manual_seed(5)).float().cuda()
    with MutationServer(device=0, prng="splitmix64", budget_bytes=1 << 30, n_slots=4, max_batch=8) as srv:
        pop = srv.population(P, seed)
        other = srv.population(P, seed + 1000)
        x = x0.clone()
        y = torch.zeros(P, L, device="cuda")
        g = torch.empty(P, L, device="cuda")
        t = [srv.submit_population(pop, x, sigma),
             srv.submit_population(other, y, 1.0),
             srv.submit_population(pop, x, sigma),
             srv.submit_population(pop, g, kind="generate")]
        for k in t:
            srv.wait(k, timeout_s=60)
        srv.release_population(pop)
        srv.release_population(other)
    zc = z.cpu().numpy()
    ref = fmaf_ref(fmaf_ref(x0.cpu().numpy(), sigma, zc[:, :L]), sigma, zc[:, L:2 * L])
    assert np.array_equal(x.cpu().numpy().view(np.int32), ref.view(np.int32))
    assert torch.equal(g, z[:, 2 * L:])


@pytest.mark.parametrize("prng", PRNGS)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_records_at_a_batch_end(Z, prng, dtype):
    # A batch takes 32 draws (31 for LCG48) and the draws a slow candidate needs past
    # them go to the row's spare slots.  With a first call as long as one batch, about
    # one stream in a hundred ends it on a slow candidate in the batch's last slot,
    # whose uniforms lie past the 32 stored slots; the record must account for them.
    n = 1 << 16
    L1 = 31 if prng == "lcg48" else 32
    seeds = W.seeds(n, base=0x3A7 + 11 * PRNGS.index(prng))
    a = np.full(n, L1, dtype=np.uint64)
    b = np.full(n, 50, dtype=np.uint64)
    got, _ = split_then_join(Z, prng, "zig128", seeds, [a, b], dtype)
    ref = stateless(Z, prng, "zig128", seeds, a + b, dtype).view(INT_VIEW[dtype]).cpu().numpy()
    assert np.array_equal(got, ref)
