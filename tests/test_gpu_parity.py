"""GPU parity: the CUDA path (through the C ABI) against the oracle, element by element.

Workload shapes follow the library's measured configurations: 64 streams x
16,384 (seeds 0x5EED + s), the bulk 2^20 x 1,024 launch (sampled streams), the
batched 10,000-stream log-uniform lengths with 2^10 chunks (sampled streams),
plus ragged and degenerate cases.  Tolerances are in tests/parity.py.
"""

import numpy as np
import pytest

import oracle as O
from paper_2405_19493_gb300 import workloads as W
from tests.parity import compare_streams, offsets_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRNGS = ["lcg48", "splitmix64", "l64x128mix", "xoroshiro128pp"]


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    return Z


def dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def gen(Z, prng, alg, seeds, lengths=None, uniform_len=0, chunk_log2=0, dtype="f64"):
    s = dev_u64(seeds)
    ln = dev_u64(lengths) if lengths is not None else None
    total = int(np.sum(lengths)) if lengths is not None else len(seeds) * uniform_len
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    out = torch.empty(max(total, 1), dtype=tdt, device="cuda")[:total]
    Z.zig_generate(prng, alg, s, out, lengths=ln, uniform_len=uniform_len,
                   chunk_log2=chunk_log2, dtype=dtype)
    torch.cuda.synchronize()
    if dtype == "bf16":
        return out.view(torch.int16).cpu().numpy().view(np.uint16)
    return out.cpu().numpy()


def check(Z, prng, alg, seeds, lengths=None, uniform_len=0, chunk_log2=0, dtype="f64"):
    g = gen(Z, prng, alg, seeds, lengths, uniform_len, chunk_log2, dtype)
    o, m, _, vl = O.generate(prng, alg, seeds, lengths=lengths, uniform_len=uniform_len,
                             chunk_log2=chunk_log2, with_margins=True, with_via_log=True)
    L = lengths if lengths is not None else np.full(len(seeds), uniform_len, dtype=np.uint64)
    return compare_streams(g, o, m, offsets_of(L), L, kind=dtype, all_inexact=(alg == "polar"),
                           via_log=vl)


# ---- uniform generators -------------------------------------------------------------

@pytest.mark.parametrize("prng", PRNGS)
@pytest.mark.parametrize("kind", ["u32", "u64", "m53"])
@pytest.mark.parametrize("skip", [0, 3 * 2 ** 32 + 5])
def test_prng_fill_bit_exact(Z, prng, kind, skip):
    seeds = W.seeds(512)
    out = torch.empty((512, 300), dtype=torch.int64, device="cuda")
    Z.zig_prng_fill(prng, dev_u64(seeds), 300, out, skip=skip, kind=kind)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    want = O.prng_fill(prng, seeds, 300, kind=kind, skip=skip)
    assert np.array_equal(got, want)


# ---- the 128-level ziggurat, binary64 ---------------------------------------------------

@pytest.mark.parametrize("prng", PRNGS)
def test_zig128_f64_small_workload(Z, prng):
    rep = check(Z, prng, "zig128", W.seeds(64), uniform_len=16384)
    assert rep.max_ulp <= 4


@pytest.mark.parametrize("prng", PRNGS)
@pytest.mark.parametrize("alg", ["polar", "zig256"])
def test_comparison_transforms_f64(Z, prng, alg):
    rep = check(Z, prng, alg, W.seeds(64), uniform_len=4096)
    assert rep.max_ulp <= 4


@pytest.mark.parametrize("prng", PRNGS)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("alg", ["zig128", "polar", "zig256"])
def test_narrow_outputs(Z, prng, dtype, alg):
    n = 16384 if alg == "zig128" else 2048
    rep = check(Z, prng, alg, W.seeds(64), uniform_len=n, dtype=dtype)
    assert rep.max_ulp <= 1 and rep.flips == 0


def full_size_sampled(Z, prng, alg, dtype="f64", n=1 << 20, L=1024, n_pick=1024):
    """The bulk launch as timed (2^20 streams x 1,024): far more warp groups than
    resident warps, so every lane runs many units; n_pick streams are compared,
    the first and the last among them."""
    seeds = W.seeds(n)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    out = torch.empty(n * L, dtype=tdt, device="cuda")
    Z.zig_generate(prng, alg, dev_u64(seeds), out, uniform_len=L, dtype=dtype)
    pick = np.sort(np.random.default_rng(5).choice(n, n_pick, replace=False))
    pick[0], pick[-1] = 0, n - 1
    rows = out.view(n, L)[torch.from_numpy(pick).cuda()]
    rows = (rows.view(torch.int16).cpu().numpy().view(np.uint16) if dtype == "bf16" else rows.cpu().numpy()).ravel()
    del out
    o, m, _, vl = O.generate(prng, alg, seeds[pick], uniform_len=L, with_margins=True, with_via_log=True)
    Ls = np.full(len(pick), L, dtype=np.uint64)
    return compare_streams(rows, o, m, offsets_of(Ls), Ls, kind=dtype, all_inexact=(alg == "polar"),
                           via_log=vl)


@pytest.mark.parametrize("prng", PRNGS)
def test_bulk_full_size_sampled(Z, prng):
    """The bulk binary64 launch as timed: 2^20 streams x 1,024 (2^30 values)."""
    full_size_sampled(Z, prng, "zig128")


@pytest.mark.parametrize("prng", PRNGS)
def test_zig256_full_size_sampled(Z, prng):
    full_size_sampled(Z, prng, "zig256")


@pytest.mark.parametrize("prng", ["lcg48", "splitmix64"])
def test_polar_full_size_sampled(Z, prng):
    full_size_sampled(Z, prng, "polar", n_pick=256)


@pytest.mark.parametrize("prng", ["splitmix64", "l64x128mix"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_narrow_full_size_sampled(Z, prng, dtype):
    rep = full_size_sampled(Z, prng, "zig128", dtype=dtype)
    assert rep.max_ulp <= 1 and rep.flips == 0


@pytest.mark.parametrize("prng", PRNGS)
def test_zig128_f64_16m_full(Z, prng):
    """2^14 streams x 1,024 (2^24 binary64) compared in full: enough lane batches that
    the rare paths all occur (tails in the last slots of a batch, rows with more than
    three rejected slots, deferred wedges beyond a lane's records)."""
    rep = check(Z, prng, "zig128", W.seeds(1 << 14), uniform_len=1024)
    assert rep.max_ulp <= 4


# ---- variable lengths, chunks, ragged and degenerate inputs -------------------------------

@pytest.mark.parametrize("prng", PRNGS)
@pytest.mark.parametrize("chunk_log2", [0, 10])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_variable_lengths(Z, prng, chunk_log2, dtype):
    L = W.batched_lengths(300, seed=7, max_log2=14)
    L[::17] = 0
    check(Z, prng, "zig128", W.seeds(300), lengths=L, chunk_log2=chunk_log2, dtype=dtype)


@pytest.mark.parametrize("alg", ["zig128", "polar", "zig256"])
def test_uniform_chunked(Z, alg):
    check(Z, "l64x128mix", alg, W.seeds(37), uniform_len=3000, chunk_log2=10)
    check(Z, "lcg48", alg, W.seeds(5), uniform_len=100, chunk_log2=4)


@pytest.mark.parametrize("n,L", [(1, 1), (1, 17), (33, 17), (31, 1), (65, 33), (2, 100003)])
def test_ragged_uniform(Z, n, L):
    check(Z, "splitmix64", "zig128", W.seeds(n), uniform_len=L)


@pytest.mark.parametrize("prng", PRNGS)
@pytest.mark.parametrize("chunk_log2", [0, 10])
def test_zig256_f64_variable_and_ragged(Z, prng, chunk_log2):
    """The batched modified-ziggurat kernel on rows that start inside a 32-byte sector,
    end mid-batch, or are empty."""
    L = W.batched_lengths(300, seed=11, max_log2=13)
    L[::13] = 0
    L[1::7] = 17
    check(Z, prng, "zig256", W.seeds(300), lengths=L, chunk_log2=chunk_log2)
    check(Z, prng, "zig256", W.seeds(33), uniform_len=17)


def test_degenerate_lengths(Z):
    L = np.zeros(50, dtype=np.uint64)
    assert gen(Z, "lcg48", "zig128", W.seeds(50), lengths=L).size == 0
    assert Z.zig_device_status(0) == 0
    # NULL output with lengths that sum above zero: nothing written, error latched
    lib = Z.load()
    s, ln = dev_u64(W.seeds(2)), dev_u64(np.array([0, 3], dtype=np.uint64))
    assert lib.zig_generate(0, 0, s.data_ptr(), ln.data_ptr(), 0, 2, 0, 0, None, None, 0, None) == 0
    assert Z.zig_device_status(0, clear=True) == 1
    assert Z.zig_device_status(0) == 0
    L[[0, 49]] = [3, 5]
    check(Z, "lcg48", "zig128", W.seeds(50), lengths=L)
    L = np.array([0, 0, 1], dtype=np.uint64)
    check(Z, "splitmix64", "zig256", W.seeds(3), lengths=L, chunk_log2=4)


def test_batched_workload_sampled(Z):
    """10,000 streams, lengths log-uniform in [1, 2^20], 2^10 chunks; sampled streams."""
    L = W.batched_lengths()
    seeds = W.seeds(len(L))
    total = int(L.sum())
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    Z.zig_generate("splitmix64", "zig128", dev_u64(seeds), out, lengths=dev_u64(L), chunk_log2=10)
    torch.cuda.synchronize()
    off = offsets_of(L)
    order = np.argsort(L)
    pick = np.unique(np.concatenate([order[:8], order[-3:], order[::800]]))
    got = np.concatenate([out[int(off[s]):int(off[s] + L[s])].cpu().numpy() for s in pick])
    del out
    o, m, _, vl = O.generate("splitmix64", "zig128", seeds[pick], lengths=L[pick], chunk_log2=10,
                             with_margins=True, with_via_log=True)
    compare_streams(got, o, m, offsets_of(L[pick]), L[pick], via_log=vl)


def test_invalid_arguments(Z):
    s = dev_u64(W.seeds(4))
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    lib = Z.load()
    INVALID = 1
    assert lib.zig_generate(7, 0, s.data_ptr(), None, 16, 4, 0, 0, out.data_ptr(), None, 0, None) == INVALID
    assert lib.zig_generate(0, 0, s.data_ptr(), None, 16, 4, 3, 0, out.data_ptr(), None, 0, None) == INVALID
    assert lib.zig_generate(0, 0, s.data_ptr(), None, 16, 4, 0, 0, out.data_ptr() + 4, None, 0, None) == INVALID
    assert lib.zig_generate(0, 0, None, None, 16, 4, 0, 0, out.data_ptr(), None, 0, None) == INVALID
    assert lib.zig_generate(0, 0, s.data_ptr(), None, 16, 0, 0, 0, out.data_ptr(), None, 0, None) == 0
    assert Z.zig_device_status(0) == 0


# ---- mutation -----------------------------------------------------------------------------

@pytest.mark.parametrize("prng", PRNGS)
def test_mutate(Z, prng):
    P, L, sigma, seed = 37, 3001, 0.3, 12345
    x0 = np.random.default_rng(3).standard_normal((P, L)).astype(np.float32)
    x = torch.from_numpy(x0.copy()).cuda()
    Z.zig_mutate(x, sigma, P, L, seed, prng)
    torch.cuda.synchronize()
    got = x.cpu().numpy()
    z, m, _ = O.generate(prng, "zig128", seed + np.arange(P, dtype=np.uint64),
                         uniform_len=L, chunk_log2=10)
    z = z.reshape(P, L)
    want = (np.float64(np.float32(sigma)) * z + x0.astype(np.float64)).astype(np.float32)
    # z enters as binary32 (<= 1 ulp from RN(z)), then one fused multiply-add
    tol = 2 * np.spacing(np.abs(want)) + abs(sigma) * 2 * np.spacing(np.abs(z).astype(np.float32))
    assert np.all(np.abs(got.astype(np.float64) - want) <= tol)


def test_mutate_large_population_sampled(Z):
    """4,096 rows of 40,000: 163,840 units of 2^10 variates, more than the resident warps
    hold at once; 48 rows compared, the first and the last among them."""
    P, L, sigma, seed = 4096, 40000, 0.25, 987654321
    x = torch.zeros((P, L), dtype=torch.float32, device="cuda")
    Z.zig_mutate(x, sigma, P, L, seed, "l64x128mix")
    torch.cuda.synchronize()
    pick = np.sort(np.random.default_rng(9).choice(P, 48, replace=False))
    pick[0], pick[-1] = 0, P - 1
    got = x[torch.from_numpy(pick).cuda()].cpu().numpy().astype(np.float64)
    del x
    z, _, _ = O.generate("l64x128mix", "zig128", np.uint64(seed) + pick.astype(np.uint64),
                         uniform_len=L, chunk_log2=10)
    z = z.reshape(len(pick), L)
    want = np.float64(np.float32(sigma)) * z
    # x starts at 0: fmaf(sigma, z32, 0) = RN32(sigma z32), z32 within 1 ulp of RN32(z)
    tol = 2 * np.spacing(np.abs(want).astype(np.float32)).astype(np.float64) + 1e-45
    assert np.all(np.abs(got - want) <= tol)


def test_device_status_clean(Z):
    assert Z.zig_device_status(0, clear=True) == 0
