"""The C-ABI boundary on the GPU: scratch, error scope, limits and stream capture.

- Variable-length calls that let the library provide their scratch run at the
  same time on two streams and still equal their serial runs (and the oracle).
- zig_generate_checked latches a call's device-side errors in the caller's own
  word, leaving other callers' words and the device's shared word alone.
- Lengths that sum to 2^40 or more are refused on the device: nothing runs.
- zig_mutate_batch refuses stream capture; a captured variable-length
  generation (its scratch allocated inside the graph) replays bit for bit.
"""

import numpy as np
import pytest

import oracle as O
from paper_2405_19493_gb300 import workloads as W
from tests.parity import compare_streams, offsets_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INVALID = 1


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    return Z


def dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _batch(n, seed, max_log2=16):
    L = W.batched_lengths(n, seed=seed, max_log2=max_log2)
    return W.seeds(n, base=0x5EED + 1000 * seed), L


def test_library_scratch_on_two_streams_at_once(Z):
    (sa, La), (sb, Lb) = _batch(3000, 3), _batch(2500, 4)
    da, db = dev_u64(sa), dev_u64(sb)
    la, lb = dev_u64(La), dev_u64(Lb)
    ref_a = torch.empty(int(La.sum()), dtype=torch.float64, device="cuda")
    ref_b = torch.empty(int(Lb.sum()), dtype=torch.float64, device="cuda")
    Z.zig_generate("splitmix64", "zig128", da, ref_a, lengths=la, chunk_log2=10)
    Z.zig_generate("l64x128mix", "zig128", db, ref_b, lengths=lb, chunk_log2=10)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for rnd in range(3):
        out_a = torch.full_like(ref_a, float("nan"))
        out_b = torch.full_like(ref_b, float("nan"))
        torch.cuda.synchronize()
        for _ in range(2):   # several calls in flight on each stream, none waiting for the other
            Z.zig_generate("splitmix64", "zig128", da, out_a, lengths=la, chunk_log2=10, stream=s1)
            Z.zig_generate("l64x128mix", "zig128", db, out_b, lengths=lb, chunk_log2=10, stream=s2)
        torch.cuda.synchronize()
        assert torch.equal(out_a.view(torch.int64), ref_a.view(torch.int64)), rnd
        assert torch.equal(out_b.view(torch.int64), ref_b.view(torch.int64)), rnd
    assert Z.zig_device_status(0) == 0
    # and the serial runs are the oracle's (sampled streams)
    pick = np.unique(np.concatenate([[0, len(La) - 1], np.argsort(La)[-2:], np.arange(0, len(La), 301)]))
    off = offsets_of(La)
    got = np.concatenate([ref_a[int(off[s]):int(off[s] + La[s])].cpu().numpy() for s in pick])
    o, m, _, vl = O.generate("splitmix64", "zig128", sa[pick], lengths=La[pick], chunk_log2=10,
                             with_margins=True, with_via_log=True)
    compare_streams(got, o, m, offsets_of(La[pick]), La[pick], via_log=vl)


def test_checked_call_has_its_own_error_word(Z):
    Z.zig_device_status(0, clear=True)
    bad_s, bad_l = dev_u64(W.seeds(2)), dev_u64(np.array([0, 3], dtype=np.uint64))
    good_s = dev_u64(W.seeds(64))
    good = torch.empty(64 * 500, dtype=torch.float64, device="cuda")
    st_bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    st_good = torch.zeros(1, dtype=torch.int32, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    # a NULL output for lengths that sum above zero: the device refuses it
    Z.zig_generate_checked("lcg48", "zig128", bad_s, empty, st_bad, lengths=bad_l, stream=s1)
    Z.zig_generate_checked("lcg48", "zig128", good_s, good, st_good, uniform_len=500, stream=s2)
    torch.cuda.synchronize()
    assert Z.zig_status_decode(int(st_bad.item())) == INVALID
    assert Z.zig_status_decode(int(st_good.item())) == 0
    assert Z.zig_device_status(0) == 0   # the shared word saw neither call
    ref = torch.empty_like(good)
    Z.zig_generate("lcg48", "zig128", good_s, ref, uniform_len=500)
    torch.cuda.synchronize()
    assert torch.equal(ref.view(torch.int64), good.view(torch.int64))
    lib = Z.load()
    assert lib.zig_generate_checked(0, 0, good_s.data_ptr(), None, 500, 64, 0, 0, good.data_ptr(),
                                    None, 0, None, None) == INVALID


def test_lengths_summing_to_2_pow_40_are_refused(Z):
    Z.zig_device_status(0, clear=True)
    s = dev_u64(W.seeds(2))
    ln = dev_u64(np.array([1 << 39, 1 << 39], dtype=np.uint64))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    Z.zig_generate_checked("splitmix64", "zig128", s, empty, st, lengths=ln)
    torch.cuda.synchronize()
    assert Z.zig_status_decode(int(st.item())) == INVALID
    assert int(st.item()) & 8   # the length-sum bit
    assert Z.zig_device_status(0) == 0


def test_mutate_batch_refuses_capture(Z):
    x = torch.zeros((4, 100), dtype=torch.float32, device="cuda")
    Z.zig_mutate_batch([(x, 0.5, 7)])   # resolves the launch facts outside capture
    x.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    err = None
    with torch.cuda.stream(st):
        g.capture_begin()
        try:
            Z.zig_mutate_batch([(x, 0.5, 7)], stream=st)
        except Z.ZigError as e:
            err = e
        x.add_(1.0)   # the graph holds this node alone
        g.capture_end()
    assert err is not None and err.status == INVALID
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, torch.ones_like(x))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_captured_variable_length_request_replays_bit_for_bit(Z, dtype):
    seeds, L = _batch(2000, 5, max_log2=15)
    ds, dl = dev_u64(seeds), dev_u64(L)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    idt = torch.int64 if dtype == "f64" else torch.int32
    ref = torch.empty(int(L.sum()), dtype=tdt, device="cuda")
    Z.zig_generate("xoroshiro128pp", "zig128", ds, ref, lengths=dl, chunk_log2=10, dtype=dtype)
    torch.cuda.synchronize()
    out = torch.full_like(ref, float("nan"))
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g.capture_begin()
        # no workspace: the call's scratch is allocated inside the graph
        Z.zig_generate("xoroshiro128pp", "zig128", ds, out, lengths=dl, chunk_log2=10, dtype=dtype,
                       stream=st)
        g.capture_end()
    for _ in range(2):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out.view(idt), ref.view(idt))
    assert Z.zig_device_status(0) == 0
