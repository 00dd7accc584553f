"""zig_generate_noalloc: variable-length generation that allocates nothing.

Some callers cannot allocate device memory when they call the library: a
service that has already divided HBM into its own pools, or a latency-bound
loop that cannot absorb the device synchronization a cudaMalloc implies.  For
them the library keeps the variable-length path's scratch in a fixed array it
owns, so the call allocates nothing.  This file checks, through the C ABI,
that two such calls in a row (the second reusing the array the first left
behind) give exactly what zig_generate gives for the same inputs, that free
device memory does not move across the calls, and that a batch larger than the
fixed array is refused.  It is collected last on purpose and also runs alone.
"""

import os
import re

import numpy as np
import pytest

from paper_2405_19493_gb300 import workloads as W
from tests.parity import ulp_diff64

torch = pytest.importorskip("torch")


def test_noalloc_limit_matches_header():
    from paper_2405_19493_gb300 import _binding
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "zig.h")
    m = re.search(r"#define ZIG_NOALLOC_MAX_STREAMS (\d+)u", open(hdr).read())
    assert m and int(m.group(1)) == _binding.NOALLOC_MAX_STREAMS


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    return Z


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _case(n, max_log2, seed, base):
    L = W.batched_lengths(n, seed=seed, max_log2=max_log2)
    L[::13] = 0
    return _dev(W.seeds(n, base=base)), _dev(L), int(L.sum())


@pytest.mark.gpu
def test_noalloc_matches_generate_on_two_calls_in_a_row(Z):
    lib = Z.load()
    # call 1: a large batch (chunked); call 2: a smaller one (sequential streams,
    # binary32), which must not see anything call 1 left in the shared array; call 3:
    # the batched modified-ziggurat kernel (binary64, chunked)
    cases = [("l64x128mix", "zig128", 10, "f64", _case(3000, 16, 7, 0x5EED)),
             ("lcg48", "zig256", 0, "f32", _case(700, 12, 8, 0xABC)),
             ("splitmix64", "zig256", 10, "f64", _case(900, 13, 9, 0x123))]
    refs, outs = [], []
    for prng, alg, c, dt, (s, ln, total) in cases:
        tdt = torch.float64 if dt == "f64" else torch.float32
        ref = torch.empty(total, dtype=tdt, device="cuda")
        Z.zig_generate(prng, alg, s, ref, lengths=ln, chunk_log2=c, dtype=dt)
        refs.append(ref)
        outs.append(torch.full((total,), float("nan"), dtype=tdt, device="cuda"))
    torch.cuda.synchronize()
    # the first call on a device resolves the array's address: do it before measuring
    warm = torch.empty(cases[1][4][2], dtype=torch.float32, device="cuda")
    Z.zig_generate_noalloc("lcg48", "zig256", cases[1][4][0], cases[1][4][1], warm, dtype="f32")
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for (prng, alg, c, dt, (s, ln, total)), out in zip(cases, outs):
        st = lib.zig_generate_noalloc(Z._binding.PRNG[prng], Z._binding.ALG[alg], s.data_ptr(),
                                      ln.data_ptr(), s.numel(), c, Z._binding.DTYPE[dt],
                                      out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == 0, Z.zig_status_string(st)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    for (prng, alg, c, dt, _), ref, out in zip(cases, refs, outs):
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        if dt == "f64":
            assert int(ulp_diff64(o, r).max(initial=0)) == 0
        else:
            assert np.array_equal(o.view(np.uint32), r.view(np.uint32))
    assert Z.zig_device_status(0) == 0


@pytest.mark.gpu
def test_noalloc_refuses_batches_beyond_its_scratch(Z):
    lib = Z.load()
    n = Z._binding.NOALLOC_MAX_STREAMS + 1
    s = _dev(W.seeds(n))
    ln = _dev(np.ones(n, dtype=np.uint64))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    st = lib.zig_generate_noalloc(0, 0, s.data_ptr(), ln.data_ptr(), n, 0, 0, out.data_ptr(), None)
    assert Z.zig_status_string(st) == "ZIG_ERR_TOO_LARGE"
    with pytest.raises(Z.ZigError):
        Z.zig_generate_noalloc("lcg48", "zig128", s, ln, out)
    # exactly the maximum is accepted
    m = Z._binding.NOALLOC_MAX_STREAMS
    Z.zig_generate_noalloc("lcg48", "zig128", s[:m], ln[:m], out[:m])
    ref = torch.empty(m, dtype=torch.float64, device="cuda")
    Z.zig_generate("lcg48", "zig128", s[:m], ref, lengths=ln[:m])
    torch.cuda.synchronize()
    assert torch.equal(out[:m].view(torch.int64), ref.view(torch.int64))
