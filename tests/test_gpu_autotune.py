"""The 128-level kernel's launch configurations and the autotuner, on the GPU.

Every configuration the autotuner may choose (block size, batch width, store
width) must give exactly the outputs of the default one, and those must match
the oracle.  Cases: the batched form (variable lengths with 2^10 chunks,
ragged lengths, zeros) and a uniform form whose rows start at every alignment.
"""

import numpy as np
import pytest

import oracle as O
from paper_2405_19493_gb300 import workloads as W
from tests.parity import compare_streams, offsets_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
IDT = {"f64": torch.int64, "f32": torch.int32, "bf16": torch.int16}


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    return Z


def dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def run(Z, prng, dtype, seeds, lengths, uniform_len, chunk_log2, cfg):
    variable = lengths is not None
    Z.zig_launch_config_set(prng, dtype, variable, cfg)
    try:
        total = int(lengths.sum().item()) if variable else seeds.numel() * uniform_len
        out = torch.full((total,), float("nan"), dtype=TDT[dtype], device="cuda")
        Z.zig_generate(prng, "zig128", seeds, out, lengths=lengths, uniform_len=uniform_len,
                       chunk_log2=chunk_log2, dtype=dtype)
        torch.cuda.synchronize()
        return out.view(IDT[dtype]).cpu().numpy()
    finally:
        Z.zig_launch_config_set(prng, dtype, variable, None)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("prng", ["lcg48", "splitmix64", "l64x128mix", "xoroshiro128pp"])
def test_every_candidate_gives_the_default_outputs(Z, prng, dtype):
    L = W.batched_lengths(400, seed=7, max_log2=13)
    L[::11] = 0
    L[1::7] = np.arange(len(L[1::7])) % 37     # short rows starting at every alignment
    seeds_np = W.seeds(len(L), base=0x5EED)
    s, ln = dev_u64(seeds_np), dev_u64(L)
    ref = run(Z, prng, dtype, s, ln, 0, 10, None)
    for cfg in Z.zig_autotune_candidates(dtype):
        got = run(Z, prng, dtype, s, ln, 0, 10, cfg)
        assert np.array_equal(got, ref), cfg
    # uniform rows of odd length: every row start has a different alignment
    su = dev_u64(W.seeds(97))
    refu = run(Z, prng, dtype, su, None, 1001, 0, None)
    for cfg in Z.zig_autotune_candidates(dtype):
        assert np.array_equal(run(Z, prng, dtype, su, None, 1001, 0, cfg), refu), cfg
    assert Z.zig_device_status(0) == 0
    # and the default matches the oracle
    o, m, _, vl = O.generate(prng, "zig128", seeds_np, lengths=L, chunk_log2=10, with_margins=True,
                             with_via_log=True)
    g = ref.view({"f64": np.float64, "f32": np.float32, "bf16": np.uint16}[dtype])
    compare_streams(g, o, m, offsets_of(L), L, kind=dtype, via_log=vl)


def test_autotune_records_the_fastest_and_keeps_outputs(Z):
    L = W.batched_lengths(2000, seed=7, max_log2=16)
    s, ln = dev_u64(W.seeds(len(L))), dev_u64(L)
    total = int(L.sum())
    ref = torch.empty(total, dtype=torch.float32, device="cuda")
    Z.zig_generate("splitmix64", "zig128", s, ref, lengths=ln, chunk_log2=10, dtype="f32")
    out = torch.empty_like(ref)
    try:
        cfg, ms = Z.zig_autotune("splitmix64", s, out, lengths=ln, chunk_log2=10, dtype="f32", reps=2)
        torch.cuda.synchronize()
        assert cfg in Z.zig_autotune_candidates("f32") and ms > 0
        assert Z.zig_launch_config_get("splitmix64", "f32", True) == cfg
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
        # zig_generate now launches with the recorded configuration: same outputs
        out.fill_(float("nan"))
        Z.zig_generate("splitmix64", "zig128", s, out, lengths=ln, chunk_log2=10, dtype="f32")
        torch.cuda.synchronize()
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
    finally:
        Z.zig_launch_config_set("splitmix64", "f32", True, None)


def test_autotune_refuses_stream_capture(Z):
    s = dev_u64(W.seeds(64))
    out = torch.empty(64 * 256, dtype=torch.float64, device="cuda")
    Z.zig_generate("lcg48", "zig128", s, out, uniform_len=256)   # warm: opt-ins resolved
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    err = None
    with torch.cuda.stream(st):
        g.capture_begin()
        try:
            Z.zig_autotune("lcg48", s, out, uniform_len=256, reps=1, stream=st)
        except Z.ZigError as e:
            err = e
        Z.zig_generate("lcg48", "zig128", s, out, uniform_len=256, stream=st)
        g.capture_end()
    assert err is not None and err.status == 1
    g.replay()
    torch.cuda.synchronize()
    assert Z.zig_device_status(0) == 0
