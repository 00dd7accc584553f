"""The C-ABI library builds, loads and exports every symbol include/zig.h declares (CPU only).

No compute call is made here (there is no GPU): only host-side entry points,
argument validation that returns before touching a device, and the tables.
"""

import os
import re

import numpy as np

import oracle as O
import paper_2405_19493_gb300 as Z
from paper_2405_19493_gb300 import _binding as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "zig.h")


def declared():
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(zig_\w+)\s*\(", txt)))


def test_exports_match_header():
    lib = Z.load()
    names = declared()
    assert names == sorted(B.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n
    assert os.path.dirname(os.path.abspath(B.library_path())).startswith(
        os.path.dirname(os.path.abspath(Z.__file__)))


def test_enums_match_header():
    txt = open(HEADER).read()
    for name, val in re.findall(r"\b(ZIG_\w+)\s*=\s*(\d+)", txt):
        key = name[4:].lower()
        if key in B.PRNG:
            assert B.PRNG[key] == int(val)
        elif key in B.ALG:
            assert B.ALG[key] == int(val)
        elif key in B.DTYPE:
            assert B.DTYPE[key] == int(val)
        elif name.startswith("ZIG_ERR") or name == "ZIG_OK":
            assert B.STATUS_NAMES[int(val)] == name


def test_tables_via_abi_equal_oracle():
    t = Z.zig_tables_get_zig128()
    o = O.read_zig128()
    assert list(t["k"]) == o["k"]
    assert list(t["w"]) == o["w"]
    assert list(t["y"]) == o["y"]
    assert t["R"] == o["R"]
    assert np.all(np.abs(t["w32"].astype(np.float64) - t["w"]) <=
                  np.spacing(t["w32"]).astype(np.float64) / 2)


def test_status_strings_and_version():
    for code, name in B.STATUS_NAMES.items():
        assert Z.zig_status_string(code) == name
    assert Z.zig_version() >= 100


def test_host_side_argument_errors():
    lib = Z.load()
    # bad enum / chunk size are rejected before any device is touched
    assert lib.zig_generate(9, 0, 8, None, 16, 4, 0, 0, 8, None, 0, None) == 1
    assert lib.zig_generate(0, 0, 8, None, 16, 4, 25, 0, 8, None, 0, None) == 1
    assert lib.zig_generate(0, 0, 8, None, 16, 0, 0, 0, 8, None, 0, None) == 0   # no streams: no-op
    assert lib.zig_mutate(None, 1.0, 0, 5, 1, 0, None) == 0                      # empty population
    assert lib.zig_mutate(8, float("nan"), 2, 5, 1, 0, None) == 1
    assert lib.zig_prng_fill(0, 8, 4, 4, 0, 5, 8, None) == 1
    assert Z.zig_generate_workspace_bytes(1000) >= 16 * 1000


def test_launch_config_validation_and_candidates():
    """Launch configurations: defaults, validation, set/reset; no CUDA call."""
    for dt in ("f64", "f32", "bf16"):
        # every output type runs in the batch kernel: the block size (and, for binary64,
        # the share of fma products) is all a configuration chooses
        want = {"block": 640, "batch": 32, "store_bytes": 0, "fma_of_4": 0}
        assert Z.zig_launch_config_get("splitmix64", dt, False, device=5) == want
        cands = Z.zig_autotune_candidates(dt)
        assert {c["batch"] for c in cands} == {32}
        assert {c["block"] for c in cands} == {256, 384, 512, 640}
        assert {c["store_bytes"] for c in cands} == {0}
        bads = [{"block": 672, "batch": 32, "store_bytes": 0},
                {"block": 100, "batch": 32, "store_bytes": 0},
                {"block": 256, "batch": 16, "store_bytes": 0},
                {"block": 256, "batch": 32, "store_bytes": 32}]
        if dt == "f64":
            assert len(cands) == 12
            assert {c["fma_of_4"] for c in cands} == {2, 3, 4}
            bads += [{"block": 256, "batch": 32, "store_bytes": 0, "fma_of_4": 1},
                     {"block": 256, "batch": 32, "store_bytes": 0, "fma_of_4": 5}]
        else:
            assert len(cands) == 4
            assert {c["fma_of_4"] for c in cands} == {0}
            bads += [{"block": 256, "batch": 32, "store_bytes": 0, "fma_of_4": 3}]
        for bad in bads:
            try:
                Z.zig_launch_config_set("lcg48", dt, True, bad, device=5)
                raise AssertionError(f"accepted {bad}")
            except Z.ZigError as e:
                assert e.status == 1
    cfg = {"block": 384, "batch": 32, "store_bytes": 0, "fma_of_4": 3}
    Z.zig_launch_config_set("l64x128mix", "f64", True, cfg, device=5)
    assert Z.zig_launch_config_get("l64x128mix", "f64", True, device=5) == cfg
    assert Z.zig_launch_config_get("l64x128mix", "f64", False, device=5)["block"] == 640
    Z.zig_launch_config_set("l64x128mix", "f64", True, None, device=5)
    assert Z.zig_launch_config_get("l64x128mix", "f64", True, device=5)["batch"] == 32


def test_more_host_side_argument_errors():
    """Limits and malformed requests are refused on the host, before any device call."""
    lib = Z.load()
    INVALID, TOO_LARGE = 1, 8
    P = 0x1000   # an aligned non-null stand-in pointer: never dereferenced on these paths
    # generators beyond the fourth, chunk sizes outside 4..24
    assert lib.zig_generate(4, 0, P, None, 16, 4, 0, 0, P, None, 0, None) == INVALID
    assert lib.zig_generate(0, 0, P, None, 16, 4, 3, 0, P, None, 0, None) == INVALID
    # the output must be aligned to its element size
    assert lib.zig_generate(0, 0, P, None, 16, 4, 0, 0, P + 4, None, 0, None) == INVALID
    assert lib.zig_generate(0, 0, P, None, 16, 4, 0, 1, P + 2, None, 0, None) == INVALID
    # uniform requests of 2^40 elements or more
    assert lib.zig_generate(0, 0, P, None, 1 << 40, 2, 0, 0, P, None, 0, None) == INVALID
    assert lib.zig_generate(0, 0, P, None, (1 << 39) + 1, 2, 0, 0, P, None, 0, None) == INVALID
    # variable-length requests of more than 2^32 streams
    assert lib.zig_generate(0, 0, P, P, 0, (1 << 32) + 1, 0, 0, P, None, 0, None) == INVALID
    # a too small or misaligned caller workspace
    assert lib.zig_generate(0, 0, P, P, 0, 100, 0, 0, P, P, 16, None) == INVALID
    # the no-allocation path refuses batches beyond its fixed scratch first
    assert lib.zig_generate_noalloc(0, 0, P, P, B.NOALLOC_MAX_STREAMS + 1, 0, 0, P, None) == TOO_LARGE
    assert lib.zig_generate_noalloc(0, 0, None, P, 4, 0, 0, P, None) == INVALID
    # mutation: population of 2^40 elements or more, misaligned rows
    assert lib.zig_mutate(P, 0.5, 1 << 20, 1 << 20, 1, 0, None) == INVALID
    assert lib.zig_mutate(P + 2, 0.5, 4, 4, 1, 0, None) == INVALID
    # batches: an unknown request kind, a NaN sigma on a mutation, a too small descriptor area
    reqs = (B.Mutation * 2)(B.Mutation(P, 4, 4, 0.5, 0, 1), B.Mutation(P, 4, 4, 0.5, 2, 2))
    assert lib.zig_mutate_batch(reqs, 2, 0, P, 4096, None) == INVALID
    reqs[1] = B.Mutation(P, 4, 4, float("nan"), 0, 2)
    assert lib.zig_mutate_batch(reqs, 2, 0, P, 4096, None) == INVALID
    reqs[1] = B.Mutation(P, 4, 4, float("nan"), 1, 2)   # generation ignores sigma
    assert lib.zig_mutate_batch(reqs, 2, 0, P, 16, None) == INVALID   # descriptor area too small
    # autotuner and self-check arguments
    assert lib.zig_autotune(0, P, None, 16, 4, 0, 0, P, None, 0, 0, None, None, None) == INVALID
    assert lib.zig_autotune(0, P, None, 16, 4, 0, 0, P, None, 0, 1001, None, None, None) == INVALID
    assert lib.zig_selfcheck(None) == INVALID
    assert lib.zig_filtercheck(None) == INVALID


def test_status_decode_and_table_sizes():
    """Error words decode to statuses; zig_tables_get reports sizes and refuses bad calls."""
    import ctypes as C
    for word, want in ((0, 0), (1, 6), (4, 1), (8, 1), (16, 1), (4 | 1, 1), (8 | 1, 1), (16 | 1, 1)):
        assert Z.zig_status_decode(word) == want
    lib = Z.load()
    n = C.c_size_t(0)
    assert lib.zig_tables_get(0, None, C.byref(n)) == 0 and n.value == C.sizeof(B.Tables128)
    assert lib.zig_tables_get(2, None, C.byref(n)) == 0 and n.value == C.sizeof(B.Tables256)
    assert lib.zig_tables_get(1, None, C.byref(n)) == 0 and n.value == 0
    small = C.c_size_t(16)
    buf = (C.c_uint8 * 16)()
    assert lib.zig_tables_get(0, buf, C.byref(small)) == 1
    assert lib.zig_tables_get(3, None, C.byref(n)) == 1
    assert lib.zig_tables_get(0, None, None) == 1


def test_stream_state_record_layout():
    import ctypes as C
    assert C.sizeof(B.StreamState) == B.STATE_BYTES == 48
    assert B.StreamState.polar_cached.offset == 32 and B.StreamState.prng.offset == 44
    assert C.sizeof(B.Mutation) == 48 and B.Mutation.state_dev.offset == 40
    lib = Z.load()
    # argument errors return before any device work
    assert lib.zig_state_init(9, None, 1, None, None) == 1
    assert lib.zig_generate_state(0, 0, None, None, 4, 4, 0, None, None, 0, None, None) == 1
    assert lib.zig_mutate_state(None, 0.5, 4, 4, None, 0, None) == 1
    assert lib.zig_generate_state(0, 0, 8, None, 4, 4, 0, 64, None, 0, None, None) == 1   # misaligned records
