"""Plain, slow, serial CPU oracle for bulk N(0,1) generation.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call, link or execute anything under ``oracle/``.  The product path (the CUDA
library ``libzig_gb300.so`` and its Python binding) never does, and fails
loudly when its own extension is missing.

Layout:
  zig_oracle.c   the samplers and PRNGs (C99, -O2 -ffp-contract=off, libm)
  tables.py      the table geometry at 50 digits (mpmath)
  gen_tables.py  writes tables/zig128.txt and tables/zig256.txt from tables.py
  tables/*.txt   the stored tables (read here; the GPU machine has no mpmath)

Parity status of each function (what pins it) is listed in the tests:
  tests/test_oracle_prng.py, test_oracle_tables.py, test_oracle_sampler.py.
Parity with the JDK and with GSL is unpinned (neither is available); the
oracle follows the definitions in zig_oracle.c's header.
"""

from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "zig_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
TABLE_DIR = os.path.join(HERE, "tables")

PRNGS = {"lcg48": 0, "splitmix64": 1, "l64x128mix": 2, "xoroshiro128pp": 3}
ALGS = {"zig128": 0, "polar": 1, "zig256": 2}
FILL_KINDS = {"u32": 0, "u64": 1, "m53": 2}


class Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "draws", "iters", "fast", "wedge", "tail", "wedge_acc", "tail_acc",
        "slow", "overhang", "overhang_quick", "overhang_acc", "tail_tries",
        "polar_pairs", "polar_tries")] + [("min_margin", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lock = threading.Lock()
_lib = None
_tabs = {}


def lib_path() -> str:
    return os.path.join(BUILD_DIR, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile zig_oracle.c with gcc (no FMA contraction).  Returns the .so path."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        u64p = C.POINTER(C.c_uint64)
        dp = C.POINTER(C.c_double)
        lib.orc_generate.argtypes = [C.c_int, C.c_int, u64p, u64p, C.c_uint64, C.c_uint64,
                                     C.c_uint32, C.c_void_p, C.c_void_p, dp, dp,
                                     C.POINTER(C.c_uint8), C.POINTER(Stats)]
        lib.orc_generate.restype = C.c_int
        lib.orc_prng_fill.argtypes = [C.c_int, u64p, C.c_uint64, C.c_uint64, C.c_uint64,
                                      C.c_int, u64p]
        lib.orc_prng_fill.restype = C.c_int
        lib.orc_zig128_tab_size.restype = C.c_size_t
        lib.orc_zig256_tab_size.restype = C.c_size_t
        lib.orc_prng_size.restype = C.c_size_t
        lib.orc_zig128_tab_set.argtypes = [C.c_void_p, C.c_double, C.POINTER(C.c_uint32), dp, dp]
        lib.orc_zig256_tab_set.argtypes = [C.c_void_p, C.c_int, C.c_double, dp, dp, dp, dp, dp,
                                           C.POINTER(C.c_int), u64p, u64p, C.POINTER(C.c_int)]
        lib.orc_zig128_scripted.argtypes = [u64p, C.c_uint64, C.c_void_p, C.c_uint64, dp,
                                            C.POINTER(Stats)]
        lib.orc_zig128_scripted.restype = C.c_int64
        lib.orc_zig256_scripted.argtypes = [u64p, C.c_uint64, C.c_void_p, C.c_uint64, dp,
                                            C.POINTER(Stats)]
        lib.orc_zig256_scripted.restype = C.c_int64
        lib.orc_seed.argtypes = [C.c_void_p, C.c_int, C.c_uint64]
        lib.orc_next_u32.argtypes = [C.c_void_p, C.c_void_p]
        lib.orc_next_u32.restype = C.c_uint32
        lib.orc_next_u64.argtypes = [C.c_void_p, C.c_void_p]
        lib.orc_next_u64.restype = C.c_uint64
        lib.orc_next_m53.argtypes = [C.c_void_p, C.c_void_p]
        lib.orc_next_m53.restype = C.c_uint64
        lib.orc_next_double.argtypes = [C.c_void_p, C.c_void_p]
        lib.orc_next_double.restype = C.c_double
        lib.orc_polar_next.argtypes = [C.c_void_p, C.c_void_p]
        lib.orc_polar_next.restype = C.c_double
        lib.orc_jump_n.argtypes = [C.c_void_p, C.c_uint64]
        lib.orc_state_get.argtypes = [C.c_void_p, u64p]
        _lib = lib
        return lib


# ---------------------------------------------------------------------------
# stored tables
# ---------------------------------------------------------------------------

def read_zig128(path=None) -> dict:
    path = path or os.path.join(TABLE_DIR, "zig128.txt")
    k, w, y = [], [], []
    R = v = None
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            if p[0] == "R":
                R = float.fromhex(p[1])
            elif p[0] == "v":
                v = float.fromhex(p[1])
            else:
                assert int(p[0]) == len(k)
                k.append(int(p[1]))
                w.append(float.fromhex(p[2]))
                y.append(float.fromhex(p[3]))
    assert len(k) == 128
    return {"R": R, "v": v, "k": k, "w": w, "y": y}


def read_zig256(path=None) -> dict:
    path = path or os.path.join(TABLE_DIR, "zig256.txt")
    t = {"xs": [], "ox": [0.0], "odx": [0.0], "oy": [0.0], "ody": [0.0], "kind": [0],
         "qa": [0], "thr": [], "alias": []}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            if p[0] == "n_r":
                t["n_r"] = int(p[1])
            elif p[0] == "x0":
                t["x0"] = float.fromhex(p[1])
            elif p[0] == "xs":
                t["xs"].append(float.fromhex(p[2]))
            elif p[0] == "oh":
                for key, val in zip(("ox", "odx", "oy", "ody"), p[2:6]):
                    t[key].append(float.fromhex(val))
                t["kind"].append(int(p[6]))
                t["qa"].append(int(p[7]))
            elif p[0] == "al":
                t["thr"].append(int(p[2]))
                t["alias"].append(int(p[3]))
    return t


def _tab128():
    if "128" not in _tabs:
        lib = load()
        t = read_zig128()
        buf = C.create_string_buffer(lib.orc_zig128_tab_size())
        k = (C.c_uint32 * 128)(*t["k"])
        w = (C.c_double * 128)(*t["w"])
        y = (C.c_double * 128)(*t["y"])
        lib.orc_zig128_tab_set(buf, t["R"], k, w, y)
        _tabs["128"] = buf
    return _tabs["128"]


def _tab256():
    if "256" not in _tabs:
        lib = load()
        t = read_zig256()
        n = t["n_r"]
        buf = C.create_string_buffer(lib.orc_zig256_tab_size())
        D = C.c_double
        lib.orc_zig256_tab_set(
            buf, n, t["x0"], (D * n)(*t["xs"]), (D * (n + 1))(*t["ox"]),
            (D * (n + 1))(*t["odx"]), (D * (n + 1))(*t["oy"]), (D * (n + 1))(*t["ody"]),
            (C.c_int * (n + 1))(*t["kind"]), (C.c_uint64 * (n + 1))(*t["qa"]),
            (C.c_uint64 * 256)(*t["thr"]), (C.c_int * 256)(*t["alias"]))
        _tabs["256"] = buf
    return _tabs["256"]


# ---------------------------------------------------------------------------
# calls
# ---------------------------------------------------------------------------

def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(C.POINTER(C.c_uint64))


def generate(prng: str, alg: str, seeds, lengths=None, uniform_len: int = 0,
             chunk_log2: int = 0, with_margins: bool = False, with_via_log: bool = False):
    """Bulk FP64 variates, stream-major packed.  Returns (out, margins|None, stats), or with
    with_via_log (out, margins|None, stats, via_log): per output 1 when its value was computed
    through log (a tail value; every polar value), else 0."""
    lib = load()
    seeds, sp = _u64(seeds)
    n = len(seeds)
    if lengths is not None:
        lengths, lp = _u64(lengths)
        total = int(lengths.sum())
    else:
        lp = None
        total = n * int(uniform_len)
    out = np.empty(total, dtype=np.float64)
    margins = np.empty(total, dtype=np.float64) if with_margins else None
    via_log = np.empty(total, dtype=np.uint8) if with_via_log else None
    st = Stats()
    rc = lib.orc_generate(
        PRNGS[prng], ALGS[alg], sp, lp, int(uniform_len), n, int(chunk_log2),
        _tab128() if alg == "zig128" else None, _tab256() if alg == "zig256" else None,
        out.ctypes.data_as(C.POINTER(C.c_double)),
        margins.ctypes.data_as(C.POINTER(C.c_double)) if with_margins else None,
        via_log.ctypes.data_as(C.POINTER(C.c_uint8)) if with_via_log else None,
        C.byref(st))
    if rc != 0:
        raise ValueError("orc_generate rejected its arguments")
    if with_via_log:
        return out, margins, st.as_dict(), via_log
    return out, margins, st.as_dict()


def prng_fill(prng: str, seeds, n: int, kind: str = "u32", skip: int = 0) -> np.ndarray:
    """Raw draws: array [n_streams, n] of uint64 (u32 values zero-extended)."""
    lib = load()
    seeds, sp = _u64(seeds)
    out = np.empty((len(seeds), n), dtype=np.uint64)
    rc = lib.orc_prng_fill(PRNGS[prng], sp, len(seeds), n, int(skip), FILL_KINDS[kind],
                           out.ctypes.data_as(C.POINTER(C.c_uint64)))
    if rc != 0:
        raise ValueError("orc_prng_fill rejected its arguments")
    return out


class Generator:
    """One oracle PRNG object (for the pin tests)."""

    def __init__(self, prng: str, seed: int):
        self._lib = load()
        self._buf = C.create_string_buffer(self._lib.orc_prng_size())
        self._lib.orc_seed(self._buf, PRNGS[prng], C.c_uint64(seed & (2**64 - 1)))

    def next_u32(self) -> int:
        return self._lib.orc_next_u32(self._buf, None)

    def next_int(self) -> int:
        """Java nextInt() as a signed value."""
        u = self.next_u32()
        return u - (1 << 32) if u >= (1 << 31) else u

    def next_u64(self) -> int:
        return self._lib.orc_next_u64(self._buf, None)

    def next_m53(self) -> int:
        return self._lib.orc_next_m53(self._buf, None)

    def next_double(self) -> float:
        return self._lib.orc_next_double(self._buf, None)

    def next_gaussian_polar(self) -> float:
        st = Stats()
        return self._lib.orc_polar_next(self._buf, C.byref(st))

    def jump(self, n: int) -> None:
        self._lib.orc_jump_n(self._buf, C.c_uint64(n))

    def state(self):
        out = (C.c_uint64 * 4)()
        self._lib.orc_state_get(self._buf, out)
        return tuple(out)


def zig128_scripted(words, n: int):
    """Run the 128-level sampler on chosen words.  Returns (values, words_used, stats)."""
    lib = load()
    words, wp = _u64(words)
    out = np.empty(n, dtype=np.float64)
    st = Stats()
    used = lib.orc_zig128_scripted(wp, len(words), _tab128(), n,
                                   out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st))
    return out, used, st.as_dict()


def zig256_scripted(words, n: int):
    lib = load()
    words, wp = _u64(words)
    out = np.empty(n, dtype=np.float64)
    st = Stats()
    used = lib.orc_zig256_scripted(wp, len(words), _tab256(), n,
                                   out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st))
    return out, used, st.as_dict()


# ---------------------------------------------------------------------------
# rounding of oracle FP64 values to the narrower output types
# ---------------------------------------------------------------------------

def round_f32(x: np.ndarray) -> np.ndarray:
    """RN-even binary64 -> binary32 (numpy's cast rounds to nearest even)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def round_bf16_bits(x: np.ndarray) -> np.ndarray:
    """RN-even binary64 -> bfloat16, returned as uint16 bit patterns.

    Rounds the binary64 value directly to 8 significant bits (no detour through
    binary32, so there is no double rounding).  Finite inputs of normal range only.
    """
    x = np.asarray(x, dtype=np.float64)
    b = x.view(np.uint64)
    sign = (b >> np.uint64(63)).astype(np.uint64)
    mag = b & np.uint64(0x7FFFFFFFFFFFFFFF)
    # keep 7 fraction bits out of 52: drop 45 bits with RN-even
    drop = np.uint64(45)
    q = mag >> drop
    rem = mag & np.uint64((1 << 45) - 1)
    half = np.uint64(1 << 44)
    up = (rem > half) | ((rem == half) & ((q & np.uint64(1)) == np.uint64(1)))
    q = q + up.astype(np.uint64)
    # q now holds (exp64 << 7) | frac7 with exp64 the binary64 biased exponent
    e64 = (q >> np.uint64(7)).astype(np.int64)
    frac = (q & np.uint64(0x7F)).astype(np.uint64)
    e16 = e64 - 1023 + 127
    zero = mag == 0
    if np.any(~zero & ((e16 <= 0) | (e16 >= 255))):
        raise ValueError("round_bf16_bits: value outside the bfloat16 normal range")
    e16 = np.where(zero, 0, e16).astype(np.uint64)
    frac = np.where(zero, np.uint64(0), frac)
    bits = (sign << np.uint64(15)) | (e16 << np.uint64(7)) | frac
    return bits.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(
        np.float32).astype(np.float64)
