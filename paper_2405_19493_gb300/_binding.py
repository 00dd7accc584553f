"""ctypes binding of libzig_gb300 (include/zig.h): argument marshalling only.

Every function named ``zig_*`` here is the C entry point of the same name;
tensors are passed as data pointers and the current torch CUDA stream as the
``cudaStream_t``.  Every step of generation runs in the library's kernels; if
the library cannot be loaded, these calls raise -- there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

ZIG_OK = 0
STATUS_NAMES = {
    0: "ZIG_OK", 1: "ZIG_ERR_INVALID_ARG", 2: "ZIG_ERR_NOT_INITIALIZED", 3: "ZIG_ERR_CUDA",
    4: "ZIG_ERR_BUDGET", 5: "ZIG_ERR_TIMEOUT", 6: "ZIG_ERR_CHUNK_OVERFLOW",
    7: "ZIG_ERR_UNSUPPORTED", 8: "ZIG_ERR_TOO_LARGE",
}
# fixed scratch capacity of zig_generate_noalloc (ZIG_NOALLOC_MAX_STREAMS in include/zig.h)
NOALLOC_MAX_STREAMS = 65536
PRNG = {"lcg48": 0, "splitmix64": 1, "l64x128mix": 2, "xoroshiro128pp": 3}
ALG = {"zig128": 0, "polar": 1, "zig256": 2}
DTYPE = {"f64": 0, "f32": 1, "bf16": 2}
ESIZE = {"f64": 8, "f32": 4, "bf16": 2}
FILL_KIND = {"u32": 0, "u64": 1, "m53": 2}

# every symbol include/zig.h declares
EXPORTS = (
    "zig_tables_init", "zig_tables_get_zig128", "zig_generate", "zig_generate_workspace_bytes",
    "zig_mutate", "zig_prng_fill", "zig_device_status", "zig_status_string", "zig_version",
    "zig_generate_noalloc", "zig_mutate_batch_desc_bytes", "zig_mutate_batch",
    "zig_server_create", "zig_server_submit", "zig_server_wait", "zig_server_query",
    "zig_server_drain", "zig_server_stats", "zig_server_destroy", "zig_server_submit_generate",
    "zig_launch_config_get", "zig_launch_config_set", "zig_autotune_candidates", "zig_autotune",
    "zig_selfcheck", "zig_filtercheck", "zig_generate_checked", "zig_status_decode", "zig_tables_get",
    "zig_state_init", "zig_generate_state", "zig_mutate_state", "zig_server_population",
    "zig_server_submit_population", "zig_server_population_release",
)

# bytes of one zig_stream_state record (include/zig.h)
STATE_BYTES = 48


REQ_KIND = {"mutate": 0, "generate": 1}   # ZIG_REQ_MUTATE, ZIG_REQ_GENERATE


class Mutation(C.Structure):
    """zig_mutation: one request of a batch (kind: ZIG_REQ_MUTATE or ZIG_REQ_GENERATE;
    state_dev: the rows' stream records, or NULL for rows seeded seed + p)."""
    _fields_ = [("x_dev", C.c_void_p), ("P", C.c_uint64), ("L", C.c_uint64),
                ("sigma", C.c_float), ("kind", C.c_uint32), ("seed", C.c_uint64),
                ("state_dev", C.c_void_p)]


class StreamState(C.Structure):
    """zig_stream_state: one stream's generator kept between calls."""
    _fields_ = [("gen", C.c_uint64 * 4), ("polar_cached", C.c_double), ("polar_have", C.c_uint32),
                ("prng", C.c_uint32)]


class LaunchConfig(C.Structure):
    """zig_launch_config: block size, batch width, store width and (binary64) fma share of the 128-level kernel."""
    _fields_ = [("block", C.c_uint32), ("batch", C.c_uint32), ("store_bytes", C.c_uint32),
                ("fma_of_4", C.c_uint32)]

    def as_dict(self):
        return {"block": self.block, "batch": self.batch, "store_bytes": self.store_bytes,
                "fma_of_4": self.fma_of_4}


class ServingStats(C.Structure):
    """zig_serving_stats."""
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("elements", C.c_uint64), ("latency_p50_us", C.c_double),
                ("latency_p99_us", C.c_double), ("span_us", C.c_double), ("batches", C.c_uint64),
                ("mean_batch", C.c_double), ("peak_inflight_bytes", C.c_uint64),
                ("peak_busy_slots", C.c_uint32), ("reserved", C.c_uint32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


class ZigError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.lib_path()


def load(build_if_missing: bool = True):
    """Load libzig_gb300 (building it first when missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.lib_path()
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libzig_gb300 is not built ({path}); run "
                              "python -m paper_2405_19493_gb300.build")
        lib = C.CDLL(path)
        u64, vp, i32 = C.c_uint64, C.c_void_p, C.c_int
        lib.zig_tables_init.argtypes = [i32]
        lib.zig_tables_get_zig128.argtypes = [vp, vp, vp, vp, vp]
        lib.zig_generate.argtypes = [i32, i32, vp, vp, u64, u64, C.c_uint32, i32, vp, vp,
                                     C.c_size_t, vp]
        lib.zig_generate_workspace_bytes.argtypes = [u64]
        lib.zig_generate_workspace_bytes.restype = C.c_size_t
        lib.zig_mutate.argtypes = [vp, C.c_float, u64, u64, u64, i32, vp]
        lib.zig_generate_noalloc.argtypes = [i32, i32, vp, vp, u64, C.c_uint32, i32, vp, vp]
        lib.zig_generate_noalloc.restype = i32
        lib.zig_prng_fill.argtypes = [i32, vp, u64, u64, u64, i32, vp, vp]
        lib.zig_mutate_batch_desc_bytes.argtypes = [C.c_uint32]
        lib.zig_mutate_batch_desc_bytes.restype = C.c_size_t
        lib.zig_mutate_batch.argtypes = [C.POINTER(Mutation), C.c_uint32, i32, vp, C.c_size_t, vp]
        lib.zig_server_create.argtypes = [i32, i32, u64, C.c_uint32, C.c_uint32, C.POINTER(vp)]
        lib.zig_server_submit.argtypes = [vp, vp, u64, u64, C.c_float, u64, C.POINTER(u64)]
        lib.zig_server_submit_generate.argtypes = [vp, vp, u64, u64, u64, C.POINTER(u64)]
        lib.zig_server_wait.argtypes = [vp, u64, C.c_double]
        lib.zig_server_query.argtypes = [vp, u64, C.POINTER(i32), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]
        lib.zig_server_drain.argtypes = [vp, C.c_double]
        lib.zig_server_stats.argtypes = [vp, C.POINTER(ServingStats)]
        lib.zig_server_destroy.argtypes = [vp]
        for name in ("zig_mutate_batch", "zig_server_create", "zig_server_submit",
                     "zig_server_submit_generate", "zig_server_wait",
                     "zig_server_query", "zig_server_drain", "zig_server_stats",
                     "zig_server_destroy"):
            getattr(lib, name).restype = i32
        lib.zig_launch_config_get.argtypes = [i32, i32, i32, i32, C.POINTER(LaunchConfig)]
        lib.zig_launch_config_set.argtypes = [i32, i32, i32, i32, C.POINTER(LaunchConfig)]
        lib.zig_autotune_candidates.argtypes = [i32, C.POINTER(LaunchConfig), C.c_uint32]
        lib.zig_autotune_candidates.restype = C.c_uint32
        lib.zig_autotune.argtypes = [i32, vp, vp, u64, u64, C.c_uint32, i32, vp, vp, C.c_size_t,
                                     C.c_uint32, C.POINTER(LaunchConfig), C.POINTER(C.c_float), vp]
        for name in ("zig_launch_config_get", "zig_launch_config_set", "zig_autotune"):
            getattr(lib, name).restype = i32
        lib.zig_selfcheck.argtypes = [C.POINTER(u64)]
        lib.zig_selfcheck.restype = i32
        lib.zig_filtercheck.argtypes = [C.POINTER(u64)]
        lib.zig_filtercheck.restype = i32
        lib.zig_device_status.argtypes = [i32, i32]
        lib.zig_generate_checked.argtypes = [i32, i32, vp, vp, u64, u64, C.c_uint32, i32, vp, vp,
                                             C.c_size_t, vp, vp]
        lib.zig_status_decode.argtypes = [C.c_uint32]
        lib.zig_tables_get.argtypes = [i32, vp, C.POINTER(C.c_size_t)]
        for name in ("zig_generate_checked", "zig_status_decode", "zig_tables_get"):
            getattr(lib, name).restype = i32
        lib.zig_state_init.argtypes = [i32, vp, u64, vp, vp]
        lib.zig_generate_state.argtypes = [i32, i32, vp, vp, u64, u64, i32, vp, vp, C.c_size_t, vp, vp]
        lib.zig_mutate_state.argtypes = [vp, C.c_float, u64, u64, vp, i32, vp]
        lib.zig_server_population.argtypes = [vp, u64, u64, C.POINTER(u64)]
        lib.zig_server_submit_population.argtypes = [vp, u64, vp, u64, C.c_float, C.c_uint32, C.POINTER(u64)]
        lib.zig_server_population_release.argtypes = [vp, u64]
        for name in ("zig_state_init", "zig_generate_state", "zig_mutate_state", "zig_server_population",
                     "zig_server_submit_population", "zig_server_population_release"):
            getattr(lib, name).restype = i32
        lib.zig_status_string.argtypes = [i32]
        lib.zig_status_string.restype = C.c_char_p
        for name in ("zig_tables_init", "zig_tables_get_zig128", "zig_generate", "zig_mutate",
                     "zig_prng_fill", "zig_device_status"):
            getattr(lib, name).restype = i32
        lib.zig_version.restype = i32
        _lib = lib
        return lib


def _check(status: int, where: str) -> None:
    if status != ZIG_OK:
        raise ZigError(status, where)


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


# ---- the C entry points --------------------------------------------------------

def zig_tables_init(device: int = 0) -> None:
    _check(load().zig_tables_init(device), "zig_tables_init")


def zig_tables_get_zig128():
    import numpy as np
    k = np.empty(128, np.uint32)
    w = np.empty(128, np.float64)
    y = np.empty(128, np.float64)
    w32 = np.empty(128, np.float32)
    R = np.empty(1, np.float64)
    _check(load().zig_tables_get_zig128(k.ctypes.data, w.ctypes.data, y.ctypes.data,
                                        w32.ctypes.data, R.ctypes.data), "zig_tables_get_zig128")
    return {"k": k, "w": w, "y": y, "w32": w32, "R": float(R[0])}


class Tables128(C.Structure):
    """zig_tables128."""
    _fields_ = [("R", C.c_double), ("V", C.c_double), ("w", C.c_double * 128), ("y", C.c_double * 128),
                ("k", C.c_uint32 * 128), ("w32", C.c_float * 128)]


class Tables256(C.Structure):
    """zig_tables256."""
    _fields_ = [("n_r", C.c_uint64), ("x0", C.c_double), ("xs", C.c_double * 256),
                ("ox", C.c_double * 256), ("odx", C.c_double * 256), ("oy", C.c_double * 256),
                ("ody", C.c_double * 256), ("qa", C.c_uint64 * 256), ("thr", C.c_uint64 * 256),
                ("kind", C.c_int32 * 256), ("alias", C.c_int32 * 256)]


def zig_tables_get(alg: str) -> dict:
    """The tables of ``alg`` as a dict of Python scalars and lists ({} for polar)."""
    lib = load()
    n = C.c_size_t(0)
    _check(lib.zig_tables_get(ALG[alg], None, C.byref(n)), "zig_tables_get")
    if n.value == 0:
        return {}
    t = Tables128() if alg == "zig128" else Tables256()
    assert C.sizeof(t) == n.value, "zig_tables_get: structure size differs from the header's"
    _check(lib.zig_tables_get(ALG[alg], C.byref(t), C.byref(n)), "zig_tables_get")
    return {name: (list(getattr(t, name)) if hasattr(getattr(t, name), "__len__") else getattr(t, name))
            for name, _ in t._fields_}


def zig_status_decode(word: int) -> int:
    return int(load().zig_status_decode(int(word) & 0xFFFFFFFF))


def zig_generate_workspace_bytes(n_streams: int) -> int:
    return int(load().zig_generate_workspace_bytes(n_streams))


def zig_generate(prng: str, alg: str, seeds, out, lengths=None, uniform_len: int = 0,
                 chunk_log2: int = 0, dtype: str = "f64", workspace=None, stream=None) -> None:
    """Fill ``out`` (a CUDA tensor of sum(lengths) elements of ``dtype``)."""
    n = int(seeds.numel())
    ws_ptr, ws_bytes = (0, 0)
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    st = load().zig_generate(PRNG[prng], ALG[alg], seeds.data_ptr(),
                             lengths.data_ptr() if lengths is not None else None,
                             int(uniform_len), n, int(chunk_log2), DTYPE[dtype], out.data_ptr(),
                             ws_ptr or None, ws_bytes, _stream_ptr(stream))
    _check(st, "zig_generate")


def zig_generate_checked(prng: str, alg: str, seeds, out, status, lengths=None, uniform_len: int = 0,
                         chunk_log2: int = 0, dtype: str = "f64", workspace=None, stream=None) -> None:
    """zig_generate whose device-side errors go to ``status`` (a CUDA int32 tensor of one element
    the caller zeroes; decode it with zig_status_decode after the stream has run the call)."""
    n = int(seeds.numel())
    ws_ptr, ws_bytes = (0, 0)
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    st = load().zig_generate_checked(PRNG[prng], ALG[alg], seeds.data_ptr(),
                                     lengths.data_ptr() if lengths is not None else None,
                                     int(uniform_len), n, int(chunk_log2), DTYPE[dtype], out.data_ptr() or None,
                                     ws_ptr or None, ws_bytes, status.data_ptr(), _stream_ptr(stream))
    _check(st, "zig_generate_checked")


def zig_state_new(n_streams: int):
    """A device buffer for n_streams zig_stream_state records (48 bytes each, 16-byte aligned)."""
    import torch
    return torch.empty(max(int(n_streams), 1) * STATE_BYTES // 8, dtype=torch.int64, device="cuda")


def zig_state_init(prng: str, seeds, state, stream=None) -> None:
    """Seed state[s] as zig_generate seeds stream s (seeds: a CUDA uint64/int64 tensor)."""
    st = load().zig_state_init(PRNG[prng], seeds.data_ptr(), int(seeds.numel()), state.data_ptr(),
                               _stream_ptr(stream))
    _check(st, "zig_state_init")


def zig_state_read(state, n_streams: int) -> list:
    """The records as dicts (copied to the host; for inspection and tests)."""
    raw = state.view(-1)[: n_streams * STATE_BYTES // 8].cpu().numpy().tobytes()
    recs = (StreamState * n_streams).from_buffer_copy(raw)
    return [{"gen": list(r.gen), "polar_cached": r.polar_cached, "polar_have": r.polar_have,
             "prng": r.prng} for r in recs]


def zig_generate_state(prng: str, alg: str, state, out, n_streams: int, lengths=None,
                       uniform_len: int = 0, dtype: str = "f64", workspace=None, status=None,
                       stream=None) -> None:
    """zig_generate continuing each stream from its record and advancing it."""
    ws_ptr, ws_bytes = (0, 0)
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    st = load().zig_generate_state(PRNG[prng], ALG[alg], state.data_ptr(),
                                   lengths.data_ptr() if lengths is not None else None,
                                   int(uniform_len), int(n_streams), DTYPE[dtype], out.data_ptr() or None,
                                   ws_ptr or None, ws_bytes, status.data_ptr() if status is not None else None,
                                   _stream_ptr(stream))
    _check(st, "zig_generate_state")


def zig_generate_noalloc(prng: str, alg: str, seeds, lengths, out, chunk_log2: int = 0,
                         dtype: str = "f64", stream=None) -> None:
    """Variable-length generation that allocates nothing, for callers that cannot
    allocate device memory at call time (a service that pre-carved HBM into its
    own pools, a latency-bound loop that cannot take cudaMalloc's device sync).
    At most NOALLOC_MAX_STREAMS streams per call; calls must not overlap on the GPU.
    """
    st = load().zig_generate_noalloc(PRNG[prng], ALG[alg], seeds.data_ptr(), lengths.data_ptr(),
                                     int(seeds.numel()), int(chunk_log2), DTYPE[dtype],
                                     out.data_ptr() or None, _stream_ptr(stream))
    _check(st, "zig_generate_noalloc")


def zig_mutate(x, sigma: float, P: int, L: int, seed: int, prng: str = "splitmix64",
               stream=None) -> None:
    st = load().zig_mutate(x.data_ptr(), float(sigma), int(P), int(L),
                           int(seed) & (2 ** 64 - 1), PRNG[prng], _stream_ptr(stream))
    _check(st, "zig_mutate")


def zig_mutate_state(x, sigma: float, P: int, L: int, state, prng: str = "splitmix64",
                     stream=None) -> None:
    """x += sigma z with row p continuing the stream record state[p] (zig_state_init)."""
    st = load().zig_mutate_state(x.data_ptr(), float(sigma), int(P), int(L), state.data_ptr(),
                                 PRNG[prng], _stream_ptr(stream))
    _check(st, "zig_mutate_state")


def zig_mutate_batch(requests, prng: str = "splitmix64", desc=None, stream=None) -> None:
    """requests: list of (x, sigma, seed), (x, sigma, seed, kind) or (x, sigma, seed, kind, state)
    with x a P x L float32 CUDA tensor, kind "mutate" (x += sigma z, the default) or
    "generate" (x = z), and state the rows' stream records (rows continue them; seed ignored)."""
    import torch
    n = len(requests)
    arr = (Mutation * max(n, 1))()
    for k, req in enumerate(requests):
        x, sigma, seed = req[:3]
        kind = REQ_KIND[req[3]] if len(req) > 3 else 0
        state = req[4] if len(req) > 4 else None
        P, L = (x.shape[0], x.shape[1]) if x.dim() == 2 else (1, x.numel())
        arr[k] = Mutation(x.data_ptr() or None, P, L, float(sigma or 0.0), kind,
                          int(seed) & (2 ** 64 - 1), state.data_ptr() if state is not None else None)
    need = int(load().zig_mutate_batch_desc_bytes(n))
    if desc is None:
        desc = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = load().zig_mutate_batch(arr, n, PRNG[prng], desc.data_ptr(), desc.numel(),
                                 _stream_ptr(stream))
    _check(st, "zig_mutate_batch")


def zig_launch_config_get(prng: str, dtype: str, variable_lengths: bool, device: int = 0) -> dict:
    c = LaunchConfig()
    _check(load().zig_launch_config_get(device, PRNG[prng], DTYPE[dtype], int(bool(variable_lengths)),
                                        C.byref(c)), "zig_launch_config_get")
    return c.as_dict()


def zig_launch_config_set(prng: str, dtype: str, variable_lengths: bool, cfg=None,
                          device: int = 0) -> None:
    """cfg: a dict with block, batch, store_bytes (and fma_of_4 for f64), or None for the default."""
    ptr = None
    if cfg is not None:
        ptr = C.byref(LaunchConfig(int(cfg["block"]), int(cfg["batch"]), int(cfg["store_bytes"]),
                                   int(cfg.get("fma_of_4", 0))))
    _check(load().zig_launch_config_set(device, PRNG[prng], DTYPE[dtype], int(bool(variable_lengths)),
                                        ptr), "zig_launch_config_set")


def zig_autotune_candidates(dtype: str) -> list:
    lib = load()
    n = int(lib.zig_autotune_candidates(DTYPE[dtype], None, 0))
    arr = (LaunchConfig * n)()
    lib.zig_autotune_candidates(DTYPE[dtype], arr, n)
    return [c.as_dict() for c in arr]


def zig_autotune(prng: str, seeds, out, lengths=None, uniform_len: int = 0, chunk_log2: int = 0,
                 dtype: str = "f64", reps: int = 3, workspace=None, stream=None):
    """Time every candidate on this request, record the fastest; returns (config, ms per call)."""
    best, ms = LaunchConfig(), C.c_float()
    ws_ptr, ws_bytes = (0, 0)
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    st = load().zig_autotune(PRNG[prng], seeds.data_ptr(),
                             lengths.data_ptr() if lengths is not None else None, int(uniform_len),
                             int(seeds.numel()), int(chunk_log2), DTYPE[dtype], out.data_ptr() or None,
                             ws_ptr or None, ws_bytes, int(reps), C.byref(best), C.byref(ms),
                             _stream_ptr(stream))
    _check(st, "zig_autotune")
    return best.as_dict(), float(ms.value)


def zig_prng_fill(prng: str, seeds, n: int, out, skip: int = 0, kind: str = "u32",
                  stream=None) -> None:
    st = load().zig_prng_fill(PRNG[prng], seeds.data_ptr(), int(seeds.numel()), int(n),
                              int(skip), FILL_KIND[kind], out.data_ptr(), _stream_ptr(stream))
    _check(st, "zig_prng_fill")


def zig_selfcheck() -> dict:
    """Exhaustive check of the fast-path product and the bfloat16 rounding (see zig.h)."""
    c = (C.c_uint64 * 6)()
    _check(load().zig_selfcheck(c), "zig_selfcheck")
    return {"product_mismatches": int(c[0]), "rounding_mismatches": int(c[1]),
            "products_checked": int(c[2]), "roundings_checked": int(c[3]),
            "logs_beyond_one_ulp": int(c[4]), "logs_not_equal": int(c[5])}


def zig_filtercheck() -> dict:
    """The slow tests' binary32 filters against their binary64 definitions (see zig.h):
    per test, inputs checked, left undecided, and decided unlike the definition."""
    c = (C.c_uint64 * 12)()
    _check(load().zig_filtercheck(c), "zig_filtercheck")
    names = ("wedge128", "tail128", "overhang256", "tail256")
    return {nm: {"checked": int(c[3 * f]), "undecided": int(c[3 * f + 1]), "wrong": int(c[3 * f + 2])}
            for f, nm in enumerate(names)}


def zig_device_status(device: int = 0, clear: bool = False) -> int:
    return int(load().zig_device_status(device, 1 if clear else 0))


def zig_status_string(status: int) -> str:
    return load().zig_status_string(status).decode()


def zig_version() -> int:
    return int(load().zig_version())


# ---- tensor-level convenience (allocation through torch, compute in the library) ----

def generate(prng: str, alg: str, seeds, lengths=None, uniform_len: int = 0, chunk_log2: int = 0,
             dtype: str = "f64", out=None, stream=None):
    """Allocate (if needed) and fill the packed stream-major output tensor."""
    import torch
    torch_dt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    if lengths is not None:
        total = int(lengths.sum().item()) if out is None else out.numel()
    else:
        total = int(seeds.numel()) * int(uniform_len)
    if out is None:
        out = torch.empty(total, dtype=torch_dt, device=seeds.device)
    zig_generate(prng, alg, seeds, out, lengths=lengths, uniform_len=uniform_len,
                 chunk_log2=chunk_log2, dtype=dtype, stream=stream)
    return out
