"""GB300-native bulk N(0,1) generation: the original 128-level ziggurat (GSL
form) over per-stream java.util.Random / SplitMix64 / L64X128Mix /
Xoroshiro128PlusPlus generators, with the polar method and a 256-slot modified
ziggurat as comparison transforms.

The compute lives in libzig_gb300.so (CUDA, sm_103a) behind the C ABI in
include/zig.h; this package only builds and binds it (``_binding``), plus the
seeded synthetic workloads (``workloads``), the request loop for Gaussian
mutation and generation (``serving``), and distribution checks of outputs
(``quality``).
"""

from ._binding import (  # noqa: F401
    ZigError, generate, load, zig_device_status, zig_generate, zig_generate_noalloc,
    zig_generate_workspace_bytes,
    zig_mutate, zig_mutate_batch, zig_prng_fill, zig_status_string, zig_tables_get_zig128, zig_tables_init,
    zig_version, zig_launch_config_get, zig_launch_config_set, zig_autotune_candidates, zig_autotune,
    zig_generate_checked, zig_status_decode, zig_tables_get, zig_state_new, zig_state_init, zig_state_read,
    zig_generate_state, zig_mutate_state,
)

__all__ = [
    "ZigError", "generate", "load", "zig_device_status", "zig_generate", "zig_generate_noalloc",
    "zig_generate_workspace_bytes", "zig_mutate", "zig_mutate_batch", "zig_prng_fill", "zig_status_string",
    "zig_tables_get_zig128", "zig_tables_init", "zig_version", "zig_launch_config_get",
    "zig_launch_config_set", "zig_autotune_candidates", "zig_autotune", "zig_generate_checked",
    "zig_status_decode", "zig_tables_get", "zig_state_new", "zig_state_init", "zig_state_read",
    "zig_generate_state", "zig_mutate_state",
]
