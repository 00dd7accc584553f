"""Gaussian-mutation serving: Python handle on the library's native service.

The scheduler, admission control (memory budget), batching and stream
management run in C++ inside libzig_gb300 (csrc/zig_server.cpp); this module
only wraps the handle and drives arrivals for measurements.
"""

from __future__ import annotations

import ctypes as C
import time

from . import _binding as B


class MutationServer:
    """Continuous-batching service for x += sigma * N(0,1) and x = N(0,1) requests.

    device < 0 runs the scheduler with simulated launches (no GPU needed).
    """

    def __init__(self, device: int = 0, prng: str = "splitmix64", budget_bytes: int = 40 << 30,
                 n_slots: int = 4, max_batch: int = 64):
        self._lib = B.load()
        h = C.c_void_p()
        B._check(self._lib.zig_server_create(device, B.PRNG[prng], int(budget_bytes), n_slots,
                                             max_batch, C.byref(h)), "zig_server_create")
        self._h = h
        self._keep = {}   # tensors referenced by in-flight tickets

    def submit(self, x, sigma: float, seed: int, P: int | None = None, L: int | None = None,
               x_ptr: int | None = None) -> int:
        """Enqueue a mutation of x (P x L float32 CUDA tensor, or a raw pointer + P, L)."""
        if x is not None:
            P, L = (x.shape[0], x.shape[1]) if x.dim() == 2 else (1, x.numel())
            ptr = x.data_ptr() or None
        else:
            ptr = x_ptr
        t = C.c_uint64()
        st = self._lib.zig_server_submit(self._h, ptr, int(P), int(L), float(sigma),
                                         int(seed) & (2 ** 64 - 1), C.byref(t))
        B._check(st, "zig_server_submit")
        if x is not None:
            self._keep[t.value] = x
        return t.value

    def submit_generate(self, out, seed: int, P: int | None = None, L: int | None = None,
                        out_ptr: int | None = None) -> int:
        """Enqueue out = N(0,1) (P x L float32 CUDA tensor, or a raw pointer + P, L)."""
        if out is not None:
            P, L = (out.shape[0], out.shape[1]) if out.dim() == 2 else (1, out.numel())
            ptr = out.data_ptr() or None
        else:
            ptr = out_ptr
        t = C.c_uint64()
        st = self._lib.zig_server_submit_generate(self._h, ptr, int(P), int(L),
                                                  int(seed) & (2 ** 64 - 1), C.byref(t))
        B._check(st, "zig_server_submit_generate")
        if out is not None:
            self._keep[t.value] = out
        return t.value

    def population(self, P: int, seed: int) -> int:
        """A population of P rows whose streams (seeded seed + p) the service keeps on the device."""
        h = C.c_uint64()
        B._check(self._lib.zig_server_population(self._h, int(P), int(seed) & (2 ** 64 - 1), C.byref(h)),
                 "zig_server_population")
        return h.value

    def submit_population(self, population: int, x, sigma: float = 0.0, kind: str = "mutate",
                          L: int | None = None, x_ptr: int | None = None) -> int:
        """Enqueue a request whose rows continue the population's streams (x: P x L float32)."""
        if x is not None:
            L = x.shape[1] if x.dim() == 2 else x.numel()
            ptr = x.data_ptr() or None
        else:
            ptr = x_ptr
        t = C.c_uint64()
        st = self._lib.zig_server_submit_population(self._h, int(population), ptr, int(L), float(sigma),
                                                    B.REQ_KIND[kind], C.byref(t))
        B._check(st, "zig_server_submit_population")
        if x is not None:
            self._keep[t.value] = x
        return t.value

    def release_population(self, population: int) -> None:
        B._check(self._lib.zig_server_population_release(self._h, int(population)),
                 "zig_server_population_release")

    def wait(self, ticket: int, timeout_s: float = -1.0) -> None:
        st = self._lib.zig_server_wait(self._h, ticket, float(timeout_s))
        self._keep.pop(ticket, None)
        B._check(st, "zig_server_wait")

    def query(self, ticket: int):
        state, lat, q = C.c_int(), C.c_double(), C.c_double()
        st = self._lib.zig_server_query(self._h, ticket, C.byref(state), C.byref(lat), C.byref(q))
        return {"state": state.value, "latency_us": lat.value, "queue_us": q.value, "status": st}

    def drain(self, timeout_s: float = -1.0) -> None:
        B._check(self._lib.zig_server_drain(self._h, float(timeout_s)), "zig_server_drain")
        self._keep.clear()

    def stats(self) -> dict:
        s = B.ServingStats()
        B._check(self._lib.zig_server_stats(self._h, C.byref(s)), "zig_server_stats")
        return s.as_dict()

    def close(self) -> None:
        if self._h:
            st = self._lib.zig_server_destroy(self._h)
            self._h = None
            self._keep.clear()
            B._check(st, "zig_server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def drive_poisson(server: MutationServer, requests, ptr_of, clock=time.perf_counter):
    """Submit requests at their arrival times (seconds from now); returns tickets.

    requests: dicts with P, L, sigma, seed, arrival (paper_2405_19493_gb300.workloads).
    ptr_of(k, req) -> device pointer of request k's population.
    """
    t0 = clock()
    tickets = []
    for k, r in enumerate(requests):
        while clock() - t0 < r["arrival"]:
            pass
        if r.get("kind", "mutate") == "generate":
            tickets.append(server.submit_generate(None, r["seed"], P=r["P"], L=r["L"],
                                                  out_ptr=ptr_of(k, r)))
        else:
            tickets.append(server.submit(None, r["sigma"], r["seed"], P=r["P"], L=r["L"],
                                         x_ptr=ptr_of(k, r)))
    return tickets
