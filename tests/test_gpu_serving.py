"""Batched mutation and the mutation service on the GPU: every request's result
is bit-identical to zig_mutate on that request alone."""

import numpy as np
import pytest

from paper_2405_19493_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_19493_gb300 as Z
    Z.zig_tables_init(0)
    return Z


def _requests(n, seed):
    reqs = W.mutation_requests(n, rate_hz=1000, seed=seed, p_range=(1, 64), l_range=(1, 5000))
    rng = np.random.default_rng(seed)
    pops = [torch.from_numpy(rng.standard_normal((r["P"], r["L"])).astype(np.float32)).cuda()
            for r in reqs]
    return reqs, pops


def _alone(Z, reqs, pops, prng):
    outs = []
    for r, x in zip(reqs, pops):
        y = x.clone()
        Z.zig_mutate(y, r["sigma"], r["P"], r["L"], r["seed"], prng)
        outs.append(y)
    torch.cuda.synchronize()
    return outs


@pytest.mark.parametrize("prng", ["lcg48", "splitmix64", "l64x128mix", "xoroshiro128pp"])
def test_mutate_batch_equals_alone(Z, prng):
    reqs, pops = _requests(37, 5)
    alone = _alone(Z, reqs, pops, prng)
    mixed = [x.clone() for x in pops]
    Z.zig_mutate_batch([(y, r["sigma"], r["seed"]) for y, r in zip(mixed, reqs)], prng=prng)
    torch.cuda.synchronize()
    for a, m in zip(alone, mixed):
        assert torch.equal(a.view(torch.int32), m.view(torch.int32))


def test_server_results_equal_alone(Z):
    from paper_2405_19493_gb300.serving import MutationServer
    reqs, pops = _requests(120, 9)
    alone = _alone(Z, reqs, pops, "splitmix64")
    mixed = [x.clone() for x in pops]
    torch.cuda.synchronize()
    biggest = max(r["P"] * r["L"] * 4 for r in reqs)
    with MutationServer(device=0, prng="splitmix64", budget_bytes=3 * biggest, n_slots=4,
                        max_batch=8) as srv:
        tickets = [srv.submit(y, r["sigma"], r["seed"]) for y, r in zip(mixed, reqs)]
        for t in tickets:
            srv.wait(t, timeout_s=60)
        st = srv.stats()
    assert st["completed"] == 120 and st["failed"] == 0
    assert st["peak_inflight_bytes"] <= 3 * biggest
    assert st["latency_p99_us"] >= st["latency_p50_us"] > 0
    for a, m in zip(alone, mixed):
        assert torch.equal(a.view(torch.int32), m.view(torch.int32))


def _generate_alone(Z, r, prng):
    """A generation request alone: row p = zig_generate(seed + p, L, chunks of 2^10, f32)."""
    seeds = (np.uint64(r["seed"]) + np.arange(r["P"], dtype=np.uint64)).view(np.int64)
    out = torch.empty(r["P"] * r["L"], dtype=torch.float32, device="cuda")
    Z.zig_generate(prng, "zig128", torch.from_numpy(seeds).cuda(), out, uniform_len=r["L"],
                   chunk_log2=10, dtype="f32")
    return out.view(r["P"], r["L"])


@pytest.mark.parametrize("prng", ["lcg48", "l64x128mix"])
def test_batch_mixing_generate_and_mutate_equals_alone(Z, prng):
    reqs, pops = _requests(29, 13)
    kinds = ["generate" if k % 3 == 1 else "mutate" for k in range(len(reqs))]
    alone = _alone(Z, reqs, pops, prng)
    for k, r in enumerate(reqs):
        if kinds[k] == "generate":
            alone[k] = _generate_alone(Z, r, prng)
    torch.cuda.synchronize()
    mixed = [x.clone() for x in pops]
    Z.zig_mutate_batch([(y, r["sigma"], r["seed"], kd) for y, r, kd in zip(mixed, reqs, kinds)],
                       prng=prng)
    torch.cuda.synchronize()
    for a, m in zip(alone, mixed):
        assert torch.equal(a.view(torch.int32), m.view(torch.int32))


def test_server_mixed_kinds_equal_alone(Z):
    from paper_2405_19493_gb300.serving import MutationServer
    reqs, pops = _requests(90, 17)
    alone = _alone(Z, reqs, pops, "splitmix64")
    for k, r in enumerate(reqs):
        if k % 2:
            alone[k] = _generate_alone(Z, r, "splitmix64")
    mixed = [x.clone() for x in pops]
    torch.cuda.synchronize()
    with MutationServer(device=0, prng="splitmix64", budget_bytes=64 << 20, n_slots=3,
                        max_batch=6) as srv:
        tickets = [srv.submit_generate(y, r["seed"]) if k % 2 else srv.submit(y, r["sigma"], r["seed"])
                   for k, (y, r) in enumerate(zip(mixed, reqs))]
        for t in tickets:
            srv.wait(t, timeout_s=60)
        st = srv.stats()
    assert st["completed"] == 90 and st["failed"] == 0
    for a, m in zip(alone, mixed):
        assert torch.equal(a.view(torch.int32), m.view(torch.int32))
