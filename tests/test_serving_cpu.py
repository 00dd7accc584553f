"""The mutation service's scheduler without a GPU (dry run: simulated launches).

Checks admission in arrival order under the memory budget, refusal of a
population larger than the budget, batching of requests that queue up, and the
latency statistics.
"""

import time

import pytest

from paper_2405_19493_gb300 import _binding as B
from paper_2405_19493_gb300.serving import MutationServer

FAKE = 1 << 20   # a non-null pointer; dry runs never dereference it


def test_dry_run_admission_and_batching():
    # 256 MiB requests: a dry launch lasts about 0.27 ms, long enough that requests
    # submitted meanwhile queue up and are batched however the submitting loop runs
    budget = 2 << 30   # 2 GiB: eight requests in flight
    with MutationServer(device=-1, budget_bytes=budget, n_slots=2, max_batch=8) as srv:
        tickets = [srv.submit(None, 0.5, k, P=2048, L=32768, x_ptr=FAKE) for k in range(40)]
        srv.drain(timeout_s=30)
        st = srv.stats()
        assert st["completed"] == 40 and st["failed"] == 0
        assert st["peak_inflight_bytes"] <= budget
        assert st["batches"] < 40 and st["mean_batch"] > 1          # requests were batched
        assert st["peak_busy_slots"] <= 2
        assert 0 < st["latency_p50_us"] <= st["latency_p99_us"]
        for t in tickets:
            q = srv.query(t)
            assert q["state"] == 2 and q["queue_us"] >= 0 and q["latency_us"] >= q["queue_us"]


def test_dry_run_budget_refusal_and_invalid():
    with MutationServer(device=-1, budget_bytes=1 << 20, n_slots=1, max_batch=4) as srv:
        with pytest.raises(B.ZigError) as e:
            srv.submit(None, 0.1, 1, P=1024, L=1024, x_ptr=FAKE)       # 4 MiB > 1 MiB
        assert e.value.status == 4                                      # ZIG_ERR_BUDGET
        t = srv.submit(None, 0.1, 2, P=16, L=16, x_ptr=FAKE)
        srv.wait(t, timeout_s=10)
        assert srv.query(t)["state"] == 2
        with pytest.raises(B.ZigError):
            srv.submit(None, float("nan"), 3, P=4, L=4, x_ptr=FAKE)
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 1


def test_dry_run_fifo_under_memory_pressure():
    # each request needs the whole budget: they must run one at a time, in order.  A dry
    # launch of 2 GiB lasts about 2 ms, so consecutive starts are 2 ms apart however the
    # submitting loop is scheduled.
    P, L = 32768, 16384                       # 2 GiB of binary32
    budget = P * L * 4
    with MutationServer(device=-1, budget_bytes=budget, n_slots=4, max_batch=16) as srv:
        tickets, t_sub = [], []
        for k in range(6):
            t_sub.append(time.perf_counter())
            tickets.append(srv.submit(None, 0.3, k, P=P, L=L, x_ptr=FAKE))
        srv.drain(timeout_s=30)
        st = srv.stats()
        assert st["peak_busy_slots"] == 1 and st["batches"] == 6
        # start = submit + queue time (the submit stamp is taken just before the call)
        start = [t_sub[k] + srv.query(t)["queue_us"] * 1e-6 for k, t in enumerate(tickets)]
        assert all(start[k] < start[k + 1] + 2e-4 for k in range(5)), start
        assert all(srv.query(t)["latency_us"] > 0 for t in tickets)


def test_dry_run_generate_and_mutate_share_queue_and_budget():
    budget = 16 << 20
    with MutationServer(device=-1, budget_bytes=budget, n_slots=2, max_batch=4) as srv:
        t = []
        for k in range(12):
            if k % 3 == 0:
                t.append(srv.submit_generate(None, k, P=32, L=32768, out_ptr=FAKE))   # 4 MiB
            else:
                t.append(srv.submit(None, 0.2, k, P=32, L=32768, x_ptr=FAKE))
        # a generation request ignores sigma, so it needs none; the budget still applies
        with pytest.raises(B.ZigError) as e:
            srv.submit_generate(None, 99, P=4096, L=4096, out_ptr=FAKE)          # 64 MiB
        assert e.value.status == 4
        srv.drain(timeout_s=30)
        st = srv.stats()
        assert st["completed"] == 12 and st["failed"] == 1
        assert st["elements"] == 12 * 32 * 32768
        assert st["peak_inflight_bytes"] <= budget
        assert all(srv.query(k)["state"] == 2 for k in t)


def test_dry_run_population_requests_run_one_at_a_time_in_order():
    # requests on one population continue its streams, so they may never share a
    # launch or overlap; requests on other populations still batch
    # 2 GiB requests: a dry launch lasts about 2 ms
    with MutationServer(device=-1, budget_bytes=16 << 30, n_slots=4, max_batch=16) as srv:
        a = srv.population(P=512, seed=1)
        b = srv.population(P=512, seed=2)
        ta = [srv.submit_population(a, None, 0.5, L=1 << 20, x_ptr=FAKE) for _ in range(5)]
        tb = [srv.submit_population(b, None, 0.5, L=1 << 20, x_ptr=FAKE) for _ in range(5)]
        srv.drain(timeout_s=30)
        st = srv.stats()
        assert st["completed"] == 10 and st["failed"] == 0
        assert st["batches"] >= 5                                      # a's five never share one
        for ts in (ta, tb):
            q = [srv.query(t) for t in ts]
            assert all(x["state"] == 2 for x in q)
            # times are from each request's own submission, and the requests were
            # submitted back to back (microseconds apart; 1 ms of slack, half a launch, for
            # a descheduled submitting thread): each launched after its predecessor finished
            done = [x["latency_us"] for x in q]
            starts = [x["queue_us"] for x in q]
            for k in range(1, len(ts)):
                assert starts[k] >= done[k - 1] - 1000.0
        srv.release_population(a)
        with pytest.raises(B.ZigError):
            srv.submit_population(a, None, 0.5, L=16, x_ptr=FAKE)    # released
        with pytest.raises(B.ZigError):
            srv.submit_population(99, None, 0.5, L=16, x_ptr=FAKE)   # no such population
        srv.release_population(b)


def test_dry_run_population_release_waits_for_its_requests():
    with MutationServer(device=-1, budget_bytes=8 << 30, n_slots=2, max_batch=4) as srv:
        a = srv.population(P=4096, seed=7)
        ts = [srv.submit_population(a, None, 0.1, L=131072, x_ptr=FAKE) for _ in range(3)]
        srv.release_population(a)             # returns once all three have run
        assert all(srv.query(t)["state"] == 2 for t in ts)
