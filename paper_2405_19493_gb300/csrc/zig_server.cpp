// Continuous-batching service for Gaussian-mutation requests (the paper's
// motivating workload, Sec. 1: Gaussian mutation in an evolutionary algorithm)
// and generation requests.
//
// Requests x += sigma * N(0,1) on device-resident binary32 populations, or
// x = N(0,1) into device buffers, arrive at any time.  A worker thread admits them in arrival order while the bytes of
// the populations in flight stay within the budget, packs up to max_batch
// admitted requests into one launch of zig_mutate_batch on a free stream slot,
// and retires a slot when its CUDA event completes.  Requests that arrive while
// others are on the GPU join the next launch on another slot, so work from
// different batches overlaps on the device.  Each request's result is exactly
// what zig_mutate computes for it alone (seeds and chunking are per request).
// A population keeps one stream record per row on the device, so that its
// requests continue the rows' streams (zig_mutate_state); requests on one
// population run one at a time, in submission order.
//
// device < 0 selects a dry run: no CUDA call is made and a launch "completes"
// after a simulated time proportional to its bytes, which lets the admission
// and batching logic be tested without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/zig.h"

namespace {

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Req {
    zig_mutation m;
    uint64_t bytes;
    double t_submit, t_launch, t_done;
    int state;
    zig_status status;
    int64_t pop;   // the population whose streams the request continues, or -1
};

// A population: P stream records on the device (none in a dry run).
struct Pop {
    zig_stream_state* state = nullptr;
    uint64_t P = 0;
    uint64_t pending = 0;   // its requests queued or running
    bool busy = false;      // one of its requests is in flight
    bool released = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* desc = nullptr;
    size_t desc_bytes = 0;
    std::vector<uint64_t> tickets;
    std::vector<zig_mutation> batch;
    uint64_t bytes = 0;
    bool busy = false;
    double t_launch = 0, sim_done = 0;
};

}  // namespace

struct zig_server {
    int device;
    bool dry;
    zig_prng prng;
    uint64_t budget;
    uint32_t max_batch;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::vector<Req> reqs;
    std::vector<Pop> pops;
    std::vector<Slot> slots;
    uint64_t inflight_bytes = 0, peak_inflight_bytes = 0;
    uint64_t batches = 0, batched_requests = 0;
    uint32_t peak_busy_slots = 0;
    bool stop = false;
    zig_status worker_error = ZIG_OK;
    std::thread worker;
};

namespace {

// Retire completed slots (caller holds the lock).
void retire(zig_server* S) {
    const double t = now_us();
    for (Slot& sl : S->slots) {
        if (!sl.busy) continue;
        bool finished;
        if (S->dry) {
            finished = t >= sl.sim_done;
        } else {
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady) continue;
            finished = true;
            if (e != cudaSuccess) S->worker_error = ZIG_ERR_CUDA;
        }
        if (!finished) continue;
        for (uint64_t k : sl.tickets) {
            Req& r = S->reqs[k];
            r.state = S->worker_error == ZIG_OK ? kDone : kFailed;
            r.status = S->worker_error;
            r.t_done = t;
            if (r.pop >= 0) {
                S->pops[r.pop].busy = false;
                S->pops[r.pop].pending -= 1;
            }
        }
        S->inflight_bytes -= sl.bytes;
        sl.busy = false;
        sl.tickets.clear();
        S->cv_done.notify_all();
    }
}

// Form a batch for a free slot from the head of the queue (caller holds the lock).
bool form_batch(zig_server* S, Slot& sl) {
    sl.tickets.clear();
    sl.batch.clear();
    sl.bytes = 0;
    while (!S->queue.empty() && sl.tickets.size() < S->max_batch) {
        const uint64_t k = S->queue.front();
        Req& r = S->reqs[k];
        if (S->inflight_bytes + sl.bytes + r.bytes > S->budget) break;   // wait for memory
        if (r.pop >= 0 && S->pops[r.pop].busy) break;   // its population's previous request first
        S->queue.pop_front();
        if (r.pop >= 0) S->pops[r.pop].busy = true;
        sl.tickets.push_back(k);
        sl.batch.push_back(r.m);
        sl.bytes += r.bytes;
    }
    return !sl.tickets.empty();
}

void worker_main(zig_server* S) {
    if (!S->dry) cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        retire(S);
        // launch into free slots while admitted work is waiting
        for (Slot& sl : S->slots) {
            if (sl.busy || S->queue.empty()) continue;
            if (!form_batch(S, sl)) break;
            const double t = now_us();
            for (uint64_t k : sl.tickets) {
                S->reqs[k].state = kRunning;
                S->reqs[k].t_launch = t;
            }
            S->inflight_bytes += sl.bytes;
            S->peak_inflight_bytes = std::max(S->peak_inflight_bytes, S->inflight_bytes);
            sl.busy = true;
            sl.t_launch = t;
            S->batches += 1;
            S->batched_requests += sl.tickets.size();
            if (S->dry) {
                sl.sim_done = t + 5.0 + (double)sl.bytes * 1e-6;   // 5 us + 1 TB/s
            } else {
                // the launch itself takes no lock-protected state; keep the lock (the
                // calls only enqueue work) so the slot cannot be retired concurrently
                zig_status st = zig_mutate_batch(sl.batch.data(), (uint32_t)sl.batch.size(), S->prng,
                                                 sl.desc, sl.desc_bytes, (void*)sl.stream);
                if (st == ZIG_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = ZIG_ERR_CUDA;
                if (st != ZIG_OK) {
                    S->worker_error = st;
                    cudaStreamSynchronize(sl.stream);
                    cudaEventRecord(sl.done, sl.stream);
                }
            }
        }
        uint32_t busy = 0;
        for (const Slot& sl : S->slots) busy += sl.busy;
        S->peak_busy_slots = std::max(S->peak_busy_slots, busy);
        if (S->stop && S->queue.empty() && busy == 0) break;
        if (busy) S->cv_work.wait_for(lk, std::chrono::microseconds(20));   // poll events
        else S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
    }
}

double percentile(std::vector<double>& v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double idx = p * (double)(v.size() - 1);
    const size_t lo = (size_t)std::floor(idx), hi = std::min(v.size() - 1, lo + 1);
    return v[lo] + (v[hi] - v[lo]) * (idx - (double)lo);
}

}  // namespace

extern "C" {

zig_status zig_server_create(int device, zig_prng prng, uint64_t budget_bytes, uint32_t n_slots,
                             uint32_t max_batch, zig_server** out) {
    if (!out || (unsigned)prng > 3u || budget_bytes == 0 || n_slots == 0 || n_slots > 64 ||
        max_batch == 0 || max_batch > (1u << 20))
        return ZIG_ERR_INVALID_ARG;
    *out = nullptr;
    zig_server* S = new zig_server();
    S->device = device;
    S->dry = device < 0;
    S->prng = prng;
    S->budget = budget_bytes;
    S->max_batch = max_batch;
    S->slots.resize(n_slots);
    if (!S->dry) {
        zig_status st = zig_tables_init(device);
        if (st != ZIG_OK) {
            delete S;
            return st;
        }
        for (Slot& sl : S->slots) {
            sl.desc_bytes = zig_mutate_batch_desc_bytes(max_batch);
            if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
                cudaMalloc(&sl.desc, sl.desc_bytes) != cudaSuccess) {
                for (Slot& t : S->slots) {
                    if (t.desc) cudaFree(t.desc);
                    if (t.done) cudaEventDestroy(t.done);
                    if (t.stream) cudaStreamDestroy(t.stream);
                }
                delete S;
                return ZIG_ERR_CUDA;
            }
        }
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return ZIG_OK;
}

}  // extern "C"

namespace {
// pop < 0: rows seeded seed + p; else rows continue population pop's records.
zig_status submit(zig_server* S, float* x_dev, uint64_t P, uint64_t L, float sigma, uint32_t kind,
                  uint64_t seed, int64_t pop, uint64_t* ticket) {
    if (!S || !ticket || kind > ZIG_REQ_GENERATE || (kind == ZIG_REQ_MUTATE && !std::isfinite(sigma)))
        return ZIG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return ZIG_ERR_INVALID_ARG;
    zig_stream_state* state = nullptr;
    if (pop >= 0) {
        if ((uint64_t)pop >= S->pops.size() || S->pops[pop].released) return ZIG_ERR_INVALID_ARG;
        P = S->pops[pop].P;
        state = S->pops[pop].state;
    }
    if ((P && L && !x_dev) || (L && P > ((1ull << 40) - 1) / L)) return ZIG_ERR_INVALID_ARG;
    const uint64_t bytes = P * L * sizeof(float);
    Req r;
    r.m = zig_mutation{x_dev, P, L, sigma, kind, seed, state};
    r.pop = pop;
    r.bytes = bytes;
    r.t_submit = now_us();
    r.t_launch = r.t_done = 0;
    r.state = kQueued;
    r.status = ZIG_OK;
    *ticket = S->reqs.size();
    if (bytes > S->budget) {   // can never be admitted
        r.state = kFailed;
        r.status = ZIG_ERR_BUDGET;
        r.t_done = r.t_submit;
        S->reqs.push_back(r);
        return ZIG_ERR_BUDGET;
    }
    S->reqs.push_back(r);
    S->queue.push_back(*ticket);
    if (pop >= 0) S->pops[pop].pending += 1;
    S->cv_work.notify_one();
    return ZIG_OK;
}
}  // namespace

extern "C" {

zig_status zig_server_submit(zig_server* S, float* x_dev, uint64_t P, uint64_t L, float sigma,
                             uint64_t seed, uint64_t* ticket) {
    return submit(S, x_dev, P, L, sigma, ZIG_REQ_MUTATE, seed, -1, ticket);
}

zig_status zig_server_submit_generate(zig_server* S, float* out_dev, uint64_t P, uint64_t L,
                                      uint64_t seed, uint64_t* ticket) {
    return submit(S, out_dev, P, L, 0.0f, ZIG_REQ_GENERATE, seed, -1, ticket);
}

zig_status zig_server_population(zig_server* S, uint64_t P, uint64_t seed, uint64_t* population) {
    if (!S || !population || P == 0 || P > (1ull << 32)) return ZIG_ERR_INVALID_ARG;
    Pop pp;
    pp.P = P;
    if (!S->dry) {
        // the records are seeded on the legacy stream and complete before this call
        // returns, so the service's streams see them initialized
        if (cudaSetDevice(S->device) != cudaSuccess) return ZIG_ERR_CUDA;
        std::vector<uint64_t> seeds(P);
        for (uint64_t p = 0; p < P; ++p) seeds[p] = seed + p;
        uint64_t* seeds_dev = nullptr;
        if (cudaMalloc(&pp.state, P * sizeof(zig_stream_state)) != cudaSuccess) return ZIG_ERR_CUDA;
        zig_status st = ZIG_OK;
        if (cudaMalloc(&seeds_dev, P * sizeof(uint64_t)) != cudaSuccess ||
            cudaMemcpy(seeds_dev, seeds.data(), P * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess)
            st = ZIG_ERR_CUDA;
        if (st == ZIG_OK) st = zig_state_init(S->prng, seeds_dev, P, pp.state, nullptr);
        if (st == ZIG_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) st = ZIG_ERR_CUDA;
        if (seeds_dev) cudaFree(seeds_dev);
        if (st != ZIG_OK) {
            cudaFree(pp.state);
            return st;
        }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    *population = S->pops.size();
    S->pops.push_back(pp);
    return ZIG_OK;
}

zig_status zig_server_submit_population(zig_server* S, uint64_t population, float* x_dev, uint64_t L,
                                        float sigma, uint32_t kind, uint64_t* ticket) {
    if (!S || population >= (1ull << 62)) return ZIG_ERR_INVALID_ARG;
    return submit(S, x_dev, 0, L, sigma, kind, 0, (int64_t)population, ticket);
}

zig_status zig_server_population_release(zig_server* S, uint64_t population) {
    if (!S) return ZIG_ERR_INVALID_ARG;
    zig_stream_state* state = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        if (population >= S->pops.size() || S->pops[population].released) return ZIG_ERR_INVALID_ARG;
        S->cv_work.notify_one();
        S->cv_done.wait(lk, [&] { return S->pops[population].pending == 0; });
        S->pops[population].released = true;
        state = S->pops[population].state;
        S->pops[population].state = nullptr;
    }
    if (state && cudaFree(state) != cudaSuccess) return ZIG_ERR_CUDA;
    return ZIG_OK;
}

zig_status zig_server_wait(zig_server* S, uint64_t ticket, double timeout_s) {
    if (!S) return ZIG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket >= S->reqs.size()) return ZIG_ERR_INVALID_ARG;
    const auto pred = [&] { return S->reqs[ticket].state >= kDone; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, pred);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return ZIG_ERR_TIMEOUT;
    }
    return S->reqs[ticket].status;
}

zig_status zig_server_query(zig_server* S, uint64_t ticket, int* state, double* latency_us,
                            double* queue_us) {
    if (!S) return ZIG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (ticket >= S->reqs.size()) return ZIG_ERR_INVALID_ARG;
    const Req& r = S->reqs[ticket];
    if (state) *state = r.state;
    if (latency_us) *latency_us = r.state >= kDone ? r.t_done - r.t_submit : -1.0;
    if (queue_us) *queue_us = r.state >= kRunning ? r.t_launch - r.t_submit : -1.0;
    return r.status;
}

zig_status zig_server_drain(zig_server* S, double timeout_s) {
    if (!S) return ZIG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto pred = [&] {
        if (!S->queue.empty()) return false;
        for (const Slot& sl : S->slots)
            if (sl.busy) return false;
        return true;
    };
    S->cv_work.notify_one();
    if (timeout_s < 0) S->cv_done.wait(lk, pred);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return ZIG_ERR_TIMEOUT;
    return S->worker_error;
}

zig_status zig_server_stats(zig_server* S, zig_serving_stats* out) {
    if (!S || !out) return ZIG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    std::vector<double> lat;
    double first = 1e300, last = 0;
    for (const Req& r : S->reqs) {
        out->submitted += 1;
        if (r.state == kDone) {
            out->completed += 1;
            out->elements += r.m.P * r.m.L;
            lat.push_back(r.t_done - r.t_submit);
            first = std::min(first, r.t_submit);
            last = std::max(last, r.t_done);
        } else if (r.state == kFailed) {
            out->failed += 1;
        }
    }
    out->latency_p50_us = percentile(lat, 0.50);
    out->latency_p99_us = percentile(lat, 0.99);
    out->span_us = out->completed ? last - first : 0.0;
    out->batches = S->batches;
    out->mean_batch = S->batches ? (double)S->batched_requests / (double)S->batches : 0.0;
    out->peak_inflight_bytes = S->peak_inflight_bytes;
    out->peak_busy_slots = S->peak_busy_slots;
    return S->worker_error;
}

zig_status zig_server_destroy(zig_server* S) {
    if (!S) return ZIG_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    S->worker.join();
    const zig_status st = S->worker_error;
    if (!S->dry) {
        for (Slot& sl : S->slots) {
            cudaStreamSynchronize(sl.stream);
            cudaFree(sl.desc);
            cudaEventDestroy(sl.done);
            cudaStreamDestroy(sl.stream);
        }
        for (Pop& pp : S->pops)
            if (pp.state) cudaFree(pp.state);
    }
    delete S;
    return st;
}

}  // extern "C"
