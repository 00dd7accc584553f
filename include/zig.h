/*
 * zig.h -- C ABI of libzig_gb300: bulk N(0,1) generation on one GB300 (sm_103a).
 *
 * The paper (Cicirello, "Fast Gaussian Distributed Pseudorandom Number
 * Generation in Java via the Ziggurat Algorithm") times one call,
 * `nextGaussian`, that draws one standard normal variate from a caller-owned
 * PRNG object which persists between calls (Sec. 2, Listing 2), for three
 * generators (Sec. 2, first list) and three transforms: the original ziggurat
 * in its GSL form, the polar method and McFarland's modified ziggurat (Sec. 2,
 * bullets; Table 3).  This library is the bulk form of that call:
 *
 *     stream s's outputs are exactly the values that repeated nextGaussian
 *     calls return on a generator seeded with seeds[s] (zig_generate), or on a
 *     generator kept between calls in a device record (zig_generate_state).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers in the current CUDA context's
 *    device memory; pointers named *_host are host pointers.  The caller owns
 *    every buffer it passes; the library keeps no pointer after a call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it asynchronously; the call returns once the
 *    launch is queued.
 *  - Argument errors are detected on the host and returned synchronously, with
 *    nothing enqueued.  Launch failures return ZIG_ERR_CUDA.  Conditions only the
 *    GPU can see (a NULL output for lengths that sum above zero, lengths that sum
 *    to 2^40 or more, a chunk overrunning its 2^32-draw budget, a stream record
 *    seeded for another generator) are latched in an
 *    error word on the device: the caller's own word for zig_generate_checked
 *    (scoped to that call), else the device's shared word, read and cleared with
 *    zig_device_status().
 *  - There is no CPU fallback: every step runs in this library's kernels.
 *  - Entry points may be called from several host threads and on distinct
 *    streams at once, with two exceptions stated where they apply: calls of
 *    zig_generate_noalloc share one fixed scratch array, and calls that latch
 *    into the device's shared error word share that word.
 */
#ifndef ZIG_GB300_H
#define ZIG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZIG_OK = 0,
    ZIG_ERR_INVALID_ARG = 1,     /* a bad enum, size, pointer or alignment */
    ZIG_ERR_NOT_INITIALIZED = 2, /* zig_tables_init was not called on this device */
    ZIG_ERR_CUDA = 3,            /* a CUDA runtime call or launch failed */
    ZIG_ERR_BUDGET = 4,          /* a request exceeds the admission budget */
    ZIG_ERR_TIMEOUT = 5,         /* a host-side wait gave up (zig_server_wait, zig_server_drain) */
    ZIG_ERR_CHUNK_OVERFLOW = 6,  /* a chunk consumed more than 2^32 raw draws */
    ZIG_ERR_UNSUPPORTED = 7,     /* the device is not sm_103 or the combination is not built */
    ZIG_ERR_TOO_LARGE = 8        /* more streams than zig_generate_noalloc's fixed scratch holds */
} zig_status;

/* Uniform generators (Sec. 2, first list; Sec. 3 for LXM). */
typedef enum {
    ZIG_LCG48 = 0,       /* java.util.Random: s <- (0x5DEECE66D s + 0xB) mod 2^48,
                            seeded (seed ^ 0x5DEECE66D) mod 2^48; nextInt = s >> 16 */
    ZIG_SPLITMIX64 = 1,  /* SplittableRandom / ThreadLocalRandom: s += 0x9E3779B97F4A7C15;
                            nextInt = mix32(s), nextLong = mix64(s) */
    ZIG_L64X128MIX = 2,  /* LXM: 64-bit LCG (M = 0xD1342543DE82EF95) + xoroshiro128
                            (24, 16, 37) + Lea's mix; seeded from 4 SplitMix64 outputs */
    ZIG_XOROSHIRO128PP = 3 /* Xoroshiro128PlusPlus, an XBG generator (Sec. 3 names the
                            XBG family): nextLong = rotl(x0 + x1, 17) + x0, then the
                            xoroshiro128 engine (49, 21, 28); seeded from 2 SplitMix64
                            outputs; nextInt = nextLong >>> 32 */
} zig_prng;

/* Gaussian transforms (Sec. 2, second list). */
typedef enum {
    ZIG_ZIG128 = 0,  /* original ziggurat, GSL form: 128 layers, 32-bit draw =
                        layer (7 b) + sign (1 b) + 24-bit abscissa */
    ZIG_POLAR = 1,   /* Marsaglia's polar method with the second variate cached */
    ZIG_ZIG256 = 2   /* modified ziggurat after McFarland: 256 slots, 64-bit draws */
} zig_alg;

typedef enum {
    ZIG_F64 = 0,  /* binary64 output (8 B per variate) */
    ZIG_F32 = 1,  /* binary32 output (4 B per variate) */
    ZIG_BF16 = 2  /* bfloat16 output (2 B per variate) */
} zig_dtype;

/*
 * zig_tables_init -- prepare `device` for the generation calls.
 * Checks that the device is compute capability 10.3 (GB300), loads the
 * library's kernels there and resolves its table and error-word symbols.  The
 * tables themselves are immutable device constants compiled into the library
 * (the geometry of Sec. 2's two ziggurats, computed at 80 digits).  Idempotent
 * and cheap after the first call; it makes `device` current.
 * Returns ZIG_ERR_UNSUPPORTED on a non-sm_103 device, ZIG_ERR_CUDA on a CUDA error.
 */
zig_status zig_tables_init(int device);

/*
 * zig_tables_get_zig128 -- copy the 128-level tables to host memory (for
 * comparison with an independent construction).  k_host: 128 uint32, w_host
 * and y_host: 128 double, w32_host: 128 float, R_host: 1 double.  Any pointer
 * may be NULL to skip that table.  Needs no device.
 */
zig_status zig_tables_get_zig128(uint32_t *k_host, double *w_host, double *y_host,
                                 float *w32_host, double *R_host);

/* The 128-level ziggurat's tables (Sec. 1; the GSL form): layer i < 127 is the
 * strip [0, x_{i+1}) x [f(x_{i+1}), f(x_i)), layer 127 the base of width R.
 * w[i] = RN(x_{i+1} / 2^24) (base: RN(v / f(R) / 2^24)), k[i] = floor(2^24 x_i / x_{i+1})
 * (base: floor(2^24 R f(R) / v)), y[i] = RN(f(x_i)), w32 the binary32 rounding of
 * x_{i+1} / 2^24; v is the common layer area. */
typedef struct {
    double R, V;
    double w[128], y[128];
    uint32_t k[128];
    float w32[128];
} zig_tables128;

/* The 256-slot modified ziggurat's tables (Sec. 2, the Java 17 bullet): slot
 * j < n_r is a rectangle of width x0-scaled xs[j] (x = xs[j] (U >> 11)); an alias
 * bin b selects region b when the draw's upper 56 bits are below thr[b], else
 * alias[b]; region 0 is the tail beyond x0, region r in 1..n_r the overhang box
 * [ox, ox + odx] x [oy, oy + ody] with its shape kind (+1 convex, -1 concave)
 * and quick-accept distance qa (all indexed by r; index 0 unused). */
typedef struct {
    uint64_t n_r;
    double x0;
    double xs[256];
    double ox[256], odx[256], oy[256], ody[256];
    uint64_t qa[256], thr[256];
    int32_t kind[256], alias[256];
} zig_tables256;

/*
 * zig_tables_get -- copy the tables of transform `alg` to host memory:
 * a zig_tables128 for ZIG_ZIG128, a zig_tables256 for ZIG_ZIG256, nothing for
 * ZIG_POLAR (it has no tables).  *bytes: in, the capacity of host_dst; out, the
 * size of the structure (0 for ZIG_POLAR).  host_dst = NULL only reports the size.
 * ZIG_ERR_INVALID_ARG for a bad enum, bytes = NULL or too small a capacity.
 * Needs no device.
 */
zig_status zig_tables_get(zig_alg alg, void *host_dst, size_t *bytes);

/*
 * zig_generate -- bulk N(0,1) variates, stream-major and packed.
 *
 * prng, alg, dtype   enums above.
 * seeds_dev          n_streams uint64 seeds (device).
 * lengths_dev        n_streams uint64 lengths (device), or NULL for every stream
 *                    having uniform_len outputs.
 * n_streams          number of streams (0 is a no-op).
 * chunk_log2         0: each stream is one sequential generator (the paper's
 *                    semantics).  c in [4, 24]: output t of stream s belongs to
 *                    chunk q = t >> c, generated from the seeded state advanced
 *                    by q * 2^32 raw generator steps (closed-form jump), so
 *                    long streams split across threads.  Outputs of chunk 0
 *                    equal the sequential ones.
 * out_dev            device buffer of sum(lengths) elements of `dtype`; stream s
 *                    occupies [off_s, off_s + L_s) with off_s the exclusive
 *                    prefix sum of the lengths.  Must be aligned to the element size.
 *                    May be NULL with lengths_dev when every length is zero; if
 *                    they sum above zero, nothing is written and the device's
 *                    error word latches ZIG_ERR_INVALID_ARG.
 * workspace_dev,     scratch for the variable-length path (lengths_dev != NULL):
 * workspace_bytes    at least zig_generate_workspace_bytes(n_streams) bytes,
 *                    16-byte aligned, owned by the caller and not used by any
 *                    other call in flight.  NULL/0 with lengths_dev != NULL makes
 *                    the call allocate its scratch on `stream` (cudaMallocAsync)
 *                    and free it there after its launch (cudaFreeAsync), so calls
 *                    on different streams never share it, and a call captured
 *                    into a graph gives the graph its own allocation.  Ignored
 *                    when lengths_dev is NULL.
 * stream             cudaStream_t.
 *
 * The sum of all lengths must be < 2^40: a variable-length batch that reaches
 * it writes nothing and latches ZIG_ERR_INVALID_ARG in the error word.  Errors:
 * ZIG_ERR_INVALID_ARG for bad enums, NULL pointers, chunk_log2 out of range,
 * misaligned buffers or too small a workspace; ZIG_ERR_NOT_INITIALIZED if
 * zig_tables_init(device) was not called for the current device.
 */
zig_status zig_generate(zig_prng prng, zig_alg alg, const uint64_t *seeds_dev,
                        const uint64_t *lengths_dev, uint64_t uniform_len, uint64_t n_streams,
                        uint32_t chunk_log2, zig_dtype dtype, void *out_dev,
                        void *workspace_dev, size_t workspace_bytes, void *stream);

/* Bytes of workspace zig_generate needs for n_streams variable-length streams. */
size_t zig_generate_workspace_bytes(uint64_t n_streams);

/*
 * zig_generate_checked -- zig_generate with its device-side errors latched in
 * the caller's own word status_dev (a uint32_t in device memory, 4-byte
 * aligned) instead of the device's shared word, so that concurrent callers
 * cannot read or clear one another's errors.  The call ORs error bits into the
 * word and never clears it: zero it before the call, read it after the stream
 * has passed the call, and turn it into a status with zig_status_decode.
 * Computes exactly what zig_generate computes; errors as zig_generate, and
 * ZIG_ERR_INVALID_ARG for a NULL or misaligned status_dev.
 */
zig_status zig_generate_checked(zig_prng prng, zig_alg alg, const uint64_t *seeds_dev,
                                const uint64_t *lengths_dev, uint64_t uniform_len, uint64_t n_streams,
                                uint32_t chunk_log2, zig_dtype dtype, void *out_dev,
                                void *workspace_dev, size_t workspace_bytes, uint32_t *status_dev,
                                void *stream);

/* The status an error word holds (the word of zig_generate_checked, or the value
 * zig_device_status reads): ZIG_OK, ZIG_ERR_INVALID_ARG (a NULL output for
 * lengths summing above zero, lengths summing to 2^40 or more, or a stream
 * record seeded for another generator) or
 * ZIG_ERR_CHUNK_OVERFLOW, in that order of precedence.  No CUDA call. */
zig_status zig_status_decode(uint32_t word);

/*
 * Streams that continue across calls.  The paper's nextGaussian draws from a
 * generator object that the caller keeps between calls (Sec. 2, Listing 2); a
 * zig_stream_state is that object for one stream, held in device memory.
 * zig_state_init seeds the records; each zig_generate_state call continues
 * every stream where its previous call stopped and advances its record, so
 * that L1 outputs followed by L2 outputs equal the first L1 + L2 outputs that
 * one call takes (and that zig_generate with chunk_log2 = 0 takes from the
 * same seed), for every transform, generator and dtype.
 *
 *  gen           the generator's state words, positioned at the stream's next
 *                raw draw: LCG48 and SplitMix64 gen[0] = s; L64X128Mix gen[0..3]
 *                = a, s, x0, x1; Xoroshiro128PlusPlus gen[0..1] = x0, x1.
 *  polar_cached  the polar method's second variate of its last pair, pending
 *  polar_have    when polar_have = 1: the next ZIG_POLAR call returns it first.
 *                A call of another transform on the stream discards it.
 *  prng          the generator the record was seeded for.  A call with another
 *                generator writes nothing for that stream and latches
 *                ZIG_ERR_INVALID_ARG in the error word.
 * 48 bytes per stream, 16-byte aligned arrays, owned by the caller.
 */
typedef struct {
    uint64_t gen[4];
    double polar_cached;
    uint32_t polar_have;
    uint32_t prng;
} zig_stream_state;

/* zig_state_init -- state_dev[s] = generator `prng` seeded with seeds_dev[s]
 * exactly as zig_generate seeds stream s, nothing pending (device buffers;
 * enqueued on stream). */
zig_status zig_state_init(zig_prng prng, const uint64_t *seeds_dev, uint64_t n_streams,
                          zig_stream_state *state_dev, void *stream);

/*
 * zig_generate_state -- zig_generate with stream s continued from state_dev[s]
 * instead of seeded, and state_dev[s] advanced past its outputs.  Each stream
 * runs as one sequential generator (no chunking), so a stream of length L is
 * one thread's work: very long streams of very uneven lengths balance worse than
 * in zig_generate's chunked form.  lengths_dev / uniform_len, n_streams, dtype,
 * out_dev, the workspace and the argument errors are those of zig_generate.
 * status_dev is the caller's error word as for zig_generate_checked, or NULL
 * for the device's shared word.  A stream of length 0 keeps its record.  The
 * records of a call must not be read or written by other work until the call
 * has completed on `stream`.
 */
zig_status zig_generate_state(zig_prng prng, zig_alg alg, zig_stream_state *state_dev,
                              const uint64_t *lengths_dev, uint64_t uniform_len, uint64_t n_streams,
                              zig_dtype dtype, void *out_dev, void *workspace_dev,
                              size_t workspace_bytes, uint32_t *status_dev, void *stream);

/*
 * zig_generate_noalloc -- zig_generate for a variable-length batch, with no
 * allocation of any kind (device or host).  The paper has no counterpart: this is an
 * integration entry point for callers that cannot allocate device memory at
 * call time, e.g. a service that has carved all of HBM into its own pools
 * before serving, a latency-bound loop that cannot absorb cudaMalloc's implicit
 * device synchronization, or a host that forbids allocations outside its
 * start-up phase.  It computes exactly what zig_generate computes for the same
 * arguments with lengths_dev != NULL (uniform batches need no scratch: use
 * zig_generate with lengths_dev = NULL).
 *
 * Its scratch (the per-stream output offsets and unit starts, 16 B per stream)
 * is a fixed array of ZIG_NOALLOC_MAX_STREAMS entries compiled into the
 * library: 1 MiB + 16 B of device memory that every GPU which loads the
 * library holds until the process exits.  The caller still owns and passes
 * seeds_dev, lengths_dev and out_dev, with the meanings and layout of
 * zig_generate.
 *  - n_streams > ZIG_NOALLOC_MAX_STREAMS returns ZIG_ERR_TOO_LARGE with nothing
 *    enqueued; split the batch or use zig_generate.
 *  - The first call on a device resolves the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.  zig_tables_init(device) must come first.
 *  - Every call shares the one array and leaves its contents behind; each call
 *    rewrites all of it that it reads, so nothing needs clearing.  Calls that
 *    overlap on the GPU (e.g. on two streams at once) race on the array and
 *    must be serialized by the caller.
 * Other errors as zig_generate.
 */
#define ZIG_NOALLOC_MAX_STREAMS 65536u
zig_status zig_generate_noalloc(zig_prng prng, zig_alg alg, const uint64_t *seeds_dev,
                                const uint64_t *lengths_dev, uint64_t n_streams,
                                uint32_t chunk_log2, zig_dtype dtype, void *out_dev,
                                void *stream);

/*
 * Launch configuration of the 128-level generation kernel (ZIG_ZIG128).  The
 * paper's single-threaded Java generator has no counterpart; these knobs only
 * change how the same work is laid out on the GPU, never the values:
 *  block        threads per block, a multiple of 32 in [64, 640] (default 640),
 *               lowered at launch to what one SM's shared memory holds for the
 *               generator.
 *  batch        slots of a lane's row per batch that a row store writes: 32, the
 *               only value (min(32, S - 2 kU) draws per batch, kU the raw steps
 *               of one nextDouble, S = 35 slots per row for 32-bit draws and 34
 *               for nextLong ones; slots past 32 hold uniforms drawn past the batch).
 *  store_bytes  0, the only value: the warp writes each row with one store per
 *               lane, the row's batch as one contiguous run, for every dtype.
 *  fma_of_4     ZIG_F64: of every 4 rows, how many rebuild their values with one
 *               binary64 fused multiply-add per value; the others use the same
 *               correctly rounded product in 32-bit integer arithmetic (GB300's
 *               binary64 pipe is narrow).  2, 3 or 4; 0 = the library's default
 *               for the generator.  Must be 0 for ZIG_F32 and ZIG_BF16, whose
 *               rows take one binary32 multiplication per value.
 * One configuration is kept per device, PRNG, dtype and input form
 * (variable_lengths = 1 for calls with a lengths array, 0 for uniform ones);
 * zig_generate and zig_generate_noalloc read it at each call.
 */
typedef struct {
    uint32_t block;
    uint32_t batch;
    uint32_t store_bytes;
    uint32_t fma_of_4;
} zig_launch_config;

/* The recorded configuration (the default if none was set). No CUDA call. */
zig_status zig_launch_config_get(int device, zig_prng prng, zig_dtype dtype, int variable_lengths,
                                 zig_launch_config *cfg);
/* Record cfg (validated as above: ZIG_ERR_INVALID_ARG otherwise); cfg = NULL
 * restores the default.  No CUDA call. */
zig_status zig_launch_config_set(int device, zig_prng prng, zig_dtype dtype, int variable_lengths,
                                 const zig_launch_config *cfg);
/* The configurations zig_autotune tries for dtype (ZIG_F64: blocks
 * 256/384/512/640 x fma_of_4 2/3/4; otherwise blocks 256/384/512/768 x both batch
 * widths x both store widths): writes up to max_cands of them to cands (may be
 * NULL) and returns how many there are. */
uint32_t zig_autotune_candidates(zig_dtype dtype, zig_launch_config *cands, uint32_t max_cands);
/*
 * zig_autotune -- time every candidate configuration on the caller's own
 * ZIG_ZIG128 request and record the fastest for the current device, prng,
 * dtype and input form.  The arguments are zig_generate's (alg = ZIG_ZIG128).
 * Each candidate runs once untimed and then `reps` times (1..1000) back to back
 * on `stream`, timed with CUDA events; the call synchronizes on the events and
 * returns the chosen configuration in *best and its mean time per call in
 * *best_ms (either may be NULL).  out_dev holds the request's outputs when it
 * returns, as after zig_generate.  ZIG_ERR_INVALID_ARG while the stream is
 * being captured into a graph; other errors as zig_generate.
 */
zig_status zig_autotune(zig_prng prng, const uint64_t *seeds_dev, const uint64_t *lengths_dev,
                        uint64_t uniform_len, uint64_t n_streams, uint32_t chunk_log2,
                        zig_dtype dtype, void *out_dev, void *workspace_dev, size_t workspace_bytes,
                        uint32_t reps, zig_launch_config *best, float *best_ms, void *stream);

/*
 * zig_mutate -- Gaussian mutation x += sigma * N(0,1) in place (the paper's
 * motivating workload, Sec. 1: Gaussian mutation in an evolutionary algorithm).
 * x_dev: P x L binary32 row-major population (device).  Row p draws its L
 * variates from stream p of the 128-level ziggurat with binary32 output, seeded
 * seed + p and split into 2^10-variate chunks, so row p's increments equal
 * zig_generate(prng, ZIG_ZIG128, seeds = {seed + p}, uniform_len = L,
 * chunk_log2 = 10, ZIG_F32) and x[p][l] = fmaf(sigma, z[p][l], x[p][l]).
 * P * L must be < 2^40; sigma must be finite.
 */
zig_status zig_mutate(float *x_dev, float sigma, uint64_t P, uint64_t L, uint64_t seed,
                      zig_prng prng, void *stream);

/*
 * zig_mutate_state -- zig_mutate whose row p continues the stream kept in
 * state_dev[p] (P records, zig_stream_state) as one sequential generator and
 * advances it: row p's increments are the next L outputs of that stream, i.e.
 * zig_generate_state(prng, ZIG_ZIG128, state_dev, uniform_len = L, ZIG_F32) on
 * it, so that mutating the same population again continues its streams.
 * Records seeded for another generator leave their rows unchanged and latch
 * ZIG_ERR_INVALID_ARG in the device's error word.
 */
zig_status zig_mutate_state(float *x_dev, float sigma, uint64_t P, uint64_t L,
                            zig_stream_state *state_dev, zig_prng prng, void *stream);

/* Request kinds of a batch (zig_mutation.kind). */
#define ZIG_REQ_MUTATE 0u   /* x_dev += sigma * N(0,1), exactly as zig_mutate */
#define ZIG_REQ_GENERATE 1u /* x_dev = N(0,1) (sigma ignored): row p equals
                               zig_generate(prng, ZIG_ZIG128, seeds = {seed + p},
                               uniform_len = L, chunk_log2 = 10, ZIG_F32) */

/* One request of a batch on a P x L binary32 row-major device buffer x_dev.
 * kind is ZIG_REQ_MUTATE (the zero default) or ZIG_REQ_GENERATE.  state_dev
 * NULL: rows seeded seed + p and chunked as zig_mutate.  Otherwise P stream
 * records: row p continues state_dev[p] as zig_mutate_state does (seed
 * ignored) and advances it; two requests of one batch must not share records. */
typedef struct {
    float *x_dev;
    uint64_t P, L;
    float sigma;
    uint32_t kind;
    uint64_t seed;
    zig_stream_state *state_dev;
} zig_mutation;

/*
 * zig_mutate_batch -- n_req mutation requests in one launch (continuous
 * batching of the Gaussian-mutation workload, Sec. 1).  Each request's result is
 * identical to zig_mutate (zig_mutate_state for a request with stream records)
 * on it alone; requests must not overlap in memory.
 * reqs_host: host array (copied before the call returns).  desc_dev: device
 * scratch of at least zig_mutate_batch_desc_bytes(n_req) bytes, 16-byte aligned,
 * not used by another call in flight.  All requests use one generator `prng`.
 * The call copies the descriptors from host memory it owns only for the call, so
 * it is refused (ZIG_ERR_INVALID_ARG) while `stream` is being captured into a graph.
 */
size_t zig_mutate_batch_desc_bytes(uint32_t n_req);
zig_status zig_mutate_batch(const zig_mutation *reqs_host, uint32_t n_req, zig_prng prng,
                            void *desc_dev, size_t desc_bytes, void *stream);

/*
 * Continuous-batching service for mutation and generation requests (serving
 * form of Sec. 1's workload); both kinds share the queue, the budget and the
 * batched launches.  A worker thread admits submitted requests in arrival order while
 * the bytes of the populations in flight stay within budget_bytes, packs up to
 * max_batch of them into one zig_mutate_batch launch on one of n_slots streams,
 * and retires a launch when its CUDA event completes; requests that arrive
 * meanwhile go to the next free slot, so launches overlap on the device.  Each
 * result equals zig_mutate (zig_mutate_state for requests on a population kept
 * by the service) on that request alone.  Populations are
 * caller-owned device memory and must not overlap while in flight.
 * device < 0 runs the scheduler without a GPU (launches complete after a
 * simulated time), for testing the admission logic.
 *
 * zig_server_create  -- start a service (allocates its streams, events and a
 *                       descriptor buffer per slot).
 * zig_server_submit  -- enqueue x += sigma * N(0,1) on P x L binary32 x_dev with
 *                       row seeds seed + p; returns a ticket.  A population larger
 *                       than the budget is refused with ZIG_ERR_BUDGET.
 * zig_server_wait    -- block until the ticket completes (timeout_s < 0: no
 *                       limit; ZIG_ERR_TIMEOUT on expiry); returns its status.
 * zig_server_query   -- state (0 queued, 1 running, 2 done, 3 failed), latency
 *                       from submit to completion and queueing time, in us.
 * zig_server_drain   -- wait until nothing is queued or running.
 * zig_server_stats   -- counts, p50 / p99 latency, batching and peak memory.
 * zig_server_destroy -- finish all work and stop.
 */
typedef struct zig_server zig_server;
typedef struct {
    uint64_t submitted, completed, failed, elements;
    double latency_p50_us, latency_p99_us, span_us;
    uint64_t batches;
    double mean_batch;
    uint64_t peak_inflight_bytes;
    uint32_t peak_busy_slots, reserved;
} zig_serving_stats;
zig_status zig_server_create(int device, zig_prng prng, uint64_t budget_bytes, uint32_t n_slots,
                             uint32_t max_batch, zig_server **out);
zig_status zig_server_submit(zig_server *server, float *x_dev, uint64_t P, uint64_t L, float sigma,
                             uint64_t seed, uint64_t *ticket);
/* A generation request (ZIG_REQ_GENERATE) into out_dev, P x L binary32; admitted,
 * batched and reported like mutation requests (the same tickets and queue). */
zig_status zig_server_submit_generate(zig_server *server, float *out_dev, uint64_t P, uint64_t L,
                                      uint64_t seed, uint64_t *ticket);
/*
 * Populations whose streams the service keeps on the device, so that repeated
 * requests on one population continue its rows' streams (an evolutionary
 * algorithm mutating the same population once per generation).
 * zig_server_population          -- P stream records seeded seed + p
 *                                   (zig_state_init; device memory the service
 *                                   owns, 48 B per row); returns a handle.
 * zig_server_submit_population   -- a request (kind ZIG_REQ_MUTATE or
 *                                   ZIG_REQ_GENERATE) on P x L binary32 x_dev
 *                                   whose rows continue the population's
 *                                   streams (zig_mutate_state).  Requests on
 *                                   one population run one at a time, in
 *                                   submission order: a request waits at the
 *                                   head of the queue while an earlier one on
 *                                   its population is in flight.
 * zig_server_population_release  -- wait until no queued or running request uses
 *                                   the population, then free its records.
 */
zig_status zig_server_population(zig_server *server, uint64_t P, uint64_t seed, uint64_t *population);
zig_status zig_server_submit_population(zig_server *server, uint64_t population, float *x_dev,
                                        uint64_t L, float sigma, uint32_t kind, uint64_t *ticket);
zig_status zig_server_population_release(zig_server *server, uint64_t population);
zig_status zig_server_wait(zig_server *server, uint64_t ticket, double timeout_s);
zig_status zig_server_query(zig_server *server, uint64_t ticket, int *state, double *latency_us,
                            double *queue_us);
zig_status zig_server_drain(zig_server *server, double timeout_s);
zig_status zig_server_stats(zig_server *server, zig_serving_stats *out);
zig_status zig_server_destroy(zig_server *server);

/*
 * zig_prng_fill -- raw uniform draws, for bit-exact checks of the generators.
 * out_dev: n_streams x n uint64 (device), stream-major.  kind 0 = nextInt
 * (32-bit, zero-extended), 1 = nextLong, 2 = the 53-bit integer behind
 * nextDouble.  Each stream is first advanced by `skip` raw steps with the
 * closed-form jump.
 */
zig_status zig_prng_fill(zig_prng prng, const uint64_t *seeds_dev, uint64_t n_streams,
                         uint64_t n, uint64_t skip, int kind, uint64_t *out_dev, void *stream);

/*
 * zig_device_status -- read (and, if clear != 0, reset) the device's shared
 * error word, which every call but zig_generate_checked latches into.
 * Synchronizes the device.  Returns zig_status_decode of the word, or
 * ZIG_ERR_CUDA.  Concurrent callers share this word (one caller's clear erases
 * another's flag): callers that need their own scope use zig_generate_checked.
 */
zig_status zig_device_status(int device, int clear);

/* Human-readable name of a status code (static storage). */
const char *zig_status_string(zig_status status);

/*
 * zig_selfcheck -- exhaustive check of the fast path's arithmetic on the current
 * device (test support; the paper has no counterpart).  Computes RN(j * w[i])
 * for every abscissa j < 2^24 of every layer i < 128 by each construction the
 * kernels use -- the fused multiply-add one, and the binary64 batch kernel's
 * fused multiply-add and 32-bit integer ones on both signed table entries
 * (+-2^52 w[i]) -- and compares each with IEEE multiplication (__dmul_rn, negated
 * for the negative entries); rounds every finite binary32 bit pattern to
 * bfloat16 by the kernel's routine and compares it with __float2bfloat16_rn,
 * 2^32 binary64 values in [2^-112, 16) of both signs to binary32 and to bfloat16
 * and compares them with __double2float_rn and __double2bfloat16, and the same
 * for 2^31 exact ties and tie neighbours each; and compares the tail step's own binary64 log
 * with CUDA's log on 2^31 uniforms in (0, 1).  Writes counts_host[0] = product
 * mismatches, [1] = rounding mismatches, [2] = products checked (5 * 2^31),
 * [3] = roundings checked, [4] = logs more than one ulp from CUDA's, [5] = logs
 * not equal to CUDA's.
 * Synchronous; allocates 48 bytes of device memory for the call.
 * ZIG_ERR_NOT_INITIALIZED without zig_tables_init.
 */
zig_status zig_selfcheck(uint64_t counts_host[6]);

/*
 * zig_filtercheck -- the slow tests' binary32 filters against their binary64
 * definitions on the current device (test support).  The kernels decide each
 * slow test first in binary32 and leave it to binary64 only inside a margin
 * that must cover every binary32 error: the 128-level wedge test (Sec. 1, the
 * GSL form's wedge comparison) and tail test, and the modified ziggurat's
 * overhang and tail tests (Sec. 2, "Java 17").  For each test f (0 wedge,
 * 1 tail, 2 overhang, 3 the 256-slot tail) 2^27 inputs: half uniform, with the
 * tails' uniforms spread over every binary scale down to 2^-53, half within
 * 2^-8 of the test's boundary.  Writes counts_host[3 f] = inputs checked,
 * [3 f + 1] = inputs the filter left undecided, [3 f + 2] = inputs the filter
 * decided unlike the binary64 definition (0 when its margin holds).
 * Synchronous; allocates 96 bytes of device memory for the call.
 * ZIG_ERR_INVALID_ARG for a NULL counts_host; ZIG_ERR_NOT_INITIALIZED without
 * zig_tables_init.
 */
zig_status zig_filtercheck(uint64_t counts_host[12]);

/* Library version as major * 10000 + minor * 100 + patch. */
int zig_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ZIG_GB300_H */
