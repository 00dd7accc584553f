// libzig_gb300: bulk N(0,1) generation on GB300 (sm_103a) behind the C ABI in
// include/zig.h.  One thread owns one (stream, chunk) unit with its generator
// state in registers; the 32 units of a warp are staged in shared memory and
// written out as coalesced rows.  The two ziggurats run in batch kernels
// (z128_batch.cuh, z256_batch.cuh); this file holds the shared device code,
// the polar kernel, the checks and the host side.
//
// Transforms (Sec. 2, second list; Table 3):
//   zig128  original ziggurat in the GSL form: a 32-bit draw gives layer i
//           (7 bits), the sign (bit 7) and j (24 bits); accept x = j * w[i] if
//           j < k[i]; else the wedge test (i < 127) or the tail (i = 127); on
//           rejection start over with a fresh draw.
//   polar   Marsaglia's polar method; the second variate of a pair is cached.
//   zig256  modified ziggurat after McFarland: 253 equal-area rectangles under
//           the curve are accepted with no test; overhangs and the tail are
//           picked by a 256-bin alias table and sampled by rejection.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "../../include/zig.h"
#include "zig_device.cuh"
#include "zig_tables.inc"

namespace zig {

// ---------------------------------------------------------------------------
// device-resident immutable tables (filled by zig_tables_init)
// ---------------------------------------------------------------------------
__device__ uint32_t d_z128_kE[128];   // K[i] | (E(w[i]) - 900) << 24
__device__ double d_z128_W[128];
__device__ double d_z128_Y[128];
__device__ float d_z128_W32[128];
__device__ double d_z256_XS[256];
__device__ double d_z256_OX[256], d_z256_ODX[256], d_z256_OY[256], d_z256_ODY[256];
__device__ float d_z256_F32[4][256];   // RN32 of OX, ODX, OY, ODY (the overhang filter's operands)
__device__ int d_z256_KIND[256];
__device__ uint64_t d_z256_QA[256];
__device__ uint64_t d_z256_THR[256];
__device__ int d_z256_ALIAS[256];
__device__ JumpTab d_jump;
__device__ unsigned d_err;

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr uint64_t kChunkDraws = 1ull << 32;   // raw steps between chunk starts

// ---------------------------------------------------------------------------
// work units
// ---------------------------------------------------------------------------
struct GenArgs {
    const uint64_t* seeds;
    const uint64_t* lengths;   // NULL: uniform
    uint64_t uniform_len;
    uint64_t n_streams;
    uint32_t chunk_log2;       // 0: one unit per stream
    void* out;
    const uint64_t* offsets;   // variable length: exclusive prefix sum of lengths
    const uint64_t* ustart;    // variable length: exclusive prefix sum of unit counts
    const uint64_t* totals;    // variable length: [0] = number of units
    uint64_t n_units;          // uniform: number of units
    uint64_t units_per_stream; // uniform: units per stream
    float sigma;               // mutation only
    uint64_t mut_seed;         // mutation only: row p is seeded mut_seed + p
    const struct MutDesc* reqs;  // batched mutation: request descriptors
    uint32_t n_req;              // batched mutation: number of requests
    unsigned* err;               // where device-side errors are latched (a caller's word or the device's)
    zig_stream_state* state;     // stream records to continue and advance (chunk_log2 = 0), or NULL
};

// One mutation request of a batch (device copy; ustart = its first unit).
struct MutDesc {
    float* x;
    uint64_t P, L, seed, upr, ustart;
    float sigma;
    uint32_t kind;   // ZIG_REQ_MUTATE: x += sigma z; ZIG_REQ_GENERATE: x = z
    zig_stream_state* state;   // rows continue these records (one unit per row), or NULL
};

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// A stream record's generator (false, and the error bit, for a record seeded
// for another generator).
template <int PRNG, class G>
__device__ __forceinline__ bool state_load(const zig_stream_state* r, G& g, unsigned* err, bool& ok) {
    if (r->prng != (uint32_t)PRNG) {
        atomicOr(err, kErrStateKind);
        ok = false;
        return false;
    }
    g.load(r->gen);
    return true;
}

// Advance a stream record past its unit: the generator at the stream's next raw
// draw, and the polar method's pending second variate (none for the others).
template <class G>
__device__ __forceinline__ void state_store(zig_stream_state* r, const G& g, bool have, double cached) {
    g.save(r->gen);
    r->polar_cached = have ? cached : 0.0;
    r->polar_have = have ? 1u : 0u;
}

// Resolve unit u to (stream s, chunk q, output offset, output count).
__device__ __forceinline__ void unit_info(const GenArgs& a, uint64_t u, uint64_t& s, uint64_t& q,
                                          uint64_t& off, uint64_t& n) {
    const uint32_t c = a.chunk_log2;
    if (a.lengths == nullptr) {
        if (c == 0) {
            s = u;
            q = 0;
            off = u * a.uniform_len;
            n = a.uniform_len;
        } else {
            s = u / a.units_per_stream;
            q = u - s * a.units_per_stream;
            uint64_t t0 = q << c;
            off = s * a.uniform_len + t0;
            n = umin64(a.uniform_len - t0, (uint64_t)1 << c);
        }
    } else {
        // last stream whose first unit is <= u (streams without units are skipped)
        uint64_t lo = 0, hi = a.n_streams;   // invariant: ustart[lo] <= u < ustart[hi]
        while (hi - lo > 1) {
            uint64_t mid = (lo + hi) >> 1;
            if (a.ustart[mid] <= u) lo = mid; else hi = mid;
        }
        s = lo;
        q = u - a.ustart[s];
        uint64_t L = a.lengths[s];
        uint64_t t0 = c ? (q << c) : 0;
        off = a.offsets[s] + t0;
        n = c ? umin64(L - t0, (uint64_t)1 << c) : L;
    }
}

__device__ __forceinline__ uint64_t units_total(const GenArgs& a) {
    return a.lengths ? a.totals[0] : a.n_units;
}

// The generator of unit (stream s, chunk q): seeded from seeds[s] and moved to
// chunk q, or continued from the stream's record a.state[s] (calls with records
// have one unit per stream).  Returns the record to advance at the unit's end
// (NULL without records); ok = false for a record of another generator, whose
// stream then gets no outputs.
template <int PRNG, class G>
__device__ __forceinline__ zig_stream_state* unit_gen(const GenArgs& a, uint64_t s, uint64_t q, G& g, bool& ok) {
    ok = true;
    if (a.state == nullptr) {
        g.seed(a.seeds[s]);
        if (q) g.jump(q * kChunkDraws, &d_jump);
        return nullptr;
    }
    zig_stream_state* r = a.state + s;
    return state_load<PRNG>(r, g, a.err, ok) ? r : nullptr;
}

// ---------------------------------------------------------------------------
// per-variate samplers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double neg_half_sq(double x) {
    return __dmul_rn(__dmul_rn(-0.5, x), x);
}

// Natural logarithm of a positive normal binary64 x, by P. T. P. Tang's
// table-driven method (ACM TOMS 16(4), 1990), all inline (no call):
// x = 2^e m with m in [1, 2); F = 1 + k/128 is the table point nearest m;
// r = (m - F)/F from f = m - F (exact) and G = RN(1/F), refined by one fused
// multiply-add step; ln(1 + r) = r + r^2 q(r) with q the Taylor series to r^7
// (|r| <= 2^-8, truncation below 2^-59 relative); and
// ln x = (e ln2_hi + ln F_hi) + (r + (r^2 q + e ln2_lo + ln F_lo)), the first
// sum exact (hi parts on the grid 2^-40).  Error about half an ulp;
// zig_selfcheck compares it with CUDA's log.
__constant__ double c_log_g[129], c_log_thi[129], c_log_tlo[129];

__device__ __forceinline__ double zlog(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const double e = (double)((int)(b >> 52) - 1023);
    const uint64_t frac = b & ((1ull << 52) - 1);
    const double m = __longlong_as_double((long long)(frac | (1023ull << 52)));
    const int k = (int)(((frac >> 44) + 1) >> 1);                  // nearest k/128: 0..128
    const double F = __dadd_rn(1.0, __dmul_rn((double)k, 0.0078125));   // exact
    const double f = __dsub_rn(m, F);                               // exact
    const double G = c_log_g[k];
    double r = __dmul_rn(f, G);
    r = __fma_rn(__fma_rn(-r, F, f), G, r);
    double q = 1.0 / 7;
    q = __fma_rn(q, r, -1.0 / 6);
    q = __fma_rn(q, r, 1.0 / 5);
    q = __fma_rn(q, r, -0.25);
    q = __fma_rn(q, r, 1.0 / 3);
    q = __fma_rn(q, r, -0.5);
    const double hi = __fma_rn(e, zigtab::LN2_HI, c_log_thi[k]);   // exact
    const double lo = __fma_rn(__dmul_rn(r, r), q, __fma_rn(e, zigtab::LN2_LO, c_log_tlo[k]));
    return __dadd_rn(hi, __dadd_rn(r, lo));
}

// binary64 value of an integer m < 2^53 (exact), scaled by 2^-k, built with
// integer operations: GB300's conversion to binary64 runs on the narrow binary64 pipe.
__device__ __forceinline__ double u53_to_double(uint64_t m, int k = 0) {
    const int lz = __clzll((long long)m);   // 11..63 (64 for m = 0)
    const uint64_t frac = ((m << (lz & 63)) >> 11) & ((1ull << 52) - 1);
    const uint64_t bits = ((uint64_t)(1086 - lz - k) << 52) | frac;
    return m ? __longlong_as_double((long long)bits) : 0.0;
}

// 2 u - 1 for u = m 2^-53 (m < 2^53): the two roundings of RN(RN(2 u) - 1) are
// exact, and the value is (m - 2^52) 2^-52, built here with integer operations
// (GB300's binary64 pipe is narrow; the polar method spends it on log, division
// and square root).
__device__ __forceinline__ double polar_v(uint64_t m) {
    const int64_t d = (int64_t)m - (1ll << 52);   // |d| < 2^52
    const double r = u53_to_double((uint64_t)(d < 0 ? -d : d), 52);
    return d < 0 ? __longlong_as_double(__double_as_longlong(r) ^ (long long)(1ull << 63)) : r;
}

// Polar method with the cached second variate (`extra` counts the raw steps).
template <class G>
__device__ __forceinline__ double polar_f64(G& g, bool& have, double& cached, uint32_t& extra) {
    if (have) {
        have = false;
        return cached;
    }
    constexpr uint32_t kStepsPerDouble = std::is_same<G, GenLcg48>::value ? 2u : 1u;
    double v1, v2, s;
    do {
        v1 = polar_v(g.next_m53());
        v2 = polar_v(g.next_m53());
        s = __dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2));
        extra += 2 * kStepsPerDouble;
    } while (s >= 1.0 || s == 0.0);
    double mult = __dsqrt_rn(__ddiv_rn(__dmul_rn(-2.0, zlog(s)), s));
    cached = __dmul_rn(v2, mult);
    have = true;
    return __dmul_rn(v1, mult);
}

// Modified ziggurat, 256 slots.
struct Z256Smem {
    double XS[256];
    uint64_t THR[256];
    int ALIAS[256];
};

__device__ __forceinline__ void z256_load(Z256Smem& t) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        t.XS[i] = d_z256_XS[i];
        t.THR[i] = d_z256_THR[i];
        t.ALIAS[i] = d_z256_ALIAS[i];
    }
}

// binary32 filter for an overhang test y < exp(-x^2/2): x = ox + odx u, y = oy + ody v
// with u, v in [0, 1).  The binary32 errors are below 3e-6 relative (x < 3.7,
// expf within 2 ulp), far inside the 2^-16 margin; returns 1 accept, 0 reject,
// -1 undecided (evaluate in binary64).
__device__ __forceinline__ int z256_overhang_filter(float ox, float odx, float oy, float ody, uint64_t m1,
                                                    uint64_t m2) {
    const float u = (float)(uint32_t)(m1 >> 29) * 0x1p-24f;
    const float v = (float)(uint32_t)(m2 >> 29) * 0x1p-24f;
    const float x = __fmaf_rn(odx, u, ox);
    const float y = __fmaf_rn(ody, v, oy);
    const float e = expf(-0.5f * x * x);
    if (y < e * (1.0f - 0x1p-16f)) return 1;
    if (y > e * (1.0f + 0x1p-16f)) return 0;
    return -1;
}

// ---------------------------------------------------------------------------
// output conversion
// ---------------------------------------------------------------------------
template <int DT> struct OutOf;
template <> struct OutOf<ZIG_F64> { using T = double; };
template <> struct OutOf<ZIG_F32> { using T = float; };
template <> struct OutOf<ZIG_BF16> { using T = uint16_t; };

template <int DT> __device__ __forceinline__ typename OutOf<DT>::T from_f64(double z);
template <> __device__ __forceinline__ double from_f64<ZIG_F64>(double z) { return z; }
template <> __device__ __forceinline__ float from_f64<ZIG_F32>(double z) { return __double2float_rn(z); }
template <> __device__ __forceinline__ uint16_t from_f64<ZIG_BF16>(double z) { return f64_to_bf16_bits(z); }

// ---------------------------------------------------------------------------
// generation kernel
// ---------------------------------------------------------------------------
// The polar method (Marsaglia), one stream per lane, outputs staged per warp.
template <int ALG, int PRNG, int DT>
__global__ void __launch_bounds__(kBlock) polar_kernel(GenArgs a) {
    using G = typename GenOf<PRNG>::T;
    using OutT = typename OutOf<DT>::T;
    static_assert(ALG == ZIG_POLAR, "the ziggurats run in their batch kernels");
    __shared__ OutT stage_all[kWarps][32 * kStageCols];

    const int lane = threadIdx.x & 31;
    OutT* stage = stage_all[threadIdx.x >> 5];
    if (a.out == nullptr) {   // only legal when every length is zero
        if (a.lengths && a.totals[1] != 0 && blockIdx.x == 0 && threadIdx.x == 0)
            atomicOr(a.err, kErrNullOutput);
        return;
    }
    const uint64_t n_units = units_total(a);
    const uint64_t n_groups = (n_units + 31) >> 5;
    const uint64_t warp_id = (uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const uint64_t warp_stride = (uint64_t)gridDim.x * kWarps;
    OutT* out = (OutT*)a.out;

    for (uint64_t grp = warp_id; grp < n_groups; grp += warp_stride) {
        uint64_t u = grp * 32 + lane;
        uint64_t rem = 0;
        OutT* dst = out;
        G g;
        g.seed(0);
        zig_stream_state* srec = nullptr;
        bool have = false;   // polar: the second variate of the last pair is pending
        double cached = 0.0;
        if (u < n_units) {
            uint64_t s, q, off, n;
            unit_info(a, u, s, q, off, n);
            bool ok;
            srec = unit_gen<PRNG>(a, s, q, g, ok);
            if (ok) {
                rem = n;
                dst = out + off;
            }
            if (ALG == ZIG_POLAR && srec && srec->polar_have) {
                have = true;
                cached = srec->polar_cached;
            }
        }
        const uint64_t n_unit = rem;
        uint32_t extra = 0;
        while (__any_sync(kFull, rem > 0)) {
            const int cnt = (int)umin64(rem, (uint64_t)kStageCols);
#pragma unroll 1
            for (int v = 0; v < kStageCols; ++v) {
                if (v < cnt) {
                    stage[stage_idx<OutT>(lane, v)] = from_f64<DT>(polar_f64(g, have, cached, extra));
                }
            }
            __syncwarp();
            stage_flush<OutT>(stage, dst, cnt, lane);
            __syncwarp();
            dst += cnt;
            rem -= cnt;
        }
        // A chunk must stay inside its 2^32-draw window; `extra` counts the raw steps.
        if (a.chunk_log2 && n_unit && (uint64_t)extra > kChunkDraws) atomicOr(a.err, kErrChunkOverflow);
        // a lane draws only for its own outputs, so g stands at the stream's next draw
        if (srec && n_unit) state_store(srec, g, have, cached);
    }
}

// ---------------------------------------------------------------------------
// 128-level ziggurat (GSL form): the slow tests shared by the batch kernel
// ---------------------------------------------------------------------------
__device__ float d_z128_Y32[128];
__device__ float d_z128_DY32[128];

// RN(j * w) with one binary64 fma, given b = 2^52 w: a = 1 + j 2^-52 (built
// from bits; j < 2^24) gives a b - b = j w exactly before the single rounding.
// (An exact zero comes out as +0; the caller sets the sign.)
__device__ __forceinline__ double mul_j_w(uint32_t j, double b) {
    return __fma_rn(__hiloint2double(0x3FF00000, (int)j), b, -b);
}

// binary32 value of m * 2^-53 for m < 2^53, correctly rounded (relative error
// at most 2^-24 at every scale: the slow tests take logarithms of uniforms far
// below 2^-8, where keeping only the top 24 of 53 bits would not do).
__device__ __forceinline__ float m53_to_float(uint64_t m) {
    return __fmul_rn(__ull2float_rn(m), 0x1p-53f);   // the scaling is exact
}

// The wedge test for layer i, abscissa j and uniform U = m1 2^-53:
// y = y[i+1] + (y[i] - y[i+1]) U < exp(-x^2/2) with x = RN(j w[i]).  Decided in
// binary32 when |y32 - e32| clears 2^-16 e32 (the binary32 errors are
// |y32/y - 1| + |e32/e - 1| <= 2.6e-6, expf within 2 ulp); inside the margin
// the binary64 definition decides.
// z128_wedge_filter: 1 accept, 0 reject, -1 inside the margin;
// z128_wedge_exact: the binary64 definition.
template <class Tab>
__device__ __forceinline__ int z128_wedge_filter(const Tab& t, uint32_t i, uint32_t j, uint64_t m1) {
    const float x32 = __fmul_rn((float)j, t.W32[i]);
    const float e32 = expf(__fmul_rn(__fmul_rn(-0.5f, x32), x32));
    const float u32 = (float)(uint32_t)(m1 >> 29) * 0x1p-24f;
    const float y32 = __fadd_rn(t.Y32[i + 1], __fmul_rn(t.DY32[i], u32));
    if (y32 < e32 * (1.0f - 0x1p-16f)) return 1;
    if (y32 > e32 * (1.0f + 0x1p-16f)) return 0;
    return -1;
}
template <class Tab>
__device__ __forceinline__ bool z128_wedge_exact(const Tab& t, uint32_t i, uint32_t j, uint64_t m1) {
    const double x = __dmul_rn((double)j, t.Wd[i]);
    const double U = m53_to_double(m1);
    const double y = __dadd_rn(t.Y[i + 1], __dmul_rn(__dsub_rn(t.Y[i], t.Y[i + 1]), U));
    return y < exp(neg_half_sq(x));
}

// RN(z / R) without a division: q = RN(z RN(1/R)) and one fused multiply-add
// correction, which gives the correctly rounded quotient (Markstein, IBM J. Res.
// Dev. 34(1), 1990).
__device__ __forceinline__ double div_by_R(double z) {
    constexpr double R = zigtab::ZIG128_R;
    constexpr double Rinv = 1.0 / zigtab::ZIG128_R;
    const double q = __dmul_rn(z, Rinv);
    return __fma_rn(__fma_rn(-q, R, z), Rinv, q);
}

// The tail test for U1 = 1 - m1 2^-53, U2 = m2 2^-53:
// y = exp(-R (x - R/2)) U2 < exp(-x^2/2) with x = R + s, s = -ln(U1)/R, which is
// ln U2 < -s^2/2 in exact arithmetic.  Decided in binary32 when that clears a
// margin of 2^-14 (1 + s^2/2 + |ln U2|), far above the binary32 errors (the
// hardware log2 within 2^-22.6 absolute on [0.5, 2] and 2 ulp elsewhere:
// below 1e-5 relative here); otherwise ln U2 < -s^2/2 decides in binary64.  The
// two tests agree except where the oracle's own rounding could flip its
// decision (a margin near 1e-16).
// z128_tail_filter: 1 accept, 0 reject, -1 inside the margin;
// z128_tail_exact: the binary64 decision.
__device__ __forceinline__ int z128_tail_filter(uint64_t m1, uint64_t m2) {
    if (m2 == 0) return 1;                            // U2 = 0: y = 0 < exp(-x^2/2)
    const uint64_t n1 = (1ull << 53) - m1;            // U1 = n1 2^-53 in (0, 1]
    constexpr float kLn2 = 0.693147180559945309f;
    constexpr float kLn2OverR = (float)(0.693147180559945309 / zigtab::ZIG128_R);
    const float s32 = -__log2f(m53_to_float(n1)) * kLn2OverR;
    const float h32 = 0.5f * s32 * s32;
    const float l32 = __log2f(m53_to_float(m2)) * kLn2;
    const float marg = 0x1p-14f * (1.0f + h32 - l32);
    if (l32 < -h32 - marg) return 1;
    if (l32 > -h32 + marg) return 0;
    return -1;
}
__device__ __forceinline__ bool z128_tail_exact(uint64_t m1, uint64_t m2) {
    const uint64_t n1 = (1ull << 53) - m1;
    const double s = -div_by_R(zlog(m53_to_double(n1)));
    return zlog(m53_to_double(m2)) < __dmul_rn(__dmul_rn(-0.5, s), s);
}

// The tail step's value for an accepted U1 = 1 - m1 2^-53: x = R - ln(U1)/R.
__device__ __forceinline__ double z128_tail_value(uint64_t m1) {
    const double U1 = __dsub_rn(1.0, m53_to_double(m1));
    return __dsub_rn(zigtab::ZIG128_R, div_by_R(zlog(U1)));
}

#include "z128_batch.cuh"
#include "z256_batch.cuh"

// Exhaustive check of the fast path's arithmetic against CUDA's IEEE operations:
// RN(j * w[i]) by the fused multiply-add construction against __dmul_rn for all
// 2^24 abscissae j of all 128 layers, and the bfloat16 rounding of every finite
// binary32 pattern against __float2bfloat16_rn.  Also the tail step's log
// against CUDA's log on 2^31 uniforms spread over (0, 1].  counts: product
// mismatches, bfloat16 mismatches, products checked, patterns checked, logs more
// than one ulp from CUDA's, logs not equal to CUDA's.
__global__ void __launch_bounds__(256) selfcheck_kernel(unsigned long long* counts) {
    unsigned long long bad_p = 0, bad_b = 0, n_p = 0, n_b = 0, far_l = 0, ne_l = 0;
    const uint64_t n = 1ull << 31;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(k >> 24), j = (uint32_t)k & 0xFFFFFFu;
        const double w = d_z128_W[i];
        const long long want = __double_as_longlong(__dmul_rn((double)j, w));
        const long long want_neg = want ^ (long long)0x8000000000000000ull;   // RN(-j w) = -RN(j w)
        bad_p += __double_as_longlong(mul_j_w(j, __dmul_rn(w, 0x1p52))) != want;
        // the binary64 batch kernel's two constructions, on both signed table entries
        // (the values its rows compute, from the entries its tables hold)
        for (uint32_t neg = 0; neg < 2; ++neg) {
            const long long b = __double_as_longlong(__dmul_rn(neg ? -w : w, 0x1p52));
            const uint32_t blo = (uint32_t)b, bhi = (uint32_t)(b >> 32);
            const uint32_t mhi = __funnelshift_l(blo, (bhi & 0xFFFFFu) | 0x100000u, 11);
            const uint32_t eh = (bhi & 0xFFF00000u) - (22u << 20);
            const long long vi = (long long)zf::int_mul_jw(j, blo << 11, mhi, eh);
            const double bd = __longlong_as_double(b);
            const long long vf = __double_as_longlong(__fma_rn(__hiloint2double(0x3FF00000, (int)j), bd, -bd)) |
                                 (long long)((uint64_t)(bhi & 0x80000000u) << 32);
            const long long wnt = neg ? want_neg : want;
            bad_p += (vi != wnt) + (vf != wnt);
        }
        n_p += 5;
        const double u = m53_to_double(((k * 0x9E3779B97F4A7C15ull) >> 11) | 1u);   // in (0, 1)
        // the binary64 -> binary32 and -> bfloat16 roundings of the narrow outputs, on u
        // scaled into [2^-112, 16) (every output's magnitude is below 15), of both
        // signs; then on exact ties and their neighbours (a fraction whose dropped
        // bits are half an ulp, +-1), which random fractions almost never give
        {
            const uint64_t e64 = (uint64_t)(0x3C4ull + (k % 64)) << 52;
            const double v = __dmul_rn(u, __longlong_as_double((long long)e64));
            bad_b += f64_to_f32_bits(v) != __float_as_uint(__double2float_rn(v));
            bad_b += f64_to_f32_bits(-v) != __float_as_uint(__double2float_rn(-v));
            bad_b += f64_to_bf16_bits(v) != __bfloat16_as_ushort(__double2bfloat16(v));
            bad_b += f64_to_bf16_bits(-v) != __bfloat16_as_ushort(__double2bfloat16(-v));
            const int64_t d = (int64_t)((k >> 6) % 3) - 1;
            const double t32 = __longlong_as_double((long long)(e64 | ((k >> 8) & 0x7FFFFFu) << 29 | (uint64_t)((1ll << 28) + d)));
            const double t16 = __longlong_as_double((long long)(e64 | ((k >> 8) & 0x7Fu) << 45 | (uint64_t)((1ll << 44) + d)));
            bad_b += f64_to_f32_bits(t32) != __float_as_uint(__double2float_rn(t32));
            bad_b += f64_to_bf16_bits(t16) != __bfloat16_as_ushort(__double2bfloat16(t16));
            n_b += 6;
        }
        const long long dl = __double_as_longlong(zlog(u)) - __double_as_longlong(log(u));
        far_l += dl > 1 || dl < -1;
        ne_l += dl != 0;
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h) {
            const float f = __uint_as_float((uint32_t)k | (h << 31));
            if (isfinite(f)) {
                bad_b += f32_to_bf16_bits(f) != __bfloat16_as_ushort(__float2bfloat16_rn(f));
                ++n_b;
            }
        }
    }
    atomicAdd(&counts[0], bad_p);
    atomicAdd(&counts[1], bad_b);
    atomicAdd(&counts[2], n_p);
    atomicAdd(&counts[3], n_b);
    atomicAdd(&counts[4], far_l);
    atomicAdd(&counts[5], ne_l);
}

// The slow tests' binary32 filters against their binary64 definitions: the
// 128-level wedge and tail tests, the 256-slot overhang and tail tests.  Half the
// inputs are uniform (the tails' uniforms spread over every binary scale), half
// sit at +-2^s units of 2^-53 (s < 45) from the test's boundary, where a filter
// error would show.  counts[3 f]: inputs checked for filter f, [3 f + 1]: left
// undecided (binary64 decides them), [3 f + 2]: decided unlike the definition.
__device__ __forceinline__ uint64_t near53(double v, int64_t off) {   // clamp(v 2^53 + off) to [0, 2^53)
    const double s = __dmul_rn(v, 0x1p53);
    const int64_t b = s >= 0x1p53 ? (int64_t)(1ll << 53) : s > 0.0 ? (int64_t)s : 0;
    const int64_t m = b + off;
    return m < 0 ? 0 : m >= (1ll << 53) ? (1ull << 53) - 1 : (uint64_t)m;
}
__global__ void __launch_bounds__(256) filtercheck_kernel(unsigned long long* counts, uint64_t n) {
    __shared__ zf::SlowTab st;
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        st.W32[i] = d_z128_W32[i];
        st.Y32[i] = d_z128_Y32[i];
        st.DY32[i] = d_z128_DY32[i];
        st.Wd[i] = d_z128_W[i];
        st.Y[i] = d_z128_Y[i];
    }
    __syncthreads();
    unsigned long long c[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) c[q] = 0;
    auto tally = [&](int f, int filt, bool exact) {
        c[3 * f] += 1;
        c[3 * f + 1] += filt < 0;
        c[3 * f + 2] += filt >= 0 && (filt == 1) != exact;
    };
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r0 = mix64(4 * k + 1), r1 = mix64(4 * k + 2), r2 = mix64(4 * k + 3), r3 = mix64(4 * k + 4);
        const bool near = r0 & 1u;
        const int s = (int)((r0 >> 1) % 45);
        const int64_t mag = (int64_t)((1ull << s) + (r3 & ((1ull << s) - 1u)));
        const int64_t off = ((r0 >> 8) & 1u) ? -mag : mag;
        // a uniform's integer at every scale: (53 random bits) >> (0 .. 52)
        const uint64_t spread1 = (r2 >> 11) >> ((r1 >> 58) % 53);
        const uint64_t spread2 = (r3 >> 11) >> ((r2 & 63) % 53);
        {   // 128-level wedge, layer i < 127, a slow abscissa j >= k[i]
            const uint32_t i = (uint32_t)(r1 % 127u);
            const uint32_t K = d_z128_kE[i] & 0xFFFFFFu;
            if (K < (1u << 24)) {
                const uint32_t j = K + (uint32_t)((r1 >> 8) % ((1u << 24) - K));
                uint64_t m1 = r2 >> 11;
                if (near) {
                    const double x = __dmul_rn((double)j, st.Wd[i]);
                    m1 = near53(__ddiv_rn(__dsub_rn(exp(neg_half_sq(x)), st.Y[i + 1]), __dsub_rn(st.Y[i], st.Y[i + 1])), off);
                }
                tally(0, z128_wedge_filter(st, i, j, m1), z128_wedge_exact(st, i, j, m1));
            }
        }
        {   // 128-level tail: U1 = 1 - m1 2^-53, U2 = m2 2^-53
            const uint64_t n1 = spread1 | 1u;
            const uint64_t m1 = (1ull << 53) - n1;
            uint64_t m2 = spread2;
            if (near) {
                const double sv = __ddiv_rn(-zlog(m53_to_double(n1)), zigtab::ZIG128_R);
                m2 = near53(exp(__dmul_rn(__dmul_rn(-0.5, sv), sv)), off);
            }
            tally(1, z128_tail_filter(m1, m2), z128_tail_exact(m1, m2));
        }
        {   // 256-slot overhang of table entry r
            const int r = (int)(r1 % (uint64_t)zigtab::ZIG256_NR);
            const uint64_t m1 = r2 >> 11;
            uint64_t m2 = r3 >> 11;
            const double x = __dadd_rn(d_z256_OX[r], __dmul_rn(d_z256_ODX[r], u53_to_double(m1, 53)));
            if (near && d_z256_ODY[r] != 0.0)
                m2 = near53(__ddiv_rn(__dsub_rn(exp(neg_half_sq(x)), d_z256_OY[r]), d_z256_ODY[r]), off);
            const double y = __dadd_rn(d_z256_OY[r], __dmul_rn(d_z256_ODY[r], u53_to_double(m2, 53)));
            tally(2, z256_overhang_filter(d_z256_F32[0][r], d_z256_F32[1][r], d_z256_F32[2][r], d_z256_F32[3][r], m1, m2),
                  y < exp(neg_half_sq(x)));
        }
        {   // 256-slot tail: U = 1 - m 2^-53 for both uniforms
            const uint64_t n1 = spread1 | 1u;
            const uint64_t m1 = (1ull << 53) - n1;
            uint64_t n2 = spread2 | 1u;
            if (near) {
                const double sv = __ddiv_rn(-zlog(m53_to_double(n1)), zigtab::ZIG256_X0);
                n2 = near53(exp(__dmul_rn(__dmul_rn(-0.5, sv), sv)), off);
                n2 = n2 ? n2 : 1u;
            }
            const uint64_t m2 = (1ull << 53) - n2;
            tally(3, zb::tail_filter(m1, m2), zb::tail_exact(m1, m2));
        }
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) atomicAdd(&counts[q], c[q]);
}

// Exclusive prefix sums of lengths and unit counts (one block).  Sums saturate
// at 2^40: a batch whose lengths reach it latches kErrLengthSum in *err and
// gets no units, so nothing is generated or written.
__global__ void __launch_bounds__(1024) scan_kernel(const uint64_t* lengths, uint64_t n,
                                                    uint32_t chunk_log2, uint64_t* offsets,
                                                    uint64_t* ustart, uint64_t* totals, unsigned* err) {
    constexpr uint64_t kLim = 1ull << 40;
    __shared__ uint64_t sl[1024], su[1024];
    const int t = threadIdx.x;
    const uint64_t per = (n + 1023) / 1024;
    const uint64_t b = umin64(n, (uint64_t)t * per), e = umin64(n, b + per);
    uint64_t accl = 0, accu = 0;
    for (uint64_t s = b; s < e; ++s) {
        const uint64_t L = umin64(lengths[s], kLim);
        accl = umin64(accl + L, kLim);
        accu += chunk_log2 ? ((L + (1ull << chunk_log2) - 1) >> chunk_log2) : (L ? 1 : 0);
    }
    sl[t] = accl;
    su[t] = accu;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {   // Hillis-Steele inclusive scan
        uint64_t vl = (t >= d) ? sl[t - d] : 0, vu = (t >= d) ? su[t - d] : 0;
        __syncthreads();
        sl[t] = umin64(sl[t] + vl, kLim);
        su[t] += vu;
        __syncthreads();
    }
    accl = t ? sl[t - 1] : 0;
    accu = t ? su[t - 1] : 0;
    for (uint64_t s = b; s < e; ++s) {
        const uint64_t L = umin64(lengths[s], kLim);
        offsets[s] = accl;
        ustart[s] = accu;
        accl = umin64(accl + L, kLim);
        accu += chunk_log2 ? ((L + (1ull << chunk_log2) - 1) >> chunk_log2) : (L ? 1 : 0);
    }
    if (t == 1023) {
        const bool over = sl[1023] >= kLim;
        totals[0] = over ? 0 : su[1023];
        totals[1] = sl[1023];
        if (over) atomicOr(err, kErrLengthSum);
    }
}

// Stream records seeded as the stateless calls seed their streams.
template <int PRNG>
__global__ void state_init_kernel(const uint64_t* seeds, uint64_t n, zig_stream_state* st) {
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    typename GenOf<PRNG>::T g;
    g.seed(seeds[s]);
    zig_stream_state r;
    r.gen[0] = r.gen[1] = r.gen[2] = r.gen[3] = 0;
    g.save(r.gen);
    r.polar_cached = 0.0;
    r.polar_have = 0;
    r.prng = PRNG;
    st[s] = r;
}

// Raw draws for generator parity checks.
template <int PRNG>
__global__ void prng_fill_kernel(const uint64_t* seeds, uint64_t n_streams, uint64_t n,
                                 uint64_t skip, int kind, uint64_t* out) {
    using G = typename GenOf<PRNG>::T;
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_streams) return;
    G g;
    g.seed(seeds[s]);
    if (skip) g.jump(skip, &d_jump);
    for (uint64_t t = 0; t < n; ++t) {
        uint64_t v = (kind == 0) ? (uint64_t)g.next_u32() : (kind == 1) ? g.next_u64() : g.next_m53();
        out[s * n + t] = v;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace host {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
bool g_init[kMaxDevices];
int g_sms[kMaxDevices];
unsigned* g_err_ptr[kMaxDevices];   // the device's own error word (d_err), per device

struct Affine { uint64_t A, C; };
static Affine compose(Affine o, Affine i) { return {o.A * i.A, o.A * i.C + o.C}; }

// One step of a xoroshiro128 linear engine with constants (a, b, c) on (x0, x1).
static void xoro_step(uint64_t& x0, uint64_t& x1, int a, int b, int c) {
    const uint64_t q1 = x1 ^ x0;
    x0 = ((x0 << a) | (x0 >> (64 - a))) ^ q1 ^ (q1 << b);
    x1 = (q1 << c) | (q1 >> (64 - c));
}

// T^(2^k), k = 0..63, of the engine (a, b, c) as GF(2) matrices stored by
// columns: column d of T^(2^k) at dst[k][2d], dst[k][2d + 1].
static void fill_gf2_powers(uint64_t (*dst)[256], int a, int b, int cc) {
    static uint64_t col[128][2], nxt[128][2];
    for (int d = 0; d < 128; ++d) {
        uint64_t x0 = d < 64 ? (1ull << d) : 0, x1 = d < 64 ? 0 : (1ull << (d - 64));
        xoro_step(x0, x1, a, b, cc);
        col[d][0] = x0;
        col[d][1] = x1;
    }
    for (int k = 0; k < 64; ++k) {
        for (int d = 0; d < 128; ++d) {
            dst[k][2 * d] = col[d][0];
            dst[k][2 * d + 1] = col[d][1];
        }
        // square the map: column d of T^2 = T applied to column d of T
        for (int d = 0; d < 128; ++d) {
            uint64_t r0 = 0, r1 = 0;
            for (int e = 0; e < 128; ++e) {
                const uint64_t bit = e < 64 ? (col[d][0] >> e) & 1 : (col[d][1] >> (e - 64)) & 1;
                if (bit) {
                    r0 ^= col[e][0];
                    r1 ^= col[e][1];
                }
            }
            nxt[d][0] = r0;
            nxt[d][1] = r1;
        }
        std::memcpy(col, nxt, sizeof(col));
    }
}

static void fill_jump(JumpTab& jt) {
    Affine l48 = {kLcgA, kLcgC};
    Affine lxm = {kLxmM, 1};
    for (int b = 0; b < 64; ++b) {
        jt.lcg48_A[b] = l48.A & kMask48;
        jt.lcg48_C[b] = l48.C & kMask48;
        jt.lxm_A[b] = lxm.A;
        jt.lxm_G[b] = lxm.C;
        l48 = compose(l48, l48);
        lxm = compose(lxm, lxm);
    }
    fill_gf2_powers(jt.xoro, 24, 16, 37);   // LXM's xoroshiro128
    fill_gf2_powers(jt.xpp, 49, 21, 28);    // Xoroshiro128PlusPlus
}

#define ZIG_CUDA(call)                               \
    do {                                             \
        if ((call) != cudaSuccess) return ZIG_ERR_CUDA; \
    } while (0)

static zig_status init_device(int device) {
    cudaDeviceProp prop;
    ZIG_CUDA(cudaSetDevice(device));
    ZIG_CUDA(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3)) return ZIG_ERR_UNSUPPORTED;
    uint32_t kE[128];
    for (int i = 0; i < 128; ++i) {
        uint64_t bits;
        std::memcpy(&bits, &zigtab::ZIG128_W[i], 8);
        int E = (int)((bits >> 52) & 0x7FF);
        if (E - 900 < 0 || E - 900 > 255) return ZIG_ERR_UNSUPPORTED;
        kE[i] = zigtab::ZIG128_K[i] | ((uint32_t)(E - 900) << 24);
    }
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_kE, kE, sizeof(kE)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_W, zigtab::ZIG128_W, sizeof(zigtab::ZIG128_W)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_Y, zigtab::ZIG128_Y, sizeof(zigtab::ZIG128_Y)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_W32, zigtab::ZIG128_W32, sizeof(zigtab::ZIG128_W32)));
    float y32[128], dy32[128];
    for (int i = 0; i < 128; ++i) {
        y32[i] = (float)zigtab::ZIG128_Y[i];
        dy32[i] = i < 127 ? (float)(zigtab::ZIG128_Y[i] - zigtab::ZIG128_Y[i + 1]) : 0.0f;
    }
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_Y32, y32, sizeof(y32)));
    ZIG_CUDA(cudaMemcpyToSymbol(c_log_g, zigtab::LOG_G, sizeof(zigtab::LOG_G)));
    ZIG_CUDA(cudaMemcpyToSymbol(c_log_thi, zigtab::LOG_THI, sizeof(zigtab::LOG_THI)));
    ZIG_CUDA(cudaMemcpyToSymbol(c_log_tlo, zigtab::LOG_TLO, sizeof(zigtab::LOG_TLO)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_DY32, dy32, sizeof(dy32)));
    const int nr = zigtab::ZIG256_NR;
    double xs[256] = {0};
    std::memcpy(xs, zigtab::ZIG256_XS, sizeof(double) * nr);
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_XS, xs, sizeof(xs)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_OX, zigtab::ZIG256_OX, sizeof(double) * nr));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_ODX, zigtab::ZIG256_ODX, sizeof(double) * nr));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_OY, zigtab::ZIG256_OY, sizeof(double) * nr));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_ODY, zigtab::ZIG256_ODY, sizeof(double) * nr));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_KIND, zigtab::ZIG256_KIND, sizeof(int) * nr));
    float f32[4][256] = {};
    for (int r = 0; r < nr; ++r) {
        f32[0][r] = (float)zigtab::ZIG256_OX[r];
        f32[1][r] = (float)zigtab::ZIG256_ODX[r];
        f32[2][r] = (float)zigtab::ZIG256_OY[r];
        f32[3][r] = (float)zigtab::ZIG256_ODY[r];
    }
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_F32, f32, sizeof(f32)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_QA, zigtab::ZIG256_QA, sizeof(uint64_t) * nr));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_THR, zigtab::ZIG256_THR, sizeof(zigtab::ZIG256_THR)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_ALIAS, zigtab::ZIG256_ALIAS, sizeof(zigtab::ZIG256_ALIAS)));
    static JumpTab jt;
    fill_jump(jt);
    ZIG_CUDA(cudaMemcpyToSymbol(d_jump, &jt, sizeof(jt)));
    unsigned zero = 0;
    ZIG_CUDA(cudaMemcpyToSymbol(d_err, &zero, sizeof(zero)));
    void* ep = nullptr;
    ZIG_CUDA(cudaGetSymbolAddress(&ep, d_err));
    ZIG_CUDA(cudaDeviceSynchronize());
    g_err_ptr[device] = (unsigned*)ep;
    g_sms[device] = prop.multiProcessorCount;
    return ZIG_OK;
}

static zig_status current_device(int& dev) {
    ZIG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return ZIG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_init[dev]) return ZIG_ERR_NOT_INITIALIZED;
    return ZIG_OK;
}

typedef void (*GenFn)(GenArgs);

// The binary64 128-level kernel with fma share `fma`: rows of every 4 whose
// products use the binary64 fma (the others use the integer product).
template <int PRNG>
static GenFn pick_zf(int fma) {
    switch (fma) {
    case 2: return zf::z128f_kernel<PRNG, ZIG_F64, 2>;
    case 3: return zf::z128f_kernel<PRNG, ZIG_F64, 3>;
    default: return zf::z128f_kernel<PRNG, ZIG_F64, 4>;
    }
}

template <int ALG, int PRNG>
static GenFn pick_dt(int dt, int fma) {
    if constexpr (ALG == ZIG_ZIG128) {
        switch (dt) {
        case ZIG_F64: return pick_zf<PRNG>(fma);
        case ZIG_F32: return zf::z128f_kernel<PRNG, ZIG_F32, 4>;
        default: return zf::z128f_kernel<PRNG, ZIG_BF16, 4>;
        }
    } else if constexpr (ALG == ZIG_ZIG256) {
        switch (dt) {
        case ZIG_F64: return zb::z256b_kernel<PRNG, ZIG_F64>;
        case ZIG_F32: return zb::z256b_kernel<PRNG, ZIG_F32>;
        default: return zb::z256b_kernel<PRNG, ZIG_BF16>;
        }
    } else {
        switch (dt) {
        case ZIG_F64: return polar_kernel<ALG, PRNG, ZIG_F64>;
        case ZIG_F32: return polar_kernel<ALG, PRNG, ZIG_F32>;
        default: return polar_kernel<ALG, PRNG, ZIG_BF16>;
        }
    }
}
template <int ALG>
static GenFn pick_prng(int prng, int dt, int fma) {
    switch (prng) {
    case ZIG_LCG48: return pick_dt<ALG, 0>(dt, fma);
    case ZIG_SPLITMIX64: return pick_dt<ALG, 1>(dt, fma);
    case ZIG_L64X128MIX: return pick_dt<ALG, 2>(dt, fma);
    default: return pick_dt<ALG, 3>(dt, fma);
    }
}
static GenFn pick(int alg, int prng, int dt, int fma) {
    switch (alg) {
    case ZIG_ZIG128: return pick_prng<ZIG_ZIG128>(prng, dt, fma);
    case ZIG_POLAR: return pick_prng<ZIG_POLAR>(prng, dt, fma);
    default: return pick_prng<ZIG_ZIG256>(prng, dt, fma);
    }
}

// Shared memory of the 128-level batch kernel: tables plus one warp area per warp.
template <int DT>
static size_t zf_smem_dt(int prng, int warps) {
    switch (prng) {
    case ZIG_LCG48: return zf::smem_bytes<0, DT>(warps);
    case ZIG_SPLITMIX64: return zf::smem_bytes<1, DT>(warps);
    case ZIG_L64X128MIX: return zf::smem_bytes<2, DT>(warps);
    default: return zf::smem_bytes<3, DT>(warps);
    }
}
static size_t zf_smem(int prng, int dt, int warps) {
    return dt == ZIG_F64 ? zf_smem_dt<ZIG_F64>(prng, warps)
         : dt == ZIG_F32 ? zf_smem_dt<ZIG_F32>(prng, warps) : zf_smem_dt<ZIG_BF16>(prng, warps);
}
// The most threads a block of that kernel can have: as many warps as one SM's
// shared memory holds (227 KB per block), at most zf::max_threads(prng).
static int zf_max_block(int prng, int dt) {
    int w = zf::max_threads(prng) / 32;
    while (w > 1 && zf_smem(prng, dt, w) > 227 * 1024) --w;
    return 32 * w;
}

// Dynamic shared memory of a generation launch (the polar kernel uses static only).
static size_t dyn_smem_of(int alg, int dt, int prng, int block) {
    if (alg == ZIG_ZIG256) return zb::smem_bytes(block / 32);
    if (alg != ZIG_ZIG128) return 0;
    return zf_smem(prng, dt, block / 32);
}

// ---- launch configuration of the 128-level generation kernel ----
// Per device, PRNG, output type and input form (uniform lengths or a lengths
// array): threads per block, batch width and store width.  Any choice gives
// the same outputs; zig_autotune times the candidates and keeps the fastest.
struct LaunchCfg {
    uint32_t block, batch, store_bytes, fma;
};
static LaunchCfg g_cfg[kMaxDevices][4][3][2];
static bool g_cfg_set[kMaxDevices][4][3][2];

static uint32_t default_batch(int dt) { (void)dt; return 32u; }
// binary64: values of every 4 whose exact product uses the binary64 fma (the
// rest use the integer product), by generator
static uint32_t default_fma(int prng) { (void)prng; return 3u; }
// every output type goes out as warp-wide row runs, one row per store (the batch
// kernel's only form); the block is lowered at launch to what shared memory holds
static LaunchCfg default_cfg(int dt) {
    (void)dt;
    return LaunchCfg{(uint32_t)zf::kMaxThreads, 32u, 0u, 0u};
}

static bool cfg_valid(int dt, const LaunchCfg& c) {
    if (!(c.block >= 64 && c.block % 32 == 0 && c.block <= (uint32_t)zf::kMaxThreads &&
          c.batch == default_batch(dt) && c.store_bytes == 0))
        return false;
    return dt == ZIG_F64 ? (c.fma == 0 || (c.fma >= 2 && c.fma <= 4)) : c.fma == 0;
}

static LaunchCfg cfg_of(int dev, int prng, int dt, bool variable) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int v = variable ? 1 : 0;
    return g_cfg_set[dev][prng][dt][v] ? g_cfg[dev][prng][dt][v] : default_cfg(dt);
}

// Opt in to the dynamic shared memory a launch needs (static + dynamic may pass
// the 48 KB default only with the attribute set).
// Per-kernel launch facts, resolved once (so a launch inside stream capture only
// enqueues work): the dynamic shared-memory opt-in and the resident blocks per SM.
struct LaunchFacts {
    const void* fn;
    int dev;
    size_t dyn;
    int block;
    int per_sm;
};
// A fixed table (no allocation at call time); when it is full, facts are
// resolved again at each launch.
constexpr int kMaxFacts = 2048;
std::mutex g_facts_mu;
LaunchFacts g_facts[kMaxFacts];
int g_n_facts = 0;

static bool allow_dyn_smem(const void* fn, size_t bytes) {
    if (bytes == 0) return true;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_facts_mu);
    // one record per kernel and device (block = -1): the largest opt-in so far
    for (int k = 0; k < g_n_facts; ++k) {
        LaunchFacts& f = g_facts[k];
        if (f.fn == fn && f.dev == dev && f.block == -1) {
            if (bytes <= f.dyn) return true;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
                return false;
            f.dyn = bytes;
            return true;
        }
    }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return false;
    if (g_n_facts < kMaxFacts) g_facts[g_n_facts++] = LaunchFacts{fn, dev, bytes, -1, 0};
    return true;
}

static int blocks_per_sm(const void* fn, int dev, size_t dyn, int block) {
    std::lock_guard<std::mutex> lk(g_facts_mu);
    for (int k = 0; k < g_n_facts; ++k) {
        const LaunchFacts& f = g_facts[k];
        if (f.fn == fn && f.dev == dev && f.dyn == dyn && f.block == block) return f.per_sm;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, dyn) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (g_n_facts < kMaxFacts) g_facts[g_n_facts++] = LaunchFacts{fn, dev, dyn, block, per_sm};
    return per_sm;
}

static int grid_for(const void* fn, int dev, uint64_t n_groups, size_t dyn = 0, int block = kBlock) {
    const int per_sm = blocks_per_sm(fn, dev, dyn, block);
    uint64_t full = (uint64_t)g_sms[dev] * per_sm;
    const uint64_t warps = (uint64_t)block / 32;
    uint64_t need = (n_groups + warps - 1) / warps;
    if (need == 0) need = 1;
    return (int)std::min<uint64_t>(full, need);
}

// Launch the generation kernel of (alg, prng, dt) for the arguments in a, with
// the configuration `force` or else the one recorded for this device.
// The batch kernel's mutation forms (MUT 1: one population, 2: a batch of requests)
// on binary32 rows, with as many warps as shared memory holds.
template <int MUT, int PRNG>
static zig_status launch_mut_p(int dev, uint64_t n_groups, GenArgs& a, cudaStream_t s) {
    const GenFn fn = zf::z128f_kernel<PRNG, ZIG_F32, 4, MUT>;
    int w = zf::max_threads(PRNG) / 32;
    while (w > 1 && zf::smem_bytes<PRNG, ZIG_F32, MUT>(w) > 227 * 1024) --w;
    const size_t dyn = zf::smem_bytes<PRNG, ZIG_F32, MUT>(w);
    if (!allow_dyn_smem((const void*)fn, dyn)) return ZIG_ERR_CUDA;
    const int grid = grid_for((const void*)fn, dev, n_groups, dyn, 32 * w);
    fn<<<grid, 32 * w, dyn, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
}
template <int MUT>
static zig_status launch_mut(int prng, int dev, uint64_t n_groups, GenArgs& a, cudaStream_t s) {
    switch (prng) {
    case ZIG_LCG48: return launch_mut_p<MUT, 0>(dev, n_groups, a, s);
    case ZIG_SPLITMIX64: return launch_mut_p<MUT, 1>(dev, n_groups, a, s);
    case ZIG_L64X128MIX: return launch_mut_p<MUT, 2>(dev, n_groups, a, s);
    default: return launch_mut_p<MUT, 3>(dev, n_groups, a, s);
    }
}

static zig_status launch_gen(int alg, int prng, int dt, int dev, bool variable, uint64_t n_groups_hint,
                             GenArgs& a, cudaStream_t s, const LaunchCfg* force) {
    const bool z128 = alg == ZIG_ZIG128;
    const LaunchCfg c = force ? *force : z128 ? cfg_of(dev, prng, dt, variable) : default_cfg(dt);
    int block = z128 ? (int)c.block : alg == ZIG_ZIG256 ? zb::kThreads : kBlock;
    if (z128) block = std::min(block, zf_max_block(prng, dt));
    const int fma = c.fma ? (int)c.fma : (int)default_fma(prng);
    GenFn fn = pick(alg, prng, dt, fma);
    const size_t dyn = dyn_smem_of(alg, dt, prng, block);
    if (!allow_dyn_smem((const void*)fn, dyn)) return ZIG_ERR_CUDA;
    const int grid = grid_for((const void*)fn, dev, n_groups_hint, dyn, block);
    fn<<<grid, block, dyn, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
}

}  // namespace host
}  // namespace zig

using namespace zig;

extern "C" {

zig_status zig_tables_init(int device) {
    if (device < 0 || device >= host::kMaxDevices) return ZIG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(host::g_mu);
    if (host::g_init[device]) {
        return cudaSetDevice(device) == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
    }
    zig_status st = host::init_device(device);
    if (st == ZIG_OK) host::g_init[device] = true;
    return st;
}

zig_status zig_tables_get_zig128(uint32_t* k_host, double* w_host, double* y_host,
                                 float* w32_host, double* R_host) {
    if (k_host) std::memcpy(k_host, zigtab::ZIG128_K, sizeof(zigtab::ZIG128_K));
    if (w_host) std::memcpy(w_host, zigtab::ZIG128_W, sizeof(zigtab::ZIG128_W));
    if (y_host) std::memcpy(y_host, zigtab::ZIG128_Y, sizeof(zigtab::ZIG128_Y));
    if (w32_host) std::memcpy(w32_host, zigtab::ZIG128_W32, sizeof(zigtab::ZIG128_W32));
    if (R_host) *R_host = zigtab::ZIG128_R;
    return ZIG_OK;
}

zig_status zig_tables_get(zig_alg alg, void* host_dst, size_t* bytes) {
    if (!bytes || (unsigned)alg > 2u) return ZIG_ERR_INVALID_ARG;
    const size_t need = alg == ZIG_ZIG128 ? sizeof(zig_tables128) : alg == ZIG_ZIG256 ? sizeof(zig_tables256) : 0;
    const size_t cap = *bytes;
    *bytes = need;
    if (!host_dst || need == 0) return ZIG_OK;
    if (cap < need) return ZIG_ERR_INVALID_ARG;
    if (alg == ZIG_ZIG128) {
        zig_tables128 t;
        std::memset(&t, 0, sizeof(t));
        t.R = zigtab::ZIG128_R;
        t.V = zigtab::ZIG128_V;
        std::memcpy(t.w, zigtab::ZIG128_W, sizeof(t.w));
        std::memcpy(t.y, zigtab::ZIG128_Y, sizeof(t.y));
        std::memcpy(t.k, zigtab::ZIG128_K, sizeof(t.k));
        std::memcpy(t.w32, zigtab::ZIG128_W32, sizeof(t.w32));
        std::memcpy(host_dst, &t, sizeof(t));
    } else {
        zig_tables256 t;
        std::memset(&t, 0, sizeof(t));
        const int nr = zigtab::ZIG256_NR;
        t.n_r = (uint64_t)nr;
        t.x0 = zigtab::ZIG256_X0;
        for (int j = 0; j < nr; ++j) t.xs[j] = zigtab::ZIG256_XS[j];
        for (int r = 1; r <= nr; ++r) {   // overhang r (1 .. n_r); index 0 is the tail
            t.ox[r] = zigtab::ZIG256_OX[r - 1];
            t.odx[r] = zigtab::ZIG256_ODX[r - 1];
            t.oy[r] = zigtab::ZIG256_OY[r - 1];
            t.ody[r] = zigtab::ZIG256_ODY[r - 1];
            t.kind[r] = zigtab::ZIG256_KIND[r - 1];
            t.qa[r] = zigtab::ZIG256_QA[r - 1];
        }
        for (int b = 0; b < 256; ++b) {
            t.thr[b] = zigtab::ZIG256_THR[b];
            t.alias[b] = zigtab::ZIG256_ALIAS[b];
        }
        std::memcpy(host_dst, &t, sizeof(t));
    }
    return ZIG_OK;
}

size_t zig_generate_workspace_bytes(uint64_t n_streams) {
    return (size_t)(16 * n_streams + 256);
}

}  // extern "C"

namespace zig {
namespace host {
// Stateless calls seed stream s from seeds_dev[s]; calls with records (state
// non-NULL, seeds_dev NULL, chunk_log2 0) continue and advance state[s].
static zig_status generate_impl(zig_prng prng, zig_alg alg, const uint64_t* seeds_dev,
                                const uint64_t* lengths_dev, uint64_t uniform_len, uint64_t n_streams,
                                uint32_t chunk_log2, zig_dtype dtype, void* out_dev, void* workspace_dev,
                                size_t workspace_bytes, unsigned* status_dev, void* stream,
                                const LaunchCfg* force, zig_stream_state* state = nullptr) {
    if ((unsigned)prng > 3u || (unsigned)alg > 2u || (unsigned)dtype > 2u) return ZIG_ERR_INVALID_ARG;
    if (chunk_log2 != 0 && (chunk_log2 < 4 || chunk_log2 > 24)) return ZIG_ERR_INVALID_ARG;
    if (state && chunk_log2 != 0) return ZIG_ERR_INVALID_ARG;
    if (n_streams == 0) return ZIG_OK;
    // out_dev may be NULL only with lengths_dev (an all-zero batch); the kernel
    // latches ZIG_ERR_INVALID_ARG in the error word if the lengths sum above zero
    if ((!seeds_dev && !state) || (!out_dev && !lengths_dev)) return ZIG_ERR_INVALID_ARG;
    const size_t esz = dtype == ZIG_F64 ? 8 : dtype == ZIG_F32 ? 4 : 2;
    if (((uintptr_t)out_dev) % esz || ((uintptr_t)seeds_dev) % 8 || ((uintptr_t)state) % 16)
        return ZIG_ERR_INVALID_ARG;
    if (lengths_dev == nullptr) {
        if (uniform_len == 0) return ZIG_OK;
        if (uniform_len >= (1ull << 40) || n_streams > ((1ull << 40) - 1) / uniform_len)
            return ZIG_ERR_INVALID_ARG;
    } else if (((uintptr_t)lengths_dev) % 8 || n_streams > (1ull << 32)) {
        return ZIG_ERR_INVALID_ARG;
    } else if (workspace_dev && (workspace_bytes < zig_generate_workspace_bytes(n_streams) ||
                                 ((uintptr_t)workspace_dev) % 16)) {
        return ZIG_ERR_INVALID_ARG;   // a caller workspace that cannot hold the scratch
    }
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    GenArgs a{};
    a.seeds = seeds_dev;
    a.state = state;
    a.lengths = lengths_dev;
    a.uniform_len = uniform_len;
    a.n_streams = n_streams;
    a.chunk_log2 = chunk_log2;
    a.out = out_dev;
    a.err = status_dev ? status_dev : host::g_err_ptr[dev];
    uint64_t n_groups_hint;
    if (lengths_dev == nullptr) {
        a.units_per_stream = chunk_log2 ? ((uniform_len + (1ull << chunk_log2) - 1) >> chunk_log2) : 1;
        a.n_units = n_streams * a.units_per_stream;
        n_groups_hint = (a.n_units + 31) / 32;
    } else {
        size_t need = zig_generate_workspace_bytes(n_streams);
        uint64_t* ws;
        void* own = nullptr;   // the call's own scratch, ordered on the stream
        if (workspace_dev) {
            if (workspace_bytes < need || ((uintptr_t)workspace_dev) % 16) return ZIG_ERR_INVALID_ARG;
            ws = (uint64_t*)workspace_dev;
        } else {
            // allocated and freed in the order of the caller's stream: calls on
            // different streams never share it, and inside stream capture the
            // graph owns the allocation
            if (cudaMallocAsync(&own, need, s) != cudaSuccess) return ZIG_ERR_CUDA;
            ws = (uint64_t*)own;
        }
        a.offsets = ws;
        a.ustart = ws + n_streams;
        a.totals = ws + 2 * n_streams;
        scan_kernel<<<1, 1024, 0, s>>>(lengths_dev, n_streams, chunk_log2, (uint64_t*)a.offsets,
                                       (uint64_t*)a.ustart, (uint64_t*)a.totals, a.err);
        st = cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
        n_groups_hint = ~0ull >> 8;   // unknown on the host: fill the device
        if (st == ZIG_OK)
            st = host::launch_gen(alg, prng, dtype, dev, true, n_groups_hint, a, s, force);
        if (own && cudaFreeAsync(own, s) != cudaSuccess && st == ZIG_OK) st = ZIG_ERR_CUDA;
        return st;
    }
    return host::launch_gen(alg, prng, dtype, dev, false, n_groups_hint, a, s, force);
}
}  // namespace host
}  // namespace zig

extern "C" {

zig_status zig_generate(zig_prng prng, zig_alg alg, const uint64_t* seeds_dev,
                        const uint64_t* lengths_dev, uint64_t uniform_len, uint64_t n_streams,
                        uint32_t chunk_log2, zig_dtype dtype, void* out_dev, void* workspace_dev,
                        size_t workspace_bytes, void* stream) {
    return host::generate_impl(prng, alg, seeds_dev, lengths_dev, uniform_len, n_streams, chunk_log2,
                               dtype, out_dev, workspace_dev, workspace_bytes, nullptr, stream, nullptr);
}

zig_status zig_generate_checked(zig_prng prng, zig_alg alg, const uint64_t* seeds_dev,
                                const uint64_t* lengths_dev, uint64_t uniform_len, uint64_t n_streams,
                                uint32_t chunk_log2, zig_dtype dtype, void* out_dev, void* workspace_dev,
                                size_t workspace_bytes, uint32_t* status_dev, void* stream) {
    if (!status_dev || ((uintptr_t)status_dev) % 4) return ZIG_ERR_INVALID_ARG;
    return host::generate_impl(prng, alg, seeds_dev, lengths_dev, uniform_len, n_streams, chunk_log2,
                               dtype, out_dev, workspace_dev, workspace_bytes, (unsigned*)status_dev, stream,
                               nullptr);
}

zig_status zig_state_init(zig_prng prng, const uint64_t* seeds_dev, uint64_t n_streams,
                          zig_stream_state* state_dev, void* stream) {
    if ((unsigned)prng > 3u || n_streams > (1ull << 32)) return ZIG_ERR_INVALID_ARG;
    if (n_streams == 0) return ZIG_OK;
    if (!seeds_dev || !state_dev || ((uintptr_t)seeds_dev) % 8 || ((uintptr_t)state_dev) % 16)
        return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)((n_streams + 255) / 256);
    switch (prng) {
    case ZIG_LCG48: state_init_kernel<0><<<grid, 256, 0, s>>>(seeds_dev, n_streams, state_dev); break;
    case ZIG_SPLITMIX64: state_init_kernel<1><<<grid, 256, 0, s>>>(seeds_dev, n_streams, state_dev); break;
    case ZIG_L64X128MIX: state_init_kernel<2><<<grid, 256, 0, s>>>(seeds_dev, n_streams, state_dev); break;
    default: state_init_kernel<3><<<grid, 256, 0, s>>>(seeds_dev, n_streams, state_dev); break;
    }
    return cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
}

zig_status zig_generate_state(zig_prng prng, zig_alg alg, zig_stream_state* state_dev,
                              const uint64_t* lengths_dev, uint64_t uniform_len, uint64_t n_streams,
                              zig_dtype dtype, void* out_dev, void* workspace_dev, size_t workspace_bytes,
                              uint32_t* status_dev, void* stream) {
    if (!state_dev || ((uintptr_t)status_dev) % 4) return ZIG_ERR_INVALID_ARG;
    return host::generate_impl(prng, alg, nullptr, lengths_dev, uniform_len, n_streams, 0, dtype, out_dev,
                               workspace_dev, workspace_bytes, (unsigned*)status_dev, stream, nullptr,
                               state_dev);
}

zig_status zig_launch_config_get(int device, zig_prng prng, zig_dtype dtype, int variable_lengths,
                                 zig_launch_config* cfg) {
    if (device < 0 || device >= host::kMaxDevices || (unsigned)prng > 3u || (unsigned)dtype > 2u || !cfg)
        return ZIG_ERR_INVALID_ARG;
    const host::LaunchCfg c = host::cfg_of(device, prng, dtype, variable_lengths != 0);
    cfg->block = c.block;
    cfg->batch = c.batch;
    cfg->store_bytes = c.store_bytes;
    cfg->fma_of_4 = c.fma;
    return ZIG_OK;
}

zig_status zig_launch_config_set(int device, zig_prng prng, zig_dtype dtype, int variable_lengths,
                                 const zig_launch_config* cfg) {
    if (device < 0 || device >= host::kMaxDevices || (unsigned)prng > 3u || (unsigned)dtype > 2u)
        return ZIG_ERR_INVALID_ARG;
    const int v = variable_lengths ? 1 : 0;
    std::lock_guard<std::mutex> lk(host::g_mu);
    if (!cfg) {
        host::g_cfg_set[device][prng][dtype][v] = false;
        return ZIG_OK;
    }
    const host::LaunchCfg c{cfg->block, cfg->batch, cfg->store_bytes, cfg->fma_of_4};
    if (!host::cfg_valid(dtype, c)) return ZIG_ERR_INVALID_ARG;
    host::g_cfg[device][prng][dtype][v] = c;
    host::g_cfg_set[device][prng][dtype][v] = true;
    return ZIG_OK;
}

uint32_t zig_autotune_candidates(zig_dtype dtype, zig_launch_config* cands, uint32_t max_cands) {
    const uint32_t b = host::default_batch((unsigned)dtype > 2u ? ZIG_F64 : dtype);
    uint32_t n = 0;
    if (dtype == ZIG_F64) {
        // blocks are clamped to what one SM's shared memory holds for the generator
        static const uint32_t blocks[] = {256, 384, 512, 640};
        for (uint32_t bl : blocks)
            for (uint32_t fm : {2u, 3u, 4u}) {
                if (cands && n < max_cands) cands[n] = zig_launch_config{bl, b, 0u, fm};
                ++n;
            }
        return n;
    }
    static const uint32_t blocks[] = {256, 384, 512, 640};
    for (uint32_t bl : blocks) {
        if (cands && n < max_cands) cands[n] = zig_launch_config{bl, b, 0u, 0u};
        ++n;
    }
    return n;
}

zig_status zig_autotune(zig_prng prng, const uint64_t* seeds_dev, const uint64_t* lengths_dev,
                        uint64_t uniform_len, uint64_t n_streams, uint32_t chunk_log2, zig_dtype dtype,
                        void* out_dev, void* workspace_dev, size_t workspace_bytes, uint32_t reps,
                        zig_launch_config* best, float* best_ms, void* stream) {
    if ((unsigned)prng > 3u || (unsigned)dtype > 2u || reps == 0 || reps > 1000) return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return ZIG_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return ZIG_ERR_INVALID_ARG;   // it synchronizes
    zig_launch_config cands[64];
    const uint32_t nc = zig_autotune_candidates(dtype, cands, 64);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ZIG_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ZIG_ERR_CUDA;
    }
    float best_t = -1.0f;
    uint32_t best_k = 0;
    for (uint32_t k = 0; k < nc && st == ZIG_OK; ++k) {
        const host::LaunchCfg c{cands[k].block, cands[k].batch, cands[k].store_bytes, cands[k].fma_of_4};
        // one untimed launch, then `reps` timed back to back on the caller's stream
        for (uint32_t r = 0; r <= reps && st == ZIG_OK; ++r) {
            if (r == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = ZIG_ERR_CUDA;
            if (st == ZIG_OK)
                st = host::generate_impl(prng, ZIG_ZIG128, seeds_dev, lengths_dev, uniform_len, n_streams,
                                         chunk_log2, dtype, out_dev, workspace_dev, workspace_bytes, nullptr,
                                         stream, &c);
        }
        float ms = 0.0f;
        if (st == ZIG_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = ZIG_ERR_CUDA;
        ms /= (float)reps;
        if (st == ZIG_OK && (best_t < 0.0f || ms < best_t)) {
            best_t = ms;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != ZIG_OK) return st;
    st = zig_launch_config_set(dev, prng, dtype, lengths_dev != nullptr, &cands[best_k]);
    if (st != ZIG_OK) return st;
    if (best) *best = cands[best_k];
    if (best_ms) *best_ms = best_t;
    return ZIG_OK;
}

}  // extern "C"

namespace zig {
namespace host {
// x += sigma z on P x L binary32 rows: row p seeded seed + p and chunked at
// 2^10 outputs, or (state non-NULL) continuing record state[p] unchunked.
static zig_status mutate_impl(float* x_dev, float sigma, uint64_t P, uint64_t L, uint64_t seed,
                              zig_stream_state* state, zig_prng prng, void* stream) {
    if ((unsigned)prng > 3u || !std::isfinite(sigma)) return ZIG_ERR_INVALID_ARG;
    if (P == 0 || L == 0) return ZIG_OK;
    if (!x_dev || ((uintptr_t)x_dev) % 4 || L >= (1ull << 40) || P > ((1ull << 40) - 1) / L ||
        ((uintptr_t)state) % 16)
        return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    const uint64_t upr = state ? 1 : (L + 1023) >> 10;
    const uint64_t groups = (P * upr + 31) / 32;
    cudaStream_t s = (cudaStream_t)stream;
    GenArgs a{};
    a.uniform_len = L;          // row length
    a.n_streams = P;
    a.chunk_log2 = state ? 0 : 10;
    a.out = x_dev;
    a.units_per_stream = upr;
    a.n_units = P * upr;
    a.sigma = sigma;
    a.seeds = nullptr;
    a.state = state;
    // without records the kernel seeds row p with a.mut_seed + p in mutation mode
    a.err = host::g_err_ptr[dev];
    GenArgs am = a;
    am.mut_seed = seed;
    return launch_mut<1>(prng, dev, groups, am, s);
}
}  // namespace host
}  // namespace zig

extern "C" {

zig_status zig_mutate(float* x_dev, float sigma, uint64_t P, uint64_t L, uint64_t seed,
                      zig_prng prng, void* stream) {
    return host::mutate_impl(x_dev, sigma, P, L, seed, nullptr, prng, stream);
}

zig_status zig_mutate_state(float* x_dev, float sigma, uint64_t P, uint64_t L, zig_stream_state* state_dev,
                            zig_prng prng, void* stream) {
    if (!state_dev) return ZIG_ERR_INVALID_ARG;
    return host::mutate_impl(x_dev, sigma, P, L, 0, state_dev, prng, stream);
}

size_t zig_mutate_batch_desc_bytes(uint32_t n_req) { return (size_t)n_req * sizeof(MutDesc) + 256; }

zig_status zig_mutate_batch(const zig_mutation* reqs_host, uint32_t n_req, zig_prng prng, void* desc_dev,
                            size_t desc_bytes, void* stream) {
    if ((unsigned)prng > 3u) return ZIG_ERR_INVALID_ARG;
    if (n_req == 0) return ZIG_OK;
    if (!reqs_host || !desc_dev || desc_bytes < zig_mutate_batch_desc_bytes(n_req) ||
        ((uintptr_t)desc_dev) % 16)
        return ZIG_ERR_INVALID_ARG;
    std::vector<MutDesc> d(n_req);
    uint64_t units = 0;
    for (uint32_t r = 0; r < n_req; ++r) {
        const zig_mutation& q = reqs_host[r];
        if (q.kind > ZIG_REQ_GENERATE || (q.kind == ZIG_REQ_MUTATE && !std::isfinite(q.sigma)) ||
            (q.P && q.L && (!q.x_dev || ((uintptr_t)q.x_dev) % 4)) || ((uintptr_t)q.state_dev) % 16 ||
            q.L >= (1ull << 40) || (q.L && q.P > ((1ull << 40) - 1) / q.L))
            return ZIG_ERR_INVALID_ARG;
        d[r].x = q.x_dev;
        d[r].P = q.P;
        d[r].L = q.L;
        d[r].seed = q.seed;
        d[r].sigma = q.sigma;
        d[r].state = q.state_dev;
        d[r].upr = (q.L && !q.state_dev) ? (q.L + 1023) >> 10 : 1;
        d[r].ustart = units;
        d[r].kind = q.kind;
        units += (q.P && q.L) ? q.P * d[r].upr : 0;
    }
    if (units == 0) return ZIG_OK;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the descriptors are copied from host memory this call owns, which a captured
    // graph would read again after it is gone: refused while the stream captures
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return ZIG_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return ZIG_ERR_INVALID_ARG;
    // pageable source: the copy is staged before this call returns, so reqs_host
    // may be reused at once
    if (cudaMemcpyAsync(desc_dev, d.data(), n_req * sizeof(MutDesc), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return ZIG_ERR_CUDA;
    GenArgs a{};
    a.err = host::g_err_ptr[dev];
    a.reqs = (const MutDesc*)desc_dev;
    a.n_req = n_req;
    a.n_units = units;
    a.chunk_log2 = 10;
    return host::launch_mut<2>(prng, dev, (units + 31) / 32, a, s);
}

zig_status zig_prng_fill(zig_prng prng, const uint64_t* seeds_dev, uint64_t n_streams, uint64_t n,
                         uint64_t skip, int kind, uint64_t* out_dev, void* stream) {
    if ((unsigned)prng > 3u || kind < 0 || kind > 2) return ZIG_ERR_INVALID_ARG;
    if (n_streams == 0 || n == 0) return ZIG_OK;
    if (!seeds_dev || !out_dev || n_streams > (1ull << 40) / n) return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned grid = (unsigned)((n_streams + 255) / 256);
    if (prng == ZIG_LCG48) prng_fill_kernel<0><<<grid, 256, 0, s>>>(seeds_dev, n_streams, n, skip, kind, out_dev);
    else if (prng == ZIG_SPLITMIX64) prng_fill_kernel<1><<<grid, 256, 0, s>>>(seeds_dev, n_streams, n, skip, kind, out_dev);
    else if (prng == ZIG_L64X128MIX) prng_fill_kernel<2><<<grid, 256, 0, s>>>(seeds_dev, n_streams, n, skip, kind, out_dev);
    else prng_fill_kernel<3><<<grid, 256, 0, s>>>(seeds_dev, n_streams, n, skip, kind, out_dev);
    return cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
}

zig_status zig_device_status(int device, int clear) {
    if (device < 0 || device >= host::kMaxDevices) return ZIG_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(host::g_mu);
        if (!host::g_init[device]) return ZIG_ERR_NOT_INITIALIZED;
    }
    if (cudaSetDevice(device) != cudaSuccess) return ZIG_ERR_CUDA;
    unsigned w = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return ZIG_ERR_CUDA;
    if (cudaMemcpyFromSymbol(&w, d_err, sizeof(w)) != cudaSuccess) return ZIG_ERR_CUDA;
    if (clear) {
        unsigned zero = 0;
        if (cudaMemcpyToSymbol(d_err, &zero, sizeof(zero)) != cudaSuccess) return ZIG_ERR_CUDA;
    }
    return zig_status_decode(w);
}

zig_status zig_status_decode(uint32_t word) {
    if (word & (kErrNullOutput | kErrLengthSum | kErrStateKind)) return ZIG_ERR_INVALID_ARG;
    if (word & kErrChunkOverflow) return ZIG_ERR_CHUNK_OVERFLOW;
    return ZIG_OK;
}

const char* zig_status_string(zig_status status) {
    switch (status) {
    case ZIG_OK: return "ZIG_OK";
    case ZIG_ERR_INVALID_ARG: return "ZIG_ERR_INVALID_ARG";
    case ZIG_ERR_NOT_INITIALIZED: return "ZIG_ERR_NOT_INITIALIZED";
    case ZIG_ERR_CUDA: return "ZIG_ERR_CUDA";
    case ZIG_ERR_BUDGET: return "ZIG_ERR_BUDGET";
    case ZIG_ERR_TIMEOUT: return "ZIG_ERR_TIMEOUT";
    case ZIG_ERR_CHUNK_OVERFLOW: return "ZIG_ERR_CHUNK_OVERFLOW";
    case ZIG_ERR_UNSUPPORTED: return "ZIG_ERR_UNSUPPORTED";
    case ZIG_ERR_TOO_LARGE: return "ZIG_ERR_TOO_LARGE";
    default: return "ZIG_ERR_UNKNOWN";
    }
}

int zig_version(void) { return 100; }

zig_status zig_selfcheck(uint64_t counts_host[6]) {
    if (!counts_host) return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    unsigned long long* d = nullptr;
    ZIG_CUDA(cudaMalloc(&d, 6 * sizeof(unsigned long long)));
    st = ZIG_OK;
    if (cudaMemset(d, 0, 6 * sizeof(unsigned long long)) != cudaSuccess) st = ZIG_ERR_CUDA;
    if (st == ZIG_OK) {
        selfcheck_kernel<<<host::g_sms[dev] * 8, 256>>>(d);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(counts_host, d, 6 * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = ZIG_ERR_CUDA;
    }
    cudaFree(d);
    return st;
}

zig_status zig_filtercheck(uint64_t counts_host[12]) {
    if (!counts_host) return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    unsigned long long* d = nullptr;
    ZIG_CUDA(cudaMalloc(&d, 12 * sizeof(unsigned long long)));
    st = ZIG_OK;
    if (cudaMemset(d, 0, 12 * sizeof(unsigned long long)) != cudaSuccess) st = ZIG_ERR_CUDA;
    if (st == ZIG_OK) {
        filtercheck_kernel<<<host::g_sms[dev] * 8, 256>>>(d, 1ull << 27);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(counts_host, d, 12 * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = ZIG_ERR_CUDA;
    }
    cudaFree(d);
    return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// zig_generate_noalloc: the variable-length path with its scratch in a fixed
// array compiled into the library, for callers that cannot allocate device
// memory at call time (see include/zig.h).
// ---------------------------------------------------------------------------
namespace zig {
// offsets[MAX] | unit starts[MAX] | totals[2]: 1 MiB + 16 B on every device
// that loads the library, held until the process exits.
static __device__ __align__(256) uint64_t g_noalloc_scratch[2 * ZIG_NOALLOC_MAX_STREAMS + 2];
namespace host {
// The array's device address, per device.  In host code the symbol name is
// only a host-side stand-in; the address comes from cudaGetSymbolAddress.
static uint64_t* g_noalloc_ptr[kMaxDevices];
}  // namespace host
}  // namespace zig

extern "C" zig_status zig_generate_noalloc(zig_prng prng, zig_alg alg, const uint64_t* seeds_dev,
                                           const uint64_t* lengths_dev, uint64_t n_streams,
                                           uint32_t chunk_log2, zig_dtype dtype, void* out_dev,
                                           void* stream) {
    if ((unsigned)prng > 3u || (unsigned)alg > 2u || (unsigned)dtype > 2u) return ZIG_ERR_INVALID_ARG;
    if (chunk_log2 != 0 && (chunk_log2 < 4 || chunk_log2 > 24)) return ZIG_ERR_INVALID_ARG;
    if (n_streams == 0) return ZIG_OK;
    if (n_streams > ZIG_NOALLOC_MAX_STREAMS) return ZIG_ERR_TOO_LARGE;
    if (!seeds_dev || !lengths_dev) return ZIG_ERR_INVALID_ARG;
    const size_t esz = dtype == ZIG_F64 ? 8 : dtype == ZIG_F32 ? 4 : 2;
    if (((uintptr_t)out_dev) % esz || ((uintptr_t)seeds_dev) % 8 || ((uintptr_t)lengths_dev) % 8)
        return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    uint64_t* scratch;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(host::g_mu);
        if (!host::g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ZIG_ERR_CUDA;
            host::g_noalloc_ptr[dev] = (uint64_t*)p;
        }
        scratch = host::g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    GenArgs a{};
    a.seeds = seeds_dev;
    a.lengths = lengths_dev;
    a.n_streams = n_streams;
    a.chunk_log2 = chunk_log2;
    a.out = out_dev;
    a.offsets = scratch;
    a.ustart = scratch + ZIG_NOALLOC_MAX_STREAMS;
    a.totals = scratch + 2 * ZIG_NOALLOC_MAX_STREAMS;
    a.err = host::g_err_ptr[dev];
    // the scan rewrites every offset, unit start and total this call reads
    scan_kernel<<<1, 1024, 0, s>>>(lengths_dev, n_streams, chunk_log2, (uint64_t*)a.offsets,
                                   (uint64_t*)a.ustart, (uint64_t*)a.totals, a.err);
    if (cudaGetLastError() != cudaSuccess) return ZIG_ERR_CUDA;
    return host::launch_gen(alg, prng, dtype, dev, true, ~0ull >> 8, a, s, nullptr);
}
