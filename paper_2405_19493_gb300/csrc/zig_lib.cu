// libzig_gb300: bulk N(0,1) generation on GB300 (sm_103a) behind the C ABI in
// include/zig.h.  One thread owns one (stream, chunk) unit with its generator
// state in registers; the 32 units of a warp are staged in shared memory and
// written out as coalesced rows.
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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/zig.h"
#include "zig_device.cuh"
#include "zig_tables.inc"

namespace zig {

// ---------------------------------------------------------------------------
// device-resident immutable tables (filled by zig_tables_init)
// ---------------------------------------------------------------------------
__device__ uint32_t d_z128_kE[128];   // K[i] | (E(w[i]) - 900) << 24
__device__ uint64_t d_z128_M[128];    // 53-bit significand of w[i], hidden bit set
__device__ double d_z128_W[128];
__device__ double d_z128_Y[128];
__device__ float d_z128_W32[128];
__device__ double d_z256_XS[256];
__device__ double d_z256_OX[256], d_z256_ODX[256], d_z256_OY[256], d_z256_ODY[256];
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
};

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

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

// ---------------------------------------------------------------------------
// per-variate samplers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double neg_half_sq(double x) {
    return __dmul_rn(__dmul_rn(-0.5, x), x);
}

// Polar method with the cached second variate.
template <class G>
__device__ __forceinline__ double polar_f64(G& g, bool& have, double& cached, uint32_t& extra) {
    if (have) {
        have = false;
        return cached;
    }
    constexpr uint32_t kStepsPerDouble = (sizeof(G) == sizeof(GenLcg48)) ? 2u : 1u;
    double v1, v2, s;
    do {
        v1 = __dsub_rn(__dmul_rn(2.0, m53_to_double(g.next_m53())), 1.0);
        v2 = __dsub_rn(__dmul_rn(2.0, m53_to_double(g.next_m53())), 1.0);
        s = __dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2));
        extra += 2 * kStepsPerDouble;
    } while (s >= 1.0 || s == 0.0);
    double mult = __dsqrt_rn(__ddiv_rn(__dmul_rn(-2.0, log(s)), s));
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

template <class G>
__device__ __forceinline__ double z256_slow(G& g, const Z256Smem& t, uint32_t& extra) {
    constexpr uint32_t kSteps64 = (sizeof(G) == sizeof(GenLcg48)) ? 2u : 1u;
    constexpr uint32_t kStepsPerDouble = kSteps64;
    const uint64_t two53 = 1ull << 53;
    uint64_t V = g.next_u64();
    extra += kSteps64;
    uint32_t b = (uint32_t)(V & 0xFF);
    int r = ((V >> 8) < t.THR[b]) ? (int)b : t.ALIAS[b];
    if (r == 0) {
        const double x0 = zigtab::ZIG256_X0;
        for (;;) {
            double U1 = __dsub_rn(1.0, m53_to_double(g.next_m53()));
            double U2 = __dsub_rn(1.0, m53_to_double(g.next_m53()));
            extra += 2 * kStepsPerDouble;
            double x = __ddiv_rn(-log(U1), x0);
            double y = -log(U2);
            if (__dadd_rn(y, y) > __dmul_rn(x, x)) return __dadd_rn(x0, x);
        }
    }
    const int kd = d_z256_KIND[r - 1];
    const double ox = d_z256_OX[r - 1], odx = d_z256_ODX[r - 1];
    const double oy = d_z256_OY[r - 1], ody = d_z256_ODY[r - 1];
    const uint64_t qa = d_z256_QA[r - 1];
    for (;;) {
        uint64_t m1 = g.next_m53();
        uint64_t m2 = g.next_m53();
        extra += 2 * kStepsPerDouble;
        if (kd > 0 && m1 + m2 > two53) {
            m1 = two53 - m1;
            m2 = two53 - m2;
        }
        double x = __dadd_rn(ox, __dmul_rn(odx, m53_to_double(m1)));
        if (kd > 0 && m1 + m2 <= two53 - qa) return x;
        if (kd < 0 && m1 + m2 < two53) return x;
        double y = __dadd_rn(oy, __dmul_rn(ody, m53_to_double(m2)));
        if (y < exp(neg_half_sq(x))) return x;
    }
}

template <class G>
__device__ __forceinline__ double z256_f64(G& g, const Z256Smem& t, uint32_t& extra) {
    uint64_t U = g.next_u64();
    uint32_t j = (uint32_t)(U & 0xFF);
    bool neg = (U >> 8) & 1;
    double x;
    if (j < (uint32_t)zigtab::ZIG256_NR) {
        x = __dmul_rn(t.XS[j], (double)(U >> 11));
    } else {
        x = z256_slow(g, t, extra);
    }
    return neg ? -x : x;
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
template <int ALG, int PRNG, int DT>
__global__ void __launch_bounds__(kBlock) gen_kernel(GenArgs a) {
    using G = typename GenOf<PRNG>::T;
    using OutT = typename OutOf<DT>::T;
    static_assert(ALG == ZIG_POLAR || ALG == ZIG_ZIG256, "zig128 runs in z128_kernel");
    __shared__ Z256Smem t256;
    __shared__ OutT stage_all[kWarps][32 * kStageCols];
    if (ALG == ZIG_ZIG256) z256_load(t256);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    OutT* stage = stage_all[threadIdx.x >> 5];
    if (a.out == nullptr) {   // only legal when every length is zero
        if (a.lengths && a.totals[1] != 0 && blockIdx.x == 0 && threadIdx.x == 0)
            atomicOr(&d_err, kErrNullOutput);
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
        if (u < n_units) {
            uint64_t s, q, off, n;
            unit_info(a, u, s, q, off, n);
            g.seed(a.seeds[s]);
            if (q) g.jump(q * kChunkDraws, &d_jump);
            rem = n;
            dst = out + off;
        }
        const uint64_t n_unit = rem;
        uint32_t extra = 0;
        bool have = false;
        double cached = 0.0;
        while (__any_sync(kFull, rem > 0)) {
            const int cnt = (int)umin64(rem, (uint64_t)kStageCols);
#pragma unroll 1
            for (int v = 0; v < kStageCols; ++v) {
                if (v < cnt) {
                    OutT z;
                    if (ALG == ZIG_POLAR) {
                        z = from_f64<DT>(polar_f64(g, have, cached, extra));
                    } else {
                        z = from_f64<DT>(z256_f64(g, t256, extra));
                    }
                    stage[stage_idx<OutT>(lane, v)] = z;
                }
            }
            __syncwarp();
            stage_flush<OutT>(stage, dst, cnt, lane);
            __syncwarp();
            dst += cnt;
            rem -= cnt;
        }
        // A chunk must stay inside its 2^32-draw window.  Each variate's first
        // draw takes `per` raw steps; `extra` counts every other step.
        if (a.chunk_log2 && n_unit) {
            const uint64_t per = (PRNG == ZIG_LCG48) ? 2 : 1;   // zig256's first draw is a nextLong
            uint64_t draws = (ALG == ZIG_POLAR) ? (uint64_t)extra : n_unit * per + extra;
            if (draws > kChunkDraws) atomicOr(&d_err, kErrChunkOverflow);
        }
    }
}

// ---------------------------------------------------------------------------
// 128-level ziggurat (GSL form): one launch per bulk request
// ---------------------------------------------------------------------------
// Each lane owns one unit (stream or chunk) with its generator in registers.
// A warp works in batches of up to 16 outputs per lane:
//  A. the lanes draw candidates in lockstep, two per step.  A fast-path
//     candidate (j < k[i]) is finished on the spot: x = RN(j * w[i]) is built
//     exactly with integer arithmetic (binary64) or as fl32(j * w32[i])
//     (binary32/bfloat16).  A slow candidate (wedge or tail) keeps a
//     placeholder slot and pushes a 16-byte record into the warp's ring: the
//     layer, j, sign, (row, slot) and either a snapshot of the generator from
//     which its uniform double is rebuilt (wedge) or the two uniforms (tail).
//     The lane's generator moves past those doubles at once and keeps drawing.
//  B. whenever 32 records wait (and at the end of a batch) all 32 lanes decide
//     32 records together: the wedge test in binary32 with a proven margin,
//     binary64 only inside it; the tail in binary64.
//  C. each row drops its rejected slots and is flushed, two rows per warp store,
//     with its own count; the stream continues in the next batch.
// The outputs of a unit are its accepted candidates in draw order: exactly the
// sequence a one-variate-at-a-time loop produces.

constexpr int kZBlock = 1024;               // one block per SM
constexpr int kZWarps = kZBlock / 32;
constexpr int kQCap = 64;                   // ring: <= 31 waiting + 32 new per step

struct Z128Tab {
    uint32_t kE[128][32];   // K[i] | (E(w[i]) - 900) << 24, one copy per lane
    uint2 M[128][16];       // significand of w[i] as (low 32, high 21 bits), 16 copies
    float W32[128];         // RN32(x_{i+1} / 2^24)
    float Y32[128];         // RN32(y[i])
    float DY32[128];        // RN32(y[i] - y[i+1])
    double W[128];
    double Y[128];
};
__device__ float d_z128_Y32[128];
__device__ float d_z128_DY32[128];

__device__ __forceinline__ void z128tab_load(Z128Tab& t) {
    for (int k = threadIdx.x; k < 128 * 32; k += blockDim.x) {
        const int i = k >> 5, c = k & 31;
        t.kE[i][c] = d_z128_kE[i];
        if (c < 16) {
            const uint64_t m = d_z128_M[i];
            t.M[i][c] = make_uint2((uint32_t)m, (uint32_t)(m >> 32));
        }
    }
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        t.W32[i] = d_z128_W32[i];
        t.Y32[i] = d_z128_Y32[i];
        t.DY32[i] = d_z128_DY32[i];
        t.W[i] = d_z128_W[i];
        t.Y[i] = d_z128_Y[i];
    }
}

// RN(j * w) as binary64 bits, w = (mh:ml) * 2^(E - 1075), j < 2^24, with
// eb = E - 900 from the table word.  Same arithmetic as mul_j_w_bits, written
// on 32-bit words and selects so that it has no branch; j = 0 gives +0.
__device__ __forceinline__ uint64_t mul_j_w_bits32(uint32_t j, uint32_t ml, uint32_t mh, uint32_t eb) {
    const uint32_t lz = __clz((int)j);                 // 8..31; 32 for j = 0
    const uint32_t jn = j << (lz & 31);
    const uint64_t A = (uint64_t)jn * ml;
    const uint64_t B = (uint64_t)jn * mh;
    const uint64_t T = B + (A >> 32);
    const uint32_t lo = (uint32_t)A;
    const uint32_t Tl = (uint32_t)T, Th = (uint32_t)(T >> 32);
    const bool s = Th < (1u << 20);                    // T < 2^52: shift one more bit in
    const uint32_t qh = s ? __funnelshift_l(Tl, Th, 1) : Th;
    const uint32_t ql = s ? __funnelshift_l(lo, Tl, 1) : Tl;
    const uint32_t rem = s ? (lo << 1) : lo;
    const uint32_t up = (uint32_t)(rem > 0x80000000u) | ((uint32_t)(rem == 0x80000000u) & ql);
    const uint64_t q = (((uint64_t)qh << 32) | ql) + (up & 1u);
    const uint32_t ex = eb + 931u - (uint32_t)s - lz;  // biased exponent - 1
    const uint64_t bits = ((uint64_t)ex << 52) + q;
    return j ? bits : 0ull;
}

// Slow-candidate record (16 bytes).
//   a: bits 53..57 row, 58..61 slot, 62 negative, 63 tail;
//      wedge: bits 0..23 j, 24..30 layer i;  tail: bits 0..52 the first uniform (m53)
//   b: wedge: the generator snapshot for its uniform;  tail: the second uniform (m53)
struct SlowRec {
    uint64_t a, b;
};

template <int DT> struct Z128Out;
template <> struct Z128Out<ZIG_F64> {
    using T = double;
    using Pair = double2;
    static __device__ __forceinline__ double fast(const Z128Tab& t, uint32_t i, uint32_t j,
                                                  uint32_t negbit, int lane, uint32_t kE) {
        const uint2 m = t.M[i][lane & 15];
        return __longlong_as_double(
            (long long)(mul_j_w_bits32(j, m.x, m.y, kE >> 24) | ((uint64_t)negbit << 63)));
    }
    static __device__ __forceinline__ double from64(double x, uint32_t neg) {
        return __longlong_as_double((long long)((uint64_t)__double_as_longlong(x) | ((uint64_t)neg << 63)));
    }
    static __device__ __forceinline__ double fast32(const Z128Tab& t, uint32_t i, uint32_t j, uint32_t neg) {
        const uint32_t kE = t.kE[i][0];
        const uint2 m = t.M[i][0];
        return __longlong_as_double(
            (long long)(mul_j_w_bits32(j, m.x, m.y, kE >> 24) | ((uint64_t)neg << 63)));
    }
};
template <> struct Z128Out<ZIG_F32> {
    using T = float;
    using Pair = float2;
    static __device__ __forceinline__ float fast(const Z128Tab& t, uint32_t i, uint32_t j,
                                                 uint32_t negbit, int, uint32_t) {
        return __uint_as_float(__float_as_uint(__fmul_rn((float)j, t.W32[i])) | (negbit << 31));
    }
    static __device__ __forceinline__ float from64(double x, uint32_t neg) {
        return __uint_as_float(__float_as_uint(__double2float_rn(x)) | (neg << 31));
    }
    static __device__ __forceinline__ float fast32(const Z128Tab& t, uint32_t i, uint32_t j, uint32_t neg) {
        return fast(t, i, j, neg, 0, 0);
    }
};
template <> struct Z128Out<ZIG_BF16> {
    using T = uint16_t;
    using Pair = uint32_t;
    static __device__ __forceinline__ uint16_t fast(const Z128Tab& t, uint32_t i, uint32_t j,
                                                    uint32_t negbit, int, uint32_t) {
        return f32_to_bf16_bits(Z128Out<ZIG_F32>::fast(t, i, j, negbit, 0, 0));
    }
    static __device__ __forceinline__ uint16_t from64(double x, uint32_t neg) {
        return f32_to_bf16_bits(Z128Out<ZIG_F32>::from64(x, neg));
    }
    static __device__ __forceinline__ uint16_t fast32(const Z128Tab& t, uint32_t i, uint32_t j, uint32_t neg) {
        return fast(t, i, j, neg, 0, 0);
    }
};

// Staging: per warp, 32 rows x 16 elements, row-major, with the pair index
// (two elements) XOR-swizzled by the row so that the per-lane pair stores and
// the per-row element reads are both bank-conflict free.
template <typename T> struct ZSw;
template <> struct ZSw<double> { static __device__ __forceinline__ int f(int r) { return r & 7; } };
template <> struct ZSw<float> { static __device__ __forceinline__ int f(int r) { return (r >> 1) & 7; } };
template <> struct ZSw<uint16_t> { static __device__ __forceinline__ int f(int r) { return (r >> 2) & 7; } };

template <typename T>
__device__ __forceinline__ int zelt(int row, int col) {   // element index of (row, col)
    return row * 16 + ((((col >> 1) ^ ZSw<T>::f(row)) << 1) | (col & 1));
}

// binary32 value of m * 2^-53 for m < 2^53 (relative error < 2^-23).
__device__ __forceinline__ float m53_to_float(uint64_t m) {
    const uint32_t hi = (uint32_t)(m >> 29);
    return hi ? (float)hi * 0x1p-24f : (float)(uint32_t)m * 0x1p-53f;
}

// Decide one queued record.  Wedge: the slot already holds RN(j * w[i]) from
// Phase A, so only the decision is made.  Tail: decision, and on acceptance
// the value x = R - ln(U1)/R goes into its slot.
template <class G, int DT>
__device__ __forceinline__ bool z128_decide(const Z128Tab& t, const SlowRec& r, bool& has_val,
                                            typename Z128Out<DT>::T& val) {
    const uint32_t neg = (uint32_t)(r.a >> 62) & 1u;
    has_val = false;
    if (!(r.a >> 63)) {
        const uint32_t j = (uint32_t)r.a & 0xFFFFFFu;
        const uint32_t i = (uint32_t)(r.a >> 24) & 0x7Fu;
        const uint64_t m1 = G::m53_of(r.b, 0, 0);
        // binary32 filter: |y32/y - 1| + |e32/e - 1| <= 2.6e-6 < 2^-16 (expf <= 2 ulp)
        const float x32 = __fmul_rn((float)j, t.W32[i]);
        const float e32 = expf(__fmul_rn(__fmul_rn(-0.5f, x32), x32));
        const float u32 = (float)(uint32_t)(m1 >> 29) * 0x1p-24f;
        const float y32 = __fadd_rn(t.Y32[i + 1], __fmul_rn(t.DY32[i], u32));
        if (y32 < e32 * (1.0f - 0x1p-16f)) return true;
        if (y32 > e32 * (1.0f + 0x1p-16f)) return false;
        // inside the margin: the binary64 test exactly as defined
        const double x = __dmul_rn((double)j, t.W[i]);
        const double U = m53_to_double(m1);
        const double y = __dadd_rn(t.Y[i + 1], __dmul_rn(__dsub_rn(t.Y[i], t.Y[i + 1]), U));
        return y < exp(neg_half_sq(x));
    }
    // Tail: y = exp(-R (x - R/2)) U2 < exp(-x^2/2) with x = R + s, s = -ln(U1)/R, is
    // ln U2 < -s^2/2 in exact arithmetic.  Decide that in binary32 when it clears a
    // margin of 2^-14 (1 + s^2/2 + |ln U2|), far above the binary32 errors (< 1e-5
    // relative); otherwise evaluate the definition in binary64.
    const double R = zigtab::ZIG128_R;
    const uint64_t m1 = r.a & ((1ull << 53) - 1);
    const uint64_t n1 = (1ull << 53) - m1;           // U1 = n1 * 2^-53 in (0, 1]
    const float s32 = -logf(m53_to_float(n1)) * (float)(1.0 / zigtab::ZIG128_R);
    const float h32 = 0.5f * s32 * s32;
    bool acc;
    if (r.b == 0) {
        acc = true;                                   // U2 = 0: y = 0 < exp(-x^2/2)
    } else {
        const float l32 = logf(m53_to_float(r.b));
        const float marg = 0x1p-14f * (1.0f + h32 - l32);
        if (l32 < -h32 - marg) acc = true;
        else if (l32 > -h32 + marg) acc = false;
        else {
            const double U1 = __dsub_rn(1.0, m53_to_double(m1));
            const double U2 = m53_to_double(r.b);
            const double x = __dsub_rn(R, __ddiv_rn(log(U1), R));
            const double y = __dmul_rn(exp(__dmul_rn(-R, __dsub_rn(x, __dmul_rn(0.5, R)))), U2);
            acc = y < exp(neg_half_sq(x));
        }
    }
    if (acc) {
        const double U1 = __dsub_rn(1.0, m53_to_double(m1));
        const double x = __dsub_rn(R, __ddiv_rn(log(U1), R));
        val = Z128Out<DT>::from64(x, neg);
        has_val = true;
    }
    return acc;
}

template <typename OutT>
__host__ __device__ constexpr size_t z128_warp_bytes() {
    // [rej u32 x 32][row info 16 B x 32][ring SlowRec x kQCap][stage OutT x 32 x 16]
    return 128 + 512 + kQCap * sizeof(SlowRec) + 32 * 16 * sizeof(OutT);
}

struct RowInfo {
    unsigned long long dst;
    int cnt;
    int pad;
};

// One candidate of Phase A.  Returns true (and fills rec) for a slow candidate.
template <class G, int DT>
__device__ __forceinline__ bool z128_candidate(G& g, const Z128Tab& t, int lane, int v,
                                               typename Z128Out<DT>::T& val, SlowRec& rec,
                                               uint64_t& draws) {
    const uint32_t w = g.next_u32();
    const uint32_t i = w & 0x7Fu;
    const uint32_t neg = (~w >> 7) & 1u;   // bit 7 set -> positive
    const uint32_t j = w >> 8;
    const uint32_t kE = t.kE[i][lane];
    val = Z128Out<DT>::fast(t, i, j, neg, lane, kE);
    if (j < (kE & 0xFFFFFFu)) return false;
    const uint64_t meta = ((uint64_t)lane << 53) | ((uint64_t)v << 58) | ((uint64_t)neg << 62);
    if (i < 127) {
        g.snap(1, rec.b, rec.a);
        rec.a = meta | (uint64_t)j | ((uint64_t)i << 24);
        draws += G::kStepsPerDouble;
    } else {
        rec.a = meta | (1ull << 63) | g.next_m53();
        rec.b = g.next_m53();
        draws += 2 * G::kStepsPerDouble;
    }
    return true;
}

// MODE 0: generation into a.out; MODE 1: mutation x += sigma * z (binary32).
template <int PRNG, int DT, int MODE>
__global__ void __launch_bounds__(kZBlock, 1) z128_kernel(GenArgs a) {
    using G = typename GenOf<PRNG>::T;
    using OutT = typename Z128Out<DT>::T;
    using Pair = typename Z128Out<DT>::Pair;
    __shared__ Z128Tab t;
    extern __shared__ __align__(16) unsigned char z128_dsm[];
    z128tab_load(t);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char* wbase = z128_dsm + (size_t)wib * z128_warp_bytes<OutT>();
    uint32_t* rej = (uint32_t*)wbase;
    RowInfo* rowinfo = (RowInfo*)(wbase + 128);
    SlowRec* q = (SlowRec*)(wbase + 640);
    OutT* stage = (OutT*)(wbase + 640 + kQCap * sizeof(SlowRec));
    const uint32_t lt_mask = (1u << lane) - 1u;
    if (MODE == 0 && a.out == nullptr) {   // only legal when every length is zero
        if (a.lengths && a.totals[1] != 0 && blockIdx.x == 0 && threadIdx.x == 0)
            atomicOr(&d_err, kErrNullOutput);
        return;
    }
    const uint64_t n_units = units_total(a);
    const uint64_t n_groups = (n_units + 31) >> 5;
    const uint64_t warp_id = (uint64_t)blockIdx.x * kZWarps + wib;
    const uint64_t warp_stride = (uint64_t)gridDim.x * kZWarps;
    OutT* out = (OutT*)a.out;

    // decide up to 32 queued records from `head`; results land in stage / rej
    auto run_pass = [&](uint32_t head, uint32_t n) {
        if ((uint32_t)lane < n) {
            const SlowRec rr = q[(head + lane) & (kQCap - 1)];
            OutT val;
            bool has_val;
            const int row = (int)(rr.a >> 53) & 31, slot = (int)(rr.a >> 58) & 15;
            if (!z128_decide<G, DT>(t, rr, has_val, val)) atomicOr(&rej[row], 1u << slot);
            else if (has_val) stage[zelt<OutT>(row, slot)] = val;
        }
    };

    for (uint64_t grp = warp_id; grp < n_groups; grp += warp_stride) {
        const uint64_t u = grp * 32 + lane;
        uint64_t rem = 0;
        OutT* dst = out;
        G g;
        g.seed(0);
        if (u < n_units) {
            uint64_t s, qd, off, n;
            unit_info(a, u, s, qd, off, n);
            g.seed(MODE == 0 ? a.seeds[s] : a.mut_seed + s);   // mutation: seed + row
            if (qd) g.jump(qd * kChunkDraws, &d_jump);
            rem = n;
            dst = out + off;
        }
        uint64_t draws = 0;   // raw steps used by this unit (chunk-overflow check)
        const bool check_chunk = a.chunk_log2 != 0 && rem != 0;
        uint32_t head = 0, tail = 0;   // warp-uniform ring indices

        while (__any_sync(kFull, rem > 0)) {
            const int cnt = (int)umin64(rem, 16);
            rej[lane] = 0;
            draws += (uint64_t)cnt;
            __syncwarp();
#pragma unroll 1
            for (int v = 0; v < 16; v += 2) {
                OutT v0, v1;
                SlowRec r0, r1;
                const bool s0 = (v < cnt) && z128_candidate<G, DT>(g, t, lane, v, v0, r0, draws);
                const bool s1 = (v + 1 < cnt) && z128_candidate<G, DT>(g, t, lane, v + 1, v1, r1, draws);
                Pair pr;
                if constexpr (DT == ZIG_BF16) pr = (uint32_t)v0 | ((uint32_t)v1 << 16);
                else pr = Pair{v0, v1};
                *(Pair*)&stage[zelt<OutT>(lane, v)] = pr;
                const uint32_t m0 = __ballot_sync(kFull, s0);
                const uint32_t m1 = __ballot_sync(kFull, s1);
                if (m0 | m1) {
                    if (s0) q[(tail + __popc(m0 & lt_mask)) & (kQCap - 1)] = r0;
                    tail += __popc(m0);
                    if (s1) q[(tail + __popc(m1 & lt_mask)) & (kQCap - 1)] = r1;
                    tail += __popc(m1);
                    if (tail - head >= 32) {
                        __syncwarp();
                        run_pass(head, 32);
                        head += 32;
                        __syncwarp();
                    }
                }
            }
            // drain the rest of this batch's records
            while (tail != head) {
                __syncwarp();
                const uint32_t n = umin64(tail - head, 32);
                run_pass(head, n);
                head += n;
            }
            __syncwarp();
            // rejected slots are skipped (each costs the stream one more layer draw,
            // which the next batch draws as a new candidate)
            const int acc = cnt - __popc(rej[lane]);
            rowinfo[lane].dst = (unsigned long long)dst;
            rowinfo[lane].cnt = acc;
            __syncwarp();
            {
                const int half = lane >> 4, c = lane & 15;
#pragma unroll 4
                for (int k = 0; k < 16; ++k) {
                    const int row = 2 * k + half;
                    const int rc = rowinfo[row].cnt;
                    OutT* rd = (OutT*)rowinfo[row].dst;
                    if (c < rc) {
                        // slot of the row's c-th accepted candidate
                        int src = c;
                        for (uint32_t m = rej[row]; m; m &= m - 1) {
                            if (__ffs(m) - 1 <= src) ++src;
                            else break;
                        }
                        const OutT z = stage[zelt<OutT>(row, src)];
                        if constexpr (MODE == 0) rd[c] = z;
                        else ((float*)rd)[c] = fmaf(a.sigma, (float)z, ((float*)rd)[c]);
                    }
                }
            }
            __syncwarp();
            dst += acc;
            rem -= (uint64_t)acc;
        }
        if (check_chunk && draws > kChunkDraws) atomicOr(&d_err, kErrChunkOverflow);
    }
}

// Exclusive prefix sums of lengths and unit counts (one block).
__global__ void __launch_bounds__(1024) scan_kernel(const uint64_t* lengths, uint64_t n,
                                                    uint32_t chunk_log2, uint64_t* offsets,
                                                    uint64_t* ustart, uint64_t* totals) {
    __shared__ uint64_t sl[1024], su[1024];
    const int t = threadIdx.x;
    const uint64_t per = (n + 1023) / 1024;
    const uint64_t b = umin64(n, (uint64_t)t * per), e = umin64(n, b + per);
    uint64_t accl = 0, accu = 0;
    for (uint64_t s = b; s < e; ++s) {
        uint64_t L = lengths[s];
        accl += L;
        accu += chunk_log2 ? ((L + (1ull << chunk_log2) - 1) >> chunk_log2) : (L ? 1 : 0);
    }
    sl[t] = accl;
    su[t] = accu;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {   // Hillis-Steele inclusive scan
        uint64_t vl = (t >= d) ? sl[t - d] : 0, vu = (t >= d) ? su[t - d] : 0;
        __syncthreads();
        sl[t] += vl;
        su[t] += vu;
        __syncthreads();
    }
    accl = t ? sl[t - 1] : 0;
    accu = t ? su[t - 1] : 0;
    for (uint64_t s = b; s < e; ++s) {
        uint64_t L = lengths[s];
        offsets[s] = accl;
        ustart[s] = accu;
        accl += L;
        accu += chunk_log2 ? ((L + (1ull << chunk_log2) - 1) >> chunk_log2) : (L ? 1 : 0);
    }
    if (t == 1023) {
        totals[0] = su[1023];
        totals[1] = sl[1023];
    }
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
void* g_ws[kMaxDevices];
size_t g_ws_bytes[kMaxDevices];

struct Affine { uint64_t A, C; };
static Affine compose(Affine o, Affine i) { return {o.A * i.A, o.A * i.C + o.C}; }

// xoroshiro128 one step on a (x0, x1) pair
static void xoro_step(uint64_t& x0, uint64_t& x1) {
    uint64_t q1 = x1 ^ x0;
    x0 = ((x0 << 24) | (x0 >> 40)) ^ q1 ^ (q1 << 16);
    x1 = (q1 << 37) | (q1 >> 27);
}

static void fill_jump(JumpTab& jt) {
    Affine l48 = {kLcgA, kLcgC};
    Affine lxm = {kLxmM, 1};
    static uint64_t col[128][2], nxt[128][2];
    for (int c = 0; c < 128; ++c) {
        uint64_t x0 = c < 64 ? (1ull << c) : 0, x1 = c < 64 ? 0 : (1ull << (c - 64));
        xoro_step(x0, x1);
        col[c][0] = x0;
        col[c][1] = x1;
    }
    for (int b = 0; b < 64; ++b) {
        jt.lcg48_A[b] = l48.A & kMask48;
        jt.lcg48_C[b] = l48.C & kMask48;
        jt.lxm_A[b] = lxm.A;
        jt.lxm_G[b] = lxm.C;
        for (int c = 0; c < 128; ++c) {
            jt.xoro[b][2 * c] = col[c][0];
            jt.xoro[b][2 * c + 1] = col[c][1];
        }
        l48 = compose(l48, l48);
        lxm = compose(lxm, lxm);
        // square the GF(2) map: column c of T^2 = T applied to column c of T
        for (int c = 0; c < 128; ++c) {
            uint64_t r0 = 0, r1 = 0;
            for (int d = 0; d < 128; ++d) {
                uint64_t bit = d < 64 ? (col[c][0] >> d) & 1 : (col[c][1] >> (d - 64)) & 1;
                if (bit) {
                    r0 ^= col[d][0];
                    r1 ^= col[d][1];
                }
            }
            nxt[c][0] = r0;
            nxt[c][1] = r1;
        }
        std::memcpy(col, nxt, sizeof(col));
    }
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
    uint64_t M[128];
    for (int i = 0; i < 128; ++i) {
        uint64_t bits;
        std::memcpy(&bits, &zigtab::ZIG128_W[i], 8);
        int E = (int)((bits >> 52) & 0x7FF);
        if (E - 900 < 0 || E - 900 > 255) return ZIG_ERR_UNSUPPORTED;
        kE[i] = zigtab::ZIG128_K[i] | ((uint32_t)(E - 900) << 24);
        M[i] = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    }
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_kE, kE, sizeof(kE)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_M, M, sizeof(M)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_W, zigtab::ZIG128_W, sizeof(zigtab::ZIG128_W)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_Y, zigtab::ZIG128_Y, sizeof(zigtab::ZIG128_Y)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_W32, zigtab::ZIG128_W32, sizeof(zigtab::ZIG128_W32)));
    float y32[128], dy32[128];
    for (int i = 0; i < 128; ++i) {
        y32[i] = (float)zigtab::ZIG128_Y[i];
        dy32[i] = i < 127 ? (float)(zigtab::ZIG128_Y[i] - zigtab::ZIG128_Y[i + 1]) : 0.0f;
    }
    ZIG_CUDA(cudaMemcpyToSymbol(d_z128_Y32, y32, sizeof(y32)));
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
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_QA, zigtab::ZIG256_QA, sizeof(uint64_t) * nr));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_THR, zigtab::ZIG256_THR, sizeof(zigtab::ZIG256_THR)));
    ZIG_CUDA(cudaMemcpyToSymbol(d_z256_ALIAS, zigtab::ZIG256_ALIAS, sizeof(zigtab::ZIG256_ALIAS)));
    static JumpTab jt;
    fill_jump(jt);
    ZIG_CUDA(cudaMemcpyToSymbol(d_jump, &jt, sizeof(jt)));
    unsigned zero = 0;
    ZIG_CUDA(cudaMemcpyToSymbol(d_err, &zero, sizeof(zero)));
    ZIG_CUDA(cudaDeviceSynchronize());
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

template <int ALG, int PRNG>
static GenFn pick_dt(int dt) {
    if constexpr (ALG == ZIG_ZIG128) {
        switch (dt) {
        case ZIG_F64: return z128_kernel<PRNG, ZIG_F64, 0>;
        case ZIG_F32: return z128_kernel<PRNG, ZIG_F32, 0>;
        default: return z128_kernel<PRNG, ZIG_BF16, 0>;
        }
    } else {
        switch (dt) {
        case ZIG_F64: return gen_kernel<ALG, PRNG, ZIG_F64>;
        case ZIG_F32: return gen_kernel<ALG, PRNG, ZIG_F32>;
        default: return gen_kernel<ALG, PRNG, ZIG_BF16>;
        }
    }
}
template <int ALG>
static GenFn pick_prng(int prng, int dt) {
    switch (prng) {
    case ZIG_LCG48: return pick_dt<ALG, 0>(dt);
    case ZIG_SPLITMIX64: return pick_dt<ALG, 1>(dt);
    default: return pick_dt<ALG, 2>(dt);
    }
}
static GenFn pick(int alg, int prng, int dt) {
    switch (alg) {
    case ZIG_ZIG128: return pick_prng<ZIG_ZIG128>(prng, dt);
    case ZIG_POLAR: return pick_prng<ZIG_POLAR>(prng, dt);
    default: return pick_prng<ZIG_ZIG256>(prng, dt);
    }
}

// Dynamic shared memory a kernel needs (0 for the kernels that use static only).
static size_t dyn_smem_of(int alg, int dt) {
    if (alg != ZIG_ZIG128) return 0;
    size_t per = dt == ZIG_F64 ? z128_warp_bytes<double>()
               : dt == ZIG_F32 ? z128_warp_bytes<float>() : z128_warp_bytes<uint16_t>();
    return per * kZWarps;
}

static int block_of(int alg) { return alg == ZIG_ZIG128 ? kZBlock : kBlock; }

// Opt in to the dynamic shared memory a launch needs (static + dynamic may pass
// the 48 KB default only with the attribute set).
static bool allow_dyn_smem(const void* fn, size_t bytes) {
    if (bytes == 0) return true;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
           cudaSuccess;
}

static int grid_for(const void* fn, int dev, uint64_t n_groups, size_t dyn = 0, int block = kBlock) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, dyn) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    uint64_t full = (uint64_t)g_sms[dev] * per_sm;
    const uint64_t warps = (uint64_t)block / 32;
    uint64_t need = (n_groups + warps - 1) / warps;
    if (need == 0) need = 1;
    return (int)std::min<uint64_t>(full, need);
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

size_t zig_generate_workspace_bytes(uint64_t n_streams) {
    return (size_t)(16 * n_streams + 256);
}

zig_status zig_generate(zig_prng prng, zig_alg alg, const uint64_t* seeds_dev,
                        const uint64_t* lengths_dev, uint64_t uniform_len, uint64_t n_streams,
                        uint32_t chunk_log2, zig_dtype dtype, void* out_dev, void* workspace_dev,
                        size_t workspace_bytes, void* stream) {
    if ((unsigned)prng > 2u || (unsigned)alg > 2u || (unsigned)dtype > 2u) return ZIG_ERR_INVALID_ARG;
    if (chunk_log2 != 0 && (chunk_log2 < 4 || chunk_log2 > 24)) return ZIG_ERR_INVALID_ARG;
    if (n_streams == 0) return ZIG_OK;
    // out_dev may be NULL only with lengths_dev (an all-zero batch); the kernel
    // latches ZIG_ERR_INVALID_ARG in the error word if the lengths sum above zero
    if (!seeds_dev || (!out_dev && !lengths_dev)) return ZIG_ERR_INVALID_ARG;
    const size_t esz = dtype == ZIG_F64 ? 8 : dtype == ZIG_F32 ? 4 : 2;
    if (((uintptr_t)out_dev) % esz || ((uintptr_t)seeds_dev) % 8) return ZIG_ERR_INVALID_ARG;
    if (lengths_dev == nullptr) {
        if (uniform_len == 0) return ZIG_OK;
        if (uniform_len > (1ull << 40) || n_streams > (1ull << 40) / uniform_len)
            return ZIG_ERR_INVALID_ARG;
    } else if (((uintptr_t)lengths_dev) % 8 || n_streams > (1ull << 32)) {
        return ZIG_ERR_INVALID_ARG;
    }
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    GenArgs a{};
    a.seeds = seeds_dev;
    a.lengths = lengths_dev;
    a.uniform_len = uniform_len;
    a.n_streams = n_streams;
    a.chunk_log2 = chunk_log2;
    a.out = out_dev;
    uint64_t n_groups_hint;
    if (lengths_dev == nullptr) {
        a.units_per_stream = chunk_log2 ? ((uniform_len + (1ull << chunk_log2) - 1) >> chunk_log2) : 1;
        a.n_units = n_streams * a.units_per_stream;
        n_groups_hint = (a.n_units + 31) / 32;
    } else {
        size_t need = zig_generate_workspace_bytes(n_streams);
        uint64_t* ws;
        if (workspace_dev) {
            if (workspace_bytes < need || ((uintptr_t)workspace_dev) % 16) return ZIG_ERR_INVALID_ARG;
            ws = (uint64_t*)workspace_dev;
        } else {
            std::lock_guard<std::mutex> lk(host::g_mu);
            if (host::g_ws_bytes[dev] < need) {
                if (host::g_ws[dev]) cudaFree(host::g_ws[dev]);
                host::g_ws[dev] = nullptr;
                host::g_ws_bytes[dev] = 0;
                if (cudaMalloc(&host::g_ws[dev], need) != cudaSuccess) return ZIG_ERR_CUDA;
                host::g_ws_bytes[dev] = need;
            }
            ws = (uint64_t*)host::g_ws[dev];
        }
        a.offsets = ws;
        a.ustart = ws + n_streams;
        a.totals = ws + 2 * n_streams;
        scan_kernel<<<1, 1024, 0, s>>>(lengths_dev, n_streams, chunk_log2, (uint64_t*)a.offsets,
                                       (uint64_t*)a.ustart, (uint64_t*)a.totals);
        if (cudaGetLastError() != cudaSuccess) return ZIG_ERR_CUDA;
        n_groups_hint = ~0ull >> 8;   // unknown on the host: fill the device
    }
    host::GenFn fn = host::pick(alg, prng, dtype);
    const size_t dyn = host::dyn_smem_of(alg, dtype);
    if (!host::allow_dyn_smem((const void*)fn, dyn)) return ZIG_ERR_CUDA;
    const int block = host::block_of(alg);
    int grid = host::grid_for((const void*)fn, dev, n_groups_hint, dyn, block);
    fn<<<grid, block, dyn, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
}

zig_status zig_mutate(float* x_dev, float sigma, uint64_t P, uint64_t L, uint64_t seed,
                      zig_prng prng, void* stream) {
    if ((unsigned)prng > 2u || !std::isfinite(sigma)) return ZIG_ERR_INVALID_ARG;
    if (P == 0 || L == 0) return ZIG_OK;
    if (!x_dev || ((uintptr_t)x_dev) % 4 || L > (1ull << 40) || P > (1ull << 40) / L)
        return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    const uint64_t upr = (L + 1023) >> 10;
    const uint64_t groups = (P * upr + 31) / 32;
    cudaStream_t s = (cudaStream_t)stream;
    GenArgs a{};
    a.uniform_len = L;          // row length
    a.n_streams = P;
    a.chunk_log2 = 10;
    a.out = x_dev;
    a.units_per_stream = upr;
    a.n_units = P * upr;
    a.sigma = sigma;
    a.seeds = nullptr;
    // the kernel seeds row p with a.uniform_len + p in mutation mode; pass seed there
    GenArgs am = a;
    host::GenFn fn = prng == ZIG_LCG48 ? z128_kernel<0, ZIG_F32, 1>
                   : prng == ZIG_SPLITMIX64 ? z128_kernel<1, ZIG_F32, 1>
                                            : z128_kernel<2, ZIG_F32, 1>;
    am.mut_seed = seed;
    const size_t dyn = host::dyn_smem_of(ZIG_ZIG128, ZIG_F32);
    if (!host::allow_dyn_smem((const void*)fn, dyn)) return ZIG_ERR_CUDA;
    int grid = host::grid_for((const void*)fn, dev, groups, dyn, kZBlock);
    fn<<<grid, kZBlock, dyn, s>>>(am);
    return cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
}

zig_status zig_prng_fill(zig_prng prng, const uint64_t* seeds_dev, uint64_t n_streams, uint64_t n,
                         uint64_t skip, int kind, uint64_t* out_dev, void* stream) {
    if ((unsigned)prng > 2u || kind < 0 || kind > 2) return ZIG_ERR_INVALID_ARG;
    if (n_streams == 0 || n == 0) return ZIG_OK;
    if (!seeds_dev || !out_dev || n_streams > (1ull << 40) / n) return ZIG_ERR_INVALID_ARG;
    int dev;
    zig_status st = host::current_device(dev);
    if (st != ZIG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned grid = (unsigned)((n_streams + 255) / 256);
    if (prng == ZIG_LCG48) prng_fill_kernel<0><<<grid, 256, 0, s>>>(seeds_dev, n_streams, n, skip, kind, out_dev);
    else if (prng == ZIG_SPLITMIX64) prng_fill_kernel<1><<<grid, 256, 0, s>>>(seeds_dev, n_streams, n, skip, kind, out_dev);
    else prng_fill_kernel<2><<<grid, 256, 0, s>>>(seeds_dev, n_streams, n, skip, kind, out_dev);
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
    if (w & kErrNullOutput) return ZIG_ERR_INVALID_ARG;
    if (w & kErrTimeout) return ZIG_ERR_TIMEOUT;
    if (w & kErrChunkOverflow) return ZIG_ERR_CHUNK_OVERFLOW;
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
    if ((unsigned)prng > 2u || (unsigned)alg > 2u || (unsigned)dtype > 2u) return ZIG_ERR_INVALID_ARG;
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
    // the scan rewrites every offset, unit start and total this call reads
    scan_kernel<<<1, 1024, 0, s>>>(lengths_dev, n_streams, chunk_log2, (uint64_t*)a.offsets,
                                   (uint64_t*)a.ustart, (uint64_t*)a.totals);
    if (cudaGetLastError() != cudaSuccess) return ZIG_ERR_CUDA;
    host::GenFn fn = host::pick(alg, prng, dtype);
    const size_t dyn = host::dyn_smem_of(alg, dtype);
    if (!host::allow_dyn_smem((const void*)fn, dyn)) return ZIG_ERR_CUDA;
    const int block = host::block_of(alg);
    int grid = host::grid_for((const void*)fn, dev, ~0ull >> 8, dyn, block);
    fn<<<grid, block, dyn, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
}
