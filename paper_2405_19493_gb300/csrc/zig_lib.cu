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
struct Z128Smem {
    uint32_t kE[128];
    uint64_t M[128];
    double W[128];
    double Y[128];
    float W32[128];
};

__device__ __forceinline__ void z128_load(Z128Smem& t) {
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        t.kE[i] = d_z128_kE[i];
        t.M[i] = d_z128_M[i];
        t.W[i] = d_z128_W[i];
        t.Y[i] = d_z128_Y[i];
        t.W32[i] = d_z128_W32[i];
    }
}

__device__ __forceinline__ double neg_half_sq(double x) {
    return __dmul_rn(__dmul_rn(-0.5, x), x);
}

// Slow path of the 128-level sampler, decided in binary64 exactly as the
// definition orders the operations.  Returns true when accepted; x is set to
// the (non-negative) value.  `extra` counts raw draws beyond the layer draw.
template <class G>
__device__ __forceinline__ bool z128_slow(G& g, const Z128Smem& t, uint32_t i, uint32_t j, double& x,
                                       uint32_t& extra) {
    const double R = zigtab::ZIG128_R;
    double y;
    constexpr uint32_t kStepsPerDouble = (sizeof(G) == sizeof(GenLcg48)) ? 2u : 1u;
    if (i < 127) {
        x = __dmul_rn((double)j, t.W[i]);
        double U = m53_to_double(g.next_m53());
        y = __dadd_rn(t.Y[i + 1], __dmul_rn(__dsub_rn(t.Y[i], t.Y[i + 1]), U));
        extra += kStepsPerDouble;
    } else {
        double U1 = __dsub_rn(1.0, m53_to_double(g.next_m53()));
        double U2 = m53_to_double(g.next_m53());
        x = __dsub_rn(R, __ddiv_rn(log(U1), R));
        y = __dmul_rn(exp(__dmul_rn(-R, __dsub_rn(x, __dmul_rn(0.5, R)))), U2);
        extra += 2 * kStepsPerDouble;
    }
    return y < exp(neg_half_sq(x));
}

// One 128-level variate as binary64 bits (sign included).
template <class G>
__device__ __forceinline__ uint64_t z128_f64(G& g, const Z128Smem& t, uint32_t& extra) {
    for (;;) {
        uint32_t u = g.next_u32();
        uint32_t i = u & 0x7Fu;
        uint64_t neg = (uint64_t)((~u >> 7) & 1u) << 63;   // bit 7 set -> positive
        uint32_t j = u >> 8;
        uint32_t kE = t.kE[i];
        if (j < (kE & 0xFFFFFFu)) {
            return mul_j_w_bits(j, t.M[i], (int)(kE >> 24) + 900) | neg;
        }
        double x;
        if (z128_slow(g, t, i, j, x, extra)) return (uint64_t)__double_as_longlong(x) | neg;
        ++extra;   // the restart's layer draw
    }
}

// One 128-level variate with binary32 arithmetic on the fast path; the slow
// path decides in binary64 and rounds its value once.
template <class G>
__device__ __forceinline__ float z128_f32(G& g, const Z128Smem& t, uint32_t& extra) {
    for (;;) {
        uint32_t u = g.next_u32();
        uint32_t i = u & 0x7Fu;
        uint32_t negbit = ((~u >> 7) & 1u) << 31;
        uint32_t j = u >> 8;
        if (j < (t.kE[i] & 0xFFFFFFu)) {
            float x = __fmul_rn((float)j, t.W32[i]);
            return __uint_as_float(__float_as_uint(x) | negbit);
        }
        double x;
        if (z128_slow(g, t, i, j, x, extra)) {
            float xf = __double2float_rn(x);
            return __uint_as_float(__float_as_uint(xf) | negbit);
        }
        ++extra;   // the restart's layer draw
    }
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
    __shared__ Z128Smem t128;
    __shared__ Z256Smem t256;
    __shared__ OutT stage_all[kWarps][32 * kStageCols];
    if (ALG == ZIG_ZIG128) z128_load(t128);
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
                    if (ALG == ZIG_ZIG128) {
                        if (DT == ZIG_F64) {
                            z = __longlong_as_double((long long)z128_f64(g, t128, extra));
                        } else if (DT == ZIG_F32) {
                            z = z128_f32(g, t128, extra);
                        } else {
                            z = f32_to_bf16_bits(z128_f32(g, t128, extra));
                        }
                    } else if (ALG == ZIG_POLAR) {
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
            const uint64_t per = (ALG == ZIG_ZIG256 && PRNG == ZIG_LCG48) ? 2 : 1;
            uint64_t draws = (ALG == ZIG_POLAR) ? (uint64_t)extra : n_unit * per + extra;
            if (draws > kChunkDraws) atomicOr(&d_err, kErrChunkOverflow);
        }
    }
}

// Mutation: x[p][l] = fmaf(sigma, z, x[p][l]) with z the binary32 128-level
// variates of stream seed + p, chunked by 2^10.
template <int PRNG>
__global__ void __launch_bounds__(kBlock) mutate_kernel(float* x, float sigma, uint64_t P,
                                                        uint64_t L, uint64_t seed,
                                                        uint64_t units_per_row) {
    using G = typename GenOf<PRNG>::T;
    __shared__ Z128Smem t128;
    __shared__ float stage_all[kWarps][32 * kStageCols];
    z128_load(t128);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float* stage = stage_all[threadIdx.x >> 5];
    const uint64_t n_units = P * units_per_row;
    const uint64_t n_groups = (n_units + 31) >> 5;
    const uint64_t warp_id = (uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const uint64_t warp_stride = (uint64_t)gridDim.x * kWarps;
    constexpr uint32_t kC = 10;
    for (uint64_t grp = warp_id; grp < n_groups; grp += warp_stride) {
        uint64_t u = grp * 32 + lane;
        uint64_t rem = 0;
        float* dst = x;
        G g;
        g.seed(0);
        if (u < n_units) {
            uint64_t p = u / units_per_row, q = u - p * units_per_row;
            g.seed(seed + p);
            if (q) g.jump(q * kChunkDraws, &d_jump);
            uint64_t t0 = q << kC;
            rem = umin64(L - t0, (uint64_t)1 << kC);
            dst = x + p * L + t0;
        }
        uint32_t extra = 0;
        while (__any_sync(kFull, rem > 0)) {
            const int cnt = (int)umin64(rem, (uint64_t)kStageCols);
#pragma unroll 1
            for (int v = 0; v < kStageCols; ++v) {
                if (v < cnt) stage[stage_idx<float>(lane, v)] = z128_f32(g, t128, extra);
            }
            __syncwarp();
            stage_flush_fma(stage, dst, cnt, lane, sigma);
            __syncwarp();
            dst += cnt;
            rem -= cnt;
        }
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
    switch (dt) {
    case ZIG_F64: return gen_kernel<ALG, PRNG, ZIG_F64>;
    case ZIG_F32: return gen_kernel<ALG, PRNG, ZIG_F32>;
    default: return gen_kernel<ALG, PRNG, ZIG_BF16>;
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

static int grid_for(const void* fn, int dev, uint64_t n_groups) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    uint64_t full = (uint64_t)g_sms[dev] * per_sm;
    uint64_t need = (n_groups + kWarps - 1) / kWarps;
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
    int grid = host::grid_for((const void*)fn, dev, n_groups_hint);
    fn<<<grid, kBlock, 0, s>>>(a);
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
    const void* fn = prng == ZIG_LCG48 ? (const void*)mutate_kernel<0>
                   : prng == ZIG_SPLITMIX64 ? (const void*)mutate_kernel<1>
                                            : (const void*)mutate_kernel<2>;
    int grid = host::grid_for(fn, dev, groups);
    if (prng == ZIG_LCG48) mutate_kernel<0><<<grid, kBlock, 0, s>>>(x_dev, sigma, P, L, seed, upr);
    else if (prng == ZIG_SPLITMIX64) mutate_kernel<1><<<grid, kBlock, 0, s>>>(x_dev, sigma, P, L, seed, upr);
    else mutate_kernel<2><<<grid, kBlock, 0, s>>>(x_dev, sigma, P, L, seed, upr);
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
    int grid = host::grid_for((const void*)fn, dev, ~0ull >> 8);
    fn<<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? ZIG_OK : ZIG_ERR_CUDA;
}
