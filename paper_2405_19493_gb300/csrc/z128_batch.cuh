// 128-level ziggurat (GSL form): the speculative batch kernel, for binary64,
// binary32 and bfloat16 output and for Gaussian mutation of binary32 rows.
// Included by zig_lib.cu after the samplers and the unit helpers.
//
// Each lane owns one unit (a stream, or a 2^c chunk of one) with its generator
// in registers; a warp works on its 32 units in batches of B draws per lane,
// B = min(32, S - 2 kU) (kU = raw steps per nextDouble), so that a batch with
// the draws a tail may need past it fits the S slots of the lane's row (35 for
// 32-bit slots, 34 for 64-bit ones, what shared memory holds for 20 warps;
// slots past the 32 a row store writes only ever hold uniforms).
//  A. Every lane takes B draws in lockstep and keeps each in its row, with no
//     branch and no vote: the fast test j < k[i] (Sec. 1; the GSL form's first
//     comparison) only sets a bit of the lane's mask nf (a carry chain: two
//     instructions a draw).  A slot holds the
//     32-bit draw w, or for the generators whose draws are nextLong outputs the
//     whole output (a wedge or tail test may read it as its uniform).
//  B. Each lane walks its nf bits in draw order and decides its own slow
//     candidates (2.8 % of draws: about 0.9 per lane and batch, so the warp's
//     loop runs about three times).  A slow candidate at draw p (j >= k[i]) consumes the next kU
//     (wedge, i < 127) or 2 kU (tail) draws as its uniforms; a consumed draw is
//     not a candidate, whatever its bit says.  Uniforms past the batch are drawn
//     at once.  The wedge and tail tests run first in binary32 with proven
//     margins.  A rejected candidate and every consumed draw are dropped.  An
//     accepted tail's value, R - ln(U1)/R in binary64, is not computed here: its
//     U1 and output address join a per-warp queue that is evaluated 32 at a time.
//  C. The warp writes its rows one at a time, all 32 lanes on one row, lane c
//     on slot c: a kept slot's output index is the number of kept slots below
//     it, so one store instruction writes the row's batch as one contiguous
//     run (about 240 bytes) at any alignment, with no close-up of the row and
//     no carry between batches.  Each lane rebuilds its value x = sign RN(j w[i])
//     from the draw: binary64, one fma, or for some rows the same correctly
//     rounded product in 32-bit integer arithmetic (the narrow binary64 pipe
//     and the integer pipes share the work); binary32 and bfloat16, one binary32
//     multiplication j w32[i].  Mutation rows read x and store x + sigma z.
// A unit's outputs are its accepted candidates in draw order: the sequence a
// one-variate-at-a-time loop produces (Sec. 2, Listing 2, repeated).
#pragma once

namespace zf {

// ---- per-generator draws ----
// SW: 32-bit words per slot.  draw(): one raw step, stored at the slot; the
// candidate w is the slot's last word.  m53(st, d, s0): the 53-bit integer of
// the nextDouble that starts at batch draw d, from the row's slots (and, for
// SplitMix64, the batch's first state s0).
// n raw steps of java.util.Random's LCG: s -> (lcg_A(n) s + lcg_C(n)) mod 2^48
__host__ __device__ constexpr uint64_t lcg_A(int n) {
    uint64_t A = 1;
    for (int k = 0; k < n; ++k) A = (A * kLcgA) & kMask48;
    return A;
}
__host__ __device__ constexpr uint64_t lcg_C(int n) {
    uint64_t C = 0;
    for (int k = 0; k < n; ++k) C = (C * kLcgA + kLcgC) & kMask48;
    return C;
}

template <int PRNG> struct Gen;
template <> struct Gen<ZIG_LCG48> {
    using G = GenLcg48;
    static constexpr int kU = 2, SW = 1;   // nextDouble = next(26), next(27)
    static __device__ __forceinline__ void draw(G& g, uint32_t* slot, uint32_t& w) { w = g.step(32); slot[0] = w; }
    // batch draw D straight from the batch's first state s0 (all draws of a batch
    // are independent of one another this way)
    template <int D>
    static __device__ __forceinline__ uint32_t draw_at(uint64_t s0) {
        return (uint32_t)(((lcg_A(D + 1) * s0 + lcg_C(D + 1)) & kMask48) >> 16);
    }
    template <int N>
    static __device__ __forceinline__ void skip(G& g) { g.s = (lcg_A(N) * g.s + lcg_C(N)) & kMask48; }
    static __device__ __forceinline__ uint64_t m53(const uint32_t* st, int d, uint64_t) {
        // next(26) = s1 >> 22 = w1 >> 6, next(27) = s2 >> 21 = w2 >> 5 (w = s >> 16)
        return ((uint64_t)(st[d] >> 6) << 27) + (st[d + 1] >> 5);
    }
    static __device__ __forceinline__ uint64_t first_state(const G& g) { return g.s; }
};
template <> struct Gen<ZIG_SPLITMIX64> {
    using G = GenSplitMix64;
    static constexpr int kU = 1, SW = 1;
    static __device__ __forceinline__ void draw(G& g, uint32_t* slot, uint32_t& w) { w = g.next_u32(); slot[0] = w; }
    static __device__ __forceinline__ uint64_t m53(const uint32_t*, int d, uint64_t s0) {
        return mix64(s0 + (uint64_t)(d + 1) * kGamma) >> 11;   // the state of draw d
    }
    static __device__ __forceinline__ uint64_t first_state(const G& g) { return g.s; }
};
template <> struct Gen<ZIG_L64X128MIX> {
    using G = GenL64X128Mix;
    static constexpr int kU = 1, SW = 2;
    // nextLong without the mixer's last z ^= z >> 32, which changes only the
    // low word (the candidate is the high word); m53 applies it.
    static __device__ __forceinline__ void draw(G& g, uint32_t* slot, uint32_t& w) {
        uint64_t z = g.s + g.x0;
        z = (z ^ (z >> 32)) * kLeaM;
        z = (z ^ (z >> 32)) * kLeaM;
        g.advance();
        *(uint64_t*)slot = z;
        w = (uint32_t)(z >> 32);
    }
    static __device__ __forceinline__ uint64_t m53(const uint32_t* st, int d, uint64_t) {
        const uint64_t z = *(const uint64_t*)(st + 2 * d);
        return (z ^ (z >> 32)) >> 11;
    }
    static __device__ __forceinline__ uint64_t first_state(const G&) { return 0; }
};
template <> struct Gen<ZIG_XOROSHIRO128PP> {
    using G = GenXoroshiro128PP;
    static constexpr int kU = 1, SW = 2;
    static __device__ __forceinline__ void draw(G& g, uint32_t* slot, uint32_t& w) {
        const uint64_t r = g.next_u64();
        *(uint64_t*)slot = r;
        w = (uint32_t)(r >> 32);
    }
    static __device__ __forceinline__ uint64_t m53(const uint32_t* st, int d, uint64_t) {
        return *(const uint64_t*)(st + 2 * d) >> 11;
    }
    static __device__ __forceinline__ uint64_t first_state(const G&) { return 0; }
};

// f(integral_constant<int, d>) for d = 0 .. N - 1, unrolled at compile time
template <int N, int D = 0, class F>
__device__ __forceinline__ void unroll(F& f) {
    if constexpr (D < N) {
        f(std::integral_constant<int, D>{});
        unroll<N, D + 1>(f);
    }
}
template <class G>
__device__ __forceinline__ uint64_t first_state_of(const G& g) {
    if constexpr (std::is_same<G, GenLcg48>::value || std::is_same<G, GenSplitMix64>::value) return g.s;
    else return 0;
}

// ---- shared memory ----
// The fast table: one 256-byte block per signed layer ix = w & 0xFF (layer
// ix & 127, positive when bit 7 is set).  Words 0..31, binary64 output: 16
// copies of the signed b = +-2^52 w[i] (low word, high word), one per lane & 15,
// so that the 16 lanes of a half warp reading 8-byte entries of random layers
// hit distinct banks; binary32 and bfloat16 output: 32 copies of the signed
// binary32 +-w32[i] = +-RN32(w[i]), one per lane.  Words 32..63: 32 copies of
// K = k[i] << 8, one per lane (j >= k[i] is w >= K).  The sign rides on the
// entry: the fma below rounds -(j w[i]) exactly as it rounds j w[i] (its zero,
// for j = 0, takes b's sign by an OR), the integer product takes it from b's
// sign bit, and the binary32 product j (-w32[i]) is -(j w32[i]), -0 for j = 0.
// The block stride of 256 bytes makes each address one byte permute of w.
// The generators whose slots are 64-bit nextLong outputs use a compact form
// instead: 128-byte blocks with half the copies (8 of b, or 16 of w32; 16 of K),
// addressed by a shift and an OR.  Their stages are twice as large, and the
// compact table is what lets 20 warps rather than 16 fit in shared memory (the
// extra copies only avoid bank conflicts).
template <int PRNG>
constexpr bool kCompactTab = Gen<PRNG>::SW == 2;
template <bool C>
struct TabT {
    uint32_t blk[256][C ? 32 : 64];
};
// byte offset of this lane's copy (copy: its byte offset in the block) in block w & 0xFF
template <bool C>
__device__ __forceinline__ uint32_t entry_off(uint32_t w, uint32_t copy) {
    if constexpr (C) return ((w & 0xFFu) << 7) | copy;
    else return __byte_perm(w, copy, 0x5504);
}
struct SlowTab {   // the wedge test's tables (z128_wedge_filter, z128_wedge_exact)
    float W32[128], Y32[128], DY32[128];
    double Wd[128], Y[128];
};

// Threads per block for a generator (the register budget is 65536 / threads:
// 102 at 640); kMaxThreads bounds them all.
__host__ __device__ constexpr int max_threads(int prng) { return prng >= 0 ? 640 : 640; }
constexpr int kMaxThreads = 640;

template <int PRNG, int DT, int MUT = 0>
struct Warp {
    static constexpr int kU = Gen<PRNG>::kU, SW = Gen<PRNG>::SW;
    static constexpr int S = SW == 1 ? 35 : 34;             // slots per row
    static constexpr int RS = SW * S;                       // row stride in words
    static constexpr int B = S - 2 * kU < 32 ? S - 2 * kU : 32;   // draws per batch
    uint32_t stage[32 * RS];   // row r, slot d: words r RS + SW d ..
    uint4 info[32];            // per row: output address (low, high), dropped slots
    uint64_t tq_addr[32];      // accepted tails waiting for their value: output address | negative
    uint64_t tq_m1[32];        // and their uniform m1 (U1 = 1 - m1 2^-53)
    uint32_t tq_sig[MUT ? 32 : 1];   // mutation: and their row's sigma bits (kGenerate: x = z)
    uint32_t tails[MUT ? 32 : 1];    // mutation: per row, the accepted tails (their queue entry updates x)
    uint32_t tq_n;
};
template <int PRNG, int DT, int MUT = 0>
__host__ __device__ constexpr size_t warp_bytes() {
    return (sizeof(Warp<PRNG, DT, MUT>) + 15) & ~(size_t)15;
}
// a mutation row's sigma word when the request generates (x = z): a NaN pattern
// no finite sigma has
constexpr uint32_t kGenerate = 0xFFFFFFFFu;
template <bool C>
__host__ __device__ constexpr size_t head_bytes() { return sizeof(TabT<C>) + ((sizeof(SlowTab) + 15) & ~(size_t)15); }
template <int PRNG, int DT, int MUT = 0>
__host__ __device__ constexpr size_t smem_bytes(int warps) {
    return head_bytes<kCompactTab<PRNG>>() + warp_bytes<PRNG, DT, MUT>() * (size_t)warps;
}

template <int DT, bool C>
__device__ __forceinline__ void tab_load(TabT<C>& t, SlowTab& s) {
    constexpr int kWords = C ? 32 : 64;   // per block; the second half holds K
    for (int k = threadIdx.x; k < 256 * kWords; k += blockDim.x) {
        const int ix = k / kWords, wd = k % kWords, i = ix & 127;
        const double wi = d_z128_W[i];
        const uint32_t K = (d_z128_kE[i] & 0xFFFFFFu) << 8;
        uint32_t v;
        if (wd >= kWords / 2) {
            v = K;
        } else if (DT == ZIG_F64) {
            const double bd = __dmul_rn(ix < 128 ? -wi : wi, 0x1p52);   // exact scaling, signed
            const long long b = __double_as_longlong(bd);
            v = (wd & 1) ? (uint32_t)(b >> 32) : (uint32_t)b;
        } else {
            const float w32 = d_z128_W32[i];
            v = __float_as_uint(ix < 128 ? -w32 : w32);
        }
        t.blk[ix][wd] = v;
    }
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        s.W32[i] = d_z128_W32[i];
        s.Y32[i] = d_z128_Y32[i];
        s.DY32[i] = d_z128_DY32[i];
        s.Wd[i] = d_z128_W[i];
        s.Y[i] = d_z128_Y[i];
    }
}

// RN(j w) for j < 2^24 and a 53-bit significand m (mlo, mhi: m << 11) in
// 32-bit integer arithmetic, returned as binary64 bits with eh's sign: the
// 77-bit product of j normalized (its top bit at bit 31) and m << 11 has its
// top bit at bit 95 or 94; its high 64 bits, shifted left when bit 95 is clear
// and with a sticky bit for the 32 bits below, round to 53 bits by adding
// 2^10 - 1 plus the last kept bit; the carry of a round-up into 2^53 moves
// into the exponent field.  j = 0 gives the signed zero.
__device__ __forceinline__ uint64_t int_mul_jw(uint32_t j, uint32_t mlo, uint32_t mhi, uint32_t eh) {
    const uint32_t s = __clz(j);
    const uint32_t jn = __funnelshift_l(0u, j, s);   // j << s, 0 for s = 32
    const uint64_t A = (uint64_t)jn * mlo;
    const uint64_t Bp = (uint64_t)jn * mhi;
    uint64_t H = Bp + (A >> 32);                      // product bits 32..95
    const uint32_t t = (uint32_t)(H >> 63);
    H <<= (1u - t);
    H |= (uint32_t)A != 0u ? 1u : 0u;                 // sticky
    const uint64_t M = (H + 0x3FFu + ((H >> 11) & 1u)) >> 11;   // in [2^52, 2^53]
    const uint32_t hi = (uint32_t)(M >> 32) + eh + ((t - s) << 20);
    return j ? ((uint64_t)hi << 32 | (uint32_t)M) : ((uint64_t)(eh & 0x80000000u) << 32);
}

// x = sign RN(j w[i]) for the draw w, as binary64 bits: one binary64 fma
// fma(1 + j 2^-52, b, -b) with the signed b = +-2^52 w[i] (exact before its one
// rounding; 1 + j 2^-52 is built from j's bits), or (kInt) int_mul_jw with the
// significand, exponent and sign read off b (E(b) = E(w[i]) + 52).
template <bool kInt, bool C>
__device__ __forceinline__ uint64_t x_of(const unsigned char* tab, uint32_t w, uint32_t copy8) {
    const uint2 e = *(const uint2*)(tab + entry_off<C>(w, copy8));   // block ix, copy
    const uint32_t j = w >> 8;
    if constexpr (kInt) {
        const uint32_t mhi = __funnelshift_l(e.x, (e.y & 0xFFFFFu) | 0x100000u, 11);
        const uint32_t eh = (e.y & 0xFFF00000u) - (22u << 20);   // sign | (E(w[i]) + 30) << 20
        return int_mul_jw(j, e.x << 11, mhi, eh);
    } else {
        const double b = __hiloint2double((int)e.y, (int)e.x);
        const double x = __fma_rn(__hiloint2double(0x3FF00000, (int)j), b, -b);
        return (uint64_t)__double_as_longlong(x) | ((uint64_t)(e.y & 0x80000000u) << 32);
    }
}

// The binary32 value RN32(j w32[i]) with the entry's sign, for the draw w
// (binary32 and bfloat16 output; j < 2^24 converts exactly).
template <bool C>
__device__ __forceinline__ uint32_t x32_of(const unsigned char* tab, uint32_t w, uint32_t copy4) {
    const float e = *(const float*)(tab + entry_off<C>(w, copy4));   // block ix, copy
    return __float_as_uint(__fmul_rn((float)(w >> 8), e));
}

// Write row r of the warp's batch: lane c takes slot c (binary64: kInt selects
// the integer product).  bfloat16 is rounded from the binary32 value.
template <int PRNG, int DT, bool kInt, class W>
__device__ __forceinline__ void write_row(const W& ws, const unsigned char* tb, int r, int lane, uint32_t lane_bit,
                                          uint32_t lt_mask, uint32_t copy) {
    using GT = Gen<PRNG>;
    const uint4 inf = ws.info[r];
    const uint32_t w = ws.stage[r * W::RS + GT::SW * lane + GT::SW - 1];
    const uint32_t e = __popc(~inf.z & lt_mask);
    const uint64_t base = (uint64_t)inf.x | (uint64_t)inf.y << 32;
    if constexpr (DT == ZIG_F64) {
        const uint64_t v = x_of<kInt, kCompactTab<PRNG>>(tb, w, copy);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.eq.u32 p, %2, 0;\n\t@p st.global.cs.b64 [%0], %1;\n\t}" ::"l"(base + 8ull * e),
            "l"(v), "r"(inf.z & lane_bit));
    } else if constexpr (DT == ZIG_F32) {
        const uint32_t v = x32_of<kCompactTab<PRNG>>(tb, w, copy);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.eq.u32 p, %2, 0;\n\t@p st.global.cs.b32 [%0], %1;\n\t}" ::"l"(base + 4ull * e),
            "r"(v), "r"(inf.z & lane_bit));
    } else {
        const uint16_t v = f32_to_bf16_bits(__uint_as_float(x32_of<kCompactTab<PRNG>>(tb, w, copy)));
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.eq.u32 p, %2, 0;\n\t@p st.global.cs.b16 [%0], %1;\n\t}" ::"l"(base + 2ull * e),
            "h"(v), "r"(inf.z & lane_bit));
    }
}

// Mutation rows r0 .. r0 + 7 (binary32 population x, row pointer and sigma word
// in the row's info): every lane loads its eight elements of x first, so that the
// loads overlap, then stores x + sigma z (fmaf, one rounding) or z.  Each element
// is read once, by the thread that then writes it; an accepted tail's element is
// left to its queue entry, which reads and writes it once its value is known.
template <int PRNG, class W>
__device__ __forceinline__ void mutate_rows8(const W& ws, const unsigned char* tb, int r0, int lane,
                                             uint32_t lane_bit, uint32_t lt_mask, uint32_t copy) {
    using GT = Gen<PRNG>;
    float* px[8];
    float xv[8];
    uint32_t sg[8];
    bool st[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint4 inf = ws.info[r0 + k];
        px[k] = (float*)((uint64_t)inf.x | (uint64_t)inf.y << 32) + __popc(~inf.z & lt_mask);
        sg[k] = inf.w;
        st[k] = !((inf.z | ws.tails[r0 + k]) & lane_bit);   // a kept slot that is no queued tail
        xv[k] = (st[k] && sg[k] != kGenerate) ? __ldcs(px[k]) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float z = __uint_as_float(x32_of<kCompactTab<PRNG>>(tb, ws.stage[(r0 + k) * W::RS + GT::SW * lane + GT::SW - 1], copy));
        if (st[k]) __stcs(px[k], sg[k] == kGenerate ? z : fmaf(__uint_as_float(sg[k]), z, xv[k]));
    }
}

// The values of queued accepted tails, 32 at a time (all 32 lanes call this):
// binary64 x, or (binary32, bfloat16) RN32(x) with the sign, rounded once more
// to bfloat16 for that output.  An entry's address carries the sign in bit 0.
template <int DT, int MUT, class W>
__device__ __forceinline__ void drain_tails(W& ws, int lane) {
    const uint32_t n = ws.tq_n;
    for (uint32_t b = 0; b < n; b += 32) {
        if (b + lane < n) {
            const uint64_t ad = ws.tq_addr[b + lane];
            const double x = z128_tail_value(ws.tq_m1[b + lane]);
            if constexpr (MUT != 0) {   // binary32 into the population: x = z, or x += sigma z
                const float z = __uint_as_float(__float_as_uint(__double2float_rn(x)) | (uint32_t)(ad & 1u) << 31);
                float* const px = (float*)(ad & ~1ull);
                const uint32_t sg = ws.tq_sig[b + lane];
                __stcs(px, sg == kGenerate ? z : fmaf(__uint_as_float(sg), z, __ldcs(px)));
            } else if constexpr (DT == ZIG_F64) {
                __stcs((unsigned long long*)(ad & ~1ull),
                       (unsigned long long)__double_as_longlong(x) | (unsigned long long)(ad & 1u) << 63);
            } else {
                const uint32_t v = __float_as_uint(__double2float_rn(x)) | (uint32_t)(ad & 1u) << 31;
                if constexpr (DT == ZIG_F32) __stcs((unsigned int*)(ad & ~1ull), v);
                else __stcs((unsigned short*)(ad & ~1ull), f32_to_bf16_bits(__uint_as_float(v)));
            }
        }
    }
    __syncwarp();
    if (lane == 0) ws.tq_n = 0;
    __syncwarp();
}

// MUT: 0 generation; 1 mutation of a P x L population (row p seeded mut_seed + p,
// or continuing state[p]); 2 a batch of mutation and generation requests.
template <int PRNG, int DT, int NDF, int MUT = 0>
__global__ void __launch_bounds__(max_threads(PRNG), 1) z128f_kernel(GenArgs a) {
    using GT = Gen<PRNG>;
    using G = typename GT::G;
    using W = Warp<PRNG, DT, MUT>;
    using OutT = typename OutOf<DT>::T;
    constexpr int kU = GT::kU, SW = GT::SW, B = W::B;
    static_assert(NDF >= 2 && NDF <= 4, "rows per 4 with the binary64 fma");
    static_assert(DT == ZIG_F64 || NDF == 4, "binary32 and bfloat16 rows have one product");
    static_assert(MUT == 0 || DT == ZIG_F32, "populations are binary32");
    extern __shared__ __align__(16) unsigned char zf_dsm[];
    constexpr bool C = kCompactTab<PRNG>;
    TabT<C>& tab = *(TabT<C>*)zf_dsm;
    SlowTab& slow = *(SlowTab*)(zf_dsm + sizeof(TabT<C>));
    tab_load<DT, C>(tab, slow);
    __syncthreads();
    const unsigned char* const tb = zf_dsm;

    const int lane = threadIdx.x & 31;
    const uint32_t lane_bit = 1u << lane, lt_mask = lane_bit - 1u;
    const int wib = threadIdx.x >> 5;
    const int n_warps = blockDim.x >> 5;
    W& ws = *(W*)(zf_dsm + head_bytes<C>() + (size_t)wib * warp_bytes<PRNG, DT, MUT>());
    uint32_t* const row = ws.stage + lane * W::RS;
    // this lane's copy of the fast entry, b (binary64) or w32, and of K
    const uint32_t copy = C ? (DT == ZIG_F64 ? (uint32_t)(lane & 7) << 3 : (uint32_t)(lane & 15) << 2)
                            : (DT == ZIG_F64 ? (uint32_t)(lane & 15) << 3 : (uint32_t)lane << 2);
    const uint32_t kcopy = C ? 0x40u + ((uint32_t)(lane & 15) << 2) : 0x80u + ((uint32_t)lane << 2);

    if (lane == 0) ws.tq_n = 0;
    __syncwarp();
    if (MUT == 0 && a.out == nullptr) {   // only legal when every length is zero
        if (a.lengths && a.totals[1] != 0 && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.err, kErrNullOutput);
        return;
    }
    const uint64_t n_units = units_total(a);
    const uint64_t n_groups = (n_units + 31) >> 5;
    const uint64_t warp_id = (uint64_t)blockIdx.x * n_warps + wib;
    const uint64_t warp_stride = (uint64_t)gridDim.x * n_warps;
    OutT* const out = (OutT*)a.out;

    for (uint64_t grp = warp_id; grp < n_groups; grp += warp_stride) {
        const uint64_t u = grp * 32 + lane;
        uint64_t rem = 0;
        OutT* dst = out;
        G g;
        g.seed(0);
        zig_stream_state* srec = nullptr;   // the record to advance when the unit ends
        uint32_t sig = 0;                    // mutation: the row's sigma bits, or kGenerate
        if (u < n_units) {
            bool ok = true;
            if constexpr (MUT == 2) {
                // the request holding unit u (the last with ustart <= u); a row has
                // units of 2^10 outputs from 2^32-draw windows, or one unit continuing
                // its record
                uint32_t lo = 0, hi = a.n_req;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (a.reqs[mid].ustart <= u) lo = mid; else hi = mid;
                }
                const MutDesc& r = a.reqs[lo];
                const uint64_t ur = u - r.ustart, p = ur / r.upr, qd = ur - p * r.upr;
                if (r.state) {
                    if (state_load<PRNG>(r.state + p, g, a.err, ok)) srec = r.state + p;
                } else {
                    g.seed(r.seed + p);
                    if (qd) g.jump(qd * kChunkDraws, &d_jump);
                }
                const uint64_t t0 = qd << 10;
                if (ok) {
                    rem = r.state ? r.L : umin64(r.L - t0, 1024);
                    dst = (OutT*)(r.x + p * r.L + t0);
                }
                sig = r.kind == ZIG_REQ_GENERATE ? kGenerate : __float_as_uint(r.sigma);
            } else {
                uint64_t s, q, off, n;
                unit_info(a, u, s, q, off, n);
                if (MUT == 1 && a.state == nullptr) {   // mutation: row s seeded mut_seed + s
                    g.seed(a.mut_seed + s);
                    if (q) g.jump(q * kChunkDraws, &d_jump);
                } else {
                    srec = unit_gen<PRNG>(a, s, q, g, ok);
                }
                if (ok) {
                    rem = n;
                    dst = out + off;
                }
                sig = __float_as_uint(a.sigma);
            }
        }
        const bool check_chunk = srec == nullptr && a.chunk_log2 != 0 && rem != 0;
        uint64_t draws = 0;   // raw steps used by this unit (chunk-overflow check)

        while (__any_sync(kFull, rem > 0)) {
            // ---- A: B draws per lane, lockstep; nf marks the slow candidates ----
            uint32_t nfr = 0;   // draw d's fast-test bit at B - 1 - d (built by doubling)
            const uint64_t sb = first_state_of(g);
            auto step = [&](auto dc) {
                constexpr int d = decltype(dc)::value;
                uint32_t w;
                if constexpr (PRNG == ZIG_LCG48) {
                    w = GT::template draw_at<d>(sb);
                    row[d] = w;
                } else {
                    GT::draw(g, row + SW * d, w);
                }
                const uint32_t K = *(const uint32_t*)(tb + entry_off<C>(w, kcopy));
                // nfr = 2 nfr + (w >= K): the carry of w - K is 1 when nothing is borrowed
                asm("{\n\t.reg .u32 t;\n\tsub.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
                    : "=r"(nfr) : "r"(w), "r"(K), "r"(nfr));
            };
            unroll<B>(step);
            const uint32_t nf = __brev(nfr) >> (32 - B);
            if constexpr (PRNG == ZIG_LCG48) GT::template skip<B>(g);
            // ---- B: each lane decides its own slow candidates, in draw order ----
            // Walking its nf bits, a lane meets each slow draw that an earlier one
            // did not consume; that draw consumes the next kU (wedge) or 2 kU (tail)
            // draws as its uniforms, taken past the batch now if need be.  The wedge
            // and tail tests run first in binary32 with proven margins (binary64 only
            // inside them).  A rejected candidate goes to the drops; an accepted
            // tail's m1 goes to the words of its first uniform for the value pass.
            uint32_t du = 0, Dr = 0, L = 0, T = 0;   // consumed uniforms, rejected, accepted tails, tails
            int ne = 0;
            for (uint32_t m = rem > 0 ? nf : 0u; m;) {
                const int p = __ffs(m) - 1;
                const uint32_t w = row[SW * p + SW - 1];
                const bool tail = (w & 0x7Fu) == 0x7Fu;
                const int need = tail ? 2 * kU : kU;
                // bits past 31 drop out: slots 32.. hold only uniforms
                const uint32_t cons = p < 31 ? ((1u << need) - 1u) << (p + 1) : 0u;
                du |= cons;
                m &= ~(cons | (1u << p));   // this candidate and the draws it consumes
                while (B + ne <= p + need) {   // uniforms past the batch (rare)
                    uint32_t wx;
                    GT::draw(g, row + SW * (B + ne), wx);
                    ++ne;
                }
                if (tail) {   // tested after the wedges (a tail is 5 % of candidates)
                    T |= 1u << p;
                    continue;
                }
                const uint64_t m1 = GT::m53(row, p + 1, sb);
                int f = z128_wedge_filter(slow, w & 0x7Fu, w >> 8, m1);
                if (f < 0) f = z128_wedge_exact(slow, w & 0x7Fu, w >> 8, m1) ? 1 : 0;
                Dr |= (f == 0 ? 1u : 0u) << p;
            }
            for (uint32_t m = T; m; m &= m - 1u) {
                const int p = __ffs(m) - 1;
                const uint64_t m1 = GT::m53(row, p + 1, sb);
                const uint64_t m2 = GT::m53(row, p + 1 + kU, sb);
                int ft = z128_tail_filter(m1, m2);
                if (ft < 0) ft = z128_tail_exact(m1, m2) ? 1 : 0;
                if (ft == 0) {
                    Dr |= 1u << p;
                } else {   // m1 goes to the first uniform's words (a dropped slot)
                    row[SW * (p + 1)] = (uint32_t)m1;
                    row[SW * (p + 1) + 1] = (uint32_t)(m1 >> 32);
                    L |= 1u << p;
                }
            }
            // ---- C: drops, the unit's end, then the rows ----
            const int n = B + ne;   // slots drawn
            uint32_t D = du | Dr | (n >= 32 ? 0u : (~0u << n));
            const int kept = 32 - __popc(D);
            int k_out = kept;
            if ((uint64_t)kept >= rem) {   // the unit ends in this batch: keep rem outputs
                k_out = (int)rem;
                uint32_t keepm = ~D;
                for (int m = 0; m < k_out; ++m) keepm &= keepm - 1u;   // the slots past the rem-th kept one
                D |= keepm;
                if ((check_chunk || srec) && k_out > 0) {
                    // the draws up to the last output and its uniforms
                    const int c = 31 - __clz(~D);   // slot of the last output
                    int used = c + 1;
                    if ((nf >> c) & 1u) {   // a slow candidate: its uniforms follow it
                        const uint32_t wc = row[SW * c + SW - 1];
                        used += (wc & 0x7Fu) == 0x7Fu ? 2 * kU : kU;
                    }
                    draws += (uint64_t)used;
                    // the stream's record: the generator after those draws (the
                    // batch drew n from the state sb)
                    if (srec) {
                        G t = g;
                        if constexpr (PRNG == ZIG_LCG48 || PRNG == ZIG_SPLITMIX64) {
                            t.s = sb;
                            t.jump((uint64_t)used, &d_jump);
                        } else {
                            for (int k = used; k < n; ++k) t.unstep();
                        }
                        state_store(srec, t, false, 0.0);
                    }
                }
            } else if (check_chunk) {
                draws += (uint64_t)n;
            }
            ws.info[lane] = make_uint4((uint32_t)(uintptr_t)dst, (uint32_t)((uintptr_t)dst >> 32), D, sig);
            if constexpr (MUT != 0) ws.tails[lane] = L & ~D;
            __syncwarp();
            if constexpr (MUT != 0) {
#pragma unroll 1
                for (int r = 0; r < 32; r += 8) mutate_rows8<PRNG>(ws, tb, r, lane, lane_bit, lt_mask, copy);
            } else {
                // products q = 0..3 of every two steps: the binary64 fma for q < NDF
#pragma unroll 4
                for (int r = 0; r < 32; r += 4) {
                    write_row<PRNG, DT, (0 >= NDF)>(ws, tb, r + 0, lane, lane_bit, lt_mask, copy);
                    write_row<PRNG, DT, (1 >= NDF)>(ws, tb, r + 1, lane, lane_bit, lt_mask, copy);
                    write_row<PRNG, DT, (2 >= NDF)>(ws, tb, r + 2, lane, lane_bit, lt_mask, copy);
                    write_row<PRNG, DT, (3 >= NDF)>(ws, tb, r + 3, lane, lane_bit, lt_mask, copy);
                }
            }
            // accepted tails join the queue (one per lane per round), evaluated 32 at a
            // time (drained first when a round would overfill it)
            uint32_t Lk = L & ~D;
            for (;;) {
                const uint32_t bal = __ballot_sync(kFull, Lk != 0);
                if (bal == 0) break;
                if (ws.tq_n + __popc(bal) > 32u) drain_tails<DT, MUT>(ws, lane);
                if (Lk) {
                    const int p = __ffs(Lk) - 1;
                    Lk &= Lk - 1u;
                    const uint32_t idx = ws.tq_n + __popc(bal & lt_mask);
                    const uint32_t w = row[SW * p + SW - 1];
                    ws.tq_addr[idx] = (uint64_t)(uintptr_t)(dst + __popc(~D & ((1u << p) - 1u))) | ((~w >> 7) & 1u);
                    ws.tq_m1[idx] = (uint64_t)row[SW * (p + 1)] | (uint64_t)row[SW * (p + 1) + 1] << 32;
                    if constexpr (MUT != 0) ws.tq_sig[idx] = sig;
                }
                __syncwarp();
                if (lane == 0) ws.tq_n += __popc(bal);
                __syncwarp();
            }
            dst += k_out;
            rem -= (uint64_t)k_out;
            __syncwarp();
        }
        if (check_chunk && draws > kChunkDraws) atomicOr(a.err, kErrChunkOverflow);
    }
    drain_tails<DT, MUT>(ws, lane);
}

}  // namespace zf
