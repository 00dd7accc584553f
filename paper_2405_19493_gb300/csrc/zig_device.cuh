// Device-side building blocks of libzig_gb300: uniform generators with state in
// registers (seeding, stepping, jumps, one step back, stream records), integer
// roundings to binary32 and bfloat16, and the warp staging of the polar kernel
// that turns per-thread streams into coalesced stores.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace zig {

constexpr uint64_t kMask48 = (1ull << 48) - 1;
constexpr uint64_t kLcgA = 0x5DEECE66Dull;           // java.util.Random multiplier
constexpr uint64_t kLcgC = 0xBull;                   // java.util.Random increment
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;   // SplitMix64 golden gamma
constexpr uint64_t kLxmM = 0xD1342543DE82EF95ull;    // L64X128Mix LCG multiplier
constexpr uint64_t kLeaM = 0xDABA0B6EB09322E3ull;    // Lea's 64-bit mix constant
constexpr unsigned kFull = 0xFFFFFFFFu;

// Error bits latched in a device error word (the caller's, or the device's own).
constexpr unsigned kErrChunkOverflow = 1u;
constexpr unsigned kErrNullOutput = 4u;   // variable lengths summed > 0 with out == NULL
constexpr unsigned kErrLengthSum = 8u;    // variable lengths summed to 2^40 or more
constexpr unsigned kErrStateKind = 16u;   // a stream record seeded for another generator

// The inverse of an odd multiplier modulo 2^64 (Newton's iteration x <- x (2 - m x),
// which doubles the number of correct low bits; m x = 1 mod 8 holds for x = m).
__host__ __device__ constexpr uint64_t inverse_mod_2_64(uint64_t m) {
    uint64_t x = m;
    for (int k = 0; k < 5; ++k) x *= 2 - m * x;
    return x;
}
constexpr uint64_t kLxmMinv = inverse_mod_2_64(kLxmM);
static_assert(kLxmM * kLxmMinv == 1, "L64X128Mix multiplier inverse");

// Jump-ahead tables for 2^b raw steps, b = 0..63 (filled on the host at init).
struct JumpTab {
    uint64_t lcg48_A[64], lcg48_C[64];   // s -> (A s + C) mod 2^48
    uint64_t lxm_A[64], lxm_G[64];       // LXM LCG: s -> A s + a G (mod 2^64)
    uint64_t xoro[64][256];              // LXM's xoroshiro128 T^(2^b): column c at [2c], [2c+1]
    uint64_t xpp[64][256];               // Xoroshiro128PlusPlus's engine, same layout
};

// ---------------------------------------------------------------------------
// mixers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t mix32(uint64_t z) {
    z = (z ^ (z >> 33)) * 0x62A9D9ED799705F5ull;
    return (uint32_t)(((z ^ (z >> 28)) * 0xCB24D0A5C88C35B3ull) >> 32);
}

__device__ __forceinline__ uint64_t mix_lea64(uint64_t z) {
    z = (z ^ (z >> 32)) * kLeaM;
    z = (z ^ (z >> 32)) * kLeaM;
    return z ^ (z >> 32);
}

__device__ __forceinline__ uint64_t rotl64(uint64_t x, int k) {
    return (x << k) | (x >> (64 - k));
}
__device__ __forceinline__ uint64_t rotr64(uint64_t x, int k) {
    return (x >> k) | (x << (64 - k));
}

// ---------------------------------------------------------------------------
// generators: one per thread, state in registers
//   next_u32 = nextInt, next_u64 = nextLong, next_m53 = the 53-bit integer of nextDouble
// ---------------------------------------------------------------------------

// load/save: the state words of a stream record (zig_stream_state.gen), in the
// order the C header states for each generator.
struct GenLcg48 {
    uint64_t s;
    __device__ __forceinline__ void seed(uint64_t x) { s = (x ^ kLcgA) & kMask48; }
    __device__ __forceinline__ void load(const uint64_t* w) { s = w[0] & kMask48; }
    __device__ __forceinline__ void save(uint64_t* w) const { w[0] = s; }
    __device__ __forceinline__ uint32_t step(int bits) {
        s = (s * kLcgA + kLcgC) & kMask48;
        return (uint32_t)(s >> (48 - bits));
    }
    __device__ __forceinline__ uint32_t next_u32() { return step(32); }
    __device__ __forceinline__ uint64_t next_u64() {
        uint64_t hi = step(32);
        int32_t lo = (int32_t)step(32);
        return (hi << 32) + (uint64_t)(int64_t)lo;
    }
    __device__ __forceinline__ uint64_t next_m53() {
        uint64_t hi = step(26);
        uint64_t lo = step(27);
        return (hi << 27) + lo;
    }
    __device__ __forceinline__ void jump(uint64_t n, const JumpTab* jt) {
        while (n) {
            int b = __ffsll((long long)n) - 1;
            s = (jt->lcg48_A[b] * s + jt->lcg48_C[b]) & kMask48;
            n &= n - 1;
        }
    }
    // Deferred doubles: snap() returns a record of the next nextDouble call and
    // moves the state past it (nextDouble = 2 steps); m53_of() rebuilds that
    // double's 53-bit integer later from the record alone.  (The kOut choice
    // only matters for L64X128Mix.)
    static constexpr uint64_t kA2 = (kLcgA * kLcgA) & kMask48;
    static constexpr uint64_t kC2 = (kLcgA * kLcgC + kLcgC) & kMask48;
    static constexpr uint32_t kStepsPerDouble = 2;
    template <bool kOut = false>
    __device__ __forceinline__ uint64_t snap() {
        const uint64_t b = s;
        s = (kA2 * s + kC2) & kMask48;
        return b;
    }
    template <bool kOut = false>
    static __device__ __forceinline__ uint64_t m53_of(uint64_t b) {
        uint64_t t = (b * kLcgA + kLcgC) & kMask48;
        const uint64_t hi = t >> 22;   // next(26)
        t = (t * kLcgA + kLcgC) & kMask48;
        const uint64_t lo = t >> 21;   // next(27)
        return (hi << 27) + lo;
    }
};

struct GenSplitMix64 {
    uint64_t s;
    __device__ __forceinline__ void seed(uint64_t x) { s = x; }
    __device__ __forceinline__ void load(const uint64_t* w) { s = w[0]; }
    __device__ __forceinline__ void save(uint64_t* w) const { w[0] = s; }
    __device__ __forceinline__ uint32_t next_u32() { s += kGamma; return mix32(s); }
    __device__ __forceinline__ uint64_t next_u64() { s += kGamma; return mix64(s); }
    __device__ __forceinline__ uint64_t next_m53() { s += kGamma; return mix64(s) >> 11; }
    __device__ __forceinline__ void jump(uint64_t n, const JumpTab*) { s += n * kGamma; }
    static constexpr uint32_t kStepsPerDouble = 1;
    // the record of the next nextDouble is the state of its step
    template <bool kOut = false>
    __device__ __forceinline__ uint64_t snap() { s += kGamma; return s; }
    template <bool kOut = false>
    static __device__ __forceinline__ uint64_t m53_of(uint64_t b) { return mix64(b) >> 11; }
};

struct GenL64X128Mix {
    uint64_t a, s, x0, x1;
    __device__ __forceinline__ void seed(uint64_t x) {
        // four consecutive SplitMix64 outputs of a generator seeded with x
        uint64_t t = x;
        t += kGamma; a = mix64(t) | 1;
        t += kGamma; s = mix64(t);
        t += kGamma; x0 = mix64(t);
        t += kGamma; x1 = mix64(t);
        if ((x0 | x1) == 0) x1 = kGamma;
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        a = w[0] | 1;
        s = w[1];
        x0 = w[2];
        x1 = w[3];
    }
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = a;
        w[1] = s;
        w[2] = x0;
        w[3] = x1;
    }
    // one raw step back (the inverse of advance): the LCG by the multiplier's
    // inverse; the xoroshiro128 step by undoing x1 = rotl(t, 37), then
    // rotl(x0, 24) = x0' ^ t ^ (t << 16), then t = x1 ^ x0
    __device__ __forceinline__ void unstep() {
        s = kLxmMinv * (s - a);
        const uint64_t t = rotr64(x1, 37);
        x0 = rotr64(x0 ^ t ^ (t << 16), 24);
        x1 = t ^ x0;
    }
    __device__ __forceinline__ uint64_t next_u64() {
        uint64_t result = mix_lea64(s + x0);
        s = kLxmM * s + a;
        uint64_t q1 = x1 ^ x0;
        x0 = rotl64(x0, 24) ^ q1 ^ (q1 << 16);
        x1 = rotl64(q1, 37);
        return result;
    }
    __device__ __forceinline__ uint32_t next_u32() { return (uint32_t)(next_u64() >> 32); }
    __device__ __forceinline__ uint64_t next_m53() { return next_u64() >> 11; }
    __device__ __forceinline__ void advance() {
        s = kLxmM * s + a;
        uint64_t q1 = x1 ^ x0;
        x0 = rotl64(x0, 24) ^ q1 ^ (q1 << 16);
        x1 = rotl64(q1, 37);
    }
    static constexpr uint32_t kStepsPerDouble = 1;
    // the record of the next nextDouble is that step's mix input s + x0, or
    // (kOut) its nextLong output itself, for a caller that computes it anyway
    template <bool kOut = false>
    __device__ __forceinline__ uint64_t snap() {
        if constexpr (kOut) {
            return next_u64();
        } else {
            const uint64_t b = s + x0;
            advance();
            return b;
        }
    }
    template <bool kOut = false>
    static __device__ __forceinline__ uint64_t m53_of(uint64_t b) {
        if constexpr (kOut) return b >> 11;
        else return mix_lea64(b) >> 11;
    }
    __device__ void jump(uint64_t n, const JumpTab* jt) {
        while (n) {
            int b = __ffsll((long long)n) - 1;
            s = jt->lxm_A[b] * s + a * jt->lxm_G[b];
            const uint64_t* m = jt->xoro[b];
            uint64_t r0 = 0, r1 = 0;
#pragma unroll 8
            for (int c = 0; c < 64; ++c) {
                uint64_t mask = 0ull - ((x0 >> c) & 1ull);
                r0 ^= m[2 * c] & mask;
                r1 ^= m[2 * c + 1] & mask;
            }
#pragma unroll 8
            for (int c = 0; c < 64; ++c) {
                uint64_t mask = 0ull - ((x1 >> c) & 1ull);
                r0 ^= m[128 + 2 * c] & mask;
                r1 ^= m[128 + 2 * c + 1] & mask;
            }
            x0 = r0;
            x1 = r1;
            n &= n - 1;
        }
    }
};

// Xoroshiro128PlusPlus, an XBG generator: nextLong = rotl(x0 + x1, 17) + x0,
// then the xoroshiro128 engine with constants (49, 21, 28).  Seeded (a
// reading) from two consecutive SplitMix64 outputs.  A deferred wedge's
// record is its nextLong output itself (the scrambler is cheap).
struct GenXoroshiro128PP {
    uint64_t x0, x1;
    __device__ __forceinline__ void seed(uint64_t x) {
        uint64_t t = x;
        t += kGamma; x0 = mix64(t);
        t += kGamma; x1 = mix64(t);
        if ((x0 | x1) == 0) x1 = kGamma;
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        x0 = w[0];
        x1 = w[1];
    }
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = x0;
        w[1] = x1;
    }
    // one raw step back: undo x1 = rotl(t, 28), then rotl(x0, 49) = x0' ^ t ^ (t << 21),
    // then t = x1 ^ x0
    __device__ __forceinline__ void unstep() {
        const uint64_t t = rotr64(x1, 28);
        x0 = rotr64(x0 ^ t ^ (t << 21), 49);
        x1 = t ^ x0;
    }
    __device__ __forceinline__ uint64_t next_u64() {
        const uint64_t s0 = x0;
        uint64_t s1 = x1;
        const uint64_t r = rotl64(s0 + s1, 17) + s0;
        s1 ^= s0;
        x0 = rotl64(s0, 49) ^ s1 ^ (s1 << 21);
        x1 = rotl64(s1, 28);
        return r;
    }
    __device__ __forceinline__ uint32_t next_u32() { return (uint32_t)(next_u64() >> 32); }
    __device__ __forceinline__ uint64_t next_m53() { return next_u64() >> 11; }
    static constexpr uint32_t kStepsPerDouble = 1;
    template <bool kOut = false>
    __device__ __forceinline__ uint64_t snap() { return next_u64(); }
    template <bool kOut = false>
    static __device__ __forceinline__ uint64_t m53_of(uint64_t r) { return r >> 11; }
    __device__ void jump(uint64_t n, const JumpTab* jt) {
        while (n) {
            const int b = __ffsll((long long)n) - 1;
            const uint64_t* m = jt->xpp[b];
            uint64_t r0 = 0, r1 = 0;
#pragma unroll 8
            for (int c = 0; c < 64; ++c) {
                const uint64_t mask = 0ull - ((x0 >> c) & 1ull);
                r0 ^= m[2 * c] & mask;
                r1 ^= m[2 * c + 1] & mask;
            }
#pragma unroll 8
            for (int c = 0; c < 64; ++c) {
                const uint64_t mask = 0ull - ((x1 >> c) & 1ull);
                r0 ^= m[128 + 2 * c] & mask;
                r1 ^= m[128 + 2 * c + 1] & mask;
            }
            x0 = r0;
            x1 = r1;
            n &= n - 1;
        }
    }
};

template <int PRNG> struct GenOf;
template <> struct GenOf<0> { using T = GenLcg48; };
template <> struct GenOf<1> { using T = GenSplitMix64; };
template <> struct GenOf<2> { using T = GenL64X128Mix; };
template <> struct GenOf<3> { using T = GenXoroshiro128PP; };

__device__ __forceinline__ double m53_to_double(uint64_t m) {
    return (double)m * 0x1p-53;   // exact: m < 2^53
}

// RN-even binary64 -> bfloat16 bits, for zero and for results in bfloat16's
// normal range, in 32-bit integer operations on the two words: the exponent and
// top 7 fraction bits, rounded on the 45 bits below them, then rebiased by
// 1023 - 127 (a rounding carry moves into the exponent first).
__device__ __forceinline__ uint16_t f64_to_bf16_bits(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t mag_hi = hi & 0x7FFFFFFFu;
    uint32_t q = mag_hi >> 13;
    const uint32_t r = hi & 0x1FFFu;   // with lo, the 45 bits below q
    const bool above = r > 0x1000u || (r == 0x1000u && lo != 0u);
    const bool tie = r == 0x1000u && lo == 0u;
    q += (above || (tie && (q & 1u))) ? 1u : 0u;
    const uint32_t sign = (hi >> 16) & 0x8000u;
    return (uint16_t)((mag_hi | lo) == 0u ? sign : (sign | (q - (896u << 7))));
}

// RN-even binary64 -> binary32 bits, for zero and for magnitudes in [2^-126, 2^128),
// in 32-bit integer operations: the exponent and top 23 fraction bits (a funnel
// shift of the two words, exact modulo 2^32 once rebiased by 1023 - 127), rounded
// on the 29 bits below them (a carry moves into the exponent).
__device__ __forceinline__ uint32_t f64_to_f32_bits(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t sign = hi & 0x80000000u;
    uint32_t q = __funnelshift_l(lo, hi, 3) - (896u << 23);
    const uint32_t rem = lo & 0x1FFFFFFFu;
    q += (rem > 0x10000000u || (rem == 0x10000000u && (q & 1u))) ? 1u : 0u;
    return ((hi & 0x7FFFFFFFu) | lo) == 0u ? sign : (sign | q);
}

// RN-even binary32 -> bfloat16 bits (finite inputs).
__device__ __forceinline__ uint16_t f32_to_bf16_bits(float x) {
    uint32_t b = __float_as_uint(x);
    uint32_t lsb = (b >> 16) & 1u;
    b += 0x7FFFu + lsb;
    return (uint16_t)(b >> 16);
}

// ---------------------------------------------------------------------------
// warp staging: 32 rows (one per lane's unit) x 16 columns, swizzled so that
// both the per-lane column writes and the per-row reads are bank-conflict free
// ---------------------------------------------------------------------------

template <typename T> struct Stage;
template <> struct Stage<double> {
    static __device__ __forceinline__ int sw(int row) { return row & 15; }
};
template <> struct Stage<float> {
    static __device__ __forceinline__ int sw(int row) { return (row >> 1) & 15; }
};
template <> struct Stage<uint16_t> {
    static __device__ __forceinline__ int sw(int row) { return ((row >> 2) & 7) << 1; }
};

constexpr int kStageCols = 16;

template <typename T>
__device__ __forceinline__ int stage_idx(int row, int col) {
    return row * kStageCols + (col ^ Stage<T>::sw(row));
}

// Write the warp's staged rows: row r has cnt_r valid columns going to dst_r.
// Two rows per step (16 lanes each).  All 32 lanes must call this.
template <typename T>
__device__ __forceinline__ void stage_flush(const T* stage, T* my_dst, int my_cnt, int lane) {
    const int half = lane >> 4, c = lane & 15;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        int row = 2 * k + half;
        T* dst = (T*)__shfl_sync(kFull, (unsigned long long)my_dst, row);
        int cnt = __shfl_sync(kFull, my_cnt, row);
        if (c < cnt) dst[c] = stage[stage_idx<T>(row, c)];
    }
}

}  // namespace zig
