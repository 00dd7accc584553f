// Modified ziggurat (McFarland's 256 slots, Sec. 2 "Java 17"), every output type:
// the batch layout of the 128-level kernel.  Included by zig_lib.cu after
// z128_batch.cuh.
//
// Each lane owns one unit with its generator in registers; a warp works on its
// 32 units in batches of 32 draws per lane.  A draw is one nextLong U (two raw
// steps for java.util.Random); a slot of the lane's row keeps it raw.
//  A. Every lane takes its 32 draws in lockstep, with no branch: the fast test
//     (slot j = U & 255 below 253) only sets a bit of the lane's mask nf.
//  B. Each lane walks its nf bits in draw order and runs the slow path of each
//     slow draw it meets (an overhang or the tail), taking that path's uniforms
//     from the slots after it (they are consumed, not candidates) and from its
//     generator once the row is used up.  The tests run in binary32 where proven
//     margins decide them, in binary64 otherwise (binary64 arithmetic runs on
//     the narrow FP64 pipe).  An accepted slow path leaves its slot r and
//     uniform in its slot; its binary64 value (an overhang's ox + odx U1, the
//     tail's x0 - ln(U1)/x0) is left to a per-warp queue that evaluates 32 at a
//     time.  A lane stops once its unit has all its outputs.  No lane waits for
//     another's slow path, and none stops early.
//  C. The warp writes its rows as the 128-level kernel does, lane c on slot c of
//     one row at a time: the output index of a kept slot is the number of kept
//     slots below it.  A fast slot's value XS[j] m (m = U >> 11) is rebuilt from
//     the raw draw with one binary64 fma; binary32 and bfloat16 outputs round
//     the binary64 value once, in integer arithmetic.  A slow slot's entry
//     joins the queue with its output address.
// A unit's outputs are its candidates' values in draw order: the sequence a
// one-variate-at-a-time loop produces (Sec. 2, Listing 2, repeated).
#pragma once

namespace zb {

// a slot's nextLong and nextDouble (53-bit integer) views; java.util.Random's
// slot keeps the two 32-bit outputs next(32) of its two steps (high, low word)
template <int PRNG>
__device__ __forceinline__ uint64_t slot_u64(uint64_t v) {
    if constexpr (PRNG == ZIG_LCG48) return (v & 0xFFFFFFFF00000000ull) + (uint64_t)(int64_t)(int32_t)(uint32_t)v;
    else return v;
}
template <int PRNG>
__device__ __forceinline__ uint64_t slot_m53(uint64_t v) {
    if constexpr (PRNG == ZIG_LCG48) return ((uint64_t)((uint32_t)(v >> 32) >> 6) << 27) + ((uint32_t)v >> 5);
    else return v >> 11;
}
// the generator's next slot
template <int PRNG, class G>
__device__ __forceinline__ uint64_t draw64(G& g) {
    if constexpr (PRNG == ZIG_LCG48) {
        const uint32_t w1 = g.step(32);
        const uint32_t w2 = g.step(32);
        return (uint64_t)w1 << 32 | w2;
    } else {
        return g.next_u64();
    }
}
template <int PRNG>
constexpr uint64_t kStepsPerSlot = PRNG == ZIG_LCG48 ? 2 : 1;

// the bits below bit p (all 32 for p >= 32)
__device__ __forceinline__ uint32_t lt_mask_of(int p) { return p >= 32 ? ~0u : (1u << p) - 1u; }

constexpr int kThreads = 640;   // 20 warps: shared memory holds no more
constexpr int kRS = 33;         // row stride in 8-byte words
constexpr int kSQ = 32;         // slow-value queue entries per warp

struct Tabs {
    double XN[256][16];   // -XS[j] 2^52, 16 copies (a half warp reads without conflicts)
    Z256Smem s;           // XS, THR, ALIAS for the slow path's slot choice
};
struct Warp {
    uint64_t stage[32 * kRS];   // row r, slot d at r kRS + d
    uint4 info[32];             // per row: output address (low, high), dropped slots
    uint64_t sq_addr[kSQ];      // accepted slow paths waiting for their value: output address | negative
    uint64_t sq_val[kSQ];       // and their slot and uniform, r << 53 | m1
    uint32_t sq_n;
};
__host__ __device__ constexpr size_t smem_bytes(int warps) {
    return ((sizeof(Tabs) + 15) & ~(size_t)15) + sizeof(Warp) * (size_t)warps;
}

// The draws of one slow path: the slots after its draw, then the generator
// (a copy, handed back with the count of draws afterwards).
template <int PRNG, class G>
struct Src {
    const uint64_t* row;
    int pos;     // the next draw's position in the batch
    int drawn;   // draws taken in the batch (the row holds the first 32)
    G g;
    __device__ __forceinline__ uint64_t next() {
        uint64_t v;
        if (pos < 32) {
            v = row[pos];
        } else {
            v = draw64<PRNG>(g);
            ++drawn;
        }
        ++pos;
        return v;
    }
};

// The tail step (Marsaglia's, beyond x0) on U = 1 - m 2^-53 in (0, 1]: x = -ln(U1)/x0,
// y = -ln(U2), accepted when 2y > x^2, which is ln U2 < -s^2/2 with s = x in exact
// arithmetic.  tail_filter decides it in binary32 when that clears a margin of
// 2^-14 (1 + s^2/2 + |ln U2|), far above the binary32 errors (correctly rounded
// conversions; the hardware log2 within 2^-22.6 absolute on [0.5, 2] and 2 ulp
// elsewhere: below 1e-5 relative here): 1 accept, 0 reject, -1 undecided.
// tail_exact is the binary64 definition.
__device__ __forceinline__ int tail_filter(uint64_t m1, uint64_t m2) {
    const uint64_t n1 = (1ull << 53) - m1, n2 = (1ull << 53) - m2;   // U = n 2^-53
    constexpr float kLn2 = 0.693147180559945309f;
    constexpr float kLn2OverX0 = (float)(0.693147180559945309 / zigtab::ZIG256_X0);
    const float s32 = -__log2f(m53_to_float(n1)) * kLn2OverX0;
    const float h32 = 0.5f * s32 * s32;
    const float l32 = __log2f(m53_to_float(n2)) * kLn2;
    const float marg = 0x1p-14f * (1.0f + h32 - l32);
    if (l32 < -h32 - marg) return 1;
    if (l32 > -h32 + marg) return 0;
    return -1;
}
__device__ __forceinline__ bool tail_exact(uint64_t m1, uint64_t m2) {
    const double U1 = __dsub_rn(1.0, m53_to_double(m1));
    const double U2 = __dsub_rn(1.0, m53_to_double(m2));
    const double x = __ddiv_rn(-zlog(U1), zigtab::ZIG256_X0);
    const double y = -zlog(U2);
    return __dadd_rn(y, y) > __dmul_rn(x, x);
}

// The value x >= 0 of an accepted slow path q = r << 53 | m1: the tail's
// x0 + RN(-ln(U1) / x0) with U1 = 1 - m1 2^-53 (r = 0), or overhang r's
// RN(ox + RN(odx U1)) with U1 = m1 2^-53.
__device__ __forceinline__ double slow_value(uint64_t q) {
    const uint64_t m1 = q & ((1ull << 53) - 1u);
    const int r = (int)(q >> 53);
    if (r == 0) {
        const double U1 = __dsub_rn(1.0, m53_to_double(m1));
        return __dadd_rn(zigtab::ZIG256_X0, __ddiv_rn(-zlog(U1), zigtab::ZIG256_X0));
    }
    return __dadd_rn(d_z256_OX[r - 1], __dmul_rn(d_z256_ODX[r - 1], u53_to_double(m1, 53)));
}

// McFarland's slow path after a slow first draw: a slot r chosen by the alias
// table from a fresh nextLong, then the tail (r = 0) or that overhang's
// rejection loop, each on fresh uniforms.  Returns the accepted slot and
// uniform, r << 53 | m1 (slow_value gives its value).
template <int PRNG, class S>
__device__ __forceinline__ uint64_t slow_path(S& src, const Z256Smem& t) {
    const uint64_t two53 = 1ull << 53;
    const uint64_t V = slot_u64<PRNG>(src.next());
    const uint32_t b = (uint32_t)(V & 0xFF);
    const int r = ((V >> 8) < t.THR[b]) ? (int)b : t.ALIAS[b];
    if (r == 0) {
        for (;;) {
            const uint64_t m1 = slot_m53<PRNG>(src.next());
            const uint64_t m2 = slot_m53<PRNG>(src.next());
            int f = tail_filter(m1, m2);
            if (f < 0) f = tail_exact(m1, m2) ? 1 : 0;
            if (f) return m1;
        }
    }
    const int kd = d_z256_KIND[r - 1];
    const uint64_t qa = d_z256_QA[r - 1];
    const float ox32 = d_z256_F32[0][r - 1], odx32 = d_z256_F32[1][r - 1];
    const float oy32 = d_z256_F32[2][r - 1], ody32 = d_z256_F32[3][r - 1];
    uint64_t m1;
    for (;;) {
        m1 = slot_m53<PRNG>(src.next());
        uint64_t m2 = slot_m53<PRNG>(src.next());
        if (kd > 0 && m1 + m2 > two53) {
            m1 = two53 - m1;
            m2 = two53 - m2;
        }
        if (kd > 0 && m1 + m2 <= two53 - qa) break;
        if (kd < 0 && m1 + m2 < two53) break;
        const int f = z256_overhang_filter(ox32, odx32, oy32, ody32, m1, m2);
        if (f == 1) break;
        if (f == 0) continue;
        const double x = __dadd_rn(d_z256_OX[r - 1], __dmul_rn(d_z256_ODX[r - 1], u53_to_double(m1, 53)));
        const double y = __dadd_rn(d_z256_OY[r - 1], __dmul_rn(d_z256_ODY[r - 1], u53_to_double(m2, 53)));
        if (y < exp(neg_half_sq(x))) break;
    }
    return (uint64_t)r << 53 | m1;
}

// The values of queued slow paths, up to 32 at once (all 32 lanes call this):
// binary64 x, or the binary32 / bfloat16 rounding of it, with the sign from bit 0
// of the entry's address.
template <int DT>
__device__ __forceinline__ void drain_slow(Warp& ws, int lane) {
    if ((uint32_t)lane < ws.sq_n) {
        const uint64_t ad = ws.sq_addr[lane];
        const double x = slow_value(ws.sq_val[lane]);
        const uint32_t neg = (uint32_t)(ad & 1u);
        if constexpr (DT == ZIG_F64) {
            __stcs((unsigned long long*)(ad & ~1ull), (unsigned long long)__double_as_longlong(x) | (unsigned long long)neg << 63);
        } else if constexpr (DT == ZIG_F32) {
            __stcs((unsigned int*)(ad & ~1ull), f64_to_f32_bits(x) | neg << 31);
        } else {
            __stcs((unsigned short*)(ad & ~1ull), (unsigned short)(f64_to_bf16_bits(x) | neg << 15));
        }
    }
    __syncwarp();
    if (lane == 0) ws.sq_n = 0;
    __syncwarp();
}

// The value of a fast slot of a row: the draw's sign XS[j] m with
// m = U >> 11 = h 2^52 + l: a = 1 + l 2^-52 from bits
// and fma(a, -XN[j], h ? 0 : XN[j]) = XS[j] 2^52 (l 2^-52 + h) before its one
// rounding (XN = -XS 2^52 in the table, so no separate negation is needed).
template <int PRNG>
__device__ __forceinline__ uint64_t value_of(const Tabs& tb, uint64_t v, int lane) {
    const uint64_t U = slot_u64<PRNG>(v);
    const uint32_t j = (uint32_t)U & 0xFFu;
    const uint64_t m = U >> 11;
    const uint32_t mh = (uint32_t)(m >> 32);
    const double xn = tb.XN[j][lane & 15];
    const double av = __hiloint2double((int)(0x3FF00000u | (mh & 0xFFFFFu)), (int)(uint32_t)m);
    const double x = __fma_rn(av, -xn, (mh >> 20) ? 0.0 : xn);
    return (uint64_t)__double_as_longlong(x) | ((U >> 8) & 1u) << 63;
}

template <int PRNG, int DT>
__global__ void __launch_bounds__(kThreads, 1) z256b_kernel(GenArgs a) {
    using GT = zf::Gen<PRNG>;
    using G = typename GT::G;
    using OutT = typename OutOf<DT>::T;
    constexpr int B = 32;
    extern __shared__ __align__(16) unsigned char zb_dsm[];
    Tabs& tb = *(Tabs*)zb_dsm;
    for (int k = threadIdx.x; k < 256 * 16; k += blockDim.x) tb.XN[k >> 4][k & 15] = __dmul_rn(d_z256_XS[k >> 4], -0x1p52);
    z256_load(tb.s);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const uint32_t lane_bit = 1u << lane, lt_mask = lane_bit - 1u;
    const int wib = threadIdx.x >> 5;
    const int n_warps = blockDim.x >> 5;
    Warp& ws = *(Warp*)(zb_dsm + ((sizeof(Tabs) + 15) & ~(size_t)15) + (size_t)wib * sizeof(Warp));
    uint64_t* const row = ws.stage + lane * kRS;
    if (lane == 0) ws.sq_n = 0;
    __syncwarp();
    if (a.out == nullptr) {   // only legal when every length is zero
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
        if (u < n_units) {
            uint64_t s, q, off, n;
            unit_info(a, u, s, q, off, n);
            bool ok;
            srec = unit_gen<PRNG>(a, s, q, g, ok);
            if (ok) {
                rem = n;
                dst = out + off;
            }
        }
        const bool check_chunk = a.chunk_log2 != 0 && rem != 0;
        uint64_t draws = 0;   // raw steps used by this unit (chunk-overflow check)

        while (__any_sync(kFull, rem > 0)) {
            // ---- A: 32 draws per lane, lockstep; nf marks the slow ones ----
            uint32_t nf = 0;
            const uint64_t sb = zf::first_state_of(g);
            auto step = [&](auto dc) {
                constexpr int d = decltype(dc)::value;
                uint64_t v;
                if constexpr (PRNG == ZIG_LCG48) {
                    v = (uint64_t)GT::template draw_at<2 * d>(sb) << 32 | GT::template draw_at<2 * d + 1>(sb);
                } else {
                    v = g.next_u64();
                }
                row[d] = v;
                nf |= (((uint32_t)slot_u64<PRNG>(v) & 0xFFu) >= (uint32_t)zigtab::ZIG256_NR ? 1u : 0u) << d;
            };
            zf::unroll<B>(step);
            if constexpr (PRNG == ZIG_LCG48) GT::template skip<2 * B>(g);
            // ---- B: each lane's slow paths, in draw order ----
            int drawn = B;
            uint32_t du = 0, Q = 0;    // consumed draws, slots of accepted slow paths
            int last_end = 0;          // the draw after the last slow path run
            for (uint32_t m = rem > 0 ? nf : 0u; m;) {
                const int p = __ffs(m) - 1;
                m &= m - 1u;
                if ((du >> p) & 1u) continue;   // a uniform of an earlier slow path
                if ((uint64_t)__popc(~du & lt_mask_of(p)) >= rem) break;   // the unit ends before p
                const uint64_t neg = (slot_u64<PRNG>(row[p]) >> 8) & 1u;
                Src<PRNG, G> src{row, p + 1, drawn, g};
                const uint64_t q = slow_path<PRNG>(src, tb.s);
                g = src.g;
                drawn = src.drawn;
                const int hi = src.pos < 32 ? src.pos : 32;
                du |= lt_mask_of(hi) & ~lt_mask_of(p + 1);
                row[p] = q | neg << 62;   // waits in the slot for the queue
                Q |= 1u << p;
                last_end = src.pos;
            }
            // ---- C: drops, the unit's end, then the rows ----
            uint32_t D = du;
            const int kept = 32 - __popc(D);
            int k_out = kept;
            if ((uint64_t)kept >= rem) {   // the unit ends in this batch: keep rem outputs
                k_out = (int)rem;
                uint32_t keepm = ~D;
                for (int mm = 0; mm < k_out; ++mm) keepm &= keepm - 1u;   // the slots past the rem-th kept one
                D |= keepm;
                if ((check_chunk || srec) && k_out > 0) {
                    const int c = 31 - __clz(~D);   // slot of the last output
                    const int used = ((Q >> c) & 1u) ? last_end : c + 1;   // draws up to it and its slow path
                    draws += (uint64_t)used * kStepsPerSlot<PRNG>;
                    if (srec) {   // the generator after those draws (the batch took `drawn` from sb)
                        G t = g;
                        if constexpr (PRNG == ZIG_LCG48 || PRNG == ZIG_SPLITMIX64) {
                            t.s = sb;
                            t.jump((uint64_t)used * kStepsPerSlot<PRNG>, &d_jump);
                        } else {
                            for (int k = used; k < drawn; ++k) t.unstep();
                        }
                        state_store(srec, t, false, 0.0);
                    }
                }
            } else if (check_chunk) {
                draws += (uint64_t)drawn * kStepsPerSlot<PRNG>;
            }
            ws.info[lane] = make_uint4((uint32_t)(uintptr_t)dst, (uint32_t)((uintptr_t)dst >> 32), D, 0u);
            __syncwarp();
#pragma unroll(DT == ZIG_F64 ? 8 : 4)   // binary64 rows: more fmas in flight; narrow rows: fewer registers
            for (int r = 0; r < 32; ++r) {
                const uint4 inf = ws.info[r];
                const uint64_t v = value_of<PRNG>(tb, ws.stage[r * kRS + lane], lane);
                const uint32_t e = __popc(~inf.z & lt_mask);
                OutT* const p = (OutT*)((uint64_t)inf.x | (uint64_t)inf.y << 32) + e;
                // a predicated store of a value computed on every lane, so that the
                // unrolled rows' loads and arithmetic overlap.  A queued slow slot
                // stores a placeholder, which its queue entry overwrites: the row's
                // run leaves no hole in a sector (a hole filled after the sector
                // left L2 would cost a read-modify-write of it).
                const uint32_t skip = inf.z & lane_bit;
                const double x = __longlong_as_double((long long)v);
                if constexpr (DT == ZIG_F64) {
                    asm volatile("{\n\t.reg .pred q;\n\tsetp.eq.u32 q, %2, 0;\n\t@q st.global.cs.b64 [%0], %1;\n\t}" ::"l"(p),
                                 "l"(v), "r"(skip));
                } else if constexpr (DT == ZIG_F32) {
                    asm volatile("{\n\t.reg .pred q;\n\tsetp.eq.u32 q, %2, 0;\n\t@q st.global.cs.b32 [%0], %1;\n\t}" ::"l"(p),
                                 "r"(f64_to_f32_bits(x)), "r"(skip));
                } else {
                    asm volatile("{\n\t.reg .pred q;\n\tsetp.eq.u32 q, %2, 0;\n\t@q st.global.cs.b16 [%0], %1;\n\t}" ::"l"(p),
                                 "h"(f64_to_bf16_bits(x)), "r"(skip));
                }
            }
            // accepted slow paths join the queue (one per lane per round)
            uint32_t Qk = Q & ~D;
            for (;;) {
                const uint32_t bal = __ballot_sync(kFull, Qk != 0);
                if (bal == 0) break;
                if (ws.sq_n + __popc(bal) > (uint32_t)kSQ) drain_slow<DT>(ws, lane);
                if (Qk) {
                    const int p = __ffs(Qk) - 1;
                    Qk &= Qk - 1u;
                    const uint32_t idx = ws.sq_n + __popc(bal & lt_mask);
                    const uint64_t v = row[p];
                    ws.sq_addr[idx] = (uint64_t)(uintptr_t)(dst + __popc(~D & ((1u << p) - 1u))) | ((v >> 62) & 1u);
                    ws.sq_val[idx] = v & ((1ull << 61) - 1u);
                }
                __syncwarp();
                if (lane == 0) ws.sq_n += __popc(bal);
                __syncwarp();
            }
            dst += k_out;
            rem -= (uint64_t)k_out;
            __syncwarp();
        }
        if (check_chunk && draws > kChunkDraws) atomicOr(a.err, kErrChunkOverflow);
    }
    drain_slow<DT>(ws, lane);
}

}  // namespace zb
