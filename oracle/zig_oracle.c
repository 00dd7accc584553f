/*
 * Serial CPU oracle for bulk N(0,1) generation.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load this code.  It shares
 * nothing with the CUDA library: its own PRNGs, its own tables (read from
 * oracle/tables/*.txt, written by oracle/gen_tables.py), its own sampler loops.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction anywhere, so
 * every binary64 expression rounds once per operation, in source order).
 * Transcendentals: the C library's exp/log/sqrt.
 *
 * What it computes, and where each part comes from:
 *  - PRNGs (Sec. 2, first list; Sec. 3 on LXM):
 *      java.util.Random 48-bit LCG (Knuth vol. 2 LCG, a = 0x5DEECE66D, c = 0xB),
 *      SplittableRandom / ThreadLocalRandom = SplitMix64 (Steele, Lea & Flood),
 *      L64X128MixRandom (LXM: 64-bit LCG + xoroshiro128 + Lea's mix), and
 *      Xoroshiro128PlusPlus (an XBG generator; Sec. 3 names the XBG family).
 *    Draw semantics follow the Java methods the paper's calls use: nextInt,
 *    nextLong, nextDouble.
 *  - Original ziggurat, GSL form (Sec. 1; Sec. 2 "Ziggurat" bullet): one 32-bit
 *    draw gives layer, sign and a 24-bit abscissa; fast test against k[i];
 *    wedge test; tail from the exponential envelope; restart on rejection.
 *  - Polar method (Sec. 1; Sec. 2 "Java 17" bullet; Listing 2: Random's
 *    nextGaussian), Knuth's Algorithm P with the second variate cached.
 *  - Modified ziggurat after McFarland (Sec. 2 "Java 17" bullet; Sec. 3):
 *    256 slots, equal-area inscribed rectangles accepted with no test,
 *    alias-selected overhangs and tail sampled by rejection.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LCG48 0
#define ORC_SPLITMIX64 1
#define ORC_L64X128MIX 2
#define ORC_XOROSHIRO128PP 3
#define ORC_SCRIPTED 9

#define ORC_ZIG128 0
#define ORC_POLAR 1
#define ORC_ZIG256 2

#define MASK48 ((UINT64_C(1) << 48) - 1)
#define LCG_A UINT64_C(0x5DEECE66D)
#define LCG_C UINT64_C(0xB)
#define GOLDEN_GAMMA UINT64_C(0x9E3779B97F4A7C15)
#define LXM_M UINT64_C(0xD1342543DE82EF95)
#define TWO_M53 (1.0 / 9007199254740992.0) /* 2^-53 */

typedef struct {
    int kind;
    uint64_t s;       /* LCG48 state, SplitMix64 seed, or LXM's LCG state */
    uint64_t a;       /* LXM additive parameter (odd) */
    uint64_t x0, x1;  /* LXM's xoroshiro128 state, or Xoroshiro128PlusPlus's state */
    const uint64_t *script; /* ORC_SCRIPTED: words returned in order */
    uint64_t script_len, script_pos;
    int script_overrun;
    int have_next;    /* polar cache: Random.haveNextNextGaussian */
    double next_gauss;
} orc_prng;

typedef struct {
    uint64_t draws;      /* raw generator steps consumed */
    uint64_t iters;      /* sampler iterations (layer draws) */
    uint64_t fast, wedge, tail, wedge_acc, tail_acc;
    uint64_t slow, overhang, overhang_quick, overhang_acc, tail_tries;
    uint64_t polar_pairs, polar_tries;
    double min_margin;   /* smallest |y - e| / e over all exp tests */
} orc_stats;

/* --------------------------------------------------------------------- */
/* PRNGs                                                                  */
/* --------------------------------------------------------------------- */

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * UINT64_C(0xBF58476D1CE4E5B9);
    z = (z ^ (z >> 27)) * UINT64_C(0x94D049BB133111EB);
    return z ^ (z >> 31);
}

static uint32_t mix32(uint64_t z) {
    z = (z ^ (z >> 33)) * UINT64_C(0x62A9D9ED799705F5);
    return (uint32_t)(((z ^ (z >> 28)) * UINT64_C(0xCB24D0A5C88C35B3)) >> 32);
}

static uint64_t mix_lea64(uint64_t z) {
    z = (z ^ (z >> 32)) * UINT64_C(0xDABA0B6EB09322E3);
    z = (z ^ (z >> 32)) * UINT64_C(0xDABA0B6EB09322E3);
    return z ^ (z >> 32);
}

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

void orc_seed(orc_prng *g, int kind, uint64_t seed) {
    memset(g, 0, sizeof(*g));
    g->kind = kind;
    if (kind == ORC_LCG48) {
        /* java.util.Random(long): initialScramble */
        g->s = (seed ^ LCG_A) & MASK48;
    } else if (kind == ORC_SPLITMIX64) {
        /* SplittableRandom(long): seed field = seed, gamma = GOLDEN_GAMMA */
        g->s = seed;
    } else if (kind == ORC_L64X128MIX) {
        /* Seed expansion: four consecutive SplitMix64 outputs of a generator
         * seeded with `seed` give a (forced odd), s, x0, x1. */
        uint64_t t = seed;
        t += GOLDEN_GAMMA; g->a = mix64(t) | 1;
        t += GOLDEN_GAMMA; g->s = mix64(t);
        t += GOLDEN_GAMMA; g->x0 = mix64(t);
        t += GOLDEN_GAMMA; g->x1 = mix64(t);
        if ((g->x0 | g->x1) == 0) g->x1 = GOLDEN_GAMMA;
    } else if (kind == ORC_XOROSHIRO128PP) {
        /* Seed expansion (reading): two consecutive SplitMix64 outputs of a
         * generator seeded with `seed` give x0, x1 (never both zero). */
        uint64_t t = seed;
        t += GOLDEN_GAMMA; g->x0 = mix64(t);
        t += GOLDEN_GAMMA; g->x1 = mix64(t);
        if ((g->x0 | g->x1) == 0) g->x1 = GOLDEN_GAMMA;
    }
}

void orc_set_script(orc_prng *g, const uint64_t *words, uint64_t n) {
    memset(g, 0, sizeof(*g));
    g->kind = ORC_SCRIPTED;
    g->script = words;
    g->script_len = n;
}

/* One LCG48 step; returns the top `bits` bits (Random.next(bits)). */
static uint32_t lcg_next(orc_prng *g, int bits) {
    g->s = (g->s * LCG_A + LCG_C) & MASK48;
    return (uint32_t)(g->s >> (48 - bits));
}

/* One LXM step (L64X128MixRandom.nextLong). */
static uint64_t lxm_next(orc_prng *g) {
    uint64_t result = mix_lea64(g->s + g->x0);
    g->s = LXM_M * g->s + g->a;
    uint64_t q0 = g->x0, q1 = g->x1;
    q1 ^= q0;
    q0 = rotl64(q0, 24) ^ q1 ^ (q1 << 16);
    q1 = rotl64(q1, 37);
    g->x0 = q0;
    g->x1 = q1;
    return result;
}
/* One Xoroshiro128PlusPlus step (the XBG generator's nextLong): the ++
 * scrambler of the current state, then the xoroshiro128 linear engine with
 * rotation/shift constants (49, 21, 28). */
static uint64_t xpp_next(orc_prng *g) {
    const uint64_t s0 = g->x0;
    uint64_t s1 = g->x1;
    const uint64_t result = rotl64(s0 + s1, 17) + s0;
    s1 ^= s0;
    g->x0 = rotl64(s0, 49) ^ s1 ^ (s1 << 21);
    g->x1 = rotl64(s1, 28);
    return result;
}

static uint64_t script_next(orc_prng *g) {
    if (g->script_pos >= g->script_len) {
        g->script_overrun = 1;
        return 0;
    }
    return g->script[g->script_pos++];
}

/* nextInt(), as an unsigned 32-bit word. */
uint32_t orc_next_u32(orc_prng *g, orc_stats *st) {
    switch (g->kind) {
    case ORC_LCG48: if (st) st->draws += 1; return lcg_next(g, 32);
    case ORC_SPLITMIX64: if (st) st->draws += 1; g->s += GOLDEN_GAMMA; return mix32(g->s);
    case ORC_L64X128MIX: if (st) st->draws += 1; return (uint32_t)(lxm_next(g) >> 32);
    case ORC_XOROSHIRO128PP: if (st) st->draws += 1; return (uint32_t)(xpp_next(g) >> 32);
    default: return (uint32_t)script_next(g);
    }
}

/* nextLong(). */
uint64_t orc_next_u64(orc_prng *g, orc_stats *st) {
    switch (g->kind) {
    case ORC_LCG48: {
        /* ((long)next(32) << 32) + next(32), the second term sign-extended */
        if (st) st->draws += 2;
        uint64_t hi = lcg_next(g, 32);
        int32_t lo = (int32_t)lcg_next(g, 32);
        return (hi << 32) + (uint64_t)(int64_t)lo;
    }
    case ORC_SPLITMIX64: if (st) st->draws += 1; g->s += GOLDEN_GAMMA; return mix64(g->s);
    case ORC_L64X128MIX: if (st) st->draws += 1; return lxm_next(g);
    case ORC_XOROSHIRO128PP: if (st) st->draws += 1; return xpp_next(g);
    default: return script_next(g);
    }
}

/* The 53-bit integer m behind nextDouble() = m * 2^-53. */
uint64_t orc_next_m53(orc_prng *g, orc_stats *st) {
    switch (g->kind) {
    case ORC_LCG48: {
        if (st) st->draws += 2;
        uint64_t hi = lcg_next(g, 26);
        uint64_t lo = lcg_next(g, 27);
        return (hi << 27) + lo;
    }
    case ORC_SPLITMIX64: if (st) st->draws += 1; g->s += GOLDEN_GAMMA; return mix64(g->s) >> 11;
    case ORC_L64X128MIX: if (st) st->draws += 1; return lxm_next(g) >> 11;
    case ORC_XOROSHIRO128PP: if (st) st->draws += 1; return xpp_next(g) >> 11;
    default: return script_next(g) >> 11;
    }
}

double orc_next_double(orc_prng *g, orc_stats *st) {
    return (double)orc_next_m53(g, st) * TWO_M53;
}

/* ---- jump-ahead by n raw generator steps -------------------------------- */

/* Affine map s -> A s + C (mod 2^64, or mod 2^48 after masking). */
typedef struct { uint64_t A, C; } affine;

static affine affine_compose(affine outer, affine inner) {
    /* outer(inner(s)) = oA (iA s + iC) + oC */
    affine r;
    r.A = outer.A * inner.A;
    r.C = outer.A * inner.C + outer.C;
    return r;
}

static affine affine_pow(affine m, uint64_t n) {
    affine r = {1, 0};
    while (n) {
        if (n & 1) r = affine_compose(m, r);
        m = affine_compose(m, m);
        n >>= 1;
    }
    return r;
}

/* GF(2) linear map on the 128-bit xoroshiro state, stored by columns:
 * col[c][0..1] = image of unit vector e_c (bit c of (x0, x1)). */
typedef struct { uint64_t col[128][2]; } gf2map;

static void gf2_apply(const gf2map *m, const uint64_t v[2], uint64_t out[2]) {
    uint64_t r0 = 0, r1 = 0;
    for (int c = 0; c < 128; c++) {
        uint64_t bit = (c < 64) ? (v[0] >> c) & 1 : (v[1] >> (c - 64)) & 1;
        if (bit) { r0 ^= m->col[c][0]; r1 ^= m->col[c][1]; }
    }
    out[0] = r0;
    out[1] = r1;
}

/* One step of a xoroshiro128 linear engine with constants (a, b, c):
 * (24, 16, 37) inside LXM, (49, 21, 28) for Xoroshiro128PlusPlus. */
static void xoro_step_vec(uint64_t v[2], int a, int b, int c) {
    uint64_t q0 = v[0], q1 = v[1];
    q1 ^= q0;
    q0 = rotl64(q0, a) ^ q1 ^ (q1 << b);
    q1 = rotl64(q1, c);
    v[0] = q0;
    v[1] = q1;
}

static void gf2_one_step(gf2map *m, int a, int b, int cc) {
    for (int c = 0; c < 128; c++) {
        uint64_t v[2] = {0, 0};
        if (c < 64) v[0] = UINT64_C(1) << c; else v[1] = UINT64_C(1) << (c - 64);
        xoro_step_vec(v, a, b, cc);
        m->col[c][0] = v[0];
        m->col[c][1] = v[1];
    }
}

static void gf2_compose(const gf2map *outer, const gf2map *inner, gf2map *out) {
    gf2map tmp;
    for (int c = 0; c < 128; c++) gf2_apply(outer, inner->col[c], tmp.col[c]);
    *out = tmp;
}

static void gf2_pow(const gf2map *m, uint64_t n, gf2map *out) {
    gf2map r, b = *m;
    memset(&r, 0, sizeof(r));
    for (int c = 0; c < 128; c++) {
        if (c < 64) r.col[c][0] = UINT64_C(1) << c; else r.col[c][1] = UINT64_C(1) << (c - 64);
    }
    while (n) {
        if (n & 1) gf2_compose(&b, &r, &r);
        gf2_compose(&b, &b, &b);
        n >>= 1;
    }
    *out = r;
}

/* Precomputed jump by a fixed number of raw steps. */
typedef struct {
    int kind;
    uint64_t n;
    affine lcg;      /* LCG48 (masked) or LXM's 64-bit LCG */
    gf2map xoro;     /* LXM and Xoroshiro128PlusPlus */
} orc_jump;

void orc_jump_init(orc_jump *j, int kind, uint64_t n) {
    memset(j, 0, sizeof(*j));
    j->kind = kind;
    j->n = n;
    if (kind == ORC_LCG48) {
        affine one = {LCG_A, LCG_C};
        j->lcg = affine_pow(one, n);
    } else if (kind == ORC_XOROSHIRO128PP) {
        gf2map one;
        gf2_one_step(&one, 49, 21, 28);
        gf2_pow(&one, n, &j->xoro);
    } else if (kind == ORC_L64X128MIX) {
        gf2map one;
        gf2_one_step(&one, 24, 16, 37);
        gf2_pow(&one, n, &j->xoro);
        /* the LCG part's additive term depends on the stream's `a`; keep A only */
        affine one_a = {LXM_M, 0};
        j->lcg = affine_pow(one_a, n);
    }
}

/* Sum_{k<n} M^k mod 2^64, for the LXM LCG increment term (a * that sum). */
static uint64_t geom_sum(uint64_t M, uint64_t n) {
    /* S(n) = 1 + M + ... + M^(n-1), via the affine map s -> M s + 1 from s = 0 */
    affine one = {M, 1};
    return affine_pow(one, n).C;
}

void orc_jump_apply(const orc_jump *j, orc_prng *g) {
    if (g->kind == ORC_LCG48) {
        g->s = (j->lcg.A * g->s + j->lcg.C) & MASK48;
    } else if (g->kind == ORC_SPLITMIX64) {
        g->s += j->n * GOLDEN_GAMMA;
    } else if (g->kind == ORC_L64X128MIX) {
        g->s = j->lcg.A * g->s + g->a * geom_sum(LXM_M, j->n);
        uint64_t v[2] = {g->x0, g->x1}, o[2];
        gf2_apply(&j->xoro, v, o);
        g->x0 = o[0];
        g->x1 = o[1];
    } else if (g->kind == ORC_XOROSHIRO128PP) {
        uint64_t v[2] = {g->x0, g->x1}, o[2];
        gf2_apply(&j->xoro, v, o);
        g->x0 = o[0];
        g->x1 = o[1];
    }
    g->have_next = 0;
}

/* Plain single-shot jump (used by tests to pin the closed forms). */
void orc_jump_n(orc_prng *g, uint64_t n) {
    orc_jump *j = (orc_jump *)malloc(sizeof(orc_jump));
    orc_jump_init(j, g->kind, n);
    orc_jump_apply(j, g);
    free(j);
}

/* --------------------------------------------------------------------- */
/* Tables                                                                 */
/* --------------------------------------------------------------------- */

typedef struct {
    double R;
    uint32_t k[128];
    double w[128];
    double y[128];
} orc_zig128_tab;

typedef struct {
    int n_r;
    double x0;
    double xs[256];
    double ox[257], odx[257], oy[257], ody[257];
    int kind[257];
    uint64_t qa[257];
    uint64_t thr[256];
    int alias[256];
} orc_zig256_tab;

size_t orc_zig128_tab_size(void) { return sizeof(orc_zig128_tab); }
size_t orc_zig256_tab_size(void) { return sizeof(orc_zig256_tab); }

void orc_zig128_tab_set(orc_zig128_tab *t, double R, const uint32_t *k, const double *w,
                        const double *y) {
    t->R = R;
    memcpy(t->k, k, sizeof(t->k));
    memcpy(t->w, w, sizeof(t->w));
    memcpy(t->y, y, sizeof(t->y));
}

void orc_zig256_tab_set(orc_zig256_tab *t, int n_r, double x0, const double *xs,
                        const double *ox, const double *odx, const double *oy,
                        const double *ody, const int *kind, const uint64_t *qa,
                        const uint64_t *thr, const int *alias) {
    memset(t, 0, sizeof(*t));
    t->n_r = n_r;
    t->x0 = x0;
    memcpy(t->xs, xs, sizeof(double) * (size_t)n_r);
    memcpy(t->ox, ox, sizeof(double) * (size_t)(n_r + 1));
    memcpy(t->odx, odx, sizeof(double) * (size_t)(n_r + 1));
    memcpy(t->oy, oy, sizeof(double) * (size_t)(n_r + 1));
    memcpy(t->ody, ody, sizeof(double) * (size_t)(n_r + 1));
    memcpy(t->kind, kind, sizeof(int) * (size_t)(n_r + 1));
    memcpy(t->qa, qa, sizeof(uint64_t) * (size_t)(n_r + 1));
    memcpy(t->thr, thr, sizeof(t->thr));
    memcpy(t->alias, alias, sizeof(t->alias));
}

/* --------------------------------------------------------------------- */
/* Samplers: one variate per call                                         */
/* --------------------------------------------------------------------- */

static void note_margin(orc_stats *st, double y, double e, double *vm) {
    double m = fabs(y - e) / e;
    if (m < st->min_margin) st->min_margin = m;
    if (vm && m < *vm) *vm = m;
}

/* Original ziggurat, GSL form.  *vm (may be NULL) receives the smallest margin
 * of the exp tests taken while producing this variate; *vlog (may be NULL) is
 * set to 1 when the value itself was computed through log (the tail), else 0. */
double orc_zig128_next(orc_prng *g, const orc_zig128_tab *t, orc_stats *st, double *vm, int *vlog) {
    if (vlog) *vlog = 0;
    for (;;) {
        uint32_t u = orc_next_u32(g, st);
        uint32_t i = u & 0xFF;
        double sign = (i & 0x80) ? 1.0 : -1.0;
        i &= 0x7F;
        uint32_t j = (u >> 8) & 0xFFFFFF;
        double x = (double)j * t->w[i];
        st->iters++;
        if (j < t->k[i]) {
            st->fast++;
            return sign * x;
        }
        double y;
        if (i < 127) {
            double y0 = t->y[i], y1 = t->y[i + 1];
            double U = orc_next_double(g, st);
            y = y1 + (y0 - y1) * U;
            st->wedge++;
        } else {
            double U1 = 1.0 - orc_next_double(g, st);
            double U2 = orc_next_double(g, st);
            x = t->R - log(U1) / t->R;
            y = exp(-t->R * (x - 0.5 * t->R)) * U2;
            st->tail++;
        }
        double e = exp(-0.5 * x * x);
        note_margin(st, y, e, vm);
        if (y < e) {
            if (i < 127) st->wedge_acc++; else st->tail_acc++;
            if (vlog) *vlog = i == 127;
            return sign * x;
        }
    }
}

/* Polar method (Knuth's Algorithm P; Random.nextGaussian with its cache). */
double orc_polar_next(orc_prng *g, orc_stats *st) {
    if (g->have_next) {
        g->have_next = 0;
        return g->next_gauss;
    }
    double v1, v2, s;
    st->polar_pairs++;
    do {
        v1 = 2 * orc_next_double(g, st) - 1;
        v2 = 2 * orc_next_double(g, st) - 1;
        s = v1 * v1 + v2 * v2;
        st->polar_tries++;
    } while (s >= 1 || s == 0);
    double multiplier = sqrt(-2 * log(s) / s);
    g->next_gauss = v2 * multiplier;
    g->have_next = 1;
    return v1 * multiplier;
}

/* Modified ziggurat, 256 slots. */
double orc_zig256_next(orc_prng *g, const orc_zig256_tab *t, orc_stats *st, double *vm, int *vlog) {
    const uint64_t two53 = UINT64_C(1) << 53;
    if (vlog) *vlog = 0;
    uint64_t U = orc_next_u64(g, st);
    unsigned j = (unsigned)(U & 0xFF);
    double sign = ((U >> 8) & 1) ? -1.0 : 1.0;
    st->iters++;
    if ((int)j < t->n_r) {
        st->fast++;
        return sign * (t->xs[j] * (double)(U >> 11));
    }
    st->slow++;
    uint64_t V = orc_next_u64(g, st);
    unsigned b = (unsigned)(V & 0xFF);
    int r = ((V >> 8) < t->thr[b]) ? (int)b : t->alias[b];
    if (r == 0) {
        /* tail beyond X_0: Marsaglia's exponential proposal, loop until accepted */
        for (;;) {
            double U1 = 1.0 - orc_next_double(g, st);
            double U2 = 1.0 - orc_next_double(g, st);
            double x = -log(U1) / t->x0;
            double y = -log(U2);
            st->tail_tries++;
            if (x > 0) note_margin(st, y + y, x * x, vm);
            if (y + y > x * x) {
                st->tail++;
                if (vlog) *vlog = 1;
                return sign * (t->x0 + x);
            }
        }
    }
    st->overhang++;
    for (;;) {
        uint64_t m1 = orc_next_m53(g, st);
        uint64_t m2 = orc_next_m53(g, st);
        int kd = t->kind[r];
        if (kd > 0 && m1 + m2 > two53) {
            /* convex overhang lies below the chord: reflect into the lower triangle */
            m1 = two53 - m1;
            m2 = two53 - m2;
        }
        double x = t->ox[r] + t->odx[r] * ((double)m1 * TWO_M53);
        if (kd > 0 && m1 + m2 <= two53 - t->qa[r]) {
            st->overhang_quick++;
            return sign * x;
        }
        if (kd < 0 && m1 + m2 < two53) {
            st->overhang_quick++;
            return sign * x;
        }
        double y = t->oy[r] + t->ody[r] * ((double)m2 * TWO_M53);
        double e = exp(-0.5 * x * x);
        note_margin(st, y, e, vm);
        if (y < e) {
            st->overhang_acc++;
            return sign * x;
        }
    }
}

/* --------------------------------------------------------------------- */
/* Bulk driver                                                            */
/* --------------------------------------------------------------------- */

/*
 * Stream-major packed output: stream s owns out[off_s .. off_s + L_s), with
 * off_s the exclusive prefix sum of the lengths.  chunk_log2 == 0: each stream
 * is one sequence of nextGaussian-style calls on a generator seeded with
 * seeds[s].  chunk_log2 == c > 0: output t of stream s belongs to chunk
 * q = t >> c, generated from the seeded state advanced by q * 2^32 raw steps.
 *
 * lengths == NULL: every stream has uniform_len outputs.
 * margins (may be NULL): per output, the smallest exp-test margin used for it
 * (+inf when no exp test was taken).
 * via_log (may be NULL): per output, 1 when the value was computed through log
 * (a tail value of either ziggurat; every polar value), else 0.
 * Returns 0, or -1 on bad arguments.
 */
int orc_generate(int prng, int alg, const uint64_t *seeds, const uint64_t *lengths,
                 uint64_t uniform_len, uint64_t n_streams, uint32_t chunk_log2,
                 const orc_zig128_tab *t128, const orc_zig256_tab *t256, double *out,
                 double *margins, unsigned char *via_log, orc_stats *st) {
    if (prng != ORC_LCG48 && prng != ORC_SPLITMIX64 && prng != ORC_L64X128MIX &&
        prng != ORC_XOROSHIRO128PP)
        return -1;
    if (alg == ORC_ZIG128 && !t128) return -1;
    if (alg == ORC_ZIG256 && !t256) return -1;
    if (alg != ORC_ZIG128 && alg != ORC_POLAR && alg != ORC_ZIG256) return -1;
    if (chunk_log2 > 40) return -1;
    orc_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof(*st));
    st->min_margin = INFINITY;
    orc_jump *jump = NULL;
    if (chunk_log2) {
        jump = (orc_jump *)malloc(sizeof(orc_jump));
        orc_jump_init(jump, prng, UINT64_C(1) << 32);
    }
    uint64_t off = 0;
    for (uint64_t s = 0; s < n_streams; s++) {
        uint64_t L = lengths ? lengths[s] : uniform_len;
        orc_prng g;
        orc_seed(&g, prng, seeds[s]);
        orc_prng chunk_start = g;
        for (uint64_t t = 0; t < L; t++) {
            if (chunk_log2 && t && (t & ((UINT64_C(1) << chunk_log2) - 1)) == 0) {
                orc_jump_apply(jump, &chunk_start);
                g = chunk_start;
            }
            double vm = INFINITY;
            int vlog = 1;
            double z;
            if (alg == ORC_ZIG128) z = orc_zig128_next(&g, t128, st, &vm, &vlog);
            else if (alg == ORC_POLAR) z = orc_polar_next(&g, st);
            else z = orc_zig256_next(&g, t256, st, &vm, &vlog);
            out[off + t] = z;
            if (margins) margins[off + t] = vm;
            if (via_log) via_log[off + t] = (unsigned char)vlog;
        }
        off += L;
    }
    free(jump);
    return 0;
}

/* Raw uniform streams for PRNG parity: kind 0 = nextInt (u32 stored in u64),
 * 1 = nextLong, 2 = nextDouble's 53-bit integer.  Stream s is advanced by
 * `skip` raw steps (closed-form jump) before its n draws. */
int orc_prng_fill(int prng, const uint64_t *seeds, uint64_t n_streams, uint64_t n,
                  uint64_t skip, int kind, uint64_t *out) {
    if (prng != ORC_LCG48 && prng != ORC_SPLITMIX64 && prng != ORC_L64X128MIX &&
        prng != ORC_XOROSHIRO128PP)
        return -1;
    orc_jump *jump = NULL;
    if (skip) {
        jump = (orc_jump *)malloc(sizeof(orc_jump));
        orc_jump_init(jump, prng, skip);
    }
    for (uint64_t s = 0; s < n_streams; s++) {
        orc_prng g;
        orc_seed(&g, prng, seeds[s]);
        if (jump) orc_jump_apply(jump, &g);
        for (uint64_t t = 0; t < n; t++) {
            uint64_t v;
            if (kind == 0) v = orc_next_u32(&g, NULL);
            else if (kind == 1) v = orc_next_u64(&g, NULL);
            else v = orc_next_m53(&g, NULL);
            out[s * n + t] = v;
        }
    }
    free(jump);
    return 0;
}

/* Single-generator helpers for the pin tests. */
size_t orc_prng_size(void) { return sizeof(orc_prng); }

void orc_state_get(const orc_prng *g, uint64_t out[4]) {
    out[0] = g->s;
    out[1] = g->a;
    out[2] = g->x0;
    out[3] = g->x1;
}

/* Scripted zig128: feed chosen words (u32 draws in the low half; doubles from
 * the top 53 bits).  Produces n outputs; returns the number of words consumed
 * or -1 if the script ran out. */
int64_t orc_zig128_scripted(const uint64_t *words, uint64_t n_words, const orc_zig128_tab *t,
                            uint64_t n, double *out, orc_stats *st) {
    orc_prng g;
    orc_set_script(&g, words, n_words);
    memset(st, 0, sizeof(*st));
    st->min_margin = INFINITY;
    for (uint64_t k = 0; k < n; k++) {
        out[k] = orc_zig128_next(&g, t, st, NULL, NULL);
        if (g.script_overrun) return -1;
    }
    return (int64_t)g.script_pos;
}

int64_t orc_zig256_scripted(const uint64_t *words, uint64_t n_words, const orc_zig256_tab *t,
                            uint64_t n, double *out, orc_stats *st) {
    orc_prng g;
    orc_set_script(&g, words, n_words);
    memset(st, 0, sizeof(*st));
    st->min_margin = INFINITY;
    for (uint64_t k = 0; k < n; k++) {
        out[k] = orc_zig256_next(&g, t, st, NULL, NULL);
        if (g.script_overrun) return -1;
    }
    return (int64_t)g.script_pos;
}
