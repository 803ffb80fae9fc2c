/*
 * synth.c -- seeded synthetic netlists and primary-input stimuli.
 *
 * This module only draws inputs: it holds none of the simulation
 * arithmetic (no cell function, no delay selection, no cancellation).
 * Both the CPU oracle and the CUDA path consume what it produces.
 *
 * Workload shapes follow the paper's re-simulation setting (Sec. 2.1 and
 * Sec. 5, Table 2): a levelized combinational DAG of library cells, given
 * waveforms on the primary inputs, each waveform a strictly time-ordered
 * list of (time, value) transitions in 4-value logic.
 *
 * Determinism: every draw comes from xoshiro256** streams seeded through
 * splitmix64; the only floating point is +,-,*,/ and sqrt (compiled with
 * -ffp-contract=off), and log/exp are written here from their series, so a
 * given seed yields the same arrays on x86_64 and aarch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* Cell codes and pin counts; the same numbering as the public C-ABI header. */
enum { C_INV, C_BUF, C_AND2, C_OR2, C_NAND2, C_NOR2, C_XOR2, C_XNOR2, C_MUX2, C_AOI21, C_OAI21, C_NCELLS };
static const int k_arity[C_NCELLS] = {1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3};

/* ---------------- random numbers ---------------- */
static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
typedef struct { uint64_t s[4]; } rng_t;
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
static void rng_seed(rng_t *r, uint64_t seed, uint64_t stream) {
    uint64_t sm = seed ^ (stream * 0xD1B54A32D192ED03ull) ^ 0x243F6A8885A308D3ull;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&sm);
}
/* uniform integer in [0, n) (Lemire's multiply-shift, 32-bit range) */
static uint32_t rng_below(rng_t *r, uint32_t n) {
    return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)n) >> 32);
}
/* uniform double in (0, 1] */
static double rng_unit(rng_t *r) {
    return (double)((rng_next(r) >> 11) + 1) * (1.0 / 9007199254740992.0);
}

/* natural log for x > 0: x = m * 2^e with m in [1,2); ln m = 2 atanh((m-1)/(m+1)) */
static double my_log(double x) {
    int e;
    double m = frexp(x, &e); /* m in [0.5, 1) */
    m *= 2.0; e -= 1;
    double s = (m - 1.0) / (m + 1.0), s2 = s * s, term = s, sum = 0.0;
    for (int k = 1; k < 60; k += 2) { sum += term / (double)k; term *= s2; }
    return 2.0 * sum + (double)e * 0.69314718055994530942;
}
/* exp via exp(x) = 2^n exp(r), |r| <= ln2/2, Taylor series */
static double my_exp(double x) {
    double n = floor(x / 0.69314718055994530942 + 0.5);
    double r = x - n * 0.69314718055994530942, term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; k++) { term *= r / (double)k; sum += term; }
    return ldexp(sum, (int)n);
}

/* ---------------- Fenwick tree for weighted choice ---------------- */
typedef struct { int64_t *t; int64_t n; } fen_t;
static void fen_add(fen_t *f, int64_t i, int64_t d) { for (i++; i <= f->n; i += i & -i) f->t[i] += d; }
static int64_t fen_prefix(const fen_t *f, int64_t i) { int64_t s = 0; for (; i > 0; i -= i & -i) s += f->t[i]; return s; }
/* smallest idx with prefix(idx+1) > target (target < total) */
static int64_t fen_find(const fen_t *f, int64_t target) {
    int64_t pos = 0, step = 1;
    while (step * 2 <= f->n) step *= 2;
    for (; step > 0; step >>= 1) {
        if (pos + step <= f->n && f->t[pos + step] <= target) { pos += step; target -= f->t[pos]; }
    }
    return pos; /* 0-based index */
}
/* draw a net in [a, b) with probability proportional to its remaining fanout
   quota; uniform when every quota in the range is spent */
static int64_t pick_net(fen_t *f, int64_t *quota, int64_t a, int64_t b, rng_t *r) {
    int64_t base = fen_prefix(f, a), tot = fen_prefix(f, b) - base, idx;
    if (tot <= 0) {
        idx = a + (int64_t)(((rng_next(r) >> 11) * (double)(b - a)) / 9007199254740992.0);
        if (idx >= b) idx = b - 1;
        return idx;
    }
    uint64_t x = rng_next(r) % (uint64_t)tot;
    idx = fen_find(f, base + (int64_t)x);
    if (quota[idx] > 0) { quota[idx]--; fen_add(f, idx, -1); }
    return idx;
}

static int64_t draw_quota(rng_t *r, int kind, double alpha, int cap) {
    int64_t q;
    if (kind == 0) { /* geometric on {1,2,...}, P(q=k) = 2^-k, mean 2 */
        uint64_t x = ~rng_next(r);
        q = 1 + (x ? __builtin_ctzll(x) : 64);
    } else { /* Pareto(alpha, x_min = 1), rounded to the nearest integer */
        double u = rng_unit(r);
        double x = (alpha == 2.0) ? 1.0 / sqrt(u) : my_exp(-my_log(u) / alpha);
        q = (x > 1e9) ? (int64_t)1e9 : (int64_t)floor(x + 0.5);
    }
    if (q < 1) q = 1;
    if (cap > 0 && q > cap) q = cap;
    return q;
}

/*
 * synth_netlist: a levelized DAG of n_gates cells over n_pi primary inputs.
 *   - levels 1..depth each get n_gates/depth gates (the first n_gates%depth
 *     levels one more); cell type uniform over the cells in cell_mask;
 *   - one randomly chosen pin of every gate reads a net of level L-1 (so the
 *     gate's level is exactly L), the other pins read nets of levels < L;
 *   - every net draws a fanout quota (fanout_kind 0: geometric mean 2;
 *     1: Pareto(alpha), rounded, capped at fanout_cap) and fanin choices are
 *     weighted by the remaining quota (uniform once a range is spent);
 *   - rise and fall delay of every arc uniform on [d_min, d_max].
 * Net ids: 0..n_pi-1 are primary inputs, n_pi+g is the output of gate g.
 * With shuffle != 0 gate ids are randomly permuted (fanins then may refer to
 * later gate ids; the DAG is unchanged).
 * Arrays: type[n_gates], fanin_off[n_gates+1], fanin_net/d_rise/d_fall[3*n_gates],
 * level[n_gates] (optional, may be NULL).  Returns the number of arcs, or
 * -1 on bad arguments, -2 on allocation failure.
 */
int64_t synth_netlist(int32_t n_pi, int32_t n_gates, int32_t depth, int32_t fanout_kind,
                      double pareto_alpha, int32_t fanout_cap, int32_t d_min, int32_t d_max,
                      uint32_t cell_mask, uint64_t seed, int32_t shuffle,
                      uint8_t *type, int32_t *fanin_off, int32_t *fanin_net,
                      int32_t *d_rise, int32_t *d_fall, int32_t *level) {
    if (n_pi < 1 || n_gates < depth || depth < 1 || d_min < 1 || d_max < d_min) return -1;
    int cells[C_NCELLS], ncell = 0;
    for (int c = 0; c < C_NCELLS; c++) if (cell_mask & (1u << c)) cells[ncell++] = c;
    if (ncell == 0) return -1;
    int64_t N = (int64_t)n_pi + n_gates;
    int64_t *quota = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    fen_t f = {(int64_t *)calloc((size_t)N + 1, sizeof(int64_t)), N};
    int32_t *lvl_start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(depth + 2));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_gates);
    if (!quota || !f.t || !lvl_start || !perm) { free(quota); free(f.t); free(lvl_start); free(perm); return -2; }
    rng_t r; rng_seed(&r, seed, 0x6E65746Cull);
    for (int64_t n = 0; n < N; n++) quota[n] = draw_quota(&r, fanout_kind, pareto_alpha, fanout_cap);
    /* internal order: nets in level order; level 0 = PIs */
    lvl_start[0] = 0; lvl_start[1] = n_pi;
    int32_t base = n_gates / depth, rem = n_gates % depth;
    for (int L = 1; L <= depth; L++) lvl_start[L + 1] = lvl_start[L] + base + (L <= rem ? 1 : 0);
    /* gate id permutation: internal gate i (level order) -> external id perm[i] */
    for (int32_t i = 0; i < n_gates; i++) perm[i] = i;
    if (shuffle) for (int32_t i = n_gates - 1; i > 0; i--) {
        int32_t j = (int32_t)rng_below(&r, (uint32_t)i + 1), t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    /* first pass: arity per external gate -> fanin_off */
    uint8_t *itype = (uint8_t *)malloc((size_t)n_gates);
    if (!itype) { free(quota); free(f.t); free(lvl_start); free(perm); return -2; }
    for (int32_t i = 0; i < n_gates; i++) itype[i] = (uint8_t)cells[rng_below(&r, (uint32_t)ncell)];
    for (int32_t i = 0; i < n_gates; i++) type[perm[i]] = itype[i];
    fanin_off[0] = 0;
    for (int32_t g = 0; g < n_gates; g++) fanin_off[g + 1] = fanin_off[g] + k_arity[type[g]];
    /* internal net id -> external net id */
    #define EXT(n) ((n) < n_pi ? (n) : n_pi + perm[(n) - n_pi])
    for (int L = 1; L <= depth; L++) {
        /* nets of levels < L are in [0, lvl_start[L]) and level L-1 is [lvl_start[L-1], lvl_start[L]) */
        int64_t prevA = lvl_start[L - 1], prevB = lvl_start[L];
        for (int64_t n = prevA; n < prevB; n++) fen_add(&f, n, quota[n]);
        for (int64_t in = lvl_start[L]; in < lvl_start[L + 1]; in++) {
            int32_t gi = (int32_t)(in - n_pi), g = perm[gi];
            int k = k_arity[itype[gi]];
            int deep = (int)rng_below(&r, (uint32_t)k);
            for (int p = 0; p < k; p++) {
                int64_t src = (p == deep) ? pick_net(&f, quota, prevA, prevB, &r)
                                          : pick_net(&f, quota, 0, prevB, &r);
                int32_t a = fanin_off[g] + p;
                fanin_net[a] = (int32_t)EXT(src);
                d_rise[a] = d_min + (int32_t)rng_below(&r, (uint32_t)(d_max - d_min + 1));
                d_fall[a] = d_min + (int32_t)rng_below(&r, (uint32_t)(d_max - d_min + 1));
            }
            if (level) level[g] = L;
        }
    }
    #undef EXT
    int64_t A = fanin_off[n_gates];
    free(quota); free(f.t); free(lvl_start); free(perm); free(itype);
    return A;
}

/* ---------------- stimulus ---------------- */
typedef struct {
    uint64_t seed; double mean, window; uint32_t th0, th1, th2;
    int32_t n_pi, n_clock, clock_period, clock_trans;
} stim_cfg;

static int is_clock(const stim_cfg *c, int32_t pi) {
    if (c->n_clock <= 0) return 0;
    int64_t stride = c->n_pi / c->n_clock;
    if (stride < 1) stride = 1;
    return (pi % stride) == 0 && pi / stride < c->n_clock;
}
static int draw_value(rng_t *r, const stim_cfg *c, int prev) {
    for (int tries = 0; tries < 64; tries++) {
        uint32_t x = (uint32_t)(rng_next(r) >> 32);
        int v = x < c->th0 ? 0 : x < c->th1 ? 1 : x < c->th2 ? 2 : 3;
        if (v != prev) return v;
    }
    return (prev + 1) & 3;
}
/* one PI waveform; writes at most 'cap' events when t/v non-NULL; returns the count */
/* times go to t (32-bit) or t64 (64-bit), whichever is non-null */
static int64_t gen_pi(const stim_cfg *c, int32_t pi, int32_t *t, int64_t *t64, uint8_t *v) {
    rng_t r; rng_seed(&r, c->seed, 0x5354494Dull + (uint64_t)pi * 0x100000001B3ull);
    int64_t n = 0;
    if (is_clock(c, pi)) {
        int64_t phase = rng_below(&r, (uint32_t)c->clock_period);
        int val = (int)(rng_next(&r) >> 63);
        int64_t half = c->clock_period / 2;
        for (int64_t j = 0; j < c->clock_trans; j++) {
            if (t) t[n] = (int32_t)(phase + half * j);
            if (t64) t64[n] = phase + half * j;
            if (v) v[n] = (uint8_t)val;
            n++; val ^= 1;
        }
        return n;
    }
    double tc = 0.0, scale = c->window / c->mean;
    int64_t last = -1; int prev = 2;
    for (;;) {
        tc += -my_log(rng_unit(&r)) * scale;
        if (tc >= c->window) break;
        int64_t ti = (int64_t)floor(tc);
        if (ti == last) continue;
        int val = draw_value(&r, c, prev);
        if (t) t[n] = (int32_t)ti;
        if (t64) t64[n] = ti;
        if (v) v[n] = (uint8_t)val;
        n++; last = ti; prev = val;
    }
    return n;
}
static void make_cfg(stim_cfg *c, int32_t n_pi, uint64_t seed, double mean, int64_t window,
                     double p0, double p1, double px, double pz,
                     int32_t n_clock, int32_t clock_period, int32_t clock_trans) {
    double tot = p0 + p1 + px + pz;
    c->seed = seed; c->mean = mean; c->window = (double)window; c->n_pi = n_pi;
    c->th0 = (uint32_t)fmin(4294967295.0, p0 / tot * 4294967296.0);
    c->th1 = (uint32_t)fmin(4294967295.0, (p0 + p1) / tot * 4294967296.0);
    c->th2 = (uint32_t)fmin(4294967295.0, (p0 + p1 + px) / tot * 4294967296.0);
    c->n_clock = n_clock; c->clock_period = clock_period; c->clock_trans = clock_trans;
}
/*
 * synth_stim_counts: per-PI transition counts.  Non-clock PIs follow a
 * Poisson process of 'mean' expected transitions over [0, window) (times
 * floored to integer ps, repeated times dropped) with values drawn from
 * (p0, p1, px, pz) and redrawn while equal to the previous value (the value
 * before the first transition is X).  n_clock PIs spread evenly over the
 * inputs are square waves of clock_trans transitions, half-period
 * clock_period/2, random phase in [0, clock_period) and random start value.
 * Returns the total.
 */
int64_t synth_stim_counts(int32_t n_pi, uint64_t seed, double mean, int64_t window,
                          double p0, double p1, double px, double pz,
                          int32_t n_clock, int32_t clock_period, int32_t clock_trans, int64_t *counts) {
    stim_cfg c; make_cfg(&c, n_pi, seed, mean, window, p0, p1, px, pz, n_clock, clock_period, clock_trans);
    int64_t tot = 0;
    /* every PI draws from its own stream, so the PIs are independent */
    #pragma omp parallel for schedule(dynamic, 64) reduction(+:tot)
    for (int32_t i = 0; i < n_pi; i++) { counts[i] = gen_pi(&c, i, NULL, NULL, NULL); tot += counts[i]; }
    return tot;
}
/* synth_stim_fill64: the same transitions with 64-bit times (windows past 2^31 ps) */
int synth_stim_fill64(int32_t n_pi, uint64_t seed, double mean, int64_t window,
                      double p0, double p1, double px, double pz,
                      int32_t n_clock, int32_t clock_period, int32_t clock_trans,
                      const int64_t *off, int64_t *t, uint8_t *v) {
    stim_cfg c; make_cfg(&c, n_pi, seed, mean, window, p0, p1, px, pz, n_clock, clock_period, clock_trans);
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 64) reduction(|:bad)
    for (int32_t i = 0; i < n_pi; i++) {
        int64_t n = gen_pi(&c, i, NULL, t + off[i], v + off[i]);
        if (n != off[i + 1] - off[i]) bad = 1;
    }
    return bad ? -1 : 0;
}
/* synth_stim_fill: the transitions themselves, PI i at [off[i], off[i+1]) */
int synth_stim_fill(int32_t n_pi, uint64_t seed, double mean, int64_t window,
                    double p0, double p1, double px, double pz,
                    int32_t n_clock, int32_t clock_period, int32_t clock_trans,
                    const int64_t *off, int32_t *t, uint8_t *v) {
    stim_cfg c; make_cfg(&c, n_pi, seed, mean, window, p0, p1, px, pz, n_clock, clock_period, clock_trans);
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 64) reduction(|:bad)
    for (int32_t i = 0; i < n_pi; i++) {
        int64_t n = gen_pi(&c, i, t + off[i], NULL, v + off[i]);
        if (n != off[i + 1] - off[i]) bad = 1;
    }
    return bad ? -1 : 0;
}
