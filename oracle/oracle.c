/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU reference for timing-aware 4-value
 * gate-level re-simulation as defined in arXiv 2304.13398.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the CUDA library never does, and this file shares no code with it.
 *
 * Definitions followed (paper sections / equations / algorithms):
 *   values      0, 1, X (=2), Z (=3); Z is read as X on inputs and X means
 *               "could be 0 or 1" (Sec. 2.2).  A cell's 4-value function is
 *               therefore the common Boolean value over every 0/1 completion
 *               of its X/Z inputs, X when completions disagree; this
 *               reproduces Table 1 for AND/OR/XOR.  Cells never output Z.
 *   delays      chosen by triggering input pin and output value (Sec. 2.3);
 *               simultaneous input changes take the minimum delay over the
 *               changed pins (Sec. 2.3, Fig. 5).  Output value 1 uses the
 *               arc's rise delay, 0 its fall delay, X the smaller of both.
 *   evaluation  Algorithm 2: all inputs start at X; the input waveforms are
 *               merged by earliest timestamp, all transitions at one time
 *               are applied together, and when the cell value changes a
 *               scheduled transition (t_d = t, t_r = t + delay) is produced.
 *   cancelling  Eq. 1 ("glitch eaten"): a new scheduled transition denies
 *               every earlier-determined one with t_r' >= t_r; a surviving
 *               transition equal to the value before it is dropped (Fig. 6).
 *
 * Readings where the paper is silent (also listed in the design notes):
 * only pins with a transition at t enter the delay minimum (an X<->Z
 * transition counts); that pin set is per timestamp; ties t_r = t_r' are
 * denied (Eq. 1 uses <=); delays are >= 1; no truncation at the window end.
 *
 * Parity pins: the test suite checks these functions against Table 1, the
 * worked examples of Fig. 5 and Fig. 6, brute force over small candidate
 * sequences, closed forms of BUF/INV chains, static settle-time evaluation,
 * and the agreement of the two independent whole-netlist simulators below.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define VX 2
#define VZ 3
#define INF64 INT64_MAX

enum { C_INV, C_BUF, C_AND2, C_OR2, C_NAND2, C_NOR2, C_XOR2, C_XNOR2, C_MUX2, C_AOI21, C_OAI21, C_NCELLS };

int oracle_arity(int type) {
    static const int ar[C_NCELLS] = {1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3};
    return (type >= 0 && type < C_NCELLS) ? ar[type] : -1;
}

/* Boolean (2-value) function of each cell, pins a, b, c. */
int oracle_cell_bool(int type, int a, int b, int c) {
    switch (type) {
    case C_INV: return !a;
    case C_BUF: return a;
    case C_AND2: return a & b;
    case C_OR2: return a | b;
    case C_NAND2: return !(a & b);
    case C_NOR2: return !(a | b);
    case C_XOR2: return a ^ b;
    case C_XNOR2: return !(a ^ b);
    case C_MUX2: return c ? b : a;          /* pins a, b, s: s selects b */
    case C_AOI21: return !((a & b) | c);
    case C_OAI21: return !((a | b) & c);
    }
    return -1;
}

/* 4-value cell function by completion (Sec. 2.2). */
int oracle_cell_eval(int type, const uint8_t *in) {
    int k = oracle_arity(type), x[3] = {0, 0, 0}, unk[3] = {0, 0, 0}, nunk = 0;
    for (int p = 0; p < k; p++) {
        if (in[p] == 0 || in[p] == 1) x[p] = in[p];
        else unk[nunk++] = p;                     /* X, and Z read as X */
    }
    int result = -1;
    for (int m = 0; m < (1 << nunk); m++) {
        for (int j = 0; j < nunk; j++) x[unk[j]] = (m >> j) & 1;
        int r = oracle_cell_bool(type, x[0], x[1], x[2]);
        if (result < 0) result = r;
        else if (result != r) return VX;
    }
    return result;
}

/* Full 4^k table of a cell, index = sum in[p] * 4^p. */
void oracle_cell_lut(int type, uint8_t *lut) {
    int k = oracle_arity(type), n = 1 << (2 * k);
    for (int i = 0; i < n; i++) {
        uint8_t in[3] = {(uint8_t)(i & 3), (uint8_t)((i >> 2) & 3), (uint8_t)((i >> 4) & 3)};
        lut[i] = (uint8_t)oracle_cell_eval(type, in);
    }
}

/* Arc delay toward output value v (Sec. 2.3): rise to 1, fall to 0, min to X. */
int64_t oracle_delay(int64_t rise, int64_t fall, int v) {
    if (v == 1) return rise;
    if (v == 0) return fall;
    return rise < fall ? rise : fall;
}

/*
 * Algorithm 2, candidate part: merge the k input waveforms by earliest
 * timestamp and produce the scheduled transitions (t_d, t_r, value), one per
 * timestamp at which the cell value changes.  Returns the count.
 */
int64_t oracle_gate_candidates(int type, const int64_t *const *in_t, const uint8_t *const *in_v,
                               const int64_t *in_n, const int64_t *rise, const int64_t *fall,
                               int64_t *cd_td, int64_t *cd_tr, uint8_t *cd_v) {
    int k = oracle_arity(type);
    uint8_t cur[3] = {VX, VX, VX};
    int64_t idx[3] = {0, 0, 0}, n = 0;
    int F = VX;                                   /* the cell value before any input event */
    for (;;) {
        int64_t t = INF64;
        for (int p = 0; p < k; p++)
            if (idx[p] < in_n[p] && in_t[p][idx[p]] < t) t = in_t[p][idx[p]];
        if (t == INF64) break;
        int changed[3] = {0, 0, 0};
        for (int p = 0; p < k; p++) {
            if (idx[p] < in_n[p] && in_t[p][idx[p]] == t) {
                cur[p] = in_v[p][idx[p]];
                idx[p]++;
                changed[p] = 1;
            }
        }
        int nF = oracle_cell_eval(type, cur);
        if (nF != F) {
            int64_t d = INF64;
            for (int p = 0; p < k; p++) {
                if (!changed[p]) continue;
                int64_t dp = oracle_delay(rise[p], fall[p], nF);
                if (dp < d) d = dp;
            }
            cd_td[n] = t; cd_tr[n] = t + d; cd_v[n] = (uint8_t)nF; n++;
        }
        F = nF;
    }
    return n;
}

/*
 * Eq. 1 in sequential form.  The list S of kept transitions is strictly
 * increasing in t_r (each push follows the removal of every element with
 * t_r' >= t_r), so "every earlier one with t_r' >= t_r" is a suffix of S.
 * After the removal the new transition is dropped when it equals the value
 * S ends with (X when S is empty), as in Fig. 6.
 */
int64_t oracle_cancel_stack(int64_t n, const int64_t *td, const int64_t *tr, const uint8_t *v,
                            int64_t *out_t, uint8_t *out_v) {
    int64_t m = 0;
    (void)td; /* candidates arrive in increasing t_d, so t_d > t_d' holds for all kept ones */
    for (int64_t i = 0; i < n; i++) {
        while (m > 0 && out_t[m - 1] >= tr[i]) m--;
        int last = m > 0 ? out_v[m - 1] : VX;
        if (v[i] != last) { out_t[m] = tr[i]; out_v[m] = v[i]; m++; }
    }
    return m;
}

/*
 * Eq. 1 in scan form: candidate i survives iff t_r(i) < t_r(j) for every
 * later j; then a survivor equal to the survivor before it (X before the
 * first) is dropped.  The tests check that this equals the stack form.
 */
int64_t oracle_cancel_scan(int64_t n, const int64_t *tr, const uint8_t *v, int64_t *out_t, uint8_t *out_v) {
    uint8_t *surv = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    int64_t sufmin = INF64, m = 0;
    for (int64_t i = n - 1; i >= 0; i--) {
        surv[i] = tr[i] < sufmin;
        if (tr[i] < sufmin) sufmin = tr[i];
    }
    int last = VX;
    for (int64_t i = 0; i < n; i++) {
        if (!surv[i]) continue;
        if (v[i] != last) { out_t[m] = tr[i]; out_v[m] = v[i]; m++; }
        last = v[i];
    }
    free(surv);
    return m;
}

/* One gate: Algorithm 2 followed by the Eq. 1 stack.  Scratch must hold
   sum(in_n) candidates; returns the number of output transitions. */
int64_t oracle_eval_gate(int type, const int64_t *const *in_t, const uint8_t *const *in_v, const int64_t *in_n,
                         const int64_t *rise, const int64_t *fall, int64_t *scratch_td, int64_t *scratch_tr,
                         uint8_t *scratch_v, int64_t *out_t, uint8_t *out_v) {
    int64_t nc = oracle_gate_candidates(type, in_t, in_v, in_n, rise, fall, scratch_td, scratch_tr, scratch_v);
    return oracle_cancel_stack(nc, scratch_td, scratch_tr, scratch_v, out_t, out_v);
}

/* ------------------------------------------------------------------ */
/* whole-netlist results                                               */
typedef struct {
    int64_t n_nets, n_events;
    int64_t *off;   /* [n_nets+1] */
    int64_t *t;     /* [n_events] */
    uint8_t *v;     /* [n_events] */
} oracle_result;

int64_t oracle_result_nevents(const oracle_result *r) { return r->n_events; }
int64_t oracle_result_nnets(const oracle_result *r) { return r->n_nets; }
void oracle_result_copy(const oracle_result *r, int64_t *off, int64_t *t, uint8_t *v) {
    memcpy(off, r->off, sizeof(int64_t) * (size_t)(r->n_nets + 1));
    memcpy(t, r->t, sizeof(int64_t) * (size_t)r->n_events);
    memcpy(v, r->v, (size_t)r->n_events);
}
void oracle_result_free(oracle_result *r) {
    if (!r) return;
    free(r->off); free(r->t); free(r->v); free(r);
}

/* per-net growable waveform */
typedef struct { int64_t *t; uint8_t *v; int64_t n, cap; } wave_t;
static int wave_push(wave_t *w, int64_t t, uint8_t v) {
    if (w->n == w->cap) {
        int64_t nc = w->cap ? w->cap * 2 : 8;
        int64_t *nt = (int64_t *)realloc(w->t, sizeof(int64_t) * (size_t)nc);
        uint8_t *nv = (uint8_t *)realloc(w->v, (size_t)nc);
        if (!nt || !nv) { if (nt) w->t = nt; if (nv) w->v = nv; return -1; }
        w->t = nt; w->v = nv; w->cap = nc;
    }
    w->t[w->n] = t; w->v[w->n] = v; w->n++;
    return 0;
}
static oracle_result *assemble(wave_t *w, int64_t N) {
    oracle_result *r = (oracle_result *)calloc(1, sizeof(oracle_result));
    if (!r) return NULL;
    r->n_nets = N;
    r->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    int64_t tot = 0;
    for (int64_t n = 0; n < N; n++) tot += w[n].n;
    r->n_events = tot;
    r->t = (int64_t *)malloc(sizeof(int64_t) * (size_t)(tot > 0 ? tot : 1));
    r->v = (uint8_t *)malloc((size_t)(tot > 0 ? tot : 1));
    if (!r->off || !r->t || !r->v) { oracle_result_free(r); return NULL; }
    int64_t o = 0;
    for (int64_t n = 0; n < N; n++) {
        r->off[n] = o;
        if (w[n].n) {
            memcpy(r->t + o, w[n].t, sizeof(int64_t) * (size_t)w[n].n);
            memcpy(r->v + o, w[n].v, (size_t)w[n].n);
        }
        o += w[n].n;
    }
    r->off[N] = o;
    return r;
}
static void free_waves(wave_t *w, int64_t N) {
    if (!w) return;
    for (int64_t n = 0; n < N; n++) { free(w[n].t); free(w[n].v); }
    free(w);
}

/* fanout lists of every net (gate, pin) */
typedef struct { int64_t *off; int32_t *gate; int8_t *pin; } fanout_t;
static int build_fanout(int32_t n_pi, int32_t G, const int32_t *fanin_off, const int32_t *fanin_net, fanout_t *fo) {
    int64_t N = (int64_t)n_pi + G, A = fanin_off[G];
    fo->off = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    fo->gate = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A > 0 ? A : 1));
    fo->pin = (int8_t *)malloc((size_t)(A > 0 ? A : 1));
    if (!fo->off || !fo->gate || !fo->pin) return -1;
    for (int64_t a = 0; a < A; a++) fo->off[fanin_net[a] + 1]++;
    for (int64_t n = 0; n < N; n++) fo->off[n + 1] += fo->off[n];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (!fill) return -1;
    memcpy(fill, fo->off, sizeof(int64_t) * (size_t)(N + 1));
    for (int32_t g = 0; g < G; g++)
        for (int32_t a = fanin_off[g]; a < fanin_off[g + 1]; a++) {
            int64_t s = fill[fanin_net[a]]++;
            fo->gate[s] = g; fo->pin[s] = (int8_t)(a - fanin_off[g]);
        }
    free(fill);
    return 0;
}
static void free_fanout(fanout_t *fo) { free(fo->off); free(fo->gate); free(fo->pin); }

/* Netlist sanity shared by the simulators below: arity matches the cell,
   net ids in range, delays >= 1.  Returns 0 or a negative code. */
static int check_netlist(int32_t n_pi, int32_t G, const uint8_t *type, const int32_t *fanin_off,
                         const int32_t *fanin_net, const int32_t *d_rise, const int32_t *d_fall) {
    int64_t N = (int64_t)n_pi + G;
    if (n_pi < 0 || G < 0 || fanin_off[0] != 0) return -1;
    for (int32_t g = 0; g < G; g++) {
        if (oracle_arity(type[g]) != fanin_off[g + 1] - fanin_off[g]) return -1;
        for (int32_t a = fanin_off[g]; a < fanin_off[g + 1]; a++) {
            if (fanin_net[a] < 0 || fanin_net[a] >= N) return -1;
            if (d_rise[a] < 1 || d_fall[a] < 1) return -1;
        }
    }
    return 0;
}

/* Topological order of the gates (Kahn); -2 if the netlist has a cycle. */
static int topo_order(int32_t n_pi, int32_t G, const int32_t *fanin_off, const int32_t *fanin_net,
                      const fanout_t *fo, int32_t *order, int32_t *level) {
    int32_t *need = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    if (!need) return -1;
    int64_t head = 0, tail = 0;
    for (int32_t g = 0; g < G; g++) {
        need[g] = 0;
        for (int32_t a = fanin_off[g]; a < fanin_off[g + 1]; a++) need[g] += fanin_net[a] >= n_pi;
        level[g] = 1;
        if (need[g] == 0) order[tail++] = g;
    }
    while (head < tail) {
        int32_t g = order[head++];
        int64_t n = (int64_t)n_pi + g;
        for (int64_t s = fo->off[n]; s < fo->off[n + 1]; s++) {
            int32_t h = fo->gate[s];
            if (level[h] < level[g] + 1) level[h] = level[g] + 1;
            if (--need[h] == 0) order[tail++] = h;
        }
    }
    free(need);
    return tail == G ? 0 : -2;
}

static void load_pis(wave_t *w, int32_t n_pi, const int64_t *soff, const int64_t *st, const uint8_t *sv) {
    for (int32_t i = 0; i < n_pi; i++)
        for (int64_t e = soff[i]; e < soff[i + 1]; e++) wave_push(&w[i], st[e], sv[e]);
}

/*
 * Whole-netlist simulation, levelized: gates in topological order, each by
 * oracle_eval_gate on its fanin waveforms.  Gates of one level are
 * independent and may be spread over nthreads OpenMP threads.
 */
int oracle_sim_levelized(int32_t n_pi, int32_t G, const uint8_t *type, const int32_t *fanin_off,
                         const int32_t *fanin_net, const int32_t *d_rise, const int32_t *d_fall,
                         const int64_t *soff, const int64_t *st, const uint8_t *sv, int nthreads,
                         oracle_result **out) {
    *out = NULL;
    if (check_netlist(n_pi, G, type, fanin_off, fanin_net, d_rise, d_fall)) return -1;
    int64_t N = (int64_t)n_pi + G;
    fanout_t fo;
    if (build_fanout(n_pi, G, fanin_off, fanin_net, &fo)) return -5;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    wave_t *w = (wave_t *)calloc((size_t)N, sizeof(wave_t));
    if (!order || !level || !w) return -5;
    int rc = topo_order(n_pi, G, fanin_off, fanin_net, &fo, order, level);
    if (rc) { free(order); free(level); free(w); free_fanout(&fo); return rc; }
    load_pis(w, n_pi, soff, st, sv);
    /* Kahn's order is level-monotone only per dependency chain; group by level */
    int32_t maxl = 0;
    for (int32_t g = 0; g < G; g++) if (level[g] > maxl) maxl = level[g];
    int64_t *lstart = (int64_t *)calloc((size_t)maxl + 2, sizeof(int64_t));
    int32_t *bylvl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    for (int32_t g = 0; g < G; g++) lstart[level[g] + 1]++;
    for (int32_t L = 0; L <= maxl; L++) lstart[L + 1] += lstart[L];
    for (int32_t i = 0; i < G; i++) { int32_t g = order[i]; bylvl[lstart[level[g]]++] = g; }
    for (int32_t L = maxl; L >= 1; L--) lstart[L] = lstart[L - 1];
    lstart[0] = 0;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int32_t L = 1; L <= maxl; L++) {
        #pragma omp parallel
        {
            int64_t cap = 0, *td = NULL, *tr = NULL, *ot = NULL; uint8_t *cv = NULL, *ov = NULL;
            #pragma omp for schedule(dynamic, 64)
            for (int64_t i = lstart[L]; i < lstart[L + 1]; i++) {
                int32_t g = bylvl[i];
                int k = oracle_arity(type[g]);
                const int64_t *it[3]; const uint8_t *iv[3]; int64_t in_n[3], ri[3], fa[3], need = 0;
                for (int p = 0; p < k; p++) {
                    int32_t a = fanin_off[g] + p; wave_t *src = &w[fanin_net[a]];
                    it[p] = src->t; iv[p] = src->v; in_n[p] = src->n; need += src->n;
                    ri[p] = d_rise[a]; fa[p] = d_fall[a];
                }
                if (need + 1 > cap) {
                    cap = (need + 1) * 2;
                    td = (int64_t *)realloc(td, sizeof(int64_t) * (size_t)cap);
                    tr = (int64_t *)realloc(tr, sizeof(int64_t) * (size_t)cap);
                    ot = (int64_t *)realloc(ot, sizeof(int64_t) * (size_t)cap);
                    cv = (uint8_t *)realloc(cv, (size_t)cap);
                    ov = (uint8_t *)realloc(ov, (size_t)cap);
                }
                int64_t m = oracle_eval_gate(type[g], it, iv, in_n, ri, fa, td, tr, cv, ot, ov);
                wave_t *dst = &w[n_pi + g];
                dst->t = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
                dst->v = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
                if (!dst->t || !dst->v) { err = 1; continue; }
                memcpy(dst->t, ot, sizeof(int64_t) * (size_t)m);
                memcpy(dst->v, ov, (size_t)m);
                dst->n = dst->cap = m;
            }
            free(td); free(tr); free(ot); free(cv); free(ov);
        }
    }
    free(lstart); free(bylvl); free(order); free(level); free_fanout(&fo);
    if (err) { free_waves(w, N); return -5; }
    *out = assemble(w, N);
    free_waves(w, N);
    return *out ? 0 : -5;
}

/* ------------------------------------------------------------------ */
/* global event-driven simulator                                       */
typedef struct { int64_t t; int64_t id; int32_t who; int8_t kind; } hev_t;  /* kind 0: PI, 1: gate */
typedef struct { hev_t *a; int64_t n, cap; } heap_t;
static int hev_less(const hev_t *x, const hev_t *y) {
    if (x->t != y->t) return x->t < y->t;
    if (x->kind != y->kind) return x->kind < y->kind;
    if (x->who != y->who) return x->who < y->who;
    return x->id < y->id;
}
static int heap_push(heap_t *h, hev_t e) {
    if (h->n == h->cap) {
        int64_t nc = h->cap ? h->cap * 2 : 1024;
        hev_t *na = (hev_t *)realloc(h->a, sizeof(hev_t) * (size_t)nc);
        if (!na) return -1;
        h->a = na; h->cap = nc;
    }
    int64_t i = h->n++;
    h->a[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hev_less(&h->a[i], &h->a[p])) break;
        hev_t tmp = h->a[i]; h->a[i] = h->a[p]; h->a[p] = tmp; i = p;
    }
    return 0;
}
static hev_t heap_pop(heap_t *h) {
    hev_t top = h->a[0];
    h->a[0] = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < h->n && hev_less(&h->a[l], &h->a[s])) s = l;
        if (r < h->n && hev_less(&h->a[r], &h->a[s])) s = r;
        if (s == i) break;
        hev_t tmp = h->a[i]; h->a[i] = h->a[s]; h->a[s] = tmp; i = s;
    }
    return top;
}
/* per-gate pending (scheduled, not yet matured) transitions, increasing t_r */
typedef struct { int64_t *t; uint8_t *v; int64_t *seq; int64_t head, n, cap; } pend_t;
static int pend_push(pend_t *q, int64_t t, uint8_t v, int64_t seq) {
    if (q->head > 0 && q->n == q->cap) {   /* slide down before growing */
        int64_t live = q->n - q->head;
        memmove(q->t, q->t + q->head, sizeof(int64_t) * (size_t)live);
        memmove(q->v, q->v + q->head, (size_t)live);
        memmove(q->seq, q->seq + q->head, sizeof(int64_t) * (size_t)live);
        q->n = live; q->head = 0;
    }
    if (q->n == q->cap) {
        int64_t nc = q->cap ? q->cap * 2 : 4;
        int64_t *nt = (int64_t *)realloc(q->t, sizeof(int64_t) * (size_t)nc);
        uint8_t *nv = (uint8_t *)realloc(q->v, (size_t)nc);
        int64_t *ns = (int64_t *)realloc(q->seq, sizeof(int64_t) * (size_t)nc);
        if (!nt || !nv || !ns) return -1;
        q->t = nt; q->v = nv; q->seq = ns; q->cap = nc;
    }
    q->t[q->n] = t; q->v[q->n] = v; q->seq[q->n] = seq; q->n++;
    return 0;
}

/*
 * Whole-netlist simulation, event-driven: one global time-ordered queue of
 * PI transitions and scheduled gate transitions.  At each time t every
 * transition maturing at t is applied first; then each gate with an input
 * transition at t is evaluated once with all of them applied.  A changed
 * cell value schedules (t + min delay over the pins with a transition at t);
 * the gate's pending transitions with t_r' >= t_r are denied (Eq. 1) and the
 * new one is dropped when it equals the last pending value, or the present
 * output value when nothing is pending.
 */
int oracle_sim_event(int32_t n_pi, int32_t G, const uint8_t *type, const int32_t *fanin_off,
                     const int32_t *fanin_net, const int32_t *d_rise, const int32_t *d_fall,
                     const int64_t *soff, const int64_t *st, const uint8_t *sv, oracle_result **out) {
    *out = NULL;
    if (check_netlist(n_pi, G, type, fanin_off, fanin_net, d_rise, d_fall)) return -1;
    int64_t N = (int64_t)n_pi + G;
    fanout_t fo;
    if (build_fanout(n_pi, G, fanin_off, fanin_net, &fo)) return -5;
    {   /* reject cycles like the levelized form */
        int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
        int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
        int rc = topo_order(n_pi, G, fanin_off, fanin_net, &fo, order, level);
        free(order); free(level);
        if (rc) { free_fanout(&fo); return rc; }
    }
    wave_t *w = (wave_t *)calloc((size_t)N, sizeof(wave_t));
    uint8_t *val = (uint8_t *)malloc((size_t)N);
    int64_t *evt = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    uint8_t *lastF = (uint8_t *)malloc((size_t)(G > 0 ? G : 1));
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G > 0 ? G : 1));
    pend_t *pq = (pend_t *)calloc((size_t)(G > 0 ? G : 1), sizeof(pend_t));
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_pi > 0 ? n_pi : 1));
    int64_t *changed = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int32_t *affected = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    heap_t h = {0};
    int err = 0;
    if (!w || !val || !evt || !lastF || !mark || !pq || !cursor || !changed || !affected) { err = -5; goto done; }
    memset(val, VX, (size_t)N);
    for (int64_t n = 0; n < N; n++) evt[n] = -1;
    memset(lastF, VX, (size_t)(G > 0 ? G : 1));
    for (int32_t g = 0; g < G; g++) mark[g] = -1;
    for (int32_t i = 0; i < n_pi; i++) {
        cursor[i] = soff[i];
        if (soff[i] < soff[i + 1]) { hev_t e = {st[soff[i]], soff[i], i, 0}; if (heap_push(&h, e)) { err = -5; goto done; } }
    }
    int64_t seq = 0;
    while (h.n > 0) {
        int64_t t = h.a[0].t, nch = 0, naff = 0;
        while (h.n > 0 && h.a[0].t == t) {
            hev_t e = heap_pop(&h);
            if (e.kind == 0) {
                int32_t i = e.who;
                int64_t ei = cursor[i]++;
                val[i] = sv[ei]; evt[i] = t;
                if (wave_push(&w[i], t, sv[ei])) { err = -5; goto done; }
                changed[nch++] = i;
                if (cursor[i] < soff[i + 1]) { hev_t nx = {st[cursor[i]], cursor[i], i, 0}; if (heap_push(&h, nx)) { err = -5; goto done; } }
            } else {
                int32_t g = e.who;
                pend_t *q = &pq[g];
                if (q->head >= q->n || q->seq[q->head] != e.id) continue;   /* denied earlier */
                int64_t n = (int64_t)n_pi + g;
                val[n] = q->v[q->head]; evt[n] = t;
                if (wave_push(&w[n], t, q->v[q->head])) { err = -5; goto done; }
                q->head++;
                changed[nch++] = n;
            }
        }
        for (int64_t c = 0; c < nch; c++) {
            int64_t n = changed[c];
            for (int64_t s = fo.off[n]; s < fo.off[n + 1]; s++) {
                int32_t g = fo.gate[s];
                if (mark[g] != t) { mark[g] = t; affected[naff++] = g; }
            }
        }
        for (int64_t a = 0; a < naff; a++) {
            int32_t g = affected[a];
            int k = oracle_arity(type[g]);
            uint8_t in[3] = {VX, VX, VX};
            for (int p = 0; p < k; p++) in[p] = val[fanin_net[fanin_off[g] + p]];
            int F = oracle_cell_eval(type[g], in);
            if (F == lastF[g]) continue;
            lastF[g] = (uint8_t)F;
            int64_t d = INF64;
            for (int p = 0; p < k; p++) {
                int32_t arc = fanin_off[g] + p;
                if (evt[fanin_net[arc]] != t) continue;
                int64_t dp = oracle_delay(d_rise[arc], d_fall[arc], F);
                if (dp < d) d = dp;
            }
            int64_t tr = t + d;
            pend_t *q = &pq[g];
            while (q->n > q->head && q->t[q->n - 1] >= tr) q->n--;          /* Eq. 1 */
            int last = (q->n > q->head) ? q->v[q->n - 1] : val[(int64_t)n_pi + g];
            if (F == last) continue;
            if (pend_push(q, tr, (uint8_t)F, seq)) { err = -5; goto done; }
            hev_t ne = {tr, seq, g, 1};
            seq++;
            if (heap_push(&h, ne)) { err = -5; goto done; }
        }
    }
    *out = assemble(w, N);
    if (!*out) err = -5;
done:
    free_waves(w, N); free(val); free(evt); free(lastF); free(mark);
    if (pq) { for (int32_t g = 0; g < G; g++) { free(pq[g].t); free(pq[g].v); free(pq[g].seq); } free(pq); }
    free(cursor); free(changed); free(affected); free(h.a); free_fanout(&fo);
    return err;
}

/*
 * Static 4-value evaluation with the final PI values (X for a PI without
 * transitions): the value every net settles to once all transitions are in.
 */
int oracle_static_eval(int32_t n_pi, int32_t G, const uint8_t *type, const int32_t *fanin_off,
                       const int32_t *fanin_net, const uint8_t *pi_val, uint8_t *net_val) {
    fanout_t fo;
    if (build_fanout(n_pi, G, fanin_off, fanin_net, &fo)) return -5;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    int rc = topo_order(n_pi, G, fanin_off, fanin_net, &fo, order, level);
    if (rc == 0) {
        memcpy(net_val, pi_val, (size_t)n_pi);
        for (int32_t i = 0; i < G; i++) {
            int32_t g = order[i];
            uint8_t in[3] = {VX, VX, VX};
            for (int p = 0; p < oracle_arity(type[g]); p++) in[p] = net_val[fanin_net[fanin_off[g] + p]];
            net_val[n_pi + g] = (uint8_t)oracle_cell_eval(type[g], in);
        }
    }
    free(order); free(level); free_fanout(&fo);
    return rc;
}

/*
 * Local check of a full simulation result given as a CSR over all nets
 * (off[n_pi+G+1], times t, values v): every gate g in [g0, g1) must carry
 * exactly oracle_eval_gate of its fanin waveforms as found in the result.
 * Together with the PI waveforms equalling the stimulus this pins the whole
 * result, by induction over any topological order.  Returns the number of
 * mismatching gates and the first one in *first_bad (-1 if none).
 */
int64_t oracle_check_gates(int32_t n_pi, int32_t G, const uint8_t *type, const int32_t *fanin_off,
                           const int32_t *fanin_net, const int32_t *d_rise, const int32_t *d_fall,
                           const int64_t *off, const int64_t *t, const uint8_t *v,
                           int32_t g0, int32_t g1, int nthreads, int64_t *first_bad) {
    int64_t bad = 0, first = INT64_MAX;
    (void)G;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel reduction(+:bad)
    {
        int64_t cap = 0, *buf = NULL, *td = NULL, *tr = NULL, *ot = NULL; uint8_t *cv = NULL, *ov = NULL;
        int64_t myfirst = INT64_MAX;
        #pragma omp for schedule(dynamic, 256)
        for (int32_t g = g0; g < g1; g++) {
            int k = oracle_arity(type[g]);
            int64_t need = 0, in_n[3], ri[3], fa[3];
            for (int p = 0; p < k; p++) {
                int32_t n = fanin_net[fanin_off[g] + p];
                in_n[p] = off[n + 1] - off[n]; need += in_n[p];
            }
            if (need + 1 > cap) {
                cap = (need + 1) * 2;
                buf = (int64_t *)realloc(buf, sizeof(int64_t) * (size_t)cap);
                td = (int64_t *)realloc(td, sizeof(int64_t) * (size_t)cap);
                tr = (int64_t *)realloc(tr, sizeof(int64_t) * (size_t)cap);
                ot = (int64_t *)realloc(ot, sizeof(int64_t) * (size_t)cap);
                cv = (uint8_t *)realloc(cv, (size_t)cap);
                ov = (uint8_t *)realloc(ov, (size_t)cap);
            }
            const int64_t *it[3]; const uint8_t *iv[3];
            int64_t o = 0;
            for (int p = 0; p < k; p++) {
                int32_t a = fanin_off[g] + p, n = fanin_net[a];
                for (int64_t e = 0; e < in_n[p]; e++) buf[o + e] = t[off[n] + e];
                it[p] = buf + o; iv[p] = v + off[n]; o += in_n[p];
                ri[p] = d_rise[a]; fa[p] = d_fall[a];
            }
            int64_t m = oracle_eval_gate(type[g], it, iv, in_n, ri, fa, td, tr, cv, ot, ov);
            int64_t n = (int64_t)n_pi + g, got = off[n + 1] - off[n];
            int ok = (got == m);
            for (int64_t e = 0; ok && e < m; e++)
                ok = (ot[e] == (int64_t)t[off[n] + e]) && (ov[e] == v[off[n] + e]);
            if (!ok) { bad++; if (g < myfirst) myfirst = g; }
        }
        #pragma omp critical
        { if (myfirst < first) first = myfirst; }
        free(buf); free(td); free(tr); free(ot); free(cv); free(ov);
    }
    *first_bad = (first == INT64_MAX) ? -1 : first;
    return bad;
}

/* ------------------------------------------------------------------ */
/* Cells with the full delay matrix, several outputs and user tables   */
/*
 * Sec. 3 ("Delay") keeps delays in a five-dimensional matrix indexed by
 * cell, input pin, output pin, edge of the input transition and value of
 * the output transition, an entry without an arc being infinite; for an
 * output k that changes at t, Algorithm 2 takes the minimum of
 * Delay[i][k][e_i][o_k] over the inputs.  Sec. 3 ("Module Function") builds
 * every cell, user-defined primitives included, from a logic function per
 * output.  Here a cell has n_in inputs (1..3) and n_out outputs; output o
 * has a 4-value table lut[o][sum v_p 4^p] with values 0, 1, X, and delays
 * D[p][o][edge][value] (edge 0 = rising, 1 = falling; value 0 = the output
 * falls to 0, 1 = it rises to 1), -1 where pin p has no arc to output o.
 *
 * Readings (the paper leaves these open):
 *   - the edge of an input transition follows Verilog's posedge / negedge
 *     classes: rising = 0->1, 0->X, 0->Z, X->1, Z->1; falling = 1->0, 1->X,
 *     1->Z, X->0, Z->0; X<->Z is neither and takes the smaller delay of the
 *     two edges;
 *   - an output changing to X takes the smaller of its value-0 and value-1
 *     delays (as the rise/fall arcs above);
 *   - as above, only pins with a transition at t enter the minimum, and the
 *     output is X before its first transition whatever the table gives for
 *     all-X inputs (Algorithm 2 starts the outputs unknown);
 *   - when none of the pins that changed at t has an arc to the output (a
 *     user table can change value through a pin without an arc, e.g. from
 *     the initial X), the output takes the smallest delay of all its arcs
 *     toward the new value;
 *   - the outputs of one cell are scheduled and cancelled (Eq. 1) each on
 *     its own, since Algorithm 2 keeps one output waveform per output pin.
 */
#define EDGE_RISE 0
#define EDGE_FALL 1
#define EDGE_NONE 2

int oracle_edge_class(int old, int nw) {
    if (old == nw) return -1;
    if (nw == 1 || old == 0) return EDGE_RISE;   /* to 1, or up from 0 */
    if (nw == 0 || old == 1) return EDGE_FALL;   /* to 0, or down from 1 */
    return EDGE_NONE;                            /* X <-> Z */
}

/* Delay of one pin's transition of class `edge` toward output value v;
   D4 = that pin's [edge][value] entries for the output, -1 = no arc. */
int64_t oracle_arc_delay4(const int64_t *D4, int edge, int v) {
    int64_t d = INF64;
    for (int e = 0; e < 2; e++) {
        if (edge != EDGE_NONE && e != edge) continue;
        for (int val = 0; val < 2; val++) {
            if (v != VX && val != v) continue;
            int64_t x = D4[2 * e + val];
            if (x >= 0 && x < d) d = x;
        }
    }
    return d;
}

/*
 * Algorithm 2 for one output of a cell: lut = that output's 4^n_in table,
 * D = the output's delays, D[p * 4 + edge * 2 + value].  Candidates as in
 * oracle_gate_candidates; returns the count, or -1 if the output has no arc
 * at all.
 */
int64_t oracle_cell_candidates(int n_in, const uint8_t *lut, const int64_t *D, const int64_t *const *in_t,
                               const uint8_t *const *in_v, const int64_t *in_n, int64_t *cd_td, int64_t *cd_tr,
                               uint8_t *cd_v) {
    uint8_t cur[3] = {VX, VX, VX};
    int64_t idx[3] = {0, 0, 0}, n = 0;
    int F = VX;                                   /* the output before any input event */
    for (;;) {
        int64_t t = INF64;
        for (int p = 0; p < n_in; p++)
            if (idx[p] < in_n[p] && in_t[p][idx[p]] < t) t = in_t[p][idx[p]];
        if (t == INF64) break;
        int edge[3] = {-1, -1, -1};
        for (int p = 0; p < n_in; p++) {
            if (idx[p] < in_n[p] && in_t[p][idx[p]] == t) {
                uint8_t nv = in_v[p][idx[p]];
                edge[p] = oracle_edge_class(cur[p], nv);
                cur[p] = nv;
                idx[p]++;
            }
        }
        int li = 0;
        for (int p = n_in - 1; p >= 0; p--) li = li * 4 + cur[p];
        int nF = lut[li];
        if (nF != F) {
            int64_t d = INF64;
            for (int p = 0; p < n_in; p++) {
                if (edge[p] < 0) continue;
                int64_t dp = oracle_arc_delay4(D + 4 * p, edge[p], nF);
                if (dp < d) d = dp;
            }
            if (d == INF64)   /* no changed pin has an arc: the fastest arc of the output */
                for (int p = 0; p < n_in; p++) {
                    int64_t dp = oracle_arc_delay4(D + 4 * p, EDGE_NONE, nF);
                    if (dp < d) d = dp;
                }
            if (d == INF64) return -1;
            cd_td[n] = t; cd_tr[n] = t + d; cd_v[n] = (uint8_t)nF; n++;
        }
        F = nF;
    }
    return n;
}

/*
 * Whole netlist of such cells, evaluated cell by cell once all fanin nets
 * are known (Kahn order).  Nets: 0..n_pi-1 primary inputs, then the outputs
 * of cell 0, cell 1, ... in order.  Cell c: inputs fanin_net[fanin_off[c]..
 * fanin_off[c+1]) (n_in = that count), n_out[c] outputs, tables at
 * luts[lut_off[c] + o * 4^n_in], delays at delays[delay_off[c] +
 * ((p * n_out + o) * 2 + edge) * 2 + value].  Returns 0, -1 for a bad
 * netlist, -2 for a cycle, -3 for a changed output without a finite delay,
 * -5 when out of memory.
 */
int oracle_sim_cells(int32_t n_pi, int32_t n_cells, const int32_t *n_out, const uint8_t *luts,
                     const int64_t *lut_off, const int32_t *fanin_off, const int32_t *fanin_net,
                     const int64_t *delays, const int64_t *delay_off, const int64_t *soff, const int64_t *st,
                     const uint8_t *sv, oracle_result **out) {
    *out = NULL;
    int64_t *obase = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cells + 1));
    if (!obase) return -5;
    obase[0] = n_pi;
    for (int32_t c = 0; c < n_cells; c++) {
        int k = fanin_off[c + 1] - fanin_off[c];
        if (k < 1 || k > 3 || n_out[c] < 1) { free(obase); return -1; }
        obase[c + 1] = obase[c] + n_out[c];
    }
    const int64_t N = obase[n_cells];
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));  /* net -> cell, -1 = PI */
    int32_t *need = (int32_t *)calloc((size_t)(n_cells > 0 ? n_cells : 1), sizeof(int32_t));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cells > 0 ? n_cells : 1));
    wave_t *w = (wave_t *)calloc((size_t)(N > 0 ? N : 1), sizeof(wave_t));
    if (!owner || !need || !queue || !w) return -5;
    for (int64_t q = 0; q < n_pi; q++) owner[q] = -1;
    for (int32_t c = 0; c < n_cells; c++)
        for (int64_t q = obase[c]; q < obase[c + 1]; q++) owner[q] = c;
    /* readers of each cell, for Kahn's algorithm */
    int64_t *roff = (int64_t *)calloc((size_t)n_cells + 1, sizeof(int64_t));
    int32_t *rd = (int32_t *)malloc(sizeof(int32_t) * (size_t)(fanin_off[n_cells] > 0 ? fanin_off[n_cells] : 1));
    for (int32_t c = 0; c < n_cells; c++)
        for (int32_t a = fanin_off[c]; a < fanin_off[c + 1]; a++) {
            int32_t net = fanin_net[a];
            if (net < 0 || net >= N) { free(obase); return -1; }
            if (owner[net] >= 0) { roff[owner[net] + 1]++; need[c]++; }
        }
    for (int32_t c = 0; c < n_cells; c++) roff[c + 1] += roff[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cells + 1));
    memcpy(fill, roff, sizeof(int64_t) * (size_t)(n_cells + 1));
    for (int32_t c = 0; c < n_cells; c++)
        for (int32_t a = fanin_off[c]; a < fanin_off[c + 1]; a++)
            if (owner[fanin_net[a]] >= 0) rd[fill[owner[fanin_net[a]]]++] = c;
    load_pis(w, n_pi, soff, st, sv);
    int32_t head = 0, tail = 0;
    for (int32_t c = 0; c < n_cells; c++) if (need[c] == 0) queue[tail++] = c;
    int rc = 0;
    int64_t cap = 0, *td = NULL, *tr = NULL, *ot = NULL; uint8_t *cv = NULL, *ov = NULL;
    while (head < tail && rc == 0) {
        int32_t c = queue[head++];
        int k = fanin_off[c + 1] - fanin_off[c];
        const int64_t *it[3]; const uint8_t *iv[3]; int64_t in_n[3], tot = 0;
        for (int p = 0; p < k; p++) {
            wave_t *src = &w[fanin_net[fanin_off[c] + p]];
            it[p] = src->t; iv[p] = src->v; in_n[p] = src->n; tot += src->n;
        }
        if (tot + 1 > cap) {
            cap = (tot + 1) * 2;
            td = (int64_t *)realloc(td, sizeof(int64_t) * (size_t)cap);
            tr = (int64_t *)realloc(tr, sizeof(int64_t) * (size_t)cap);
            ot = (int64_t *)realloc(ot, sizeof(int64_t) * (size_t)cap);
            cv = (uint8_t *)realloc(cv, (size_t)cap);
            ov = (uint8_t *)realloc(ov, (size_t)cap);
        }
        const int nl = 1 << (2 * k);
        for (int o = 0; o < n_out[c]; o++) {
            int64_t D[12];
            for (int p = 0; p < k; p++)
                for (int j = 0; j < 4; j++) D[4 * p + j] = delays[delay_off[c] + ((int64_t)p * n_out[c] + o) * 4 + j];
            int64_t nc = oracle_cell_candidates(k, luts + lut_off[c] + (int64_t)o * nl, D, it, iv, in_n, td, tr, cv);
            if (nc < 0) { rc = -3; break; }
            int64_t m = oracle_cancel_stack(nc, td, tr, cv, ot, ov);
            wave_t *dst = &w[obase[c] + o];
            dst->t = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
            dst->v = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
            if (!dst->t || !dst->v) { rc = -5; break; }
            memcpy(dst->t, ot, sizeof(int64_t) * (size_t)m);
            memcpy(dst->v, ov, (size_t)m);
            dst->n = dst->cap = m;
        }
        for (int64_t s = roff[c]; s < roff[c + 1]; s++)
            if (--need[rd[s]] == 0) queue[tail++] = rd[s];
    }
    if (rc == 0 && tail != n_cells) rc = -2;
    free(td); free(tr); free(ot); free(cv); free(ov);
    free(obase); free(owner); free(need); free(queue); free(roff); free(rd); free(fill);
    if (rc) { free_waves(w, N); return rc; }
    *out = assemble(w, N);
    free_waves(w, N);
    return *out ? 0 : -5;
}
