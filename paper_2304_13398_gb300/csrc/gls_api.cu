// gls_api.cu -- host side of libgls.so: validation, levelization, device
// layout, run graphs and read-back.  Every entry point declared in gls.h is
// defined here; no exception crosses the C boundary.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gls_internal.h"
#include "../../include/gls.h"

using namespace gls;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(GLS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr int kArity[GLS_NCELLS] = {1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3};
constexpr int32_t kMaxDelay = 1 << 29;

// ---- 4-value cell tables -------------------------------------------------
// Each cell is written as the disjunction of all its prime implicants; Kleene
// evaluation of that cover (AND: 0 if a literal is 0, 1 if all are 1, else X;
// OR: 1 if a term is 1, 0 if all are 0, else X) gives 1 exactly when every
// 0/1 completion of the unknown inputs gives 1, and 0 exactly when every
// completion gives 0 -- the reading of X as "either 0 or 1" of Sec. 2.2.
// Literal per pin: +1 the pin, -1 its complement, 0 absent.
struct Cover { int nterms; int8_t lit[3][3]; };
const Cover kCovers[GLS_NCELLS] = {
    {1, {{-1, 0, 0}}},                              // INV   !a
    {1, {{+1, 0, 0}}},                              // BUF   a
    {1, {{+1, +1, 0}}},                             // AND2  ab
    {2, {{+1, 0, 0}, {0, +1, 0}}},                  // OR2   a + b
    {2, {{-1, 0, 0}, {0, -1, 0}}},                  // NAND2 !a + !b
    {1, {{-1, -1, 0}}},                             // NOR2  !a!b
    {2, {{+1, -1, 0}, {-1, +1, 0}}},                // XOR2  a!b + !ab
    {2, {{+1, +1, 0}, {-1, -1, 0}}},                // XNOR2 ab + !a!b
    {3, {{+1, 0, -1}, {0, +1, +1}, {+1, +1, 0}}},   // MUX2  a!c + bc + ab
    {2, {{-1, 0, -1}, {0, -1, -1}}},                // AOI21 !a!c + !b!c
    {2, {{-1, -1, 0}, {0, 0, -1}}},                 // OAI21 !a!b + !c
};

int kleene_cover(const Cover &c, const int in[3]) {
    int any_x = 0;
    for (int t = 0; t < c.nterms; t++) {
        int term = 1;  // 1, 0 or 2 (X)
        for (int p = 0; p < 3; p++) {
            if (!c.lit[t][p]) continue;
            int v = in[p];                         // 0, 1 or 2
            if (v != 2 && c.lit[t][p] < 0) v = 1 - v;
            if (v == 0) { term = 0; break; }
            if (v == 2) term = 2;
        }
        if (term == 1) return 1;
        if (term == 2) any_x = 1;
    }
    return any_x ? 2 : 0;
}

void build_luts(uint64_t lut[GLS_NCELLS][2]) {
    for (int c = 0; c < GLS_NCELLS; c++) {
        lut[c][0] = lut[c][1] = 0;
        for (int idx = 0; idx < 64; idx++) {
            int in[3];
            for (int p = 0; p < 3; p++) {
                int v = (idx >> (2 * p)) & 3;
                in[p] = v == 3 ? 2 : v;            // Z is read as X
            }
            uint64_t f = (uint64_t)kleene_cover(kCovers[c], in);
            lut[c][idx >> 5] |= f << (2 * (idx & 31));
        }
    }
}

// ---- host netlist analysis ------------------------------------------------
struct Levelized {
    int32_t depth = 0;
    std::vector<int32_t> level;        // per external gate
    std::vector<int32_t> order;        // internal position -> external gate
    std::vector<int32_t> pos;          // external gate -> internal position
    std::vector<int32_t> level_begin;  // [depth+2], gates of level L at [level_begin[L], level_begin[L+1])
    int64_t max_path_delay = 0;
};

// Per-arc delays of the general form: d4[a * 4 + edge * 2 + value] (edge 0
// rising, 1 falling; value 0 the output falls, 1 it rises); all four -1 for
// a pin without an arc.
int check_arcs(int32_t n_pi, int32_t G, const int32_t *fanin_off, const int32_t *fanin_net, const int32_t *d4) {
    if (n_pi < 0 || G < 0) return fail(GLS_EINVAL, "negative n_pi or n_gates");
    if (G > 0 && (!fanin_off || !fanin_net || !d4)) return fail(GLS_EINVAL, "NULL netlist array");
    if ((int64_t)n_pi + G >= (int64_t)INT32_MAX) return fail(GLS_EINVAL, "too many nets");
    const int64_t N = (int64_t)n_pi + G;
    if (G > 0 && fanin_off[0] != 0) return fail(GLS_EINVAL, "fanin_off[0] must be 0");
    for (int32_t g = 0; g < G; g++) {
        const int32_t k = fanin_off[g + 1] - fanin_off[g];
        if (k < 1 || k > 3) return fail(GLS_EINVAL, "gate %d: %d input pins (1..3 supported)", g, k);
        int32_t lo = INT32_MAX, hi = 0, arcs = 0;
        for (int32_t a = fanin_off[g]; a < fanin_off[g + 1]; a++) {
            if (fanin_net[a] < 0 || fanin_net[a] >= N) return fail(GLS_EINVAL, "gate %d: net %d out of range", g, fanin_net[a]);
            if (fanin_net[a] == n_pi + g) return fail(GLS_ECYCLE, "gate %d reads its own output", g);
            const int32_t *d = d4 + 4 * (int64_t)a;
            const bool none = d[0] == -1 && d[1] == -1 && d[2] == -1 && d[3] == -1;
            if (none) continue;
            arcs++;
            for (int j = 0; j < 4; j++) {
                if (d[j] < 1 || d[j] >= kMaxDelay)
                    return fail(GLS_EINVAL, "gate %d pin %d: delay %d out of [1, 2^29) (all four -1 = no arc)", g,
                                a - fanin_off[g], d[j]);
                lo = std::min(lo, d[j]);
                hi = std::max(hi, d[j]);
            }
        }
        if (arcs == 0) return fail(GLS_EINVAL, "gate %d: no pin has an arc to the output", g);
        if (hi - lo > GLS_MAX_DELAY_SPREAD)
            return fail(GLS_ERANGE, "gate %d: delay spread %d exceeds %d", g, hi - lo, GLS_MAX_DELAY_SPREAD);
    }
    return GLS_OK;
}

// The classic form -- a built-in cell per gate, rise/fall per arc for both
// input edges -- checked and put in the general per-arc layout.
int classic_arcs(int32_t n_pi, int32_t G, const uint8_t *type, const int32_t *fanin_off, const int32_t *fanin_net,
                 const int32_t *d_rise, const int32_t *d_fall, std::vector<int32_t> &d4) {
    if (n_pi < 0 || G < 0) return fail(GLS_EINVAL, "negative n_pi or n_gates");
    if (G > 0 && (!type || !fanin_off || !fanin_net || !d_rise || !d_fall))
        return fail(GLS_EINVAL, "NULL netlist array");
    if (G > 0 && fanin_off[0] != 0) return fail(GLS_EINVAL, "fanin_off[0] must be 0");
    for (int32_t g = 0; g < G; g++) {
        if (type[g] >= GLS_NCELLS) return fail(GLS_EINVAL, "gate %d: unknown cell %d", g, type[g]);
        if (fanin_off[g + 1] - fanin_off[g] != kArity[type[g]])
            return fail(GLS_EINVAL, "gate %d: %d fanins for a %d-pin cell", g, fanin_off[g + 1] - fanin_off[g],
                        kArity[type[g]]);
        for (int32_t a = fanin_off[g]; a < fanin_off[g + 1]; a++)
            if (d_rise[a] < 1 || d_fall[a] < 1 || d_rise[a] >= kMaxDelay || d_fall[a] >= kMaxDelay)
                return fail(GLS_EINVAL, "gate %d: delay out of [1, 2^29)", g);
    }
    const int64_t A = G > 0 ? fanin_off[G] : 0;
    d4.resize((size_t)std::max<int64_t>(4 * A, 4));
    for (int64_t a = 0; a < A; a++) {
        d4[4 * a + 0] = d4[4 * a + 2] = d_fall[a];
        d4[4 * a + 1] = d4[4 * a + 3] = d_rise[a];
    }
    return GLS_OK;
}

// Levels, level order and the longest path delay of a checked netlist.
int analyse_netlist(int32_t n_pi, int32_t G, const int32_t *fanin_off, const int32_t *fanin_net, const int32_t *d4,
                    Levelized *out) {
    int rc = check_arcs(n_pi, G, fanin_off, fanin_net, d4);
    if (rc) return rc;
    // Kahn's algorithm over gate->gate arcs; level = 1 + max fanin level
    std::vector<int32_t> need(G, 0), level(G, 1), fo_cnt(G + 1, 0);
    for (int32_t g = 0; g < G; g++)
        for (int32_t a = fanin_off[g]; a < fanin_off[g + 1]; a++)
            if (fanin_net[a] >= n_pi) { need[g]++; fo_cnt[fanin_net[a] - n_pi + 1]++; }
    for (int32_t g = 0; g < G; g++) fo_cnt[g + 1] += fo_cnt[g];
    std::vector<int32_t> fo(fo_cnt[G]), fill(fo_cnt.begin(), fo_cnt.end() - 1);
    for (int32_t g = 0; g < G; g++)
        for (int32_t a = fanin_off[g]; a < fanin_off[g + 1]; a++)
            if (fanin_net[a] >= n_pi) fo[fill[fanin_net[a] - n_pi]++] = g;
    std::vector<int32_t> queue;
    queue.reserve(G);
    for (int32_t g = 0; g < G; g++) if (need[g] == 0) queue.push_back(g);
    for (size_t h = 0; h < queue.size(); h++) {
        int32_t g = queue[h];
        for (int32_t s = fo_cnt[g]; s < fo_cnt[g + 1]; s++) {
            int32_t x = fo[s];
            level[x] = std::max(level[x], level[g] + 1);
            if (--need[x] == 0) queue.push_back(x);
        }
    }
    if ((int64_t)queue.size() != G) return fail(GLS_ECYCLE, "netlist has a cycle (%lld gates on or behind it)",
                                                (long long)(G - (int64_t)queue.size()));
    if (!out) return GLS_OK;
    out->depth = 0;
    for (int32_t g = 0; g < G; g++) out->depth = std::max(out->depth, level[g]);
    out->level_begin.assign(out->depth + 2, 0);
    for (int32_t g = 0; g < G; g++) out->level_begin[level[g] + 1]++;
    for (int32_t L = 0; L <= out->depth; L++) out->level_begin[L + 1] += out->level_begin[L];
    out->order.resize(G);
    out->pos.resize(G);
    std::vector<int32_t> f2(out->level_begin.begin(), out->level_begin.end());
    for (int32_t g = 0; g < G; g++) {
        int32_t p = f2[level[g]]++;
        out->order[p] = g;
        out->pos[g] = p;
    }
    // longest path delay (max over arcs of the largest entry)
    std::vector<int64_t> pd(G, 0);
    int64_t best = 0;
    for (int32_t p = 0; p < G; p++) {
        int32_t g = out->order[p];
        int64_t m = 0;
        for (int32_t a = fanin_off[g]; a < fanin_off[g + 1]; a++) {
            int64_t in = fanin_net[a] >= n_pi ? pd[fanin_net[a] - n_pi] : 0;
            const int32_t *d = d4 + 4 * (int64_t)a;
            m = std::max(m, in + std::max(std::max(d[0], d[1]), std::max(d[2], d[3])));
        }
        pd[g] = m;
        best = std::max(best, m);
    }
    out->max_path_delay = best;
    out->level = std::move(level);
    return GLS_OK;
}

int check_stimulus_host(int32_t n_pi, const int64_t *off, const int32_t *t, const uint8_t *v, bool deep) {
    if (n_pi < 0 || !off) return fail(GLS_EINVAL, "bad stimulus arguments");
    if (off[0] != 0) return fail(GLS_ESTIM, "off[0] must be 0");
    for (int32_t i = 0; i < n_pi; i++)
        if (off[i + 1] < off[i]) return fail(GLS_ESTIM, "off not monotone at PI %d", i);
    if (off[n_pi] > 0 && (!t || !v)) return fail(GLS_EINVAL, "NULL stimulus arrays");
    if (off[n_pi] >= ((int64_t)1 << 32)) return fail(GLS_ESTIM, "more than 2^32 stimulus transitions");
    if (!deep) return GLS_OK;
    for (int32_t i = 0; i < n_pi; i++)
        for (int64_t e = off[i]; e < off[i + 1]; e++) {
            if (t[e] < 0 || (uint32_t)t[e] >= kTimeLimit) return fail(GLS_ESTIM, "PI %d: time %d out of [0, 2^30-1)", i, t[e]);
            if (v[e] > 3) return fail(GLS_ESTIM, "PI %d: value %d", i, v[e]);
            if (e > off[i] && t[e] <= t[e - 1]) return fail(GLS_ESTIM, "PI %d: times not increasing", i);
            if (e > off[i] && v[e] == v[e - 1]) return fail(GLS_ESTIM, "PI %d: repeated value", i);
        }
    return GLS_OK;
}

// The same rules for 64-bit times: 0 <= t < 2^62.
int check_stimulus64_host(int32_t n_pi, const int64_t *off, const int64_t *t, const uint8_t *v, int64_t *max_t) {
    if (n_pi < 0 || !off) return fail(GLS_EINVAL, "bad stimulus arguments");
    if (off[0] != 0) return fail(GLS_ESTIM, "off[0] must be 0");
    for (int32_t i = 0; i < n_pi; i++)
        if (off[i + 1] < off[i]) return fail(GLS_ESTIM, "off not monotone at PI %d", i);
    if (off[n_pi] > 0 && (!t || !v)) return fail(GLS_EINVAL, "NULL stimulus arrays");
    if (off[n_pi] >= ((int64_t)1 << 32)) return fail(GLS_ESTIM, "more than 2^32 stimulus transitions");
    int64_t mx = 0;
    for (int32_t i = 0; i < n_pi; i++)
        for (int64_t e = off[i]; e < off[i + 1]; e++) {
            if (t[e] < 0 || t[e] >= ((int64_t)1 << 62))
                return fail(GLS_ESTIM, "PI %d: time %lld out of [0, 2^62)", i, (long long)t[e]);
            if (v[e] > 3) return fail(GLS_ESTIM, "PI %d: value %d", i, v[e]);
            if (e > off[i] && t[e] <= t[e - 1]) return fail(GLS_ESTIM, "PI %d: times not increasing", i);
            if (e > off[i] && v[e] == v[e - 1]) return fail(GLS_ESTIM, "PI %d: repeated value", i);
            mx = std::max(mx, t[e]);
        }
    *max_t = mx;
    return GLS_OK;
}

// ---- objects --------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct UserCell {
    int32_t n_in = 0, n_out = 0;
    std::vector<uint8_t> tables;       // n_out tables of 4^n_in values
};

struct NetlistObj {
    int32_t n_pi = 0, n_gates = 0;
    bool general = false;              // a record needs the windowed kernels (kGateGeneral)
    Levelized lv;
    GateRec *d_gates = nullptr;
    int32_t *d_ext2int = nullptr;      // [N] caller net id -> internal net id
    std::vector<int32_t> ext2int;      // host copy
    std::vector<GateRec> recs;         // host copy of the level-ordered records (batches)
    int32_t *d_level_begin = nullptr;  // [depth + 2] device copy of lv.level_begin (replicated items)
    GateRec *d_plan = nullptr;         // records in the planned order (dependency schedule), or null
    std::vector<GateRec *> plans;      // every planned copy, kept until the netlist is released
};

struct StimObj {
    int32_t n_pi = 0;
    int64_t n_events = 0, cap_events = 0;
    uint32_t max_time = 0;
    bool wide = false;                 // 64-bit times (gls_load_stimulus64): sliced runs only
    int64_t max_time64 = 0;
    int64_t *d_t64 = nullptr;
    int64_t *d_off = nullptr;
    int32_t *d_t = nullptr;
    uint8_t *d_v = nullptr;
    uint32_t *d_packed = nullptr;
};

// One (netlist, stimulus) instance of a run; its nets occupy the combined
// net ids [net_base, net_base + n_pi + n_gates) in internal order.
struct RunItem {
    int32_t netlist_id = 0, stim_id = 0;
    int64_t net_base = 0;
    uint32_t t_limit = kTimeInf;       // stimulus transitions at or after this time are left out
};

struct RunObj {
    std::vector<RunItem> items;
    int64_t n_nets = 0;                 // all instances
    int32_t n_gates = 0;
    int32_t depth = 0;                  // deepest instance
    std::vector<int32_t> level_begin;   // gates of level L at [level_begin[L], level_begin[L+1])
    GateRec *d_gates = nullptr;         // level-ordered records of all instances
    bool owns_gates = false;            // batches own a combined copy
    RunDev dev{};
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    unsigned long long *d_sum = nullptr;
    unsigned long long *d_pi_total = nullptr;
    int64_t *d_off = nullptr;          // [max nets + 1] for read-back
    int64_t off_cap = 0;
    int64_t *d_scan_tmp = nullptr;
    size_t scan_tmp = 0;
    uint32_t *d_gather = nullptr;
    int64_t gather_cap = 0;
    int schedule = 0;
    uint32_t *h_arena = nullptr;        // pinned host mirror of the arena (GLS_OPT_HOST_MIRROR)
    uint32_t *d_glen = nullptr;         // [gates] scratch of gls_read_host
    int64_t glen_cap = 0;
    // time-sliced runs (task division over time)
    int64_t slice_ps = 0;               // 0: not sliced
    int32_t slice_group = 1;            // most slices one launch evaluates
    int32_t launch_slices = 1;          // slices the last launch evaluated (descriptor sets to count)
    uint32_t *d_slice_packed = nullptr; // primary-input transitions of one launch's slices
    uint32_t *d_st[3] = {nullptr, nullptr, nullptr};    // gate state at slice boundaries: a launch's
                                                        // input and the two it alternates between
    uint32_t *d_pend[3] = {nullptr, nullptr, nullptr};  // pending transitions, kPendCap per net
    struct Slice {
        int64_t t0;                     // start of the slice (local time 0)
        std::vector<int64_t> off;       // [n_nets + 1] caller net order
        // slice-local (t << 2) | v, off[n_nets] words: carved from the
        // pinned host pool when the context has one (the copies from the
        // device then run at the link's rate), else ordinary host memory
        // that is not zero-filled first (the copy writes all of it)
        std::unique_ptr<uint32_t[]> heap;
        uint32_t *pinned = nullptr;
        const uint32_t *words() const { return pinned ? pinned : heap.get(); }
    };
    std::vector<Slice> slices;
    int64_t sliced_total = 0, sliced_demand = 0;
    double sliced_ms = 0.0;
};

}  // namespace

// One region carved first-fit into 256-byte aligned blocks.
struct Pool {
    char *base = nullptr;
    uint64_t bytes = 0;
    std::map<uint64_t, uint64_t> free;            // offset -> size of free ranges
    std::unordered_map<void *, uint64_t> allocs;  // block -> size
};

struct gls_ctx {
    int device = 0;
    uint64_t budget = 0, used = 0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    int sm_count = 0;
    LevelCfg cfg{4, 0, kVariantWindowedWide};
    int schedule = GLS_SCHEDULE_DEPENDENCY;
    uint64_t wait_limit_ns = 10ull * 1000 * 1000 * 1000;
    int32_t withhold_gate = -1;
    uint32_t seg_target = 32;
    int32_t slice_group = kMaxSliceGroup;   // GLS_OPT_SLICE_GROUP
    bool host_mirror = false;           // GLS_OPT_HOST_MIRROR
    int32_t next_id = 1;
    std::unordered_map<int32_t, std::unique_ptr<NetlistObj>> netlists;
    std::unordered_map<int32_t, std::unique_ptr<StimObj>> stims;
    std::unordered_map<int32_t, std::unique_ptr<RunObj>> runs;
    std::unordered_map<void *, size_t> allocs;       // cudaMalloc'd blocks
    // optional device pool: one region carved first-fit into 256-byte aligned blocks
    Pool pool;
    // optional pinned host pool for the host mirrors of runs (GLS_OPT_HOST_POOL_BYTES),
    // mapped into the device's address space at hpool_dev
    Pool hpool;
    char *hpool_dev = nullptr;
    uint32_t *d_status = nullptr;       // scratch for stimulus packing (3 words)
    std::vector<UserCell> cells;        // gls_define_cell, type GLS_USER_CELL_BASE + index
};

namespace {

// First-fit allocation from the context's pool (no CUDA call, so creating
// and freeing run buffers never synchronises the device).
// Long-lived objects (netlists, stimuli, planned orders) are carved from the
// top of the pool and runs from the bottom, so releasing a run leaves one
// large free range instead of gaps between persistent blocks.
void *pool_take(Pool &pl, uint64_t bytes, bool persistent) {
    bytes = (bytes + 255) & ~255ull;
    if (persistent) {
        for (auto it = pl.free.rbegin(); it != pl.free.rend(); ++it) {
            if (it->second < bytes) continue;
            const uint64_t off = it->first, size = it->second;
            if (size > bytes) it->second = size - bytes;
            else pl.free.erase(std::next(it).base());
            void *p = pl.base + off + size - bytes;
            pl.allocs[p] = bytes;
            return p;
        }
        return nullptr;
    }
    for (auto it = pl.free.begin(); it != pl.free.end(); ++it) {
        if (it->second < bytes) continue;
        const uint64_t off = it->first, size = it->second;
        pl.free.erase(it);
        if (size > bytes) pl.free[off + bytes] = size - bytes;
        void *p = pl.base + off;
        pl.allocs[p] = bytes;
        return p;
    }
    return nullptr;
}

bool pool_give(Pool &pl, void *p) {
    auto a = pl.allocs.find(p);
    if (a == pl.allocs.end()) return false;
    uint64_t off = (uint64_t)((char *)p - pl.base), size = a->second;
    pl.allocs.erase(a);
    auto next = pl.free.lower_bound(off);
    if (next != pl.free.end() && next->first == off + size) {   // merge with the following range
        size += next->second;
        next = pl.free.erase(next);
    }
    if (next != pl.free.begin()) {                               // and with the preceding one
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += size;
            return true;
        }
    }
    pl.free[off] = size;
    return true;
}

uint64_t pool_largest_free(const Pool &pl) {
    uint64_t m = 0;
    for (auto &kv : pl.free) m = std::max(m, kv.second);
    return m;
}

int dalloc(gls_ctx *c, void **p, size_t bytes, bool persistent = false) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->pool.base) {
        *p = pool_take(c->pool, bytes, persistent);
        if (!*p)
            return fail(GLS_ENOMEM, "device pool of %llu bytes has no free block of %llu bytes",
                        (unsigned long long)c->pool.bytes, (unsigned long long)bytes);
        return GLS_OK;
    }
    if (c->used + bytes > c->budget)
        return fail(GLS_ENOMEM, "device budget exceeded (%llu + %llu > %llu bytes)", (unsigned long long)c->used,
                    (unsigned long long)bytes, (unsigned long long)c->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(GLS_ENOMEM, "cudaMalloc(%llu): %s", (unsigned long long)bytes, cudaGetErrorString(e));
    }
    c->used += bytes;
    c->allocs[*p] = bytes;
    return GLS_OK;
}

template <class T>
int dalloc_n(gls_ctx *c, T **p, size_t n, bool persistent = false) {
    void *q = nullptr;
    int rc = dalloc(c, &q, n * sizeof(T), persistent);
    *p = static_cast<T *>(q);
    return rc;
}

void dfree(gls_ctx *c, void *p) {
    if (!p) return;
    if (pool_give(c->pool, p)) return;
    auto it = c->allocs.find(p);
    if (it != c->allocs.end()) {
        c->used -= it->second;
        c->allocs.erase(it);
    }
    cudaFree(p);
}

void free_netlist(gls_ctx *c, NetlistObj *n) {
    for (GateRec *p : n->plans) dfree(c, p);
    dfree(c, n->d_gates);
    dfree(c, n->d_ext2int);
    dfree(c, n->d_level_begin);
}
void free_stim(gls_ctx *c, StimObj *s) {
    dfree(c, s->d_off);
    dfree(c, s->d_t);
    dfree(c, s->d_v);
    dfree(c, s->d_packed);
    dfree(c, s->d_t64);
}
// The host copies of a sliced run's slices (pool blocks back to the pinned pool).
void release_slices(gls_ctx *c, RunObj *r) {
    for (auto &sl : r->slices)
        if (sl.pinned) pool_give(c->hpool, sl.pinned);
    r->slices.clear();
}

void free_run(gls_ctx *c, RunObj *r) {
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->ev0) cudaEventDestroy(r->ev0);
    if (r->ev1) cudaEventDestroy(r->ev1);
    if (r->owns_gates) dfree(c, r->d_gates);
    dfree(c, r->dev.net_ptr);
    dfree(c, r->dev.net_len);
    dfree(c, r->dev.arena);
    dfree(c, r->dev.arena_top);
    dfree(c, r->dev.status);
    dfree(c, r->dev.level_ctr);
    dfree(c, r->dev.done);
    dfree(c, r->d_sum);
    dfree(c, r->d_pi_total);
    dfree(c, r->d_off);
    dfree(c, r->d_scan_tmp);
    dfree(c, r->d_gather);
    dfree(c, r->d_slice_packed);
    dfree(c, r->d_glen);
    if (r->h_arena && !pool_give(c->hpool, r->h_arena)) cudaFreeHost(r->h_arena);
    release_slices(c, r);
    for (int k = 0; k < 3; k++) {
        dfree(c, r->d_st[k]);
        dfree(c, r->d_pend[k]);
    }
}

cudaStream_t pick_stream(gls_ctx *c, void *s) { return s ? static_cast<cudaStream_t>(s) : c->stream; }

int upload_stimulus(gls_ctx *c, StimObj *s, const int64_t *off, const int32_t *t, const uint8_t *v) {
    const int64_t E = off[s->n_pi];
    CK(cudaMemcpyAsync(s->d_off, off, sizeof(int64_t) * (size_t)(s->n_pi + 1), cudaMemcpyHostToDevice, c->stream));
    if (E > 0) {
        CK(cudaMemcpyAsync(s->d_t, t, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(s->d_v, v, (size_t)E, cudaMemcpyHostToDevice, c->stream));
    }
    const uint32_t init[3] = {0u, 0xFFFFFFFFu, 0u};
    CK(cudaMemcpyAsync(c->d_status, init, sizeof init, cudaMemcpyHostToDevice, c->stream));
    CK(launch_pack_stimulus(s->d_off, s->d_t, s->d_v, s->n_pi, s->d_packed, c->d_status, c->stream));
    uint32_t st[3];
    CK(cudaMemcpyAsync(st, c->d_status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st[0]) {
        // the device found a violation; name the first rule broken on the host
        int rc = check_stimulus_host(s->n_pi, off, t, v, true);
        return rc ? rc : fail(GLS_ESTIM, "stimulus rule violated at PI %u", st[1]);
    }
    s->n_events = E;
    s->max_time = st[2];
    return GLS_OK;
}

NetlistObj *find_netlist(gls_ctx *c, int32_t id) {
    auto it = c->netlists.find(id);
    return it == c->netlists.end() ? nullptr : it->second.get();
}
StimObj *find_stim(gls_ctx *c, int32_t id) {
    auto it = c->stims.find(id);
    return it == c->stims.end() ? nullptr : it->second.get();
}
RunObj *find_run(gls_ctx *c, int32_t id) {
    auto it = c->runs.find(id);
    return it == c->runs.end() ? nullptr : it->second.get();
}

// The gate kernels of one evaluation: one persistent launch (dependency
// schedule) or one launch per level.
cudaError_t launch_gates(gls_ctx *c, const RunObj *r, const RunDev &dev, cudaStream_t cs) {
    if (r->schedule == GLS_SCHEDULE_DEPENDENCY) return launch_dependency(r->d_gates, r->n_gates, r->depth, dev, c->cfg, cs);
    cudaError_t e = cudaSuccess;
    for (int32_t L = 1; L <= r->depth && e == cudaSuccess; L++) {
        const int32_t b = r->level_begin[L], cnt = r->level_begin[L + 1] - b;
        e = launch_level(r->d_gates, b, cnt, L - 1, dev, c->cfg, cs);
    }
    return e;
}

int build_run_graph(gls_ctx *c, RunObj *r) {
    cudaGraph_t graph = nullptr;
    const bool dep = r->schedule == GLS_SCHEDULE_DEPENDENCY;
    cudaStream_t cs = c->cap_stream;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(r->dev.level_ctr, 0, sizeof(int32_t) * ((size_t)r->depth + 1), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->dev.arena_top, 0, sizeof(unsigned long long), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->dev.status, 0, sizeof(uint32_t), cs);
    if (e == cudaSuccess && dep) e = cudaMemsetAsync(r->dev.done, 0, sizeof(uint32_t) * (size_t)r->n_nets, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d_pi_total, 0, sizeof(unsigned long long), cs);
    for (const RunItem &it : r->items) {
        if (e != cudaSuccess) break;
        NetlistObj *n = find_netlist(c, it.netlist_id);
        StimObj *s = find_stim(c, it.stim_id);
        e = launch_pi_init(s->d_off, s->d_packed, n->n_pi, it.net_base, it.t_limit, r->dev.net_ptr, r->dev.net_len,
                           dep ? r->dev.done : nullptr, r->d_pi_total, cs);
    }
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(r->ev0, cs, cudaEventRecordExternal);
    if (e == cudaSuccess) e = launch_gates(c, r, r->dev, cs);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(r->ev1, cs, cudaEventRecordExternal);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(GLS_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&r->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(GLS_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    return GLS_OK;
}

int apply_launch_cfg(gls_ctx *c, int variant, int warps_per_cta) {
    const int per_sm = gate_max_ctas_per_sm(variant, warps_per_cta);
    CK(cudaGetLastError());
    if (per_sm < 1) return fail(GLS_EINVAL, "%d warps per CTA do not fit on an SM", warps_per_cta);
    c->cfg.variant = variant;
    c->cfg.warps_per_cta = warps_per_cta;
    c->cfg.ctas = per_sm * c->sm_count;
    return GLS_OK;
}

int time_range_check(NetlistObj *n, StimObj *s) {
    if ((int64_t)s->max_time + n->lv.max_path_delay >= (int64_t)kTimeLimit)
        return fail(GLS_ERANGE, "latest input time %u + longest path delay %lld reaches 2^30-1", s->max_time,
                    (long long)n->lv.max_path_delay);
    return GLS_OK;
}

int items_time_range_check(gls_ctx *c, const RunObj *r) {
    for (const RunItem &it : r->items) {
        int rc = time_range_check(find_netlist(c, it.netlist_id), find_stim(c, it.stim_id));
        if (rc) return rc;
    }
    return GLS_OK;
}

// Validate the instances, lay out their nets and gates, allocate the store and
// capture the run's graph; the run is launched by the caller.
int create_run(gls_ctx *c, const int32_t *netlist_ids, const int32_t *stim_ids, const int32_t *t_limits,
               int32_t n_items, int64_t arena_events, std::unique_ptr<RunObj> &out, int64_t slice_ps = 0) {
    auto r = std::make_unique<RunObj>();
    r->schedule = c->schedule;
    r->slice_ps = slice_ps;
    if (slice_ps > 0) {
        if (n_items != 1) return fail(GLS_EINVAL, "a sliced run has one item");
        if (c->cfg.variant == kVariantSegmented)
            return fail(GLS_EINVAL, "sliced runs use the windowed kernels (GLS_KERNEL_WINDOWED or _WIDE)");
    }
    int64_t stim_events = 0, base = 0;
    for (int32_t i = 0; i < n_items; i++) {
        NetlistObj *n = find_netlist(c, netlist_ids[i]);
        StimObj *s = find_stim(c, stim_ids[i]);
        if (!n) return fail(GLS_EINVAL, "item %d: unknown netlist id %d", i, netlist_ids[i]);
        if (!s) return fail(GLS_EINVAL, "item %d: unknown stimulus id %d", i, stim_ids[i]);
        if (s->n_pi != n->n_pi) return fail(GLS_EINVAL, "item %d: stimulus has %d PIs, netlist %d", i, s->n_pi, n->n_pi);
        if (n->general && c->cfg.variant == kVariantSegmented)
            return fail(GLS_EINVAL, "item %d: the netlist has edge-dependent delays, pins without arcs or a cell that "
                        "is not X for all-X inputs; these run on the windowed kernels", i);
        if (slice_ps > 0) {
            // slice-local times: inputs below slice_ps, outputs below slice_ps + the longest path
            if (slice_ps + n->lv.max_path_delay >= (int64_t)kTimeLimit)
                return fail(GLS_ERANGE, "slice of %lld ps + longest path delay %lld reaches 2^30-1",
                            (long long)slice_ps, (long long)n->lv.max_path_delay);
            const int64_t mt = s->wide ? s->max_time64 : (int64_t)s->max_time;
            if (mt / slice_ps >= (1 << 20)) return fail(GLS_EINVAL, "more than 2^20 slices of %lld ps", (long long)slice_ps);
        } else {
            if (s->wide) return fail(GLS_EINVAL, "item %d: a stimulus with 64-bit times runs only in time slices", i);
            int rc = time_range_check(n, s);
            if (rc) return rc;
        }
        uint32_t tl = kTimeInf;
        if (t_limits) {
            if (t_limits[i] < 0) return fail(GLS_EINVAL, "item %d: negative time limit", i);
            tl = (uint32_t)t_limits[i];
        }
        r->items.push_back(RunItem{netlist_ids[i], stim_ids[i], base, tl});
        base += (int64_t)n->n_pi + n->n_gates;
        r->n_gates += n->n_gates;
        r->depth = std::max(r->depth, n->lv.depth);
        stim_events += s->n_events;
    }
    if (base >= (int64_t)INT32_MAX) return fail(GLS_EINVAL, "a run holds at most 2^31 - 1 nets");
    r->n_nets = base;
    int rc = GLS_OK;
    bool same = true;
    for (int32_t i = 1; i < n_items; i++) same &= netlist_ids[i] == netlist_ids[0];
    if (same) {   // one netlist (once or replicated): its own records, decoded per replica on the device
        NetlistObj *n = find_netlist(c, netlist_ids[0]);
        r->d_gates = n->d_gates;
        r->level_begin = n->lv.level_begin;
        for (int32_t &x : r->level_begin) x *= n_items;
        r->dev.rep = n_items;
        r->dev.rep_nets = (int64_t)n->n_pi + n->n_gates;
        r->dev.lb = n->d_level_begin;
        if (r->schedule == GLS_SCHEDULE_DEPENDENCY && n->d_plan) {
            r->d_gates = n->d_plan;
            r->dev.planned = 1;
        }
    } else {      // records of all instances interleaved by level, net ids shifted
        std::vector<GateRec> comb((size_t)std::max(r->n_gates, 1));
        r->level_begin.assign(r->depth + 2, 0);
        size_t at = 0;
        for (int32_t L = 1; L <= r->depth; L++) {
            r->level_begin[L] = (int32_t)at;
            for (const RunItem &it : r->items) {
                NetlistObj *n = find_netlist(c, it.netlist_id);
                if (L > n->lv.depth) continue;
                for (int32_t q = n->lv.level_begin[L]; q < n->lv.level_begin[L + 1]; q++) {
                    GateRec g = n->recs[q];
                    for (int k = 0; k < g.k; k++) g.fin[k] += (int32_t)it.net_base;
                    g.out_net += (uint32_t)it.net_base;
                    comb[at++] = g;
                }
            }
        }
        r->level_begin[r->depth + 1] = (int32_t)at;
        r->level_begin[0] = 0;
        rc = dalloc_n(c, &r->d_gates, comb.size());
        if (rc) return rc;
        r->owns_gates = true;
        CK(cudaMemcpy(r->d_gates, comb.data(), sizeof(GateRec) * comb.size(), cudaMemcpyHostToDevice));
    }
    if (arena_events <= 0) {
        // default: 256 words per stimulus transition plus 1 Mi, at most half
        // of what is left of the budget (GLS_EOVERFLOW reports the demand)
        uint64_t left = c->budget > c->used ? c->budget - c->used : 0;
        if (c->pool.base) left = pool_largest_free(c->pool);
        uint64_t meta = (uint64_t)r->n_nets * 16 + (uint64_t)r->depth * 4 + 4096;
        uint64_t cap = left > meta ? (left - meta) / 2 / 4 : 0;
        uint64_t want = 256ull * (uint64_t)stim_events + (1ull << 20);
        if (slice_ps > 0) {   // about one launch's share; a launch that overflows is rerun with more
            const StimObj *s = find_stim(c, stim_ids[0]);
            const int64_t mt = s->wide ? s->max_time64 : (int64_t)s->max_time;
            const int64_t ns = mt / slice_ps + 1;
            const int64_t per = std::min<int64_t>(ns, r->schedule == GLS_SCHEDULE_DEPENDENCY ? c->slice_group : 1);
            want = 256ull * (uint64_t)(stim_events / ns + 1) * (uint64_t)per + (1ull << 20);
        }
        arena_events = (int64_t)std::min(cap, want);
    }
    const int64_t N = r->n_nets;
    if (slice_ps > 0 && r->schedule == GLS_SCHEDULE_DEPENDENCY) {
        // a warp evaluates its gate over up to slice_group slices per launch
        // (a descriptor set per slice)
        const StimObj *s = find_stim(c, stim_ids[0]);
        const int64_t mt = s->wide ? s->max_time64 : (int64_t)s->max_time;
        const int64_t ns = s->n_events > 0 ? mt / slice_ps + 1 : 1;
        r->slice_group = (int32_t)std::max<int64_t>(1, std::min<int64_t>(ns, c->slice_group));
    }
    const int64_t NS = N * r->slice_group;   // descriptors of one launch
    r->dev.arena_cap = (uint64_t)arena_events;
    {   // warps claim the arena in blocks of a quarter of their share per launch,
        // at most 256 Ki words (1 MiB): large against a gate's Eq. 2 bound, so
        // little of a block is left behind when a gate's bound does not fit
        // its rest; below one line every gate claims its own slot
        const uint64_t warps = (uint64_t)std::max(1, c->cfg.ctas * c->cfg.warps_per_cta);
        const uint64_t launches = r->schedule == GLS_SCHEDULE_DEPENDENCY ? 1 : (uint64_t)std::max(1, r->depth);
        const uint64_t blk = std::min<uint64_t>((uint64_t)arena_events / (4 * warps * launches), 262144);
        r->dev.arena_blk = (uint32_t)(blk & ~(uint64_t)(kSlotAlign - 1));
    }
    r->dev.n_pi = 0;
    r->dev.n_gates = r->n_gates;
    r->dev.wait_limit_ns = c->wait_limit_ns;
    r->dev.withhold_gate = c->withhold_gate;
    r->dev.seg_target = c->seg_target;
    rc = dalloc_n(c, &r->dev.net_ptr, (size_t)std::max<int64_t>(NS, 1));
    if (!rc) rc = dalloc_n(c, &r->dev.net_len, (size_t)std::max<int64_t>(NS, 1));
    // padded by one slot line: readers round a waveform's end up to 4 words
    if (!rc) rc = dalloc_n(c, &r->dev.arena, (size_t)arena_events + 2 * kSlotAlign);
    if (!rc) rc = dalloc_n(c, &r->dev.arena_top, 1);
    if (!rc) rc = dalloc_n(c, &r->dev.status, 1);
    if (!rc) rc = dalloc_n(c, &r->dev.level_ctr, (size_t)r->depth + 1);
    if (!rc) rc = dalloc_n(c, &r->dev.done, (size_t)std::max<int64_t>(N, 1));
    if (!rc) rc = dalloc_n(c, &r->d_sum, 1);
    if (!rc) rc = dalloc_n(c, &r->d_pi_total, 1);
    if (rc) { free_run(c, r.get()); return rc; }
    r->dev.pi_total = r->d_pi_total;
    if (c->host_mirror && slice_ps == 0) {
        if (c->cfg.variant == kVariantSegmented) {
            free_run(c, r.get());
            return fail(GLS_EINVAL, "host-mirrored results need the windowed kernels");
        }
        const size_t mbytes = sizeof(uint32_t) * ((size_t)arena_events + 2 * kSlotAlign);
        void *h = nullptr, *d = nullptr;
        if (c->hpool.base) {   // carved from the pinned host pool: no allocation call per run
            h = pool_take(c->hpool, mbytes, false);
            if (!h) {
                free_run(c, r.get());
                return fail(GLS_ENOMEM, "host pool of %llu bytes has no free block for a mirror of %zu bytes",
                            (unsigned long long)c->hpool.bytes, mbytes);
            }
            d = c->hpool_dev + ((char *)h - c->hpool.base);
        } else {
            cudaError_t e = cudaHostAlloc(&h, mbytes, cudaHostAllocMapped);
            if (e == cudaSuccess) e = cudaHostGetDevicePointer(&d, h, 0);
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (h) cudaFreeHost(h);
                free_run(c, r.get());
                return fail(GLS_ENOMEM, "pinned host mirror of %lld words: %s", (long long)arena_events,
                            cudaGetErrorString(e));
            }
        }
        r->h_arena = static_cast<uint32_t *>(h);
        r->dev.harena = static_cast<uint32_t *>(d);
    }
    if (slice_ps > 0) {
        const StimObj *s = find_stim(c, stim_ids[0]);
        rc = dalloc_n(c, &r->d_slice_packed, (size_t)slice_words(s->cap_events, s->n_pi, r->slice_group));
        for (int k = 0; k < 3 && !rc; k++) {
            rc = dalloc_n(c, &r->d_st[k], (size_t)std::max<int64_t>(N, 1));
            if (!rc) rc = dalloc_n(c, &r->d_pend[k], (size_t)std::max<int64_t>(N, 1) * kPendCap);
        }
        if (rc) { free_run(c, r.get()); return rc; }
    }
    cudaError_t e = cudaEventCreate(&r->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev1);
    if (e != cudaSuccess) { free_run(c, r.get()); return fail(GLS_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e)); }
    if (slice_ps == 0) {
        rc = build_run_graph(c, r.get());
        if (rc) { free_run(c, r.get()); return rc; }
    }
    out = std::move(r);
    return GLS_OK;
}

// Dense CSR of one instance of a run (its nets in caller order) into host memory.
// (net_shift: the descriptor set of slice j of a launch over several time
// slices)
int read_item(gls_ctx *c, RunObj *r, int32_t item, int64_t *off, uint32_t *packed, int64_t cap,
              int64_t net_shift = 0) {
    if (item < 0 || item >= (int32_t)r->items.size()) return fail(GLS_EINVAL, "item %d out of range", item);
    const RunItem &it = r->items[item];
    NetlistObj *n = find_netlist(c, it.netlist_id);
    const int64_t N = (int64_t)n->n_pi + n->n_gates;
    const int64_t net_base = it.net_base + net_shift;
    CK(cudaEventSynchronize(r->ev1));
    int rc = GLS_OK;
    if (r->off_cap < N + 1) {
        dfree(c, r->d_off);
        dfree(c, r->d_scan_tmp);
        r->d_off = nullptr;
        r->d_scan_tmp = nullptr;
        r->off_cap = 0;
        r->scan_tmp = scan_tmp_elems(N + 1);
        rc = dalloc_n(c, &r->d_off, (size_t)N + 1);
        if (!rc) rc = dalloc_n(c, &r->d_scan_tmp, r->scan_tmp);
        if (rc) return rc;
        r->off_cap = N + 1;
    }
    CK(launch_gather_lengths(r->dev.net_len, n->d_ext2int, N, r->d_off, c->stream, net_base));
    CK(launch_exclusive_scan_i64(r->d_off, N + 1, r->d_scan_tmp, r->scan_tmp, c->stream));
    CK(cudaMemcpyAsync(off, r->d_off, sizeof(int64_t) * (size_t)(N + 1), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int64_t total = off[N];
    if (total > cap) return fail(GLS_EOVERFLOW, "%lld transitions, cap %lld", (long long)total, (long long)cap);
    if (total == 0) return GLS_OK;
    if (!packed) return fail(GLS_EINVAL, "NULL packed array");
    if (total > r->gather_cap) {
        dfree(c, r->d_gather);
        r->d_gather = nullptr;
        r->gather_cap = 0;
        rc = dalloc_n(c, &r->d_gather, (size_t)total);
        if (rc) return rc;
        r->gather_cap = total;
    }
    CK(launch_gather_events(r->dev.net_ptr, r->dev.net_len, n->d_ext2int, r->d_off, N, r->d_gather, c->stream,
                            net_base));
    CK(cudaMemcpyAsync(packed, r->d_gather, sizeof(uint32_t) * (size_t)total, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return GLS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch of gls_simulate_noalloc: per-level work counters, the arena bump
// pointer and the status word of a run, in one statically allocated device
// array (words [0,1] arena top, [2] status, [64, 64 + GLS_NOALLOC_MAX_LEVELS)
// level counters).  Every GPU that loads this library holds it until exit.
static __device__ __align__(256) uint32_t g_noalloc_scratch[GLS_NOALLOC_SCRATCH_WORDS];

namespace {

constexpr int kNoallocMaxDevices = 128;
std::mutex g_noalloc_mu;
uint32_t *g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
int noalloc_scratch(int device, uint32_t **out) {
    if (device < 0 || device >= kNoallocMaxDevices) return fail(GLS_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(GLS_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_noalloc_addr[device] = static_cast<uint32_t *>(p);
    }
    *out = g_noalloc_addr[device];
    return GLS_OK;
}

// Copy the run's status and arena demand from the scratch array to the
// caller's report words.
__global__ void noalloc_report_kernel(uint32_t *report) {
    const unsigned long long top = *reinterpret_cast<const unsigned long long *>(g_noalloc_scratch);
    report[0] = g_noalloc_scratch[2];
    report[1] = (uint32_t)(top & 0xFFFFFFFFull);
    report[2] = (uint32_t)(top >> 32);
    report[3] = 0u;
}

}  // namespace

// ===========================================================================
extern "C" {

int gls_version(void) { return 100; }

int gls_cell_arity(int cell) { return (cell >= 0 && cell < GLS_NCELLS) ? kArity[cell] : GLS_EINVAL; }

int gls_check_netlist(int32_t n_pi, int32_t n_gates, const uint8_t *type, const int32_t *fanin_off,
                      const int32_t *fanin_net, const int32_t *d_rise, const int32_t *d_fall, int32_t *depth_out,
                      int32_t *level_out) {
    try {
        Levelized lv;
        std::vector<int32_t> d4;
        int rc = classic_arcs(n_pi, n_gates, type, fanin_off, fanin_net, d_rise, d_fall, d4);
        if (!rc) rc = analyse_netlist(n_pi, n_gates, fanin_off, fanin_net, d4.data(), &lv);
        if (rc) return rc;
        if (depth_out) *depth_out = lv.depth;
        if (level_out) std::copy(lv.level.begin(), lv.level.end(), level_out);
        return GLS_OK;
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_check_stimulus(int32_t n_pi, const int64_t *off, const int32_t *t, const uint8_t *v) {
    return check_stimulus_host(n_pi, off, t, v, true);
}

int gls_create(gls_ctx **out, int device, uint64_t hbm_budget_bytes) {
    if (!out) return fail(GLS_EINVAL, "out is NULL");
    *out = nullptr;
    try {
        int ndev = 0;
        CK(cudaGetDeviceCount(&ndev));
        if (device < 0 || device >= ndev) return fail(GLS_EINVAL, "device %d of %d", device, ndev);
        CK(cudaSetDevice(device));
        auto c = std::make_unique<gls_ctx>();
        c->device = device;
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        c->budget = hbm_budget_bytes ? hbm_budget_bytes : (uint64_t)(0.9 * (double)fr);
        CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        CK(cudaGetLastError());
        int rc = apply_launch_cfg(c.get(), kVariantWindowedWide, 4);
        if (rc) return rc;
        rc = dalloc_n(c.get(), &c->d_status, 4);
        if (rc) return rc;
        *out = c.release();
        return GLS_OK;
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

void gls_destroy(gls_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->runs) free_run(c, kv.second.get());
    for (auto &kv : c->stims) free_stim(c, kv.second.get());
    for (auto &kv : c->netlists) free_netlist(c, kv.second.get());
    dfree(c, c->d_status);
    if (c->pool.base) cudaFree(c->pool.base);
    if (c->hpool.base) cudaFreeHost(c->hpool.base);
    cudaStreamDestroy(c->stream);
    cudaStreamDestroy(c->cap_stream);
    delete c;
}

const char *gls_last_error(gls_ctx *) { return g_err.c_str(); }

// A netlist in the general form: gate g (one cell output) reads
// fanin_net[fanin_off[g]..fanin_off[g+1]] with per-arc delays d4 (see
// check_arcs), its function is the 64-entry table lut[g] and types[g] is
// its built-in cell id (255 for user cells).
static int load_general(gls_ctx *c, int32_t n_pi, int32_t n_gates, const int32_t *fanin_off, const int32_t *fanin_net,
                        const int32_t *d4, const uint64_t (*lut)[2], const uint8_t *types, int32_t *netlist_id) {
    try {
        CK(cudaSetDevice(c->device));
        auto n = std::make_unique<NetlistObj>();
        int rc = analyse_netlist(n_pi, n_gates, fanin_off, fanin_net, d4, &n->lv);
        if (rc) return rc;
        n->n_pi = n_pi;
        n->n_gates = n_gates;
        const int64_t N = (int64_t)n_pi + n_gates;
        std::vector<GateRec> recs(std::max<int32_t>(n_gates, 1));
        for (int32_t p = 0; p < n_gates; p++) {
            const int32_t g = n->lv.order[p];
            GateRec &r = recs[p];
            std::memset(&r, 0, sizeof r);
            r.lut_lo = lut[g][0];
            r.lut_hi = lut[g][1];
            r.type = types[g];
            r.k = (uint8_t)(fanin_off[g + 1] - fanin_off[g]);
            r.out_net = (uint32_t)(n_pi + p);
            int32_t dmin = INT32_MAX;
            for (int q = 0; q < r.k; q++) {
                const int32_t *d = d4 + 4 * ((int64_t)fanin_off[g] + q);
                if (d[0] >= 0) for (int j = 0; j < 4; j++) dmin = std::min(dmin, d[j]);
            }
            r.dmin = dmin;
            bool edge = false;
            for (int q = 0; q < r.k; q++) {
                const int32_t a = fanin_off[g] + q, net = fanin_net[a];
                r.fin[q] = net < n_pi ? net : n_pi + n->lv.pos[net - n_pi];
                const int32_t *d = d4 + 4 * (int64_t)a;
                const bool arc = d[0] >= 0;
                if (arc) r.arcs |= (uint8_t)(1u << q);
                for (int e = 0; e < 2; e++)
                    for (int v = 0; v < 2; v++) r.doff[q][e][v] = arc ? (uint8_t)(d[e * 2 + v] - dmin) : kNoArc;
                edge |= arc && (d[0] != d[2] || d[1] != d[3]);
            }
            const bool all_x_is_x = ((r.lut_hi >> (2 * (42 - 32))) & 3u) == 2u;   // inputs X, X, X
            if (edge) r.flags |= kGateEdge;
            if (edge || r.arcs != (uint8_t)((1u << r.k) - 1) || !all_x_is_x) r.flags |= kGateGeneral;
            if (r.flags & kGateGeneral) n->general = true;
        }
        n->ext2int.resize(N);
        for (int32_t i = 0; i < n_pi; i++) n->ext2int[i] = i;
        for (int32_t g = 0; g < n_gates; g++) n->ext2int[n_pi + g] = n_pi + n->lv.pos[g];
        rc = dalloc_n(c, &n->d_gates, recs.size(), true);
        if (!rc) rc = dalloc_n(c, &n->d_ext2int, (size_t)std::max<int64_t>(N, 1), true);
        if (!rc) rc = dalloc_n(c, &n->d_level_begin, n->lv.level_begin.size(), true);
        if (rc) { free_netlist(c, n.get()); return rc; }
        CK(cudaMemcpyAsync(n->d_level_begin, n->lv.level_begin.data(), sizeof(int32_t) * n->lv.level_begin.size(),
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(n->d_gates, recs.data(), sizeof(GateRec) * recs.size(), cudaMemcpyHostToDevice, c->stream));
        n->recs = recs;
        if (N > 0)
            CK(cudaMemcpyAsync(n->d_ext2int, n->ext2int.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const int32_t id = c->next_id++;
        c->netlists[id] = std::move(n);
        *netlist_id = id;
        return GLS_OK;
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_load_netlist(gls_ctx *c, int32_t n_pi, int32_t n_gates, const uint8_t *type, const int32_t *fanin_off,
                     const int32_t *fanin_net, const int32_t *d_rise, const int32_t *d_fall, int32_t *netlist_id) {
    if (!c || !netlist_id) return fail(GLS_EINVAL, "NULL argument");
    try {
        std::vector<int32_t> d4;
        int rc = classic_arcs(n_pi, n_gates, type, fanin_off, fanin_net, d_rise, d_fall, d4);
        if (rc) return rc;
        uint64_t bl[GLS_NCELLS][2];
        build_luts(bl);
        std::vector<uint64_t> lut(2 * (size_t)std::max(n_gates, 1));
        for (int32_t g = 0; g < n_gates; g++) {
            lut[2 * (size_t)g] = bl[type[g]][0];
            lut[2 * (size_t)g + 1] = bl[type[g]][1];
        }
        return load_general(c, n_pi, n_gates, fanin_off, fanin_net, d4.data(),
                            reinterpret_cast<const uint64_t (*)[2]>(lut.data()), type, netlist_id);
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_cell_table(int32_t cell, uint8_t *table) {
    if (cell < 0 || cell >= GLS_NCELLS || !table) return fail(GLS_EINVAL, "built-in cell id %d", cell);
    uint64_t bl[GLS_NCELLS][2];
    build_luts(bl);
    const int k = kArity[cell];
    for (int i = 0; i < (1 << (2 * k)); i++) {
        // pins beyond k read X in the 64-entry table
        int idx = i;
        for (int p = k; p < 3; p++) idx |= 2 << (2 * p);
        table[i] = (uint8_t)((bl[cell][idx >> 5] >> (2 * (idx & 31))) & 3u);
    }
    return GLS_OK;
}

int gls_define_cell(gls_ctx *c, int32_t n_inputs, int32_t n_outputs, const uint8_t *tables, int32_t *cell_type) {
    if (!c || !tables || !cell_type) return fail(GLS_EINVAL, "NULL argument");
    if (n_inputs < 1 || n_inputs > 3) return fail(GLS_EINVAL, "%d inputs (1..3 supported)", n_inputs);
    if (n_outputs < 1 || n_outputs > GLS_MAX_CELL_OUTPUTS)
        return fail(GLS_EINVAL, "%d outputs (1..%d supported)", n_outputs, GLS_MAX_CELL_OUTPUTS);
    const int n4 = 1 << (2 * n_inputs);
    for (int i = 0; i < n_outputs * n4; i++)
        if (tables[i] > 2) return fail(GLS_EINVAL, "table entry %d: value %d (0, 1 or 2 = X)", i, tables[i]);
    try {
        UserCell u;
        u.n_in = n_inputs;
        u.n_out = n_outputs;
        u.tables.assign(tables, tables + (size_t)n_outputs * n4);
        c->cells.push_back(std::move(u));
        *cell_type = GLS_USER_CELL_BASE + (int32_t)c->cells.size() - 1;
        return GLS_OK;
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_load_netlist_cells(gls_ctx *c, int32_t n_pi, int32_t n_cells, const int32_t *cell_type,
                           const int32_t *fanin_off, const int32_t *fanin_net, const int32_t *delays,
                           int32_t *netlist_id) {
    if (!c || !netlist_id) return fail(GLS_EINVAL, "NULL argument");
    if (n_pi < 0 || n_cells < 0) return fail(GLS_EINVAL, "negative n_pi or n_cells");
    if (n_cells > 0 && (!cell_type || !fanin_off || !fanin_net || !delays)) return fail(GLS_EINVAL, "NULL netlist array");
    if (n_cells > 0 && fanin_off[0] != 0) return fail(GLS_EINVAL, "fanin_off[0] must be 0");
    try {
        uint64_t bl[GLS_NCELLS][2];
        build_luts(bl);
        // every cell output becomes one gate; its nets keep the caller's numbering
        std::vector<int32_t> goff(1, 0), gnet, d4;
        std::vector<uint64_t> lut;
        std::vector<uint8_t> types;
        int64_t dpos = 0;
        for (int32_t cc = 0; cc < n_cells; cc++) {
            const int32_t T = cell_type[cc];
            int n_in, n_out;
            const UserCell *u = nullptr;
            if (T >= 0 && T < GLS_NCELLS) { n_in = kArity[T]; n_out = 1; }
            else if (T >= GLS_USER_CELL_BASE && T - GLS_USER_CELL_BASE < (int32_t)c->cells.size()) {
                u = &c->cells[T - GLS_USER_CELL_BASE];
                n_in = u->n_in;
                n_out = u->n_out;
            } else return fail(GLS_EINVAL, "cell %d: unknown cell type %d", cc, T);
            if (fanin_off[cc + 1] - fanin_off[cc] != n_in)
                return fail(GLS_EINVAL, "cell %d: %d fanins for a %d-input cell", cc, fanin_off[cc + 1] - fanin_off[cc], n_in);
            const int n4 = 1 << (2 * n_in);
            for (int o = 0; o < n_out; o++) {
                for (int p = 0; p < n_in; p++) {
                    gnet.push_back(fanin_net[fanin_off[cc] + p]);
                    for (int j = 0; j < 4; j++) d4.push_back(delays[dpos + ((int64_t)p * n_out + o) * 4 + j]);
                }
                goff.push_back((int32_t)gnet.size());
                uint64_t w[2] = {0, 0};
                for (int idx = 0; idx < 64; idx++) {
                    const int i = idx & (n4 - 1);   // the cell's own pins; the others read X in the kernel
                    const uint64_t v = u ? u->tables[(size_t)o * n4 + i] : ((bl[T][idx >> 5] >> (2 * (idx & 31))) & 3u);
                    w[idx >> 5] |= v << (2 * (idx & 31));
                }
                lut.push_back(w[0]);
                lut.push_back(w[1]);
                types.push_back(u ? (uint8_t)255 : (uint8_t)T);
            }
            dpos += (int64_t)n_in * n_out * 4;
        }
        const int64_t G = (int64_t)types.size();
        if ((int64_t)n_pi + G >= (int64_t)INT32_MAX) return fail(GLS_EINVAL, "too many nets");
        if (G == 0) { d4.assign(4, 0); lut.assign(2, 0); types.assign(1, 0); }
        return load_general(c, n_pi, (int32_t)G, goff.data(), gnet.data(), d4.data(),
                            reinterpret_cast<const uint64_t (*)[2]>(lut.data()), types.data(), netlist_id);
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_load_stimulus(gls_ctx *c, int32_t n_pi, const int64_t *off, const int32_t *t, const uint8_t *v,
                      int32_t *stim_id) {
    if (!c || !stim_id) return fail(GLS_EINVAL, "NULL argument");
    try {
        CK(cudaSetDevice(c->device));
        int rc = check_stimulus_host(n_pi, off, t, v, false);
        if (rc) return rc;
        auto s = std::make_unique<StimObj>();
        s->n_pi = n_pi;
        s->cap_events = off[n_pi];
        rc = dalloc_n(c, &s->d_off, (size_t)n_pi + 1, true);
        if (!rc) rc = dalloc_n(c, &s->d_t, (size_t)std::max<int64_t>(s->cap_events, 1), true);
        if (!rc) rc = dalloc_n(c, &s->d_v, (size_t)std::max<int64_t>(s->cap_events, 1), true);
        if (!rc) rc = dalloc_n(c, &s->d_packed, (size_t)stim_words(s->cap_events, n_pi), true);
        if (!rc) rc = upload_stimulus(c, s.get(), off, t, v);
        if (rc) { free_stim(c, s.get()); return rc; }
        const int32_t id = c->next_id++;
        c->stims[id] = std::move(s);
        *stim_id = id;
        return GLS_OK;
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_update_stimulus(gls_ctx *c, int32_t stim_id, const int64_t *off, const int32_t *t, const uint8_t *v) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    StimObj *s = find_stim(c, stim_id);
    if (!s) return fail(GLS_EINVAL, "unknown stimulus id %d", stim_id);
    if (s->wide) return fail(GLS_EINVAL, "stimulus %d has 64-bit times; load a new one", stim_id);
    CK(cudaSetDevice(c->device));
    int rc = check_stimulus_host(s->n_pi, off, t, v, false);
    if (rc) return rc;
    if (off[s->n_pi] > s->cap_events)
        return fail(GLS_EOVERFLOW, "%lld transitions exceed the stimulus capacity %lld", (long long)off[s->n_pi],
                    (long long)s->cap_events);
    // runs reading this stimulus may still be in flight on other streams
    CK(cudaDeviceSynchronize());
    return upload_stimulus(c, s, off, t, v);
}

int gls_simulate(gls_ctx *c, int32_t netlist_id, int32_t stim_id, int64_t arena_events, void *cuda_stream,
                 int32_t *run_id) {
    return gls_simulate_batch(c, 1, &netlist_id, &stim_id, nullptr, arena_events, cuda_stream, run_id);
}

int gls_simulate_batch(gls_ctx *c, int32_t n_items, const int32_t *netlist_ids, const int32_t *stim_ids,
                       const int32_t *t_limits, int64_t arena_events, void *cuda_stream, int32_t *run_id) {
    if (!c || !run_id || !netlist_ids || !stim_ids) return fail(GLS_EINVAL, "NULL argument");
    if (n_items < 1) return fail(GLS_EINVAL, "a run needs at least one item");
    try {
        CK(cudaSetDevice(c->device));
        std::unique_ptr<RunObj> r;
        int rc = create_run(c, netlist_ids, stim_ids, t_limits, n_items, arena_events, r);
        if (rc) return rc;
        cudaError_t e = cudaGraphLaunch(r->exec, pick_stream(c, cuda_stream));
        if (e != cudaSuccess) { free_run(c, r.get()); return fail(GLS_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e)); }
        const int32_t id = c->next_id++;
        c->runs[id] = std::move(r);
        *run_id = id;
        return GLS_OK;
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int run_sliced(gls_ctx *c, RunObj *r, cudaStream_t cs);

int gls_rerun(gls_ctx *c, int32_t run_id, void *cuda_stream) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    if (r->slice_ps > 0) {
        CK(cudaSetDevice(c->device));
        try {
            return run_sliced(c, r, pick_stream(c, cuda_stream));
        } catch (const std::bad_alloc &) {
            return fail(GLS_ENOMEM, "host allocation failed");
        }
    }
    int rc = items_time_range_check(c, r);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    CK(cudaGraphLaunch(r->exec, pick_stream(c, cuda_stream)));
    return GLS_OK;
}

int gls_run_query(gls_ctx *c, int32_t run_id) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    CK(cudaSetDevice(c->device));
    const cudaError_t e = cudaEventQuery(r->ev1);
    if (e == cudaSuccess) return GLS_OK;
    if (e == cudaErrorNotReady) return GLS_EAGAIN;
    return fail(GLS_ECUDA, "cudaEventQuery: %s", cudaGetErrorString(e));
}

int gls_run_info(gls_ctx *c, int32_t run_id, int64_t *arena_demand, int64_t *arena_capacity) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    CK(cudaSetDevice(c->device));
    CK(cudaEventSynchronize(r->ev1));
    unsigned long long top = 0;
    CK(cudaMemcpy(&top, r->dev.arena_top, sizeof top, cudaMemcpyDeviceToHost));
    if (r->slice_ps > 0) top = (unsigned long long)r->sliced_demand;   // largest slice
    if (arena_demand) *arena_demand = (int64_t)top;
    if (arena_capacity) *arena_capacity = (int64_t)r->dev.arena_cap;
    return GLS_OK;
}

int run_stats_impl(gls_ctx *c, RunObj *r, int64_t *total_events, double *kernel_ms);

int gls_run_stats(gls_ctx *c, int32_t run_id, int64_t *total_events, double *kernel_ms) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    CK(cudaSetDevice(c->device));
    if (r->slice_ps > 0) {   // evaluated synchronously; errors were returned then
        if (total_events) *total_events = r->sliced_total;
        if (kernel_ms) *kernel_ms = r->sliced_ms;
        return GLS_OK;
    }
    return run_stats_impl(c, r, total_events, kernel_ms);
}

int run_stats_impl(gls_ctx *c, RunObj *r, int64_t *total_events, double *kernel_ms) {
    CK(cudaEventSynchronize(r->ev1));
    uint32_t status = 0;
    unsigned long long top = 0, sum = 0;
    CK(cudaMemcpyAsync(&status, r->dev.status, sizeof status, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&top, r->dev.arena_top, sizeof top, cudaMemcpyDeviceToHost, c->stream));
    // every net, minus the primary inputs (their transitions within the time limits)
    CK(launch_sum_gate_lengths(r->dev.net_len, 0, r->n_nets * r->launch_slices, r->d_sum, c->stream));
    unsigned long long pi_events = 0;
    CK(cudaMemcpyAsync(&pi_events, r->d_pi_total, sizeof pi_events, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&sum, r->d_sum, sizeof sum, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (kernel_ms) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r->ev0, r->ev1));
        *kernel_ms = ms;
    }
    if (status & kStArenaOverflow) {
        if (total_events) *total_events = (int64_t)top;
        return fail(GLS_EOVERFLOW, "event arena of %llu transitions too small; the run needs %llu",
                    (unsigned long long)r->dev.arena_cap, top);
    }
    if (total_events) *total_events = (int64_t)(sum - pi_events);
    if (status & kStPendingOverflow) return fail(GLS_ERANGE, "a cell's pending transitions exceeded the device buffer");
    if (status & kStTimeRange) return fail(GLS_ERANGE, "a computed time reached 2^30-1");
    if (status & kStTimeout) return fail(GLS_ETIMEOUT, "a wait for a fanin gate exceeded %.3f s",
                                         (double)r->dev.wait_limit_ns * 1e-9);
    return GLS_OK;
}

// Task division over time: the stimulus is cut at T_k = k * slice_ps and the
// slices are evaluated in order, each on the primary-input transitions
// inside it, in slice-local time.  Every gate carries its state across a
// boundary (input pin values, last output value, the scheduled transitions
// at or past the boundary, which later inputs may still cancel by Eq. 1); a
// transition scheduled before the boundary is final, because a later input
// can only schedule at or after boundary + dmin.  So the slices' outputs,
// concatenated, are the unsliced waveforms.  Under the dependency schedule
// one launch evaluates up to slice_group consecutive slices, a warp taking
// its gate through all of them in turn once the gate's fanins are done for
// all of them, so the per-gate costs are paid once per launch; under the
// level schedule each slice is one set of level launches.  The waveforms of
// a launch's slices are copied to host memory once it completes; a launch
// whose arena overflows is evaluated again with a larger one (its input
// state is never written by the launch).
int run_sliced(gls_ctx *c, RunObj *r, cudaStream_t cs) {
    const RunItem &it = r->items[0];
    NetlistObj *n = find_netlist(c, it.netlist_id);
    StimObj *s = find_stim(c, it.stim_id);
    const int64_t S = r->slice_ps, N = r->n_nets;
    const int64_t mt = s->wide ? s->max_time64 : (int64_t)s->max_time;
    const int32_t ns = s->n_events > 0 ? (int32_t)(mt / S + 1) : 1;
    const bool dep = r->schedule == GLS_SCHEDULE_DEPENDENCY;
    release_slices(c, r);
    r->sliced_total = 0;
    r->sliced_demand = 0;
    r->sliced_ms = 0.0;
    int in = 0;   // the state buffers holding the state at the next launch's start
    CK(cudaMemsetAsync(r->d_st[0], 0, sizeof(uint32_t) * (size_t)N, cs));   // start state
    for (int32_t k0 = 0; k0 < ns;) {
        const int32_t L = std::min(r->slice_group, ns - k0);
        const int o = (in + 1) % 3, a = (in + 2) % 3;
        RunDev d = r->dev;
        d.st_in = r->d_st[in];
        d.st_out = r->d_st[o];
        d.st_alt = r->d_st[a];
        d.pend_in = r->d_pend[in];
        d.pend_out = r->d_pend[o];
        d.pend_alt = r->d_pend[a];
        d.slices = L;
        d.slice_nets = N;
        d.slice_len = (uint32_t)S;
        d.slice_end = k0 + L == ns ? kTimeInf : (uint32_t)S;   // of the launch's last slice
        d.slice_shift = k0 == 0 ? 0u : (uint32_t)S;            // of its first
        r->launch_slices = L;
        int64_t total = 0;
        double ms = 0.0;
        for (int attempt = 0;; attempt++) {
            CK(cudaMemsetAsync(d.level_ctr, 0, sizeof(int32_t) * ((size_t)r->depth + 1), cs));
            CK(cudaMemsetAsync(d.arena_top, 0, sizeof(unsigned long long), cs));
            CK(cudaMemsetAsync(d.status, 0, sizeof(uint32_t), cs));
            if (dep) CK(cudaMemsetAsync(d.done, 0, sizeof(uint32_t) * (size_t)N, cs));
            CK(cudaMemsetAsync(r->d_pi_total, 0, sizeof(unsigned long long), cs));
            CK(launch_slice_pack(s->d_off, s->wide ? nullptr : s->d_t, s->wide ? s->d_t64 : nullptr, s->d_v, n->n_pi,
                                 (int64_t)k0 * S, S, L, k0 + L == ns, N, r->d_slice_packed, d.net_ptr, d.net_len,
                                 dep ? d.done : nullptr, r->d_pi_total, cs));
            CK(cudaEventRecord(r->ev0, cs));
            CK(launch_gates(c, r, d, cs));
            CK(cudaEventRecord(r->ev1, cs));
            const int rc = run_stats_impl(c, r, &total, &ms);
            if (rc == GLS_OK) break;
            if (rc != GLS_EOVERFLOW || attempt >= 8) return rc;
            // total is a lower bound of this launch's demand: grow and evaluate it again
            const uint64_t want = std::max<uint64_t>(2 * r->dev.arena_cap, (uint64_t)total + total / 4 + (1u << 20));
            dfree(c, r->dev.arena);
            r->dev.arena = nullptr;
            r->dev.arena_cap = 0;
            int arc = dalloc_n(c, &r->dev.arena, (size_t)want + 2 * kSlotAlign);
            if (arc) return arc;
            r->dev.arena_cap = want;
            d.arena = r->dev.arena;
            d.arena_cap = want;
        }
        unsigned long long top = 0;
        CK(cudaMemcpy(&top, d.arena_top, sizeof top, cudaMemcpyDeviceToHost));
        r->sliced_demand = std::max<int64_t>(r->sliced_demand, (int64_t)top);
        r->sliced_total += total;
        r->sliced_ms += ms;
        for (int32_t j = 0; j < L; j++) {
            RunObj::Slice sl;
            sl.t0 = (int64_t)(k0 + j) * S;
            sl.off.assign((size_t)N + 1, 0);
            int rc = read_item(c, r, 0, sl.off.data(), nullptr, 0, (int64_t)j * N);
            if (rc != GLS_OK && rc != GLS_EOVERFLOW) return rc;
            uint32_t *dst = nullptr;
            const int64_t n_words = sl.off[N];
            if (n_words > 0) {
                if (c->hpool.base)
                    dst = static_cast<uint32_t *>(pool_take(c->hpool, sizeof(uint32_t) * (uint64_t)n_words, false));
                if (dst) sl.pinned = dst;
                else sl.heap.reset(dst = new uint32_t[(size_t)n_words]);
            }
            r->slices.push_back(std::move(sl));   // the run owns the storage (and its pool block) from here
            if (dst) {
                rc = read_item(c, r, 0, r->slices.back().off.data(), dst, n_words, (int64_t)j * N);
                if (rc) return rc;
            }
        }
        in = (L & 1) ? o : a;   // slice L - 1 wrote st_out when L - 1 is even, st_alt when odd
        k0 += L;
    }
    return GLS_OK;
}

int gls_read_host(gls_ctx *c, int32_t run_id, int32_t item, const uint32_t **arena, int64_t *gate_off,
                  uint32_t *gate_len) {
    if (!c || !arena || !gate_off || !gate_len) return fail(GLS_EINVAL, "NULL argument");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    if (!r->h_arena) return fail(GLS_EINVAL, "run %d has no host mirror (set GLS_OPT_HOST_MIRROR before creating it)", run_id);
    if (item < 0 || item >= (int32_t)r->items.size()) return fail(GLS_EINVAL, "item %d out of range", item);
    CK(cudaSetDevice(c->device));
    int rc = run_stats_impl(c, r, nullptr, nullptr);   // waits; a failed run has no complete result
    if (rc) return rc;
    const RunItem &it = r->items[item];
    NetlistObj *n = find_netlist(c, it.netlist_id);
    const int64_t G = n->n_gates, N = (int64_t)n->n_pi + G;
    if (r->off_cap < N + 1) {
        dfree(c, r->d_off);
        dfree(c, r->d_scan_tmp);
        r->d_off = nullptr;
        r->d_scan_tmp = nullptr;
        r->off_cap = 0;
        r->scan_tmp = scan_tmp_elems(N + 1);
        rc = dalloc_n(c, &r->d_off, (size_t)N + 1);
        if (!rc) rc = dalloc_n(c, &r->d_scan_tmp, r->scan_tmp);
        if (rc) return rc;
        r->off_cap = N + 1;
    }
    if (r->glen_cap < G) {
        dfree(c, r->d_glen);
        r->d_glen = nullptr;
        r->glen_cap = 0;
        rc = dalloc_n(c, &r->d_glen, (size_t)std::max<int64_t>(G, 1));
        if (rc) return rc;
        r->glen_cap = G;
    }
    CK(launch_gather_descriptors(r->dev.net_ptr, r->dev.net_len, n->d_ext2int, n->n_pi, G, it.net_base, r->dev.arena,
                                 r->d_off, r->d_glen, c->stream));
    if (G > 0) {
        CK(cudaMemcpyAsync(gate_off, r->d_off, sizeof(int64_t) * (size_t)G, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(gate_len, r->d_glen, sizeof(uint32_t) * (size_t)G, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    *arena = r->h_arena;
    return GLS_OK;
}

// Critical-path-first order for the dependency schedule: w(g) = 64 + the
// transitions on g's fanin pins in the calibration run, b(g) = w(g) + max b
// over g's readers (longest weighted path to an output), gates by decreasing
// b.  b of a fanin gate exceeds b of its reader (w >= 64), so the order is
// topological, which keeps Algorithm 1's waits finite: every fanin gate of a
// handed-out gate was handed out earlier.
int gls_plan_order(gls_ctx *c, int32_t netlist_id, int32_t run_id, int32_t item) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    NetlistObj *n = find_netlist(c, netlist_id);
    if (!n) return fail(GLS_EINVAL, "unknown netlist id %d", netlist_id);
    CK(cudaSetDevice(c->device));
    if (run_id == -1) {
        n->d_plan = nullptr;
        return GLS_OK;
    }
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    if (item < 0 || item >= (int32_t)r->items.size()) return fail(GLS_EINVAL, "item %d out of range", item);
    if (r->items[item].netlist_id != netlist_id)
        return fail(GLS_EINVAL, "item %d of run %d is not an instance of netlist %d", item, run_id, netlist_id);
    int rc = gls_run_stats(c, run_id, nullptr, nullptr);
    if (rc) return rc;
    const int32_t P = n->n_pi, G = n->n_gates;
    std::vector<uint32_t> len((size_t)P + G);
    CK(cudaMemcpy(len.data(), r->dev.net_len + r->items[item].net_base, sizeof(uint32_t) * len.size(),
                  cudaMemcpyDeviceToHost));
    std::vector<int64_t> w((size_t)G), b((size_t)G);
    for (int32_t q = 0; q < G; q++) {
        const GateRec &g = n->recs[q];
        int64_t x = 64;
        for (int k = 0; k < g.k; k++) x += len[g.fin[k]];
        w[q] = b[q] = x;
    }
    for (int32_t q = G - 1; q >= 0; q--) {   // readers come later in level order
        const GateRec &g = n->recs[q];
        for (int k = 0; k < g.k; k++)
            if (g.fin[k] >= P) {
                const int32_t f = g.fin[k] - P;
                b[f] = std::max(b[f], w[f] + b[q]);
            }
    }
    std::vector<int32_t> order((size_t)G);
    for (int32_t q = 0; q < G; q++) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return b[x] > b[y]; });
    std::vector<GateRec> recs((size_t)std::max(G, 1));
    for (int32_t q = 0; q < G; q++) recs[q] = n->recs[order[q]];
    GateRec *d = nullptr;
    rc = dalloc_n(c, &d, recs.size(), true);
    if (rc) return rc;
    n->plans.push_back(d);
    CK(cudaMemcpy(d, recs.data(), sizeof(GateRec) * recs.size(), cudaMemcpyHostToDevice));
    n->d_plan = d;
    return GLS_OK;
}

int gls_read_waveform(gls_ctx *c, int32_t run_id, int32_t net, int32_t *t, uint8_t *v, int64_t cap, int64_t *n_out) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    if (r->slice_ps > 0) return fail(GLS_EINVAL, "run %d is sliced: read it with gls_read_waveform64", run_id);
    NetlistObj *n = find_netlist(c, r->items[0].netlist_id);
    const int64_t N = (int64_t)n->n_pi + n->n_gates;
    if (net < 0 || net >= N) return fail(GLS_EINVAL, "net %d out of range", net);
    CK(cudaSetDevice(c->device));
    CK(cudaEventSynchronize(r->ev1));
    const int64_t in = r->items[0].net_base + n->ext2int[net];
    uint64_t ptr = 0;
    uint32_t len = 0;
    CK(cudaMemcpy(&ptr, r->dev.net_ptr + in, sizeof ptr, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&len, r->dev.net_len + in, sizeof len, cudaMemcpyDeviceToHost));
    if (n_out) *n_out = len;
    if ((int64_t)len > cap) return fail(GLS_EOVERFLOW, "net %d has %u transitions, cap %lld", net, len, (long long)cap);
    if (len == 0) return GLS_OK;
    if (!t || !v) return fail(GLS_EINVAL, "NULL output arrays");
    try {
        std::vector<uint32_t> buf(len);
        CK(cudaMemcpy(buf.data(), reinterpret_cast<const void *>(ptr), sizeof(uint32_t) * len, cudaMemcpyDeviceToHost));
        for (uint32_t i = 0; i < len; i++) {
            t[i] = (int32_t)(buf[i] >> 2);
            v[i] = (uint8_t)(buf[i] & 3u);
        }
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
    return GLS_OK;
}

int gls_read_all(gls_ctx *c, int32_t run_id, int64_t *off, uint32_t *packed, int64_t cap) {
    return gls_read_item(c, run_id, 0, off, packed, cap);
}

int gls_read_item(gls_ctx *c, int32_t run_id, int32_t item, int64_t *off, uint32_t *packed, int64_t cap) {
    if (!c || !off) return fail(GLS_EINVAL, "NULL argument");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    if (r->slice_ps > 0) return fail(GLS_EINVAL, "run %d is sliced: read it with gls_read_all64", run_id);
    CK(cudaSetDevice(c->device));
    try {
        return read_item(c, r, item, off, packed, cap);
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_set_option(gls_ctx *c, int option, int64_t value) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    CK(cudaSetDevice(c->device));
    switch (option) {
    case GLS_OPT_SCHEDULE:
        if (value != GLS_SCHEDULE_LEVELS && value != GLS_SCHEDULE_DEPENDENCY)
            return fail(GLS_EINVAL, "unknown schedule %lld", (long long)value);
        c->schedule = (int)value;
        return GLS_OK;
    case GLS_OPT_WARPS_PER_CTA:
        if (value < 1 || value > 32) return fail(GLS_EINVAL, "warps per CTA must be in [1, 32]");
        return apply_launch_cfg(c, c->cfg.variant, (int)value);
    case GLS_OPT_WAIT_LIMIT_MS:
        if (value < 1) return fail(GLS_EINVAL, "wait limit must be >= 1 ms");
        c->wait_limit_ns = (uint64_t)value * 1000000ull;
        return GLS_OK;
    case GLS_OPT_KERNEL:
        if (value != GLS_KERNEL_SEGMENTED && value != GLS_KERNEL_WINDOWED && value != GLS_KERNEL_WINDOWED_WIDE)
            return fail(GLS_EINVAL, "unknown kernel variant %lld", (long long)value);
        return apply_launch_cfg(c, value == GLS_KERNEL_SEGMENTED ? kVariantSegmented
                                   : value == GLS_KERNEL_WINDOWED ? kVariantWindowed : kVariantWindowedWide,
                                c->cfg.warps_per_cta);
    case GLS_OPT_SEGMENT:
        if (value < 1 || value > (1 << 20)) return fail(GLS_EINVAL, "segment target must be in [1, 2^20]");
        c->seg_target = (uint32_t)value;
        return GLS_OK;
    case GLS_OPT_SLICE_GROUP:
        if (value < 1 || value > kMaxSliceGroup) return fail(GLS_EINVAL, "slice group must be in [1, %d]", kMaxSliceGroup);
        c->slice_group = (int32_t)value;
        return GLS_OK;
    case GLS_OPT_HOST_MIRROR:
        if (value != 0 && value != 1) return fail(GLS_EINVAL, "host mirror must be 0 or 1");
        c->host_mirror = value == 1;
        return GLS_OK;
    case GLS_OPT_POOL_BYTES: {
        if (value < 0) return fail(GLS_EINVAL, "pool size must be >= 0");
        if (!c->pool.allocs.empty()) return fail(GLS_EINVAL, "the pool still holds %zu blocks", c->pool.allocs.size());
        if (c->pool.base) {
            CK(cudaFree(c->pool.base));
            c->used -= c->pool.bytes;
            c->pool = Pool{};
        }
        if (value == 0) return GLS_OK;
        const uint64_t bytes = ((uint64_t)value + 255) & ~255ull;
        if (c->used + bytes > c->budget)
            return fail(GLS_ENOMEM, "pool of %llu bytes exceeds the device budget", (unsigned long long)bytes);
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GLS_ENOMEM, "cudaMalloc(pool %llu): %s", (unsigned long long)bytes, cudaGetErrorString(e));
        }
        c->pool.base = static_cast<char *>(p);
        c->pool.bytes = bytes;
        c->used += bytes;
        c->pool.free[0] = bytes;
        return GLS_OK;
    }
    case GLS_OPT_HOST_POOL_BYTES: {
        if (value < 0) return fail(GLS_EINVAL, "host pool size must be >= 0");
        if (!c->hpool.allocs.empty())
            return fail(GLS_EINVAL, "the host pool still holds %zu blocks (run mirrors or sliced results)",
                        c->hpool.allocs.size());
        if (c->hpool.base) {
            CK(cudaFreeHost(c->hpool.base));
            c->hpool = Pool{};
            c->hpool_dev = nullptr;
        }
        if (value == 0) return GLS_OK;
        const uint64_t bytes = ((uint64_t)value + 255) & ~255ull;
        void *h = nullptr, *d = nullptr;
        cudaError_t e = cudaHostAlloc(&h, bytes, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&d, h, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (h) cudaFreeHost(h);
            return fail(GLS_ENOMEM, "pinned host pool of %llu bytes: %s", (unsigned long long)bytes,
                        cudaGetErrorString(e));
        }
        c->hpool.base = static_cast<char *>(h);
        c->hpool.bytes = bytes;
        c->hpool.free[0] = bytes;
        c->hpool_dev = static_cast<char *>(d);
        return GLS_OK;
    }
    case GLS_OPT_TEST_WITHHOLD_GATE:
        if (value < -1 || value > INT32_MAX) return fail(GLS_EINVAL, "gate index out of range");
        c->withhold_gate = (int32_t)value;
        return GLS_OK;
    }
    return fail(GLS_EINVAL, "unknown option %d", option);
}

int gls_simulate_noalloc(gls_ctx *c, int32_t netlist_id, int32_t stim_id, uint64_t *d_net_ptr,
                         uint32_t *d_net_len, uint32_t *d_arena, int64_t arena_words, uint32_t *d_report,
                         void *cuda_stream) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    if (!d_net_ptr || !d_net_len || !d_arena || !d_report) return fail(GLS_EINVAL, "NULL device buffer");
    NetlistObj *n = find_netlist(c, netlist_id);
    StimObj *s = find_stim(c, stim_id);
    if (!n) return fail(GLS_EINVAL, "unknown netlist id %d", netlist_id);
    if (!s) return fail(GLS_EINVAL, "unknown stimulus id %d", stim_id);
    if (s->n_pi != n->n_pi) return fail(GLS_EINVAL, "stimulus has %d PIs, netlist %d", s->n_pi, n->n_pi);
    if (s->wide) return fail(GLS_EINVAL, "a stimulus with 64-bit times runs only in time slices");
    if (n->general && c->cfg.variant == kVariantSegmented)
        return fail(GLS_EINVAL, "the netlist needs the windowed kernels");
    if (n->lv.depth > GLS_NOALLOC_MAX_LEVELS)
        return fail(GLS_ERANGE, "netlist depth %d exceeds the %d levels of the no-allocation scratch",
                    n->lv.depth, GLS_NOALLOC_MAX_LEVELS);
    if (reinterpret_cast<uintptr_t>(d_arena) & 15u) return fail(GLS_EINVAL, "d_arena must be 16-byte aligned");
    if (arena_words < 2 * (int64_t)kSlotAlign)
        return fail(GLS_EINVAL, "arena of %lld words is below the %u-word minimum", (long long)arena_words,
                    2 * kSlotAlign);
    int rc = time_range_check(n, s);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    uint32_t *scratch = nullptr;
    rc = noalloc_scratch(c->device, &scratch);
    if (rc) return rc;
    RunDev r{};
    r.net_ptr = d_net_ptr;
    r.net_len = d_net_len;
    r.arena = d_arena;
    r.arena_cap = (uint64_t)arena_words - 2 * kSlotAlign;   // the last words stay as read padding
    r.arena_top = reinterpret_cast<unsigned long long *>(scratch);
    r.status = scratch + 2;
    r.level_ctr = reinterpret_cast<int32_t *>(scratch + 64);
    r.done = nullptr;
    r.n_pi = n->n_pi;
    r.n_gates = n->n_gates;
    r.wait_limit_ns = c->wait_limit_ns;
    r.withhold_gate = -1;
    r.seg_target = c->seg_target;
    cudaStream_t st = pick_stream(c, cuda_stream);
    // run_init zeroes the counters (one per level, all inside the array because
    // depth <= GLS_NOALLOC_MAX_LEVELS), the arena top and the status left by
    // the previous call
    CK(launch_run_init(s->d_off, s->d_packed, r, n->lv.depth, st));
    for (int32_t L = 1; L <= n->lv.depth; L++) {
        const int32_t b = n->lv.level_begin[L], cnt = n->lv.level_begin[L + 1] - b;
        CK(launch_level(n->d_gates, b, cnt, L - 1, r, c->cfg, st));
    }
    noalloc_report_kernel<<<1, 1, 0, st>>>(d_report);
    CK(cudaGetLastError());
    return GLS_OK;
}

int gls_release(gls_ctx *c, int32_t id) {
    if (!c) return fail(GLS_EINVAL, "NULL context");
    cudaSetDevice(c->device);
    if (auto it = c->runs.find(id); it != c->runs.end()) {
        cudaEventSynchronize(it->second->ev1);
        free_run(c, it->second.get());
        c->runs.erase(it);
        return GLS_OK;
    }
    for (auto &kv : c->runs)
        for (const RunItem &it : kv.second->items)
            if (it.netlist_id == id || it.stim_id == id)
                return fail(GLS_EINVAL, "id %d is still used by run %d", id, kv.first);
    if (auto it = c->stims.find(id); it != c->stims.end()) {
        free_stim(c, it->second.get());
        c->stims.erase(it);
        return GLS_OK;
    }
    if (auto it = c->netlists.find(id); it != c->netlists.end()) {
        free_netlist(c, it->second.get());
        c->netlists.erase(it);
        return GLS_OK;
    }
    return fail(GLS_EINVAL, "unknown id %d", id);
}


int gls_load_stimulus64(gls_ctx *c, int32_t n_pi, const int64_t *off, const int64_t *t, const uint8_t *v,
                        int32_t *stim_id) {
    if (!c || !stim_id) return fail(GLS_EINVAL, "NULL argument");
    try {
        CK(cudaSetDevice(c->device));
        int64_t mx = 0;
        int rc = check_stimulus64_host(n_pi, off, t, v, &mx);
        if (rc) return rc;
        auto s = std::make_unique<StimObj>();
        s->n_pi = n_pi;
        s->wide = true;
        s->cap_events = s->n_events = off[n_pi];
        s->max_time64 = mx;
        const size_t E = (size_t)std::max<int64_t>(s->cap_events, 1);
        rc = dalloc_n(c, &s->d_off, (size_t)n_pi + 1, true);
        if (!rc) rc = dalloc_n(c, &s->d_t64, E, true);
        if (!rc) rc = dalloc_n(c, &s->d_v, E, true);
        if (rc) { free_stim(c, s.get()); return rc; }
        cudaError_t e = cudaMemcpy(s->d_off, off, sizeof(int64_t) * ((size_t)n_pi + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && s->n_events > 0)
            e = cudaMemcpy(s->d_t64, t, sizeof(int64_t) * (size_t)s->n_events, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && s->n_events > 0) e = cudaMemcpy(s->d_v, v, (size_t)s->n_events, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { free_stim(c, s.get()); return fail(GLS_ECUDA, "stimulus upload: %s", cudaGetErrorString(e)); }
        const int32_t id = c->next_id++;
        c->stims[id] = std::move(s);
        *stim_id = id;
        return GLS_OK;
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_simulate_sliced(gls_ctx *c, int32_t netlist_id, int32_t stim_id, int64_t slice_ps, int64_t arena_events,
                        void *cuda_stream, int32_t *run_id) {
    if (!c || !run_id) return fail(GLS_EINVAL, "NULL argument");
    if (slice_ps < 1) return fail(GLS_EINVAL, "slice_ps must be >= 1");
    try {
        CK(cudaSetDevice(c->device));
        std::unique_ptr<RunObj> r;
        int rc = create_run(c, &netlist_id, &stim_id, nullptr, 1, arena_events, r, slice_ps);
        if (rc) return rc;
        rc = run_sliced(c, r.get(), pick_stream(c, cuda_stream));
        if (rc) { free_run(c, r.get()); return rc; }
        const int32_t id = c->next_id++;
        c->runs[id] = std::move(r);
        *run_id = id;
        return GLS_OK;
    } catch (const std::bad_alloc &) {
        return fail(GLS_ENOMEM, "host allocation failed");
    }
}

int gls_run_slices(gls_ctx *c, int32_t run_id, int32_t *n_slices) {
    if (!c || !n_slices) return fail(GLS_EINVAL, "NULL argument");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    *n_slices = r->slice_ps > 0 ? (int32_t)r->slices.size() : 0;
    return GLS_OK;
}

int gls_read_all64(gls_ctx *c, int32_t run_id, int64_t *off, int64_t *t, uint8_t *v, int64_t cap) {
    if (!c || !off) return fail(GLS_EINVAL, "NULL argument");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    if (r->slice_ps == 0) return fail(GLS_EINVAL, "run %d is not sliced: read it with gls_read_all", run_id);
    const int64_t N = r->n_nets;
    off[0] = 0;
    for (int64_t q = 0; q < N; q++) {
        int64_t len = 0;
        for (const auto &sl : r->slices) len += sl.off[q + 1] - sl.off[q];
        off[q + 1] = off[q] + len;
    }
    if (off[N] > cap) return fail(GLS_EOVERFLOW, "%lld transitions, cap %lld", (long long)off[N], (long long)cap);
    if (off[N] > 0 && (!t || !v)) return fail(GLS_EINVAL, "NULL output arrays");
    // widen every slice's words into the caller's arrays, nets split over the
    // host's cores when there is enough to do (each net's range is its own)
    auto widen = [&](int64_t q0, int64_t q1) {
        for (int64_t q = q0; q < q1; q++) {
            int64_t o = off[q];
            for (const auto &sl : r->slices) {
                const uint32_t *w = sl.words();
                for (int64_t e = sl.off[q]; e < sl.off[q + 1]; e++, o++) {
                    t[o] = sl.t0 + (int64_t)(w[e] >> 2);
                    v[o] = (uint8_t)(w[e] & 3u);
                }
            }
        }
    };
    const int64_t nt = off[N] < (1 << 22) ? 1 : std::min<int64_t>(16, std::max(1u, std::thread::hardware_concurrency()));
    if (nt == 1) {
        widen(0, N);
        return GLS_OK;
    }
    std::vector<std::thread> pool;
    int64_t done_to = 0;   // nets widened by this thread when a worker cannot be started
    try {
        for (int64_t k = 0; k < nt; k++) {
            pool.emplace_back(widen, N * k / nt, N * (k + 1) / nt);
            done_to = N * (k + 1) / nt;
        }
    } catch (const std::exception &) {
        widen(done_to, N);
    }
    for (auto &th : pool) th.join();
    return GLS_OK;
}

int gls_read_waveform64(gls_ctx *c, int32_t run_id, int32_t net, int64_t *t, uint8_t *v, int64_t cap,
                        int64_t *n_out) {
    if (!c || !n_out) return fail(GLS_EINVAL, "NULL argument");
    RunObj *r = find_run(c, run_id);
    if (!r) return fail(GLS_EINVAL, "unknown run id %d", run_id);
    if (r->slice_ps == 0) return fail(GLS_EINVAL, "run %d is not sliced: read it with gls_read_waveform", run_id);
    if (net < 0 || net >= r->n_nets) return fail(GLS_EINVAL, "net %d out of range", net);
    int64_t len = 0;
    for (const auto &sl : r->slices) len += sl.off[net + 1] - sl.off[net];
    *n_out = len;
    if (len > cap) return fail(GLS_EOVERFLOW, "%lld transitions, cap %lld", (long long)len, (long long)cap);
    if (len > 0 && (!t || !v)) return fail(GLS_EINVAL, "NULL output arrays");
    int64_t o = 0;
    for (const auto &sl : r->slices) {
        const uint32_t *w = sl.words();
        for (int64_t e = sl.off[net]; e < sl.off[net + 1]; e++, o++) {
            t[o] = sl.t0 + (int64_t)(w[e] >> 2);
            v[o] = (uint8_t)(w[e] & 3u);
        }
    }
    return GLS_OK;
}

}  // extern "C"
