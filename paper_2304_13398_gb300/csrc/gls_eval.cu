// gls_eval.cu -- gate evaluation kernels: one warp evaluates one gate at a time.
//
// For a gate with K <= 3 fanin waveforms the warp streams the fanins in
// chunks through shared memory.  Per chunk:
//   1. a window of up to 3 CH / K transitions of every pin sits in shared
//      memory (one bulk copy per pin, completed on an mbarrier, issued as
//      soon as the previous chunk's walk was done with the windows, so it
//      overlaps that chunk's commit); the chunk is cut at T_end, the earliest
//      window end among pins with more transitions left, so every transition
//      at t <= T_end is present and a timestamp never straddles two chunks;
//   2. the pins are merged by time with merge-path partitions (pins a and b
//      first for 3-input cells), each lane taking an equal share; an
//      all-ones sentinel after every window removes bounds checks;
//   3. each lane walks its share in time order, applying all transitions of
//      one timestamp together, and when the cell value changes produces the
//      scheduled transition (t + min delay over the pins with a transition
//      at t, new value) -- Algorithm 2, minimum delay of Sec. 2.3;
//   4. Eq. 1: a transition survives iff its t_r is below the t_r of every
//      later one.  Each lane keeps a monotone stack of its own share, a warp
//      suffix minimum across lanes finishes the test, and transitions carried
//      over from the previous chunk are filtered by the chunk minimum;
//   5. every survivor with t_r < T_end + 1 + dmin is final (no later
//      transition of this gate can reach back that far): it is written out
//      unless it equals the value before it (Fig. 6); the rest is carried to
//      the next chunk (at most dmax - dmin transitions).
// Step 4's scan form equals the sequential "deny and replace" of Sec. 2.3:
// a transition is denied iff a later-determined one has t_r <= its t_r.
//
// Output allocation: before evaluating, the warp reserves the Eq. 2 bound
// (sum of fanin lengths >= distinct input timestamps >= output length),
// rounded up to 32 words, from the run's event arena with one atomicAdd and
// records (address, length) in the net descriptors when done.
//
// Two schedules share the gate code:
//   level mode       one launch per level (captured in one CUDA graph); the
//                    launch boundary orders a level after the one before;
//   dependency mode  one persistent launch for all gates (Algorithm 1): a
//                    warp takes the next gate in a topological order and waits, with
//                    a bounded spin, until each fanin gate has published its
//                    waveform (release/acquire flags), so no level barrier
//                    holds work back behind the longest gate of a level.
#include "gls_internal.h"

namespace gls {

namespace {

constexpr int PCAP = kPendCap;          // carried (pending) transitions, > GLS_MAX_DELAY_SPREAD

// Window size of the default ('wide') variant and its register cap in the
// persistent kernel (compile-time tuning knobs).
#ifndef GLS_WIDE_CH
#define GLS_WIDE_CH 352
#endif
#ifndef GLS_WIDE_MAXNREG
#define GLS_WIDE_MAXNREG 128
#endif
constexpr int kWideCH = GLS_WIDE_CH;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t EINF = 0xFFFFFFFFu;  // sentinel event; its time 2^30-1 exceeds every real time

// Shared memory of one warp of the windowed variant with CH transitions per
// pin window.
template <int CH>
struct __align__(16) WarpSmem {
    static constexpr int WIN = CH + 8;     // aligned lead (<= 3) + CH + sentinel, multiple of 4
    uint32_t win[1][3][WIN];  // pin windows (refilled while the chunk's survivors are committed)
    // per-lane stacks of scheduled transitions (t_r << 2 | v), column by
    // column: entry k of lane l at cand[32 k + l] (cslot), so that the lanes'
    // pushes, pops and reads fall into distinct banks; a lane's share of a
    // chunk holds at most 3 CH / 32 transitions, hence at most that many
    // entries
    uint32_t cand[3 * CH];
    // Q: carried transitions (front, at most PCAP) + this chunk's survivors
    // (at most 3 CH).  The survivors are written only after the walk, so the
    // part past PCAP also holds the 3-input cells' merged pins a+b during the
    // walk: B (2 CH + 4 words, sentinel-terminated) and Binfo (source of B[i]:
    // pin b flag (bit 15) | index in its window; 2 CH + 8 halves).
    uint32_t Q[PCAP + 3 * CH + 8];
    // cells whose delays depend on the input edge: delay - dmin by output
    // value (0, 1, X) and set of (pin, edge) pairs changed at the timestamp
    // (bit 2p: pin p rose, bit 2p+1: it fell; both for X<->Z)
    uint8_t dtab[3][64];
    // two-input cells: (delay - dmin) << 2 | new value, by changed-pin set
    // (bits 4-5) and pin values (bits 0-3)
    uint16_t ftab[64];
    uint8_t f3[64];           // three-input cells: the value for each of the 64 pin-value states
    uint64_t mbar[1];         // completion barrier of the window buffer
    __device__ __forceinline__ uint32_t *B() { return Q + PCAP; }
    __device__ __forceinline__ uint16_t *Binfo() { return reinterpret_cast<uint16_t *>(Q + PCAP + 2 * CH + 4); }
    // A K-pin cell spreads the three windows of a buffer over its K pins:
    // chunk<K>() transitions per pin (3 CH, 1.5 CH rounded to 32, CH), so
    // one- and two-input cells take fewer, longer chunks.
    template <int K>
    __host__ __device__ static constexpr int chunk() { return K == 3 ? CH : (K == 2 ? (3 * CH / 2) & ~31 : 3 * CH); }
    template <int K>
    __device__ __forceinline__ uint32_t *window(int b, int p) { return &win[0][0][0] + p * (chunk<K>() + 8); }
};

// A warp's current block of the event arena, [cur, end).  The gates a warp
// evaluates take their output slots from it one after another: a slot is the
// gate's Eq. 2 bound (rounded up to whole 128-byte lines) while the gate
// runs and shrinks to its actual length (rounded up likewise) when the gate
// is done, so the arena holds about the real output instead of the bounds.
// A gate whose bound does not fit the rest of the block claims a new block of
// max(bound, r.arena_blk) words with one atomicAdd on the arena top (the rest
// of the old block stays unused); r.arena_blk = 0 gives every gate a slot of
// its own, exactly its bound.
struct WarpArena {
    unsigned long long cur, end;
};

// Word of stack entry k of a lane (column-major per-lane stacks).
__device__ __forceinline__ int cslot(int k, int lane) { return (k << 5) + lane; }

// Running state of one gate's output between chunks.
struct CommitState {
    uint32_t outCount;   // transitions written
    uint32_t lastV;      // value of the last final survivor (kept or dropped)
    int np;              // carried transitions in Q[0..np)
};

// Bulk (TMA) copies of pin windows into shared memory, completed on the
// window buffer's mbarrier: lane 0 announces the bytes, lane p issues pin
// p's copy, every lane waits for the barrier's phase.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// Orders this thread's generic-proxy accesses of global memory with its
// async-proxy (bulk copy) accesses: a waveform written with ordinary stores
// by one warp is read with cp.async.bulk by another in the same launch.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
constexpr uint64_t kWindowWaitNs = 2000000000ull;   // bound on one window wait (2 s; a copy takes microseconds)


__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Once per warp before its first gate: the window barrier (phase parity 0).
template <int CH>
__device__ __forceinline__ void init_window_barriers(WarpSmem<CH> &sm, int lane) {
    if (lane == 0) {
        mbar_init(&sm.mbar[0]);
        mbar_init_fence();
    }
    __syncwarp();
}

// Wait for window buffer b (parity bit b of par, flipped on completion);
// false if the copies did not complete within kWindowWaitNs.
template <int CH>
__device__ __forceinline__ bool wait_window(WarpSmem<CH> &sm, int b, uint32_t &par) {
    const uint32_t ph = (par >> b) & 1u;
    if (!mbar_try_wait(&sm.mbar[b], ph)) {
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&sm.mbar[b], ph))
            if (globaltimer() - t0 > kWindowWaitNs) return false;
    }
    par ^= 1u << b;
    return true;
}

// Number of elements of L among the first d elements of merge(L, R), where an
// element of L precedes an element of R at equal time.
__device__ __forceinline__ int corank(int d, const uint32_t *L, int nL, const uint32_t *R, int nR) {
    int lo = max(0, d - nR), hi = min(d, nL);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (L[mid] <= (R[d - mid - 1] | 3u)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t setpin(uint32_t st, int pin, uint32_t v) {
    return (st & ~(3u << (2 * pin))) | (v << (2 * pin));
}

struct GateCtx {
    const uint32_t *src[3];
    uint32_t len[3];
    uint32_t rise[3], fall[3], dx[3];   // pin 0's arc (one-input cells)
    uint32_t dmin, dmax;
    uint64_t lut_lo, lut_hi;
    // min over the pins of a pin set of (delay - dmin), one byte per set
    // (bit p = pin p; byte 0, the empty set, is 0): sets 0-3 in *_lo,
    // 4-7 in *_hi; for a fall (f), a rise (r) and a change to X (x)
    uint32_t df_lo, df_hi, dr_lo, dr_hi, dx_lo, dx_hi;
};

// Delay of a timestamp at which the pins of set `grp` changed and the cell's
// value became F (min over those pins with an arc, Sec. 3 delay rule; the
// output's fastest arc when none has one).  Byte grp of the table pair; the
// other bytes of the permute read byte 0, which is 0.
template <int K>
__device__ __forceinline__ uint32_t group_delay(const GateCtx &g, uint32_t F, uint32_t grp) {
    const uint32_t lo = F == 1u ? g.dr_lo : (F == 0u ? g.df_lo : g.dx_lo);
    const uint32_t hi = K == 3 ? (F == 1u ? g.dr_hi : (F == 0u ? g.df_hi : g.dx_hi)) : 0u;
    return g.dmin + __byte_perm(lo, hi, grp);
}

__device__ __forceinline__ uint32_t pin_delay(const GateCtx &g, int p, uint32_t F) {
    return F == 1u ? g.rise[p] : (F == 0u ? g.fall[p] : g.dx[p]);
}

// Edge class of a pin transition old -> new, index old * 4 + new, 2 bits
// each: 1 rising (0->1, 0->X, 0->Z, X->1, Z->1), 2 falling (the mirror
// images), 3 neither (X<->Z, counted as both edges).
constexpr uint32_t kEdgeLut = 0x36C6A254u;
__device__ __forceinline__ uint32_t edge_class(uint32_t old, uint32_t nw) {
    return (kEdgeLut >> (2u * ((old << 2) | nw))) & 3u;
}

// Issue the asynchronous copies of every pin's next window into buffer b.
// Window p covers transitions [cur[p], cur[p] + n[p]); the copy starts at the
// 16-byte boundary below cur[p] (lead[p] <= 3 words) and ends at a multiple
// of 4 words, which stays inside the net's slot (slots are padded).
template <int K, int CH>
__device__ __forceinline__ bool issue_windows(WarpSmem<CH> &sm, int b, const GateCtx &g, const uint32_t *cur,
                                              int *lead, int *n, int lane) {
    uint32_t bytes[3] = {0u, 0u, 0u}, total = 0;
#pragma unroll
    for (int p = 0; p < K; p++) {
        const int np = (int)min((uint32_t)WarpSmem<CH>::template chunk<K>(), g.len[p] - cur[p]);
        n[p] = np;
        lead[p] = (int)(cur[p] & 3u);
        if (np > 0) {
            bytes[p] = (uint32_t)((lead[p] + np + 3) >> 2) * 16u;
            total += bytes[p];
        }
    }
    if (total > 0 && lane < K) {
        fence_proxy_async();   // the warp's earlier reads and writes of buffer b precede the copies
        if (lane == 0) mbar_arrive_expect_tx(&sm.mbar[b], total);
        // one lane per pin
        const uint32_t by = lane == 0 ? bytes[0] : (lane == 1 ? bytes[1] : bytes[2]);
        const uint32_t cu = lane == 0 ? cur[0] : (lane == 1 ? cur[1] : cur[2]);
        const uint32_t *src = lane == 0 ? g.src[0] : (lane == 1 ? g.src[1] : g.src[2]);
        if (by) bulk_load(sm.template window<K>(b, lane), src + (cu & ~3u), by, &sm.mbar[b]);
    }
    return total > 0;
}

// Steps 4 and 5 of a chunk, shared by every pin count.  Lane l's stack
// holds top - d0 entries (cand[cslot(0, l)] at the bottom).  Returns false
// when more than PCAP transitions would be carried.
template <int CH, bool MIRROR>
__device__ __forceinline__ bool commit_chunk(WarpSmem<CH> &sm, int lane, int d0, int top, uint32_t Tfin, uint32_t *out,
                                          uint32_t *hout, CommitState &cs) {
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    // Eq. 1 across lanes (suffix minimum of the later lanes' smallest t_r)
    // and against the carried transitions (minimum over the whole chunk)
    const uint32_t mn = top > d0 ? (sm.cand[cslot(0, lane)] >> 2) : kTimeInf;
    uint32_t inc = mn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_down_sync(FULL, inc, o);
        if (lane + o < 32) inc = min(inc, y);
    }
    uint32_t after = __shfl_down_sync(FULL, inc, 1);
    if (lane == 31) after = kTimeInf;
    const uint32_t Mall = __shfl_sync(FULL, inc, 0);
    while (top > d0 && (sm.cand[cslot(top - 1 - d0, lane)] >> 2) >= after) top--;
    const int np = cs.np;
    int npk = 0;
    for (int b0 = 0; b0 < np; b0 += 32) {
        const int idx = b0 + lane;
        npk += __popc(__ballot_sync(FULL, idx < np && (sm.Q[idx] >> 2) < Mall));
    }
    // survivors, in order, behind the carried ones that survive
    const uint32_t cnt = (uint32_t)(top - d0);
    uint32_t pre = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, pre, o);
        if (lane >= o) pre += y;
    }
    const int total = (int)__shfl_sync(FULL, pre, 31);
    const int pos = npk + (int)(pre - cnt);
    __syncwarp();
#pragma unroll 4
    for (uint32_t x = 0; x < cnt; x++) sm.Q[pos + x] = sm.cand[cslot((int)x, lane)];
    const int nQ = npk + total;
    __syncwarp();
    // commit the final prefix (t_r < Tfin), dropping repeats (Fig. 6)
    int nf = 0;
    uint32_t outCount = cs.outCount;
    uint32_t vlast = cs.lastV;   // value of the element before this round
    // two batches of 32 per round, independent but for the carried values;
    // t_r increases along Q, so the final ones are a prefix and the second
    // batch has none unless the first is all final
    for (int b0 = 0; b0 < nQ; b0 += 64) {
        const int i1 = b0 + lane, i2 = b0 + 32 + lane;
        const uint32_t e1 = i1 < nQ ? sm.Q[i1] : 0u, e2 = i2 < nQ ? sm.Q[i2] : 0u;
        const bool f1 = i1 < nQ && (e1 >> 2) < Tfin, f2 = i2 < nQ && (e2 >> 2) < Tfin;
        const uint32_t v1 = e1 & 3u, v2 = e2 & 3u;
        const uint32_t up1 = __shfl_up_sync(FULL, v1, 1), up2 = __shfl_up_sync(FULL, v2, 1);
        const uint32_t last1 = __shfl_sync(FULL, v1, 31);
        const bool k1 = f1 && v1 != (lane == 0 ? vlast : up1);
        const bool k2 = f2 && v2 != (lane == 0 ? last1 : up2);
        vlast = __shfl_sync(FULL, v2, 31);
        const uint32_t bk1 = __ballot_sync(FULL, k1), bk2 = __ballot_sync(FULL, k2);
        const uint32_t n1 = __popc(bk1);
        if (k1) {
            const uint32_t at = outCount + __popc(bk1 & lanemask_lt);
            out[at] = e1;
        }
        if (k2) {
            const uint32_t at = outCount + n1 + __popc(bk2 & lanemask_lt);
            out[at] = e2;
        }
        outCount += n1 + __popc(bk2);
        const uint32_t bf1 = __ballot_sync(FULL, f1), bf2 = __ballot_sync(FULL, f2);
        nf += __popc(bf1) + __popc(bf2);
        if ((bf1 & bf2) != FULL) break;   // the rest stays pending
    }
    cs.outCount = outCount;
    if (nf > 0) cs.lastV = sm.Q[nf - 1] & 3u;
    // carry the rest to the front of Q
    const int npn = nQ - nf;
    if (npn > PCAP) return false;
    for (int b0 = 0; b0 < npn; b0 += 32) {
        const int idx = b0 + lane;
        const uint32_t e = idx < npn ? sm.Q[nf + idx] : 0u;
        __syncwarp();
        if (idx < npn) sm.Q[idx] = e;
    }
    cs.np = npn;
    return true;
}

// Steps 1-5 for every chunk of one gate's inputs (or of one time slice's):
// the chunk cut, the merge and per-lane walk, the window refill and the
// commit, until the windows are exhausted.  Returns false only when a window
// copy did not complete within its poll bound.
template <int K, int CH, bool EDGE, bool MIRROR>
__device__ __forceinline__ bool run_chunks(const RunDev &r, WarpSmem<CH> &sm, GateCtx &g, int lane, uint32_t &par,
                                           bool &more, uint32_t (&cur)[3], int (&lead)[3], int (&n)[3],
                                           uint32_t &carry, bool &started, CommitState &cs, uint32_t send,
                                           uint32_t *out, uint32_t *hout, bool &failed) {
    const int b = 0;   // the one window buffer
    // 4-value tables: K == 1 uses f(a) with b = c = X (entries 40..43),
    // K == 2 uses f(a, b) with c = X (entries 32..47), K == 3 all 64
    const uint32_t lut1 = (uint32_t)(g.lut_hi >> 16) & 0xFFu;
    const uint32_t lut2 = (uint32_t)g.lut_hi;

    while (more) {
        if (!wait_window(sm, b, par)) {   // the copies never completed: stop this warp
            if (lane == 0) atomicOr(r.status, kStTimeout);
            return false;
        }
        const uint32_t *A[3];
#pragma unroll
        for (int p = 0; p < 3; p++) A[p] = sm.template window<K>(b, p < K ? p : 0) + (p < K ? lead[p] : 0);

        // ---- 1. chunk cut ----
        uint32_t Tend = kTimeInf;
#pragma unroll
        for (int p = 0; p < K; p++)
            if (n[p] > 0 && cur[p] + (uint32_t)n[p] < g.len[p]) Tend = min(Tend, A[p][n[p] - 1] >> 2);
        const bool last = (Tend == kTimeInf);
        int m[3] = {0, 0, 0};
        if (last) {
#pragma unroll
            for (int p = 0; p < K; p++) m[p] = n[p];
        } else {
            // m[p] = transitions of window p at or before Tend (a prefix):
            // count the S-blocks whose last transition qualifies, then the
            // qualifying transitions of the first block that does not (its
            // last one does not qualify, so S - 1 <= 32 tests suffice).  S is
            // odd, so the 32 block ends fall into 32 different banks.
            constexpr int S = ((WarpSmem<CH>::template chunk<K>() + 31) / 32) | 1;
            static_assert(32 * S >= WarpSmem<CH>::template chunk<K>() && S <= 33, "cut blocks");
            int q[3];
#pragma unroll
            for (int p = 0; p < K; p++) {
                const int x = S * lane + S - 1;
                q[p] = __popc(__ballot_sync(FULL, x < n[p] && (A[p][x] >> 2) <= Tend));
            }
#pragma unroll
            for (int p = 0; p < K; p++) {
                const int x = S * q[p] + lane;
                m[p] = S * q[p] + __popc(__ballot_sync(FULL, lane < S && x < n[p] && (A[p][x] >> 2) <= Tend));
            }
        }
        if (lane == 0) {   // every t_r of this chunk is below the latest input time + dmax
            uint32_t tmx = 0;
#pragma unroll
            for (int p = 0; p < K; p++)
                if (m[p] > 0) tmx = max(tmx, A[p][m[p] - 1] >> 2);
            if (tmx + g.dmax >= kTimeLimit) atomicOr(r.status, kStTimeRange);
        }
        uint32_t ncur[3] = {cur[0], cur[1], cur[2]};
#pragma unroll
        for (int p = 0; p < K; p++) ncur[p] += (uint32_t)m[p];
        int nlead[3] = {0, 0, 0}, nn[3] = {0, 0, 0};
        if (lane < K) {   // sentinels after the consumed part of every window
            const int at = lane == 0 ? lead[0] + m[0] : (lane == 1 ? lead[1] + m[1] : lead[2] + m[2]);
            sm.template window<K>(b, lane)[at] = EINF;
        }
        __syncwarp();

        // ---- 2./3. merge and per-lane walk (Algorithm 2 + local Eq. 1 stack) ----
        const uint32_t *L = A[0];
        const uint32_t *R = A[K - 1];
        int nL = m[0], nR = K >= 2 ? m[K - 1] : 0;
        if (K == 3) {
            const int M1 = m[0] + m[1];
            const int d0 = (lane * M1) >> 5, d1 = ((lane + 1) * M1) >> 5;
            int i = corank(d0, A[0], m[0], A[1], m[1]), j = d0 - i;
            uint32_t hl = A[0][i], hr = A[1][j];
            for (int s = d0; s < d1; s++) {
                const bool tl = hl <= (hr | 3u);
                sm.B()[s] = tl ? hl : hr;
                sm.Binfo()[s] = tl ? (uint16_t)i : (uint16_t)(0x8000u | (uint32_t)j);
                if (tl) { i++; hl = A[0][i]; } else { j++; hr = A[1][j]; }
            }
            if (lane == 0) sm.B()[M1] = EINF;
            __syncwarp();
            L = sm.B();
            nL = M1;
        }
        const int M = nL + nR;
        const int d0 = (lane * M) >> 5, d1 = ((lane + 1) * M) >> 5;
        int top = d0;
        // The walks are branch-free apart from the Eq. 1 pop loop: state
        // updates are selects, the stack top sits in a register, and a
        // candidate is always written one entry above the stack top (scratch
        // inside the lane's column) and kept by advancing the top.
        if (K == 1) {
            // one pin: every transition is its own timestamp
            uint32_t vprev = d0 > 0 ? (L[d0 - 1] & 3u) : (carry & 3u);   // pin value before the share
            // the output before the first input transition is X (Algorithm 2)
            uint32_t Fprev = (d0 == 0 && !started) ? kVX : (lut1 >> (2 * vprev)) & 3u;
            uint32_t topv = 0;   // cand[top - 1] when top > d0
            for (int s = d0; s < d1; s++) {
                const uint32_t e = L[s], t = e >> 2;
                const uint32_t F = (lut1 >> (2 * (e & 3u))) & 3u;
                const bool chg = F != Fprev;
                uint32_t dl;
                if (EDGE) {
                    dl = g.dmin + sm.dtab[F][edge_class(vprev, e & 3u)];
                    vprev = e & 3u;
                } else {
                    dl = pin_delay(g, 0, F);
                }
                const uint32_t key = (t + dl) << 2;
                while (chg && top > d0 && topv >= key) {
                    top--;
                    topv = top > d0 ? sm.cand[cslot(top - 1 - d0, lane)] : 0u;
                }
                sm.cand[cslot(top - d0, lane)] = key | F;
                top += chg;
                topv = chg ? (key | F) : topv;
                Fprev = F;
            }
        } else {
            int i = corank(d0, L, nL, R, nR);
            const int j = d0 - i;
            int c0, c1, c2;   // transitions of pins a, b, c consumed before d0
            if (K == 3) {
                if (i == 0) { c0 = 0; c1 = 0; }
                else {
                    const uint32_t inf = sm.Binfo()[i - 1], idx = inf & 0x7FFFu;
                    if (inf & 0x8000u) { c1 = (int)idx + 1; c0 = i - c1; }
                    else { c0 = (int)idx + 1; c1 = i - c0; }
                }
                c2 = j;
            } else { c0 = i; c1 = j; c2 = 0; }
            const int cc[3] = {c0, c1, c2};
            uint32_t st = carry;
            uint32_t ltp[3] = {kTimeInf, kTimeInf, kTimeInf};
#pragma unroll
            for (int p = 0; p < K; p++)
                if (cc[p] > 0) {
                    const uint32_t e = A[p][cc[p] - 1];
                    st = setpin(st, p, e & 3u);
                    ltp[p] = e >> 2;
                }
            uint32_t hl = L[i], hr = R[j];
            uint32_t hinfo = K == 3 ? sm.Binfo()[i] : 0u;   // source of the L head (3-pin cells)
            uint32_t Fprev = 0;
            // pins with a transition at the current timestamp: one bit per pin,
            // or, for edge-dependent delays, the (pin, edge) bits of dtab
            uint32_t grp = 0;
            if (d0 < d1) {
                // cell value just before the first timestamp of this share, and
                // the pins whose transitions at that timestamp precede the share
                const uint32_t tf = min(hl, hr) >> 2;
                uint32_t sb = st;
                int npre = 0;   // transitions at tf before the share
#pragma unroll
                for (int p = 0; p < K; p++)
                    if (cc[p] > 0 && ltp[p] == tf) {
                        const uint32_t v = cc[p] >= 2 ? (A[p][cc[p] - 2] & 3u) : ((carry >> (2 * p)) & 3u);
                        sb = setpin(sb, p, v);
                        grp |= EDGE ? edge_class(v, A[p][cc[p] - 1] & 3u) << (2 * p) : 1u << p;
                        npre++;
                    }
                Fprev = K == 3 ? (uint32_t)(((sb & 32u) ? g.lut_hi : g.lut_lo) >> (2 * (sb & 31u))) & 3u
                               : (lut2 >> (2 * (sb & 15u))) & 3u;
                // tf is the gate's first timestamp: the output is still at its X
                // start (Algorithm 2), whatever the table gives for X inputs
                if (!started && d0 == npre) Fprev = kVX;
            }
            bool gend = false;   // the previous transition closed its timestamp
            uint32_t topv = 0;   // cand[top - 1] when top > d0
            for (int s = d0; s < d1; s++) {
                const bool tl = hl <= (hr | 3u);
                const uint32_t e = tl ? hl : hr;
                const uint32_t pin = tl ? (K == 3 ? (hinfo >> 15) : 0u) : (uint32_t)(K - 1);
                i += tl;   // s + 1 transitions consumed: i of L, s + 1 - i of R
                const uint32_t y = tl ? L[i] : R[s + 1 - i];
                hl = tl ? y : hl;
                hr = tl ? hr : y;
                if (K == 3) hinfo = sm.Binfo()[i];
                const uint32_t t = e >> 2, v = e & 3u;
                uint32_t bit;
                if (EDGE) bit = edge_class((st >> (2 * pin)) & 3u, v) << (2 * pin);
                else bit = K == 2 ? (tl ? 1u : 2u) : 1u << pin;
                if (K == 2) st = tl ? ((st & ~3u) | v) : ((st & ~12u) | (v << 2));
                else st = setpin(st, (int)pin, v);
                grp = (gend ? 0u : grp) | bit;
                const bool end = (min(hl, hr) >> 2) != t;   // last transition at this time
                uint32_t F, key;
                if (K == 2 && !EDGE) {
                    const uint32_t te = sm.ftab[(grp << 4) | (st & 15u)];
                    F = te & 3u;
                    key = (t + g.dmin + (te >> 2)) << 2;
                } else {
                    F = K == 3 ? (EDGE ? (uint32_t)(((st & 32u) ? g.lut_hi : g.lut_lo) >> (2 * (st & 31u))) & 3u
                                       : (uint32_t)sm.f3[st & 63u])
                               : (lut2 >> (2 * (st & 15u))) & 3u;
                    key = (t + (EDGE || K == 3 ? g.dmin + sm.dtab[F][grp] : group_delay<K>(g, F, grp))) << 2;
                }
                const bool chg = end && F != Fprev;
                while (chg && top > d0 && topv >= key) {
                    top--;
                    topv = top > d0 ? sm.cand[cslot(top - 1 - d0, lane)] : 0u;
                }
                sm.cand[cslot(top - d0, lane)] = key | F;
                top += chg;
                topv = chg ? (key | F) : topv;
                Fprev = end ? F : Fprev;
                gend = end;
            }
        }

        // the windows are consumed: refill them for the next chunk while this
        // one's survivors are committed
#pragma unroll
        for (int p = 0; p < K; p++)
            if (m[p] > 0) carry = setpin(carry, p, A[p][m[p] - 1] & 3u);
        __syncwarp();
        more = issue_windows<K, CH>(sm, 0, g, ncur, nlead, nn, lane);

        // ---- 4./5. Eq. 1 across lanes, commit, carry ----
        const uint32_t Tfin = min(last ? kTimeInf : Tend + 1u + g.dmin, send);
        if (!commit_chunk<CH, MIRROR>(sm, lane, d0, top, Tfin, out, hout, cs)) { failed = true; break; }
        started = true;
#pragma unroll
        for (int p = 0; p < 3; p++) { cur[p] = ncur[p]; lead[p] = nlead[p]; n[p] = nn[p]; }
        __syncwarp();
    }
    // leave no copy in flight into this warp's buffers
    if (failed && more && !wait_window(sm, b, par)) {
        if (lane == 0) atomicOr(r.status, kStTimeout);
        return false;
    }
    return true;
}

// A gate's delay and value tables from its record: the register part
// (GateCtx) and the shared-memory tables of two- and three-input cells and
// of edge-dependent delays.
template <int K, int CH, bool EDGE>
__device__ __forceinline__ void build_tables(const GateRec &gr, GateCtx &g, WarpSmem<CH> &sm, int lane) {
    g.dmin = (uint32_t)gr.dmin;
    g.lut_lo = gr.lut_lo;
    g.lut_hi = gr.lut_hi;
    // delay tables from the record's [pin][edge][value] offsets
    const uint32_t arcs = gr.arcs;
    uint32_t fb_f = 255u, fb_r = 255u, omax = 0;   // fastest arcs to 0 / to 1, slowest arc
#pragma unroll
    for (int p = 0; p < K; p++)
        if ((arcs >> p) & 1u)
#pragma unroll
            for (int e = 0; e < 2; e++) {
                fb_f = min(fb_f, (uint32_t)gr.doff[p][e][0]);
                fb_r = min(fb_r, (uint32_t)gr.doff[p][e][1]);
                omax = max(omax, max((uint32_t)gr.doff[p][e][0], (uint32_t)gr.doff[p][e][1]));
            }
    g.dmax = g.dmin + omax;
    g.rise[0] = g.dmin + gr.doff[0][0][1];
    g.fall[0] = g.dmin + gr.doff[0][0][0];
    g.dx[0] = min(g.rise[0], g.fall[0]);
    g.df_lo = g.df_hi = g.dr_lo = g.dr_hi = 0;
    if (!EDGE) {
#pragma unroll
        for (int set = 1; set < 8; set++) {
            uint32_t f = 255u, rr = 255u;   // sets with a pin >= K never occur
            const uint32_t in = (uint32_t)set & arcs;
#pragma unroll
            for (int p = 0; p < K; p++)
                if ((in >> p) & 1u) { f = min(f, (uint32_t)gr.doff[p][0][0]); rr = min(rr, (uint32_t)gr.doff[p][0][1]); }
            if (in == 0) { f = fb_f; rr = fb_r; }
            if (set < 4) { g.df_lo |= f << (8 * set); g.dr_lo |= rr << (8 * set); }
            else { g.df_hi |= f << (8 * (set - 4)); g.dr_hi |= rr << (8 * (set - 4)); }
        }
        g.dx_lo = __vminu4(g.df_lo, g.dr_lo);
        g.dx_hi = __vminu4(g.df_hi, g.dr_hi);
        if (K == 3) {   // delay - dmin by new value and changed-pin set; value by pin values
            for (int x = lane; x < 24; x += 32) {
                const uint32_t F = (uint32_t)x >> 3, grp = (uint32_t)x & 7u;
                sm.dtab[F][grp] = (uint8_t)(group_delay<3>(g, F, grp) - g.dmin);
            }
            for (int x = lane; x < 64; x += 32)
                sm.f3[x] = (uint8_t)((((x & 32) ? g.lut_hi : g.lut_lo) >> (2 * (x & 31))) & 3u);
            __syncwarp();
        }
        if (K == 2) {
            const uint32_t l2 = (uint32_t)g.lut_hi;
            for (int x = lane; x < 64; x += 32) {
                const uint32_t F = (l2 >> (2 * (x & 15))) & 3u, grp = (uint32_t)x >> 4;
                sm.ftab[x] = (uint16_t)(((group_delay<2>(g, F, grp) - g.dmin) << 2) | F);
            }
            __syncwarp();
        }
    } else {
        for (int x = lane; x < 192; x += 32) {
            const int F = x >> 6, vm = x & 63;
            uint32_t d = 255u;
            bool any = false;
#pragma unroll
            for (int p = 0; p < K; p++)
#pragma unroll
                for (int e = 0; e < 2; e++)
                    if (((vm >> (2 * p + e)) & 1) && ((arcs >> p) & 1u)) {
                        const uint32_t d0 = gr.doff[p][e][0], d1 = gr.doff[p][e][1];
                        d = min(d, F == 0 ? d0 : (F == 1 ? d1 : min(d0, d1)));
                        any = true;
                    }
            if (!any) d = F == 0 ? fb_f : (F == 1 ? fb_r : min(fb_f, fb_r));
            sm.dtab[F][vm] = (uint8_t)d;
        }
        __syncwarp();
    }
}

// Returns false only when a window copy did not complete within its poll
// bound (the warp then stops: its buffers may still be written).
template <int K, bool DEP, int CH, bool EDGE, bool MIRROR>
__device__ bool eval_gate(const GateRec &gr, const RunDev &r, WarpSmem<CH> &sm, int lane, uint32_t &par,
                          WarpArena &wa) {
    GateCtx g;
    uint64_t bound = 0;
#pragma unroll
    for (int p = 0; p < 3; p++) {
        if (p < K) {
            const int32_t n = gr.fin[p];
            uint64_t ptr;
            uint32_t len;
            if (DEP) {  // written during this launch: read through L2
                ptr = __ldcg(reinterpret_cast<const unsigned long long *>(r.net_ptr) + n);
                len = __ldcg(r.net_len + n);
            } else {
                ptr = __ldg(reinterpret_cast<const unsigned long long *>(r.net_ptr) + n);
                len = __ldg(r.net_len + n);
            }
            g.src[p] = reinterpret_cast<const uint32_t *>(ptr);
            g.len[p] = len;
        } else {
            g.src[p] = nullptr;
            g.len[p] = 0;
        }
        bound += g.len[p];
    }
    const uint32_t out_net = gr.out_net;

    // state before the first input transition: pins at X, output X, nothing
    // pending -- or, in a time slice, where the previous slice left the gate
    uint32_t carry = 0x2Au;
    CommitState cs{0u, kVX, 0};
    uint32_t send = kTimeInf;   // transitions with t_r >= send stay pending
    bool started = false;       // an input transition was evaluated (else the output is still at its X start)
    if (r.st_in) {
        const uint32_t h = r.st_in[out_net];
        carry = (h & 63u) ^ 0x2Au;
        started = (h >> 7) & 1u;
        cs.lastV = ((h >> 8) & 3u) ^ kVX;
        cs.np = (int)(h >> 16);
        bound += (uint64_t)cs.np;   // each carried transition may become an output
        send = r.slice_end;
    }
    if (bound == 0) {   // no input transition: the output stays as it is (X at the start, Algorithm 2)
        if (lane == 0) {
            r.net_ptr[out_net] = 0;
            r.net_len[out_net] = 0;
            if (r.st_in) r.st_out[out_net] = r.st_in[out_net];
        }
        return true;
    }

    // Claim the output slot and start the first window copies before the
    // per-gate tables are built, so that the atomic's and the copies'
    // latencies overlap that work.
    const uint64_t need = (bound + kSlotAlign - 1) & ~(uint64_t)(kSlotAlign - 1);
    const bool claim = wa.cur + need > wa.end;   // the same on every lane
    const uint64_t blk = need > r.arena_blk ? need : (uint64_t)r.arena_blk;
    unsigned long long base = 0;
    if (claim && lane == 0) base = atomicAdd(r.arena_top, (unsigned long long)blk);
    uint32_t cur[3] = {0, 0, 0};
    bool failed = false;
    const int b = 0;   // the one window buffer
    int lead[3] = {0, 0, 0}, n[3] = {0, 0, 0};
    __syncwarp();      // the previous gate's reads of the buffer precede the copies
    bool more = issue_windows<K, CH>(sm, 0, g, cur, lead, n, lane);
    const bool any_input = more;

    build_tables<K, CH, EDGE>(gr, g, sm, lane);
    if (claim) {
        base = __shfl_sync(FULL, base, 0);
        wa.end = base + blk;
    } else {
        base = wa.cur;
    }
    if (base + bound > r.arena_cap) {
        wa.cur = wa.end = 0;   // past the arena: the next gate claims again (and counts its demand)
        if (lane == 0) {
            atomicOr(r.status, kStArenaOverflow);
            r.net_ptr[out_net] = 0;
            r.net_len[out_net] = 0;
        }
        // the copies already issued land in this warp's buffer: let them finish
        if (more && !wait_window(sm, b, par)) {
            if (lane == 0) atomicOr(r.status, kStTimeout);
            return false;
        }
        return true;
    }
    uint32_t *out = r.arena + base;
    uint32_t *hout = MIRROR ? r.harena + base : nullptr;
    if (cs.np > 0) {   // carried transitions, moved to this slice's local time
        const uint32_t *pp = r.pend_in + (size_t)out_net * PCAP;
        for (int x = lane; x < cs.np; x += 32) sm.Q[x] = pp[x] - (r.slice_shift << 2);
        __syncwarp();
    }

    if (!run_chunks<K, CH, EDGE, MIRROR>(r, sm, g, lane, par, more, cur, lead, n, carry, started, cs, send, out, hout,
                                         failed))
        return false;
    if (r.st_in && !failed) {
        // no input transition in this slice: settle the carried ones alone
        if (!any_input) failed = !commit_chunk<CH, MIRROR>(sm, lane, 0, 0, send, out, hout, cs);
        if (!failed) {
            if (lane == 0)
                r.st_out[out_net] = (carry ^ 0x2Au) | ((uint32_t)(started || any_input) << 7) | ((cs.lastV ^ kVX) << 8) |
                                    ((uint32_t)cs.np << 16);
            uint32_t *pp = r.pend_out + (size_t)out_net * PCAP;
            for (int x = lane; x < cs.np; x += 32) pp[x] = sm.Q[x];
        }
    }
    if (MIRROR && !failed && cs.outCount > 0) {
        // the waveform to the pinned host mirror in whole, aligned 16-byte
        // words (the slot is line-aligned and padded, so the rounded-up copy
        // stays inside it); the lanes' stores precede it through the barrier
        __syncwarp();
        const uint32_t n16 = (cs.outCount + 3u) >> 2;
        const uint4 *src = reinterpret_cast<const uint4 *>(out);
        uint4 *dst = reinterpret_cast<uint4 *>(hout);
        for (uint32_t x = (uint32_t)lane; x < n16; x += 32) dst[x] = __ldcg(src + x);
    }
    if (lane == 0) {
        if (failed) atomicOr(r.status, kStPendingOverflow);
        r.net_ptr[out_net] = reinterpret_cast<uint64_t>(out);
        r.net_len[out_net] = failed ? 0u : cs.outCount;
    }
    // the slot shrinks to the waveform, whole lines (no two nets share one)
    wa.cur = base + (failed ? need : (((uint64_t)cs.outCount + kSlotAlign - 1) & ~(uint64_t)(kSlotAlign - 1)));
    return true;
}

template <bool DEP, int CH, bool MIRROR>
__device__ __forceinline__ bool eval_windowed(const GateRec &gr, const RunDev &r, WarpSmem<CH> &sm, int lane,
                                              uint32_t &par, WarpArena &wa) {
    if (gr.flags & kGateEdge) {
        switch (gr.k) {
        case 1: return eval_gate<1, DEP, CH, true, MIRROR>(gr, r, sm, lane, par, wa);
        case 2: return eval_gate<2, DEP, CH, true, MIRROR>(gr, r, sm, lane, par, wa);
        default: return eval_gate<3, DEP, CH, true, MIRROR>(gr, r, sm, lane, par, wa);
        }
    }
    switch (gr.k) {
    case 1: return eval_gate<1, DEP, CH, false, MIRROR>(gr, r, sm, lane, par, wa);
    case 2: return eval_gate<2, DEP, CH, false, MIRROR>(gr, r, sm, lane, par, wa);
    default: return eval_gate<3, DEP, CH, false, MIRROR>(gr, r, sm, lane, par, wa);
    }
}

// ===========================================================================
// Segmented variant: the lanes of the warp split one gate's input timeline
// into consecutive segments [T_l, T_l+1) of about equal transition counts
// (quantiles of the longest fanin waveform).  Each lane runs Algorithm 2 and
// the sequential Eq. 1 stack (deny every scheduled transition with
// t_r' >= t_r, drop a transition equal to the one below it) on its own
// segment, streaming its inputs with 16-byte loads and keeping the stack in
// its private part of the gate's output slot.  Segments interact only
// through Eq. 1 across a boundary, resolved once per gate:
//   - a lane's stack tail is denied by any transition of a later segment with
//     a smaller or equal t_r: pop while t_r >= (suffix minimum of the later
//     lanes' smallest candidate t_r);
//   - the bottom of each lane's stack was pushed onto an empty local stack, so
//     whether it repeats the value before it is decided against the last
//     surviving transition of the nearest earlier non-empty lane (X if none);
// and a warp-wide copy packs the lanes' stacks into one contiguous waveform.
// There is no per-chunk work and no shared memory.
namespace seg {


template <bool DEP>
__device__ __forceinline__ uint4 ld16(const uint4 *p) {
    if (DEP) {   // produced during this launch: coherent load after the acquire
        uint4 v;
        asm volatile("ld.v4.u32 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
        return v;
    }
    return __ldg(p);
}
template <bool DEP>
__device__ __forceinline__ uint32_t ld4(const uint32_t *p) {
    if (DEP) {
        uint32_t v;
        asm volatile("ld.u32 %0, [%1];\n" : "=r"(v) : "l"(p));
        return v;
    }
    return __ldg(p);
}
__device__ __forceinline__ uint32_t pick(const uint4 &b, uint32_t i) {
    return i == 0 ? b.x : (i == 1 ? b.y : (i == 2 ? b.z : b.w));
}

// Transitions [s, e) of one pin, read 16 bytes at a time through L1; the
// 128-byte line after the current one is prefetched into L1 when the stream
// enters a line.  Reads and prefetches stay inside the net's slot: they start
// at the 16-byte boundary below s and never pass the multiple of 4 words at
// or above e (slots are padded to whole lines).
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.L1 [%0];\n" ::"l"(p));
}
template <bool DEP>
struct PinStream {
    const uint32_t *base;
    uint32_t idx, end, head;   // current index, end index, current transition (EINF at the end)
    uint4 buf;
    __device__ __forceinline__ void init(const uint32_t *b, uint32_t s, uint32_t e) {
        base = b;
        idx = s;
        end = e;
        head = EINF;
        if (s >= e) return;
        const uint32_t a = s & ~3u;
        buf = ld16<DEP>(reinterpret_cast<const uint4 *>(b + a));
        const uint32_t nl = (a & ~31u) + 32;   // next line
        if (nl < e) prefetch_l1(b + nl);
        head = pick(buf, s & 3u);
    }
    __device__ __forceinline__ void advance() {
        if (++idx >= end) { head = EINF; return; }
        if ((idx & 3u) == 0) {
            buf = ld16<DEP>(reinterpret_cast<const uint4 *>(base + idx));
            if ((idx & 31u) == 0 && idx + 32 < end) prefetch_l1(base + idx + 32);
        }
        head = pick(buf, idx & 3u);
    }
};

// first index of a[0..n) with time >= T
template <bool DEP>
__device__ __forceinline__ uint32_t lower_bound_t(const uint32_t *a, uint32_t n, uint32_t T) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((ld4<DEP>(a + mid) >> 2) < T) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int K, bool DEP>
__device__ void eval_gate_seg(const GateRec &gr, const RunDev &r, int lane, WarpArena &wa) {
    const uint32_t *src[3];
    uint32_t len[3], rise[3], fall[3];
    uint64_t bound = 0;
#pragma unroll
    for (int p = 0; p < K; p++) {
        const int32_t n = gr.fin[p];
        uint64_t ptr;
        if (DEP) {
            ptr = __ldcg(reinterpret_cast<const unsigned long long *>(r.net_ptr) + n);
            len[p] = __ldcg(r.net_len + n);
        } else {
            ptr = __ldg(reinterpret_cast<const unsigned long long *>(r.net_ptr) + n);
            len[p] = __ldg(r.net_len + n);
        }
        src[p] = reinterpret_cast<const uint32_t *>(ptr);
        rise[p] = (uint32_t)gr.dmin + gr.doff[p][0][1];
        fall[p] = (uint32_t)gr.dmin + gr.doff[p][0][0];
        bound += len[p];
    }
    const uint32_t out_net = gr.out_net;
    if (bound == 0) {   // no input transition: the output stays X
        if (lane == 0) { r.net_ptr[out_net] = 0; r.net_len[out_net] = 0; }
        return;
    }
    const uint64_t need = (bound + kSlotAlign - 1) & ~(uint64_t)(kSlotAlign - 1);
    unsigned long long base = 0;
    if (wa.cur + need > wa.end) {   // claim a new block (the same decision on every lane)
        const uint64_t blk = need > r.arena_blk ? need : (uint64_t)r.arena_blk;
        if (lane == 0) base = atomicAdd(r.arena_top, (unsigned long long)blk);
        base = __shfl_sync(FULL, base, 0);
        wa.end = base + blk;
    } else {
        base = wa.cur;
    }
    if (base + bound > r.arena_cap) {
        wa.cur = wa.end = 0;
        if (lane == 0) {
            atomicOr(r.status, kStArenaOverflow);
            r.net_ptr[out_net] = 0;
            r.net_len[out_net] = 0;
        }
        return;
    }
    uint32_t *const slot = r.arena + base;
    const uint64_t lut_lo = gr.lut_lo, lut_hi = gr.lut_hi;

    // ---- segments: lane l takes input times [T_l, T_l+1) ----
    const uint32_t S = (uint32_t)min((uint64_t)32, (bound + r.seg_target - 1) / r.seg_target);
    int pilot = 0;
#pragma unroll
    for (int p = 1; p < K; p++)
        if (len[p] > len[pilot]) pilot = p;
    uint32_t lp = len[0];
    const uint32_t *ps = src[0];
#pragma unroll
    for (int p = 1; p < K; p++)
        if (p == pilot) { lp = len[p]; ps = src[p]; }
    uint32_t sidx[3];
    if ((uint32_t)lane < S && lane > 0) {
        const uint32_t q = (uint32_t)(((uint64_t)lane * lp) / S);
        const uint32_t T = ld4<DEP>(ps + q) >> 2;
#pragma unroll
        for (int p = 0; p < K; p++) sidx[p] = (p == pilot) ? q : lower_bound_t<DEP>(src[p], len[p], T);
    } else {
#pragma unroll
        for (int p = 0; p < K; p++) sidx[p] = lane == 0 ? 0u : len[p];
    }
    uint32_t eidx[3], nseg = 0;
#pragma unroll
    for (int p = 0; p < K; p++) {
        eidx[p] = __shfl_down_sync(FULL, sidx[p], 1);
        if (lane == 31) eidx[p] = len[p];
        nseg += eidx[p] - sidx[p];
    }
    uint32_t segoff = nseg;   // exclusive prefix of segment sizes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, segoff, o);
        if (lane >= o) segoff += y;
    }
    segoff -= nseg;
    uint32_t *const out = slot + segoff;

    // ---- per-lane Algorithm 2 + Eq. 1 stack ----
    uint32_t st = 0x2Au;
    PinStream<DEP> in[K];
#pragma unroll
    for (int p = 0; p < K; p++) {
        // value of pin p just before the segment (X before its first transition)
        st = setpin(st, p, sidx[p] > 0 ? (ld4<DEP>(src[p] + sidx[p] - 1) & 3u) : kVX);
        in[p].init(src[p], sidx[p], eidx[p]);
    }
    auto lut = [&](uint32_t x) -> uint32_t {
        return (uint32_t)(((x & 32u) ? lut_hi : lut_lo) >> (2 * (x & 31u))) & 3u;
    };
    uint32_t Fprev = lut(st);
    uint32_t pos = 0, top = 0, top2 = 0, mintr = kTimeInf, trmax = 0;   // top, top2: out[pos-1], out[pos-2]
    for (;;) {
        uint32_t h = in[0].head;
#pragma unroll
        for (int p = 1; p < K; p++) h = min(h, in[p].head);
        if (h == EINF) break;
        const uint32_t t = h >> 2;
        uint32_t ch = 0;
#pragma unroll
        for (int p = 0; p < K; p++) {
            if ((in[p].head >> 2) == t) {
                st = setpin(st, p, in[p].head & 3u);
                ch |= 1u << p;
                in[p].advance();
            }
        }
        const uint32_t F = lut(st);
        if (F != Fprev) {
            uint32_t d = kTimeInf;
#pragma unroll
            for (int p = 0; p < K; p++)
                if (ch & (1u << p)) d = min(d, F == 1u ? rise[p] : (F == 0u ? fall[p] : min(rise[p], fall[p])));
            const uint32_t tr = t + d;
            trmax = max(trmax, tr);
            mintr = min(mintr, tr);
            const uint32_t key = tr << 2;
            while (pos > 0 && top >= key) {   // Eq. 1: deny t_r' >= t_r
                pos--;
                top = top2;
                top2 = pos >= 2 ? out[pos - 2] : 0u;
            }
            if (pos == 0 || (top & 3u) != F) {   // a repeat of the value below is dropped
                top2 = top;
                top = key | F;
                out[pos++] = top;
            }
        }
        Fprev = F;
    }
    if (trmax >= kTimeLimit) atomicOr(r.status, kStTimeRange);

    // ---- Eq. 1 across segments ----
    uint32_t inc = mintr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_down_sync(FULL, inc, o);
        if (lane + o < 32) inc = min(inc, y);
    }
    uint32_t after = __shfl_down_sync(FULL, inc, 1);
    if (lane == 31) after = kTimeInf;
    while (pos > 0 && (top >> 2) >= after) {
        pos--;
        top = top2;
        top2 = pos >= 2 ? out[pos - 2] : 0u;
    }
    // value before each lane's bottom: last survivor of the nearest earlier non-empty lane
    bool hv = pos > 0;
    uint32_t vv = top & 3u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const bool h2 = __shfl_up_sync(FULL, (int)hv, o);
        const uint32_t v2 = __shfl_up_sync(FULL, vv, o);
        if (lane >= o && !hv) { hv = h2; vv = v2; }
    }
    bool ph = __shfl_up_sync(FULL, (int)hv, 1);
    uint32_t pv = __shfl_up_sync(FULL, vv, 1);
    if (lane == 0) { ph = false; }
    const uint32_t before = ph ? pv : kVX;
    const uint32_t drop = (pos > 0 && (out[0] & 3u) == before) ? 1u : 0u;
    const uint32_t flen = pos - drop;
    uint32_t foff = flen;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, foff, o);
        if (lane >= o) foff += y;
    }
    const uint32_t total = __shfl_sync(FULL, foff, 31);
    foff -= flen;
    // pack the lanes' stacks in lane order (destinations never pass sources)
    __syncwarp();
    for (uint32_t l = 0; l < S; l++) {
        const uint32_t so = __shfl_sync(FULL, segoff + drop, l);
        const uint32_t dof = __shfl_sync(FULL, foff, l);
        const uint32_t n = __shfl_sync(FULL, flen, l);
        if (so == dof) continue;
        for (uint32_t b0 = 0; b0 < n; b0 += 32) {
            const uint32_t i = b0 + lane;
            const uint32_t v = i < n ? slot[so + i] : 0u;
            __syncwarp();
            if (i < n) slot[dof + i] = v;
            __syncwarp();
        }
    }
    if (lane == 0) {
        r.net_ptr[out_net] = reinterpret_cast<uint64_t>(slot);
        r.net_len[out_net] = total;
    }
    wa.cur = base + (((uint64_t)total + kSlotAlign - 1) & ~(uint64_t)(kSlotAlign - 1));
}

template <bool DEP>
__device__ __forceinline__ void eval_segmented(const GateRec &gr, const RunDev &r, int lane, WarpArena &wa) {
    switch (gr.k) {
    case 1: eval_gate_seg<1, DEP>(gr, r, lane, wa); break;
    case 2: eval_gate_seg<2, DEP>(gr, r, lane, wa); break;
    default: eval_gate_seg<3, DEP>(gr, r, lane, wa); break;
    }
}

}  // namespace seg

// V = kVariantSegmented or kVariantWindowed
template <int V, bool DEP, bool MIRROR>
__device__ __forceinline__ bool eval_variant(const GateRec &gr, const RunDev &r, unsigned char *smem_raw,
                                             int warp, int lane, uint32_t &par, WarpArena &wa) {
    if (V == kVariantSegmented) {
        seg::eval_segmented<DEP>(gr, r, lane, wa);
        return true;
    }
    if (V == kVariantWindowedWide)
        return eval_windowed<DEP, kWideCH, MIRROR>(gr, r, reinterpret_cast<WarpSmem<kWideCH> *>(smem_raw)[warp], lane,
                                                   par, wa);
    return eval_windowed<DEP, 128, MIRROR>(gr, r, reinterpret_cast<WarpSmem<128> *>(smem_raw)[warp], lane, par, wa);
}

template <int V>
__device__ __forceinline__ void init_variant(unsigned char *smem_raw, int warp, int lane) {
    if (V == kVariantWindowedWide) init_window_barriers(reinterpret_cast<WarpSmem<kWideCH> *>(smem_raw)[warp], lane);
    else if (V == kVariantWindowed) init_window_barriers(reinterpret_cast<WarpSmem<128> *>(smem_raw)[warp], lane);
}

// Gate record of work index g.  With rep > 1 replicas of one netlist the work
// order is level by level and, inside a level, replica by replica (L is the
// caller's running level hint: work indices only grow per warp), or, for
// records in a planned order, record by record and replica by replica; the
// net ids of replica i are shifted by i * rep_nets.
__device__ __forceinline__ GateRec fetch_gate(const GateRec *__restrict__ gates, const RunDev &r, int64_t g,
                                              int32_t &L) {
    if (r.rep <= 1) return gates[g];
    int64_t item;
    GateRec gr;
    if (r.planned) {
        const int64_t q = g / r.rep;
        item = g - q * r.rep;
        gr = gates[q];
    } else {
        while (g >= (int64_t)r.rep * __ldg(r.lb + L + 1)) L++;
        const int32_t b = __ldg(r.lb + L), cnt = __ldg(r.lb + L + 1) - b;
        const int64_t off = g - (int64_t)r.rep * b;
        item = off / cnt;
        gr = gates[b + (int32_t)(off - item * cnt)];
    }
    const int32_t sh = (int32_t)(item * r.rep_nets);
#pragma unroll
    for (int k = 0; k < 3; k++) gr.fin[k] += sh;
    gr.out_net += (uint32_t)sh;
    return gr;
}

template <int V, bool MIRROR>
__global__ void level_kernel(const GateRec *__restrict__ gates, int32_t g_begin, int32_t g_count,
                             int32_t level, RunDev r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t L = level + 1;
    init_variant<V>(smem_raw, warp, lane);
    uint32_t par = 0;   // phase parities of the warp's window barriers
    WarpArena wa{0, 0};  // no block yet
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(r.level_ctr + level, 1);
        g = __shfl_sync(FULL, g, 0);
        if (g >= g_count) break;
        const GateRec gr = fetch_gate(gates, r, (int64_t)g_begin + g, L);
        if (!eval_variant<V, false, MIRROR>(gr, r, smem_raw, warp, lane, par, wa)) break;
        __syncwarp();
    }
}

// A gate over the consecutive time slices of a launch, one after the other:
// each slice is evaluated as a gate of its own (its descriptor set, its state
// buffers, its end and shift), and the state one slice leaves is where the
// next one starts.  The gate's fanins are done for every slice of the launch
// before it starts, so the per-gate costs (work claim, record, fanin waits,
// publication) are paid once per launch instead of once per slice.
template <int V, bool MIRROR>
__device__ __forceinline__ bool eval_slices(const GateRec &gr, const RunDev &r, unsigned char *smem_raw, int warp,
                                            int lane, uint32_t &par, WarpArena &wa) {
    for (int j = 0; j < r.slices; j++) {
        RunDev rj = r;
        rj.net_ptr = r.net_ptr + (size_t)j * (size_t)r.slice_nets;
        rj.net_len = r.net_len + (size_t)j * (size_t)r.slice_nets;
        const bool odd = j & 1;
        rj.st_in = j == 0 ? r.st_in : (odd ? r.st_out : r.st_alt);
        rj.pend_in = j == 0 ? r.pend_in : (odd ? r.pend_out : r.pend_alt);
        rj.st_out = odd ? r.st_alt : r.st_out;
        rj.pend_out = odd ? r.pend_alt : r.pend_out;
        rj.slice_end = j == r.slices - 1 ? r.slice_end : r.slice_len;
        rj.slice_shift = j == 0 ? r.slice_shift : r.slice_len;
        // the start state until this slice writes its own: a slice that does
        // not (its arena overflowed, or its pending transitions did, and the
        // launch is evaluated again or fails) hands the next one nothing to
        // carry instead of an unwritten word
        if (lane == 0) rj.st_out[gr.out_net] = 0u;
        if (!eval_variant<V, true, MIRROR>(gr, rj, smem_raw, warp, lane, par, wa)) return false;
        __syncwarp();   // this slice's state stores precede the next slice's loads
    }
    return true;
}

// Algorithm 1 without level barriers: gates are handed out in a topological
// order (level order, or a planned critical-path-first order), so every fanin
// gate of a handed-out gate was handed out earlier to a running warp and the
// waits always end (the bound only guards against faults).  72 registers a
// thread let 28 warps of the 128-transition windowed variant share an SM
// (shared memory admits 7 CTAs of 4 warps).
// Completion flags are per net: primary inputs start done, a gate's output
// net is released once its waveform and descriptor are written (with MS, a
// launch over several time slices: once all of its slices are).
template <int V, bool MIRROR, bool MS>
__global__ void __maxnreg__(V == kVariantWindowed ? 72 : GLS_WIDE_MAXNREG) dependency_kernel(const GateRec *__restrict__ gates, int32_t n_gates, int32_t ctr_slot, RunDev r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t L = 1;
    init_variant<V>(smem_raw, warp, lane);
    uint32_t par = 0;   // phase parities of the warp's window barriers
    WarpArena wa{0, 0};  // no block yet
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(r.level_ctr + ctr_slot, 1);
        g = __shfl_sync(FULL, g, 0);
        if (g >= n_gates) break;
        const GateRec gr = fetch_gate(gates, r, g, L);
        bool ok = true;
        if (lane < gr.k) {   // primary-input flags are set before the launch
            const uint32_t *flag = r.done + (lane == 0 ? gr.fin[0] : (lane == 1 ? gr.fin[1] : gr.fin[2]));
            if (ld_acquire(flag) == 0u) {
                const uint64_t t0 = globaltimer();
                while (ld_acquire(flag) == 0u) {
                    if (globaltimer() - t0 > r.wait_limit_ns) { ok = false; break; }
                    __nanosleep(100);
                }
            }
        }
        ok = __all_sync(FULL, ok);
        // Every lane reads the fanin descriptors that lanes 0..k-1 acquired:
        // the barrier carries their acquires to the whole warp.  The fanin
        // waveforms were written by generic stores and are fetched by bulk
        // copies (async proxy) issued by the lane that acquired the pin's
        // flag, so that lane orders the two proxies first.
        __syncwarp();
        if (lane < gr.k) fence_proxy_async_global();
        if (ok) {
            // a window copy that never completed stops the warp (its readers
            // then give up their bounded waits)
            if constexpr (MS) {
                if (!eval_slices<V, MIRROR>(gr, r, smem_raw, warp, lane, par, wa)) break;
            } else {
                if (!eval_variant<V, true, MIRROR>(gr, r, smem_raw, warp, lane, par, wa)) break;
            }
        } else if (lane == 0) {
            atomicOr(r.status, kStTimeout);
            if constexpr (MS) {
                for (int j = 0; j < r.slices; j++) {
                    r.net_ptr[(size_t)j * (size_t)r.slice_nets + gr.out_net] = 0;
                    r.net_len[(size_t)j * (size_t)r.slice_nets + gr.out_net] = 0;
                }
            } else {
                r.net_ptr[gr.out_net] = 0;
                r.net_len[gr.out_net] = 0;
            }
        }
        // publish: this lane's output stores are ordered for the readers' bulk
        // copies (async proxy) and, through the warp barrier (which orders the
        // lanes' memory accesses among them) and lane 0's release (cumulative
        // at GPU scope), for their acquire of the completion flag
        fence_proxy_async_global();
        __syncwarp();
        if (lane == 0 && g != r.withhold_gate) st_release(r.done + gr.out_net, 1u);
    }
}

}  // namespace

size_t gate_smem_bytes(int variant, int warps_per_cta) {
    if (variant == kVariantSegmented) return 0;
    return (variant == kVariantWindowedWide ? sizeof(WarpSmem<kWideCH>) : sizeof(WarpSmem<128>)) * (size_t)warps_per_cta;
}

template <int V>
static int max_ctas(int warps_per_cta) {
    const size_t sm = gate_smem_bytes(V, warps_per_cta);
    cudaFuncSetAttribute(level_kernel<V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(dependency_kernel<V, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(level_kernel<V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(dependency_kernel<V, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (sm > 0) {   // the windowed variants are limited by shared memory: prefer the largest carveout
        cudaFuncSetAttribute(level_kernel<V, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(dependency_kernel<V, false, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(level_kernel<V, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(dependency_kernel<V, true, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    int a = 0, b = 0, c = 1 << 30;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, level_kernel<V, false>, warps_per_cta * 32, sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, dependency_kernel<V, false, false>, warps_per_cta * 32, sm);
    if constexpr (V != kVariantSegmented) {   // time slices per gate: the windowed variants only
        cudaFuncSetAttribute(dependency_kernel<V, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(dependency_kernel<V, false, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, dependency_kernel<V, false, true>, warps_per_cta * 32, sm);
    }
    const int ab = a < b ? a : b;
    return ab < c ? ab : c;
}

int gate_max_ctas_per_sm(int variant, int warps_per_cta) {
    if (variant == kVariantSegmented) return max_ctas<kVariantSegmented>(warps_per_cta);
    if (variant == kVariantWindowedWide) return max_ctas<kVariantWindowedWide>(warps_per_cta);
    return max_ctas<kVariantWindowed>(warps_per_cta);
}

cudaError_t launch_level(const GateRec *d_gates, int32_t g_begin, int32_t g_count, int32_t level,
                         const RunDev &r, const LevelCfg &cfg, cudaStream_t s) {
    if (g_count <= 0) return cudaSuccess;
    const int ctas = min(cfg.ctas, (g_count + cfg.warps_per_cta - 1) / cfg.warps_per_cta);
    const size_t sm = gate_smem_bytes(cfg.variant, cfg.warps_per_cta);
    if (cfg.variant == kVariantSegmented)
        level_kernel<kVariantSegmented, false><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, g_begin, g_count, level, r);
    else if (cfg.variant == kVariantWindowedWide) {
        if (r.harena) level_kernel<kVariantWindowedWide, true><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, g_begin, g_count, level, r);
        else level_kernel<kVariantWindowedWide, false><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, g_begin, g_count, level, r);
    } else {
        if (r.harena) level_kernel<kVariantWindowed, true><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, g_begin, g_count, level, r);
        else level_kernel<kVariantWindowed, false><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, g_begin, g_count, level, r);
    }
    return cudaGetLastError();
}

cudaError_t launch_dependency(const GateRec *d_gates, int32_t n_gates, int32_t ctr_slot, const RunDev &r,
                              const LevelCfg &cfg, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    const int ctas = min(cfg.ctas, (n_gates + cfg.warps_per_cta - 1) / cfg.warps_per_cta);
    const size_t sm = gate_smem_bytes(cfg.variant, cfg.warps_per_cta);
    const bool ms = r.slices > 1;   // several time slices per gate (windowed variants, no host mirror)
    if (ms && (cfg.variant == kVariantSegmented || r.harena)) return cudaErrorInvalidValue;
    if (cfg.variant == kVariantSegmented)
        dependency_kernel<kVariantSegmented, false, false><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, n_gates, ctr_slot, r);
    else if (cfg.variant == kVariantWindowedWide) {
        if (ms) dependency_kernel<kVariantWindowedWide, false, true><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, n_gates, ctr_slot, r);
        else if (r.harena) dependency_kernel<kVariantWindowedWide, true, false><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, n_gates, ctr_slot, r);
        else dependency_kernel<kVariantWindowedWide, false, false><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, n_gates, ctr_slot, r);
    } else {
        if (ms) dependency_kernel<kVariantWindowed, false, true><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, n_gates, ctr_slot, r);
        else if (r.harena) dependency_kernel<kVariantWindowed, true, false><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, n_gates, ctr_slot, r);
        else dependency_kernel<kVariantWindowed, false, false><<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, n_gates, ctr_slot, r);
    }
    return cudaGetLastError();
}

}  // namespace gls
