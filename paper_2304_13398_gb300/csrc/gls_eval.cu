// gls_eval.cu -- the level kernel: one warp evaluates one gate at a time.
//
// For a gate with k <= 3 fanin waveforms the warp streams the fanins in
// chunks through shared memory and, per chunk:
//   1. loads a window of up to CH transitions of every pin and cuts the chunk
//      at T_end, the earliest window end among pins with more transitions
//      left, so every transition at t <= T_end is present (a timestamp never
//      straddles two chunks);
//   2. merges the pins by time with merge-path partitions (pins a and b are
//      merged first for 3-input cells), each lane taking an equal share;
//   3. walks its share in time order, applying all transitions of one
//      timestamp together and, when the cell value changes, producing the
//      scheduled transition (t + min delay over the pins with a transition at
//      t, new value) -- Algorithm 2 (Sec. 4.2), minimum delay of Sec. 2.3;
//   4. applies Eq. 1: a transition survives iff its t_r is below the t_r of
//      every later one.  Each lane keeps a monotone stack of its own share,
//      a warp suffix-minimum across lanes finishes the test, and transitions
//      carried over from the previous chunk are filtered by the chunk minimum;
//   5. commits every survivor whose t_r is below T_end + 1 + dmin (no later
//      transition of this gate can reach back that far), dropping one equal
//      to the value before it (Fig. 6), and carries the rest to the next
//      chunk (at most dmax - dmin of them).
// Step 4's scan form equals the paper's sequential "deny and replace": a
// transition is denied iff a later-determined one has t_r <= its t_r.
//
// Output allocation: before evaluating, the warp reserves the Eq. 2 bound
// (sum of fanin lengths, >= the number of distinct input timestamps >= the
// output length) from the run's event arena with one atomicAdd, writes the
// waveform into it and records (address, length) in the net descriptors.  Net
// descriptors are read by the next levels only, so all waveform loads may go
// through the read-only path.
#include "gls_internal.h"

namespace gls {

__constant__ uint64_t c_lut[16][2];

void set_luts(const uint64_t lut[][2], int ncells) {
    cudaMemcpyToSymbol(c_lut, lut, sizeof(uint64_t) * 2 * ncells);
}

namespace {

constexpr int CH = 128;                 // transitions per pin window
constexpr int PCAP = 256;               // carried (pending) transitions, > GLS_MAX_DELAY_SPREAD
constexpr int QCAP = PCAP + 3 * CH;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t EINF = 0xFFFFFFFFu;  // sentinel event; its time 2^30-1 exceeds every real time

struct WarpSmem {
    uint32_t A[3][CH];      // pin windows
    uint32_t B[2 * CH];     // pins a+b merged (3-input cells)
    uint16_t Binfo[2 * CH]; // source of B[i]: pin b flag (bit 15) | index in its window
    uint32_t cand[3 * CH];  // per-lane stacks of scheduled transitions (t_r << 2 | v)
    uint32_t Q[QCAP];       // carried + surviving transitions of the chunk
};

__device__ __forceinline__ uint32_t lut_eval(uint64_t lo, uint64_t hi, uint32_t st) {
    uint64_t w = (st & 32u) ? hi : lo;
    return (uint32_t)(w >> ((st & 31u) * 2u)) & 3u;
}

// Number of elements of L among the first d elements of merge(L, R), where an
// element of L precedes an element of R at equal time.
__device__ __forceinline__ int corank(int d, const uint32_t *L, int nL, const uint32_t *R, int nR) {
    int lo = max(0, d - nR), hi = min(d, nL);
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((L[mid] >> 2) <= (R[d - mid - 1] >> 2)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// count of a[0..n) with time <= T (a sorted by time)
__device__ __forceinline__ int upper_count(const uint32_t *a, int n, uint32_t T) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((a[mid] >> 2) <= T) lo = mid + 1;
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
    uint32_t rise[3], fall[3], dx[3];
    uint32_t dmin;
    int k;
    uint64_t lut_lo, lut_hi;
};

__device__ __forceinline__ uint32_t pin_delay(const GateCtx &g, int p, uint32_t F) {
    return F == 1u ? g.rise[p] : (F == 0u ? g.fall[p] : g.dx[p]);
}

__device__ void eval_gate(const GateRec &gr, const RunDev &r, WarpSmem &sm, int lane) {
    GateCtx g;
    g.k = gr.k;
    uint64_t bound = 0;
#pragma unroll
    for (int p = 0; p < 3; p++) {
        if (p < g.k) {
            int32_t n = gr.fin[p];
            g.src[p] = reinterpret_cast<const uint32_t *>(__ldg(reinterpret_cast<const unsigned long long *>(r.net_ptr) + n));
            g.len[p] = __ldg(r.net_len + n);
            g.rise[p] = (uint32_t)gr.rise[p];
            g.fall[p] = (uint32_t)gr.fall[p];
            g.dx[p] = min(g.rise[p], g.fall[p]);
        } else {
            g.src[p] = nullptr;
            g.len[p] = 0;
            g.rise[p] = g.fall[p] = g.dx[p] = 0;
        }
        bound += g.len[p];
    }
    g.dmin = (uint32_t)gr.dmin;
    g.lut_lo = c_lut[gr.type][0];
    g.lut_hi = c_lut[gr.type][1];
    const uint32_t out_net = gr.out_net;

    if (bound == 0) {   // no input transition: the output stays X (Algorithm 2 starts at X)
        if (lane == 0) { r.net_ptr[out_net] = 0; r.net_len[out_net] = 0; }
        return;
    }
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(r.arena_top, (unsigned long long)((bound + 3) & ~3ull));
    base = __shfl_sync(FULL, base, 0);
    if (base + bound > r.arena_cap) {
        if (lane == 0) {
            atomicOr(r.status, kStArenaOverflow);
            r.net_ptr[out_net] = 0;
            r.net_len[out_net] = 0;
        }
        return;
    }
    uint32_t *out = r.arena + base;

    uint32_t carry = 0x2Au;           // pins a, b, c at X (2 | 2<<2 | 2<<4)
    uint32_t lastV = kVX;             // value of the last committed survivor
    uint32_t outCount = 0;
    int np = 0;                       // carried transitions in Q[0..np)
    uint32_t cur[3] = {0, 0, 0};
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    bool failed = false;

    for (;;) {
        // ---- 1. windows and chunk cut ----
        int n[3], m[3];
        bool any = false;
#pragma unroll
        for (int p = 0; p < 3; p++) {
            n[p] = (p < g.k) ? (int)min((uint32_t)CH, g.len[p] - cur[p]) : 0;
            any |= n[p] > 0;
        }
        if (!any) break;
#pragma unroll
        for (int p = 0; p < 3; p++) {
            const uint32_t *s = g.src[p] + cur[p];
            for (int x = lane; x < n[p]; x += 32) sm.A[p][x] = __ldg(s + x);
        }
        __syncwarp();
        uint32_t Tend = kTimeInf;
#pragma unroll
        for (int p = 0; p < 3; p++)
            if (n[p] > 0 && cur[p] + (uint32_t)n[p] < g.len[p]) Tend = min(Tend, sm.A[p][n[p] - 1] >> 2);
        const bool last = (Tend == kTimeInf);
#pragma unroll
        for (int p = 0; p < 3; p++) m[p] = last ? n[p] : upper_count(sm.A[p], n[p], Tend);

        // ---- 2. merge inputs: L (pin a, or a+b merged) and R (last pin) ----
        const uint32_t *L = sm.A[0];
        const uint32_t *R = sm.A[g.k - 1];
        int nL = m[0], nR = (g.k >= 2) ? m[g.k - 1] : 0;
        if (g.k == 3) {
            const int M1 = m[0] + m[1];
            const int d0 = (lane * M1) >> 5, d1 = ((lane + 1) * M1) >> 5;
            int i = corank(d0, sm.A[0], m[0], sm.A[1], m[1]), j = d0 - i;
            uint32_t hl = i < m[0] ? sm.A[0][i] : EINF, hr = j < m[1] ? sm.A[1][j] : EINF;
            for (int s = d0; s < d1; s++) {
                if ((hl >> 2) <= (hr >> 2)) {
                    sm.B[s] = hl; sm.Binfo[s] = (uint16_t)i; i++;
                    hl = i < m[0] ? sm.A[0][i] : EINF;
                } else {
                    sm.B[s] = hr; sm.Binfo[s] = (uint16_t)(0x8000u | (uint32_t)j); j++;
                    hr = j < m[1] ? sm.A[1][j] : EINF;
                }
            }
            __syncwarp();
            L = sm.B; nL = M1;
        }

        // ---- 3. per-lane walk: Algorithm 2 with a local Eq. 1 stack ----
        const int M = nL + nR;
        const int d0 = (lane * M) >> 5, d1 = ((lane + 1) * M) >> 5;
        int i = corank(d0, L, nL, R, nR), j = d0 - i;
        int c0, c1, c2;   // transitions of pins a, b, c consumed before d0
        if (g.k == 3) {
            if (i == 0) { c0 = 0; c1 = 0; }
            else {
                uint32_t inf = sm.Binfo[i - 1], idx = inf & 0x7FFFu;
                if (inf & 0x8000u) { c1 = (int)idx + 1; c0 = i - c1; }
                else { c0 = (int)idx + 1; c1 = i - c0; }
            }
            c2 = j;
        } else if (g.k == 2) { c0 = i; c1 = j; c2 = 0; }
        else { c0 = i; c1 = 0; c2 = 0; }
        const int cc[3] = {c0, c1, c2};
        uint32_t st = carry, lt[3] = {kTimeInf, kTimeInf, kTimeInf};
#pragma unroll
        for (int p = 0; p < 3; p++)
            if (p < g.k && cc[p] > 0) {
                uint32_t e = sm.A[p][cc[p] - 1];
                st = setpin(st, p, e & 3u);
                lt[p] = e >> 2;
            }
        uint32_t hl = i < nL ? L[i] : EINF, hr = j < nR ? R[j] : EINF;
        uint32_t Fprev = 0;
        if (d0 < d1) {
            // cell value just before the first timestamp of this share
            uint32_t tf = min(hl >> 2, hr >> 2), sb = st;
#pragma unroll
            for (int p = 0; p < 3; p++)
                if (p < g.k && cc[p] > 0 && lt[p] == tf) {
                    uint32_t v = cc[p] >= 2 ? (sm.A[p][cc[p] - 2] & 3u) : ((carry >> (2 * p)) & 3u);
                    sb = setpin(sb, p, v);
                }
            Fprev = lut_eval(g.lut_lo, g.lut_hi, sb);
        }
        int top = d0;
        uint32_t trmax = 0;
        for (int s = d0; s < d1; s++) {
            uint32_t e;
            int pin;
            if ((hl >> 2) <= (hr >> 2)) {
                e = hl;
                pin = (g.k == 3) ? (int)(sm.Binfo[i] >> 15) : 0;
                i++;
                hl = i < nL ? L[i] : EINF;
            } else {
                e = hr;
                pin = g.k - 1;
                j++;
                hr = j < nR ? R[j] : EINF;
            }
            const uint32_t t = e >> 2;
            st = setpin(st, pin, e & 3u);
            lt[0] = pin == 0 ? t : lt[0];
            lt[1] = pin == 1 ? t : lt[1];
            lt[2] = pin == 2 ? t : lt[2];
            if (min(hl >> 2, hr >> 2) == t) continue;   // more transitions at this time
            const uint32_t F = lut_eval(g.lut_lo, g.lut_hi, st);
            if (F != Fprev) {
                uint32_t d = kTimeInf;
#pragma unroll
                for (int p = 0; p < 3; p++)
                    if (p < g.k && lt[p] == t) d = min(d, pin_delay(g, p, F));
                const uint32_t tr = t + d;
                trmax = max(trmax, tr);
                const uint32_t key = tr << 2;
                while (top > d0 && sm.cand[top - 1] >= key) top--;
                sm.cand[top++] = key | F;
            }
            Fprev = F;
        }
        if (trmax >= kTimeLimit) atomicOr(r.status, kStTimeRange);

        // ---- 4. Eq. 1 across lanes and against the carried transitions ----
        uint32_t mn = top > d0 ? (sm.cand[d0] >> 2) : kTimeInf;
        uint32_t inc = mn;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_down_sync(FULL, inc, o);
            if (lane + o < 32) inc = min(inc, y);
        }
        uint32_t after = __shfl_down_sync(FULL, inc, 1);
        if (lane == 31) after = kTimeInf;
        const uint32_t Mall = __shfl_sync(FULL, inc, 0);
        while (top > d0 && (sm.cand[top - 1] >> 2) >= after) top--;
        int npk = 0;
        for (int b = 0; b < np; b += 32) {
            int idx = b + lane;
            bool f = idx < np && (sm.Q[idx] >> 2) < Mall;
            npk += __popc(__ballot_sync(FULL, f));
        }
        const uint32_t cnt = (uint32_t)(top - d0);
        uint32_t pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, pre, o);
            if (lane >= o) pre += y;
        }
        const int total = (int)__shfl_sync(FULL, pre, 31);
        const int pos = npk + (int)(pre - cnt);
        __syncwarp();
        for (uint32_t x = 0; x < cnt; x++) sm.Q[pos + x] = sm.cand[d0 + x];
        const int nQ = npk + total;
        __syncwarp();

        // ---- 5. commit what no later transition can deny; drop repeats ----
        const uint32_t Tfin = last ? kTimeInf : Tend + 1u + g.dmin;
        int nf = 0;
        for (int b = 0; b < nQ; b += 32) {
            const int idx = b + lane;
            const uint32_t e = idx < nQ ? sm.Q[idx] : 0u;
            const bool fin = idx < nQ && (e >> 2) < Tfin;
            const uint32_t pv = idx == 0 ? lastV : (idx < nQ ? (sm.Q[idx - 1] & 3u) : 0u);
            const bool keep = fin && ((e & 3u) != pv);
            const uint32_t bk = __ballot_sync(FULL, keep);
            if (keep) out[outCount + __popc(bk & lanemask_lt)] = e;
            outCount += __popc(bk);
            nf += __popc(__ballot_sync(FULL, fin));
        }
        if (nf > 0) lastV = sm.Q[nf - 1] & 3u;
        const int npn = nQ - nf;
        if (npn > PCAP) { failed = true; break; }
        for (int b = 0; b < npn; b += 32) {
            const int idx = b + lane;
            const uint32_t e = idx < npn ? sm.Q[nf + idx] : 0u;
            __syncwarp();
            if (idx < npn) sm.Q[idx] = e;
        }
        np = npn;
#pragma unroll
        for (int p = 0; p < 3; p++)
            if (m[p] > 0) {
                carry = setpin(carry, p, sm.A[p][m[p] - 1] & 3u);
                cur[p] += (uint32_t)m[p];
            }
        __syncwarp();
    }
    if (lane == 0) {
        if (failed) atomicOr(r.status, kStPendingOverflow);
        r.net_ptr[out_net] = reinterpret_cast<uint64_t>(out);
        r.net_len[out_net] = failed ? 0u : outCount;
    }
}

__global__ void level_kernel(const GateRec *__restrict__ gates, int32_t g_begin, int32_t g_count,
                             int32_t level, RunDev r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem &sm = reinterpret_cast<WarpSmem *>(smem_raw)[warp];
    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(r.level_ctr + level, 1);
        g = __shfl_sync(FULL, g, 0);
        if (g >= g_count) break;
        const GateRec gr = gates[g_begin + g];
        eval_gate(gr, r, sm, lane);
        __syncwarp();
    }
}

}  // namespace

size_t level_smem_bytes(int warps_per_cta) { return sizeof(WarpSmem) * (size_t)warps_per_cta; }

int level_max_ctas_per_sm(int warps_per_cta) {
    int n = 0;
    size_t sm = level_smem_bytes(warps_per_cta);
    cudaFuncSetAttribute(level_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, level_kernel, warps_per_cta * 32, sm);
    return n;
}

cudaError_t launch_level(const GateRec *d_gates, int32_t g_begin, int32_t g_count, int32_t level,
                         const RunDev &r, const LevelCfg &cfg, cudaStream_t s) {
    if (g_count <= 0) return cudaSuccess;
    int ctas = min(cfg.ctas, (g_count + cfg.warps_per_cta - 1) / cfg.warps_per_cta);
    size_t sm = level_smem_bytes(cfg.warps_per_cta);
    level_kernel<<<ctas, cfg.warps_per_cta * 32, sm, s>>>(d_gates, g_begin, g_count, level, r);
    return cudaGetLastError();
}

}  // namespace gls
