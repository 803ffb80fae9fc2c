// gls_kernels.cu -- stimulus packing, run initialisation and result gather.
#include "gls_internal.h"

namespace gls {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// One warp per primary input: check the stimulus rules (time in range and
// strictly increasing, value <= 3, no value equal to the previous one) and
// pack each transition into (t << 2) | v at its 16-byte aligned slot.
// status[0] |= 1 on a violation, status[1] = min bad PI, status[2] = max time.
__global__ void pack_stimulus_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ t,
                                     const uint8_t *__restrict__ v, int32_t n_pi, uint32_t *__restrict__ packed,
                                     uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint32_t tmax = 0;
    for (int64_t pi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pi < n_pi; pi += warps) {
        const int64_t a = off[pi], b = off[pi + 1];
        uint32_t *dst = packed + stim_slot(a, pi);
        bool bad = false;
        for (int64_t e = a + lane; e < b; e += 32) {
            const int32_t te = t[e];
            const uint32_t ve = v[e];
            bool ok = te >= 0 && (uint32_t)te < kTimeLimit && ve <= 3u;
            if (e > a) ok = ok && t[e - 1] < te && v[e - 1] != ve;
            bad |= !ok;
            if (ok) tmax = max(tmax, (uint32_t)te);
            dst[e - a] = ((uint32_t)te << 2) | (ve & 3u);
        }
        if (__any_sync(FULL, bad) && lane == 0) {
            atomicOr(status, 1u);
            atomicMin(status + 1, (uint32_t)pi);
        }
    }
    for (int o = 16; o > 0; o >>= 1) tmax = max(tmax, __shfl_xor_sync(FULL, tmax, o));
    if (lane == 0) atomicMax(status + 2, tmax);
}

// First index of a[0..n) whose time is >= T.
template <typename TT>
__device__ __forceinline__ int64_t first_at_or_after(const TT *a, int64_t n, int64_t T) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)a[mid] < T) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One warp per primary input: the PI's transitions in each of L consecutive
// time slices, moved to slice-local time (t - slice start fits 30 bits,
// checked on the host) and packed at their aligned place (slice_base).  The
// L + 1 slice boundaries are found by binary searches, one per lane, and
// kept in shared memory.
template <typename TT>
__global__ void __launch_bounds__(256) slice_pack_kernel(const int64_t *__restrict__ off, const TT *__restrict__ t,
                                                         const uint8_t *__restrict__ v, int32_t n_pi, int64_t T0,
                                                         int64_t S, int32_t L, bool open_end, int64_t slice_nets,
                                                         uint32_t *__restrict__ packed, uint64_t *net_ptr,
                                                         uint32_t *net_len, uint32_t *done,
                                                         unsigned long long *pi_total) {
    __shared__ int64_t bnd_all[8][kMaxSliceGroup + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t *bnd = bnd_all[w];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long tot = 0;
    for (int64_t pi = (int64_t)blockIdx.x * (blockDim.x >> 5) + w; pi < n_pi; pi += warps) {
        const int64_t a = off[pi], n = off[pi + 1] - a;
        __syncwarp();   // the previous PI's reads of bnd are done
        for (int j = lane; j <= L; j += 32)
            bnd[j] = j == L && open_end ? n : first_at_or_after(t + a, n, T0 + (int64_t)j * S);
        __syncwarp();
        uint32_t *region = packed + slice_base(a, pi, L);
        for (int j = 0; j < L; j++) {
            const int64_t lo = bnd[j], hi = bnd[j + 1], tj = T0 + (int64_t)j * S;
            uint32_t *dst = region + ((lo - bnd[0] + 4 * j + 3) & ~(int64_t)3);
            for (int64_t e = lo + lane; e < hi; e += 32)
                dst[e - lo] = ((uint32_t)((int64_t)t[a + e] - tj) << 2) | (v[a + e] & 3u);
            if (lane == (j & 31)) {
                const int64_t q = (int64_t)j * slice_nets + pi;
                net_ptr[q] = reinterpret_cast<uint64_t>(dst);
                net_len[q] = (uint32_t)(hi - lo);
            }
        }
        if (lane == 0) {
            if (done) done[pi] = 1u;
            tot += (unsigned long long)(bnd[L] - bnd[0]);
        }
    }
    if (lane == 0 && tot) atomicAdd(pi_total, tot);
}

__global__ void gather_descriptors_kernel(const uint64_t *__restrict__ net_ptr, const uint32_t *__restrict__ net_len,
                                          const int32_t *__restrict__ ext2int, int32_t n_pi, int64_t n_gates,
                                          int64_t net_base, const uint32_t *arena, int64_t *off, uint32_t *len) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_gates; g += stride) {
        const int64_t n = net_base + ext2int[n_pi + g];
        const uint32_t l = net_len[n];
        len[g] = l;
        off[g] = l ? (int64_t)((net_ptr[n] - reinterpret_cast<uint64_t>(arena)) >> 2) : 0;
    }
}

// PI net descriptors point into the packed stimulus; everything a run
// accumulates (counters, status, completion flags) is reset.
__global__ void run_init_kernel(const int64_t *__restrict__ off, const uint32_t *packed, RunDev r, int32_t n_ctr) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < r.n_pi; i += stride) {
        const int64_t a = off[i];
        r.net_ptr[i] = reinterpret_cast<uint64_t>(packed + stim_slot(a, i));
        r.net_len[i] = (uint32_t)(off[i + 1] - a);
    }
    for (int64_t i = tid; i < n_ctr; i += stride) r.level_ctr[i] = 0;
    if (r.done)
        for (int64_t i = tid; i < r.n_gates; i += stride) r.done[i] = 0u;
    if (tid == 0) { *r.arena_top = 0; *r.status = 0; }
}

// Descriptors of one instance's primary inputs (nets net_base + i) and, in
// the dependency schedule, their completion flags.  Only transitions before
// t_limit belong to the instance (a prefix of each waveform).
__global__ void pi_init_kernel(const int64_t *__restrict__ off, const uint32_t *packed, int32_t n_pi, int64_t net_base,
                               uint32_t t_limit, uint64_t *net_ptr, uint32_t *net_len, uint32_t *done,
                               unsigned long long *pi_total) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long tot = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pi; i += stride) {
        const int64_t a = off[i];
        const uint32_t *w = packed + stim_slot(a, i);
        uint32_t lo = 0, hi = (uint32_t)(off[i + 1] - a);
        if (t_limit != kTimeInf)
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if ((w[mid] >> 2) < t_limit) lo = mid + 1;
                else hi = mid;
            }
        else lo = hi;
        net_ptr[net_base + i] = reinterpret_cast<uint64_t>(w);
        net_len[net_base + i] = lo;
        if (done) done[net_base + i] = 1u;
        tot += lo;
    }
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(pi_total, tot);
}

__global__ void gather_lengths_kernel(const uint32_t *__restrict__ net_len, const int32_t *__restrict__ ext2int,
                                      int64_t n, int64_t *__restrict__ off, int64_t net_base) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride)
        off[i] = i < n ? (int64_t)net_len[net_base + ext2int[i]] : 0;
}

constexpr int SCAN_T = 512;            // threads per scan block
constexpr int SCAN_E = 4;              // elements per thread
constexpr int SCAN_TILE = SCAN_T * SCAN_E;

// Exclusive scan of one tile per block, writing the tile total to sums[block].
__global__ void scan_tile_kernel(int64_t *data, int64_t n, int64_t *sums) {
    __shared__ int64_t warp_tot[SCAN_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_E;
    int64_t x[SCAN_E], run = 0;
#pragma unroll
    for (int e = 0; e < SCAN_E; e++) {
        x[e] = (base + e < n) ? data[base + e] : 0;
        const int64_t y = x[e];
        x[e] = run;
        run += y;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < SCAN_T / 32 ? warp_tot[lane] : 0, si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, si, o);
            if (lane >= o) si += y;
        }
        if (lane < SCAN_T / 32) warp_tot[lane] = si - s;
        if (lane == SCAN_T / 32 - 1 && sums) sums[blockIdx.x] = si;
    }
    __syncthreads();
    const int64_t pre = warp_tot[w] + inc - run;
#pragma unroll
    for (int e = 0; e < SCAN_E; e++)
        if (base + e < n) data[base + e] = x[e] + pre;
}

__global__ void scan_add_kernel(int64_t *data, int64_t n, const int64_t *offs) {
    const int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    const int64_t add = offs[blockIdx.x];
#pragma unroll
    for (int e = 0; e < SCAN_E; e++) {
        const int64_t k = i + (int64_t)e * SCAN_T;
        if (k < n) data[k] += add;
    }
}

// One warp per net (in the caller's net order): copy its waveform to the
// dense CSR position.
__global__ void gather_events_kernel(const uint64_t *__restrict__ net_ptr, const uint32_t *__restrict__ net_len,
                                     const int32_t *__restrict__ ext2int, const int64_t *__restrict__ off, int64_t n,
                                     uint32_t *__restrict__ out, int64_t net_base) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int64_t in = net_base + ext2int[i];
        const uint32_t len = net_len[in];
        const uint32_t *src = reinterpret_cast<const uint32_t *>(net_ptr[in]);
        uint32_t *dst = out + off[i];
        for (uint32_t e = lane; e < len; e += 32) dst[e] = src[e];
    }
}

__global__ void sum_lengths_kernel(const uint32_t *__restrict__ net_len, int64_t a, int64_t b,
                                   unsigned long long *sum) {
    unsigned long long s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += stride) s += net_len[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, s);
}

int grid_for(int64_t work, int per_block) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    return (int)g;
}

}  // namespace

cudaError_t launch_pack_stimulus(const int64_t *d_off, const int32_t *d_t, const uint8_t *d_v, int32_t n_pi,
                                 uint32_t *d_packed, uint32_t *d_status, cudaStream_t s) {
    if (n_pi <= 0) return cudaSuccess;
    pack_stimulus_kernel<<<grid_for(n_pi, 8), 256, 0, s>>>(d_off, d_t, d_v, n_pi, d_packed, d_status);
    return cudaGetLastError();
}

cudaError_t launch_slice_pack(const int64_t *d_off, const int32_t *d_t32, const int64_t *d_t64, const uint8_t *d_v,
                              int32_t n_pi, int64_t T0, int64_t S, int32_t L, bool open_end, int64_t slice_nets,
                              uint32_t *d_packed, uint64_t *net_ptr, uint32_t *net_len, uint32_t *done,
                              unsigned long long *pi_total, cudaStream_t s) {
    if (n_pi <= 0) return cudaSuccess;
    if (L < 1 || L > kMaxSliceGroup) return cudaErrorInvalidValue;
    if (d_t64)
        slice_pack_kernel<int64_t><<<grid_for(n_pi, 8), 256, 0, s>>>(d_off, d_t64, d_v, n_pi, T0, S, L, open_end,
                                                                     slice_nets, d_packed, net_ptr, net_len, done,
                                                                     pi_total);
    else
        slice_pack_kernel<int32_t><<<grid_for(n_pi, 8), 256, 0, s>>>(d_off, d_t32, d_v, n_pi, T0, S, L, open_end,
                                                                     slice_nets, d_packed, net_ptr, net_len, done,
                                                                     pi_total);
    return cudaGetLastError();
}

cudaError_t launch_gather_descriptors(const uint64_t *d_net_ptr, const uint32_t *d_net_len, const int32_t *d_ext2int,
                                      int32_t n_pi, int64_t n_gates, int64_t net_base, const uint32_t *arena,
                                      int64_t *d_off, uint32_t *d_len, cudaStream_t s) {
    if (n_gates <= 0) return cudaSuccess;
    gather_descriptors_kernel<<<grid_for(n_gates, 256), 256, 0, s>>>(d_net_ptr, d_net_len, d_ext2int, n_pi, n_gates,
                                                                      net_base, arena, d_off, d_len);
    return cudaGetLastError();
}

cudaError_t launch_run_init(const int64_t *d_stim_off, const uint32_t *d_stim_packed, const RunDev &r,
                            int32_t n_ctr, cudaStream_t s) {
    int64_t work = r.n_pi;
    if (r.done && r.n_gates > work) work = r.n_gates;
    if (n_ctr > work) work = n_ctr;
    run_init_kernel<<<grid_for(work, 256), 256, 0, s>>>(d_stim_off, d_stim_packed, r, n_ctr);
    return cudaGetLastError();
}

cudaError_t launch_pi_init(const int64_t *d_stim_off, const uint32_t *d_stim_packed, int32_t n_pi, int64_t net_base,
                           uint32_t t_limit, uint64_t *net_ptr, uint32_t *net_len, uint32_t *done,
                           unsigned long long *pi_total, cudaStream_t s) {
    if (n_pi <= 0) return cudaSuccess;
    pi_init_kernel<<<grid_for(n_pi, 256), 256, 0, s>>>(d_stim_off, d_stim_packed, n_pi, net_base, t_limit, net_ptr,
                                                         net_len, done, pi_total);
    return cudaGetLastError();
}

cudaError_t launch_gather_lengths(const uint32_t *d_net_len, const int32_t *d_ext2int, int64_t n, int64_t *d_off,
                                  cudaStream_t s, int64_t net_base) {
    gather_lengths_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(d_net_len, d_ext2int, n, d_off, net_base);
    return cudaGetLastError();
}

size_t scan_tmp_elems(int64_t n) {
    size_t tot = 0;
    while (n > 1) {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        tot += (size_t)n;
        if (n == 1) break;
    }
    return tot + 1;
}

cudaError_t launch_exclusive_scan_i64(int64_t *d_data, int64_t n, int64_t *d_tmp, size_t tmp_elems, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        scan_tile_kernel<<<1, SCAN_T, 0, s>>>(d_data, n, nullptr);
        return cudaGetLastError();
    }
    if ((size_t)nb > tmp_elems) return cudaErrorInvalidValue;
    scan_tile_kernel<<<(unsigned)nb, SCAN_T, 0, s>>>(d_data, n, d_tmp);
    cudaError_t e = launch_exclusive_scan_i64(d_tmp, nb, d_tmp + nb, tmp_elems - (size_t)nb, s);
    if (e != cudaSuccess) return e;
    scan_add_kernel<<<(unsigned)nb, SCAN_T, 0, s>>>(d_data, n, d_tmp);
    return cudaGetLastError();
}

cudaError_t launch_gather_events(const uint64_t *d_net_ptr, const uint32_t *d_net_len, const int32_t *d_ext2int,
                                 const int64_t *d_off, int64_t n, uint32_t *d_out, cudaStream_t s, int64_t net_base) {
    if (n <= 0) return cudaSuccess;
    gather_events_kernel<<<grid_for(n, 8), 256, 0, s>>>(d_net_ptr, d_net_len, d_ext2int, d_off, n, d_out, net_base);
    return cudaGetLastError();
}

cudaError_t launch_sum_gate_lengths(const uint32_t *d_net_len, int32_t n_pi, int64_t n, unsigned long long *d_sum,
                                    cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_sum, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    sum_lengths_kernel<<<grid_for(n - n_pi, 256 * 8), 256, 0, s>>>(d_net_len, n_pi, n, d_sum);
    return cudaGetLastError();
}

}  // namespace gls
