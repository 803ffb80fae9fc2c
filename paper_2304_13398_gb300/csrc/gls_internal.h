// gls_internal.h -- device data layout and launch wrappers shared by the
// translation units of libgls.so.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gls {

// One transition on the device: (time << 2) | value.  Every time must stay
// below kTimeLimit = 2^30 - 1 so that it fits 30 bits and stays below the
// time field of the all-ones sentinel word.  Values: 0, 1, 2 = X, 3 = Z.
constexpr uint32_t kVX = 2;
constexpr uint32_t kTimeLimit = (1u << 30) - 1u;   // exclusive
constexpr uint32_t kTimeInf = 0xFFFFFFFFu;         // "no more transitions"

// Device gate record: one output of one cell, records in level order (64
// bytes, 16-byte aligned).  fin[] are internal net ids: 0..n_pi-1 primary
// inputs, n_pi+i the output of record i.
//   lut      the output's 4-value function over pins a, b, c: entry
//            sum v_p 4^p (2 bits: 0, 1, X) of lut_lo (entries 0..31) and
//            lut_hi (32..63); the pins a cell does not have read X
//   doff     delay - dmin by [pin][input edge (0 rising, 1 falling)]
//            [output value (0 falls, 1 rises)]; kNoArc where the pin has no
//            arc to this output
//   flags    kGateEdge: the delays depend on the input edge;
//            kGateGeneral: the record needs the windowed kernels (edge
//            delays, a pin without an arc, or an output that is not X for
//            all-X inputs)
struct __align__(16) GateRec {
    uint64_t lut_lo, lut_hi;
    int32_t fin[3];
    int32_t dmin;        // smallest delay over the arcs
    uint32_t out_net;    // internal net id of the output (n_pi + i)
    uint8_t doff[3][2][2];
    uint8_t type;        // built-in cell id, or 255 for a user-defined cell
    uint8_t k;           // input pins
    uint8_t flags;
    uint8_t arcs;        // bit p: pin p has an arc to this output
    uint32_t pad[2];
};
static_assert(sizeof(GateRec) == 64, "GateRec layout");
constexpr uint8_t kNoArc = 255;
enum : uint8_t { kGateEdge = 1, kGateGeneral = 2 };

// Status bits a run's kernels may raise.
enum : uint32_t {
    kStArenaOverflow = 1u,    // output arena too small
    kStPendingOverflow = 2u,  // a cell's pending transitions exceeded the buffer
    kStTimeRange = 4u,        // a computed time reached 2^30 - 1
    kStTimeout = 8u,          // a bounded wait for a fanin gave up
};

// Per-run device state.
struct RunDev {
    uint64_t *net_ptr;        // [N] device address of net n's first transition
    uint32_t *net_len;        // [N] transition count of net n
    uint32_t *arena;          // [arena_cap] gate output transitions
    uint64_t arena_cap;       // capacity in transitions
    unsigned long long *arena_top;  // bump pointer (transitions), counts demand past cap
    uint32_t arena_blk;       // words a warp claims from the arena at a time, a multiple of kSlotAlign
                              // (0: every gate claims exactly its own slot)
    uint32_t *status;         // kSt* bits
    int32_t *level_ctr;       // [depth + 1] work counters, zeroed per run (last: dependency mode)
    uint32_t *done;           // [N] per-net completion flags (dependency mode): PIs 1, gates 0 per run
    int32_t n_pi;
    int32_t n_gates;
    uint64_t wait_limit_ns;   // bound on one wait for a fanin (dependency mode)
    int32_t withhold_gate;    // test hook: this gate never publishes its flag (-1: none)
    uint32_t seg_target;      // segmented variant: target transitions per lane segment
    // replicated items: rep > 1 instances of one netlist (level_begin lb[],
    // rep_nets nets each) are evaluated without a copy of its gate records;
    // work index g -> (level L, replica, gate) level by level, replica by replica
    int32_t rep;
    int64_t rep_nets;
    const int32_t *lb;
    // planned order (dependency schedule): the records are in a planned
    // topological order and work index g is record g / rep of replica g % rep
    int32_t planned;
    // Time-sliced runs (task division over time), else null: every gate's
    // state at the start (st_in, pend_in) and end (st_out, pend_out) of the
    // slice, per net.  st = (input pins ^ 0x2A) | started << 7 | (output
    // value ^ X) << 8 | pending count << 16, so all-zero is the start state
    // (inputs X, no input transition yet, output X, nothing pending); pend
    // holds kPendCap pending transitions per net in the previous slice's
    // local time.
    uint32_t *st_in, *st_out, *pend_in, *pend_out;
    uint32_t *harena;         // device view of a pinned host mirror of arena (every output word is
                              // stored there too), or null
    uint32_t slice_end;       // local end of the slice: a t_r at or past it stays pending
    uint32_t slice_shift;     // start of this slice minus start of the previous one
    // A dependency launch over `slices` > 1 consecutive time slices: a warp
    // evaluates its gate over slice 0, 1, ... in turn.  Slice j's descriptors
    // are net_ptr / net_len + j * slice_nets; slice 0 reads (st_in, pend_in)
    // and writes (st_out, pend_out), slice j > 0 reads what slice j - 1
    // wrote and writes the other buffer of the (out, alt) pair, so the
    // launch's input state is never overwritten.  slice_end and slice_shift
    // then hold the values of the launch's last and first slice.
    int32_t slices;
    uint32_t slice_len;       // slice length (local end of every slice but the run's last)
    int64_t slice_nets;       // nets of one slice's descriptor set
    uint32_t *st_alt, *pend_alt;
    unsigned long long *pi_total;   // primary-input transitions of the run (after time limits)
};

// Pending (scheduled, not yet final) transitions a gate carries from one
// input chunk or time slice to the next; more than the delay spread of a
// cell fits (GLS_MAX_DELAY_SPREAD).
constexpr int kPendCap = 256;

// Output slots are padded to whole 128-byte lines so that no two nets share a
// cache line (a reader's L1 can then never hold a stale copy of a line that a
// gate on another SM writes later in the same launch).
constexpr uint32_t kSlotAlign = 32;   // words

// Gate kernel variants: warp-wide shared-memory windows of 128 or 352
// (default) transitions per pin of 3-input cells, or per-lane time segments.
enum { kVariantSegmented = 0, kVariantWindowed = 1, kVariantWindowedWide = 2 };

// Launch configuration of the gate kernels.
struct LevelCfg {
    int warps_per_cta;
    int ctas;                 // resident CTAs on the whole GPU
    int variant;
};

// Stimulus device layout: PI i's packed transitions start at word
// stim_slot(off[i], i) = (off[i] + 3 i + 3) & ~3 (16-byte aligned, disjoint,
// and every read rounded up to a multiple of 4 words stays inside the buffer
// of stim_words(E, n_pi) words).
__host__ __device__ inline uint64_t stim_slot(int64_t off_i, int64_t i) {
    return (uint64_t)((off_i + 3 * i + 3) & ~(int64_t)3);
}
__host__ __device__ inline uint64_t stim_words(int64_t n_events, int64_t n_pi) {
    return (uint64_t)(n_events + 3 * n_pi + 8);
}

// Most time slices one launch evaluates.
constexpr int kMaxSliceGroup = 64;

// Primary-input layout of a launch over L time slices: PI i's region starts
// at word slice_base(off[i], i, L) = (off[i] + (4 L + 8) i + 3) & ~3, and the
// slice-local transitions of its slice j, transitions lo..hi-1 of the PI
// counted from its first transition in the launch's first slice, start at
// region + ((lo + 4 j + 3) & ~3): 16-byte aligned, disjoint for consecutive
// slices, and every read rounded up to 4 words stays inside the buffer of
// slice_words(E, n_pi, L) words.
__host__ __device__ inline uint64_t slice_base(int64_t off_i, int64_t i, int64_t L) {
    return (uint64_t)((off_i + (4 * L + 8) * i + 3) & ~(int64_t)3);
}
__host__ __device__ inline uint64_t slice_words(int64_t n_events, int64_t n_pi, int64_t L) {
    return (uint64_t)(n_events + (4 * L + 8) * n_pi + 8);
}

// ---- launch wrappers ----
size_t gate_smem_bytes(int variant, int warps_per_cta);
int gate_max_ctas_per_sm(int variant, int warps_per_cta);
// one level: gates [g_begin, g_begin + g_count) of the level-ordered array
cudaError_t launch_level(const GateRec *d_gates, int32_t g_begin, int32_t g_count, int32_t level,
                         const RunDev &r, const LevelCfg &cfg, cudaStream_t s);
// all gates in one persistent launch, each gate started once its fanin gates
// are done (Algorithm 1 scheduling without level barriers)
cudaError_t launch_dependency(const GateRec *d_gates, int32_t n_gates, int32_t ctr_slot, const RunDev &r,
                              const LevelCfg &cfg, cudaStream_t s);

// Primary-input descriptors of L consecutive time slices [T0 + j S, T0 +
// (j + 1) S), j < L (the last one open-ended if open_end): each PI's
// transitions in slice j, as slice-local packed transitions at their aligned
// place of d_packed (slice_base), described at net j * slice_nets + i; the
// PIs' completion flags set (one per PI); pi_total accumulates the PI
// transitions of the L slices.  Exactly one of t32 / t64 is set;
// 1 <= L <= kMaxSliceGroup.
cudaError_t launch_slice_pack(const int64_t *d_off, const int32_t *d_t32, const int64_t *d_t64, const uint8_t *d_v,
                              int32_t n_pi, int64_t T0, int64_t S, int32_t L, bool open_end, int64_t slice_nets,
                              uint32_t *d_packed, uint64_t *net_ptr, uint32_t *net_len, uint32_t *done,
                              unsigned long long *pi_total, cudaStream_t s);
cudaError_t launch_pack_stimulus(const int64_t *d_off, const int32_t *d_t, const uint8_t *d_v, int32_t n_pi,
                                 uint32_t *d_packed, uint32_t *d_status, cudaStream_t s);
cudaError_t launch_run_init(const int64_t *d_stim_off, const uint32_t *d_stim_packed, const RunDev &r,
                            int32_t n_ctr, cudaStream_t s);
// primary-input descriptors (and completion flags) of one instance whose nets
// start at net_base
// (transitions at or after t_limit are left out of the instance)
cudaError_t launch_pi_init(const int64_t *d_stim_off, const uint32_t *d_stim_packed, int32_t n_pi, int64_t net_base,
                           uint32_t t_limit, uint64_t *net_ptr, uint32_t *net_len, uint32_t *done,
                           unsigned long long *pi_total, cudaStream_t s);
// gather of nets net_base + ext2int[i], i < n
cudaError_t launch_gather_lengths(const uint32_t *d_net_len, const int32_t *d_ext2int, int64_t n,
                                  int64_t *d_off, cudaStream_t s, int64_t net_base = 0);
cudaError_t launch_exclusive_scan_i64(int64_t *d_data, int64_t n, int64_t *d_tmp, size_t tmp_elems,
                                      cudaStream_t s);
size_t scan_tmp_elems(int64_t n);
// Word offset of each gate output (nets net_base + ext2int[n_pi + g]) in the
// arena and its length, in caller gate order.
cudaError_t launch_gather_descriptors(const uint64_t *d_net_ptr, const uint32_t *d_net_len, const int32_t *d_ext2int,
                                      int32_t n_pi, int64_t n_gates, int64_t net_base, const uint32_t *arena,
                                      int64_t *d_off, uint32_t *d_len, cudaStream_t s);
cudaError_t launch_gather_events(const uint64_t *d_net_ptr, const uint32_t *d_net_len, const int32_t *d_ext2int,
                                 const int64_t *d_off, int64_t n, uint32_t *d_out, cudaStream_t s,
                                 int64_t net_base = 0);
cudaError_t launch_sum_gate_lengths(const uint32_t *d_net_len, int32_t n_pi, int64_t n, unsigned long long *d_sum,
                                    cudaStream_t s);

}  // namespace gls
