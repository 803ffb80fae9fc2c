/*
 * gls.h -- C-ABI of libgls.so: timing-aware 4-value gate-level re-simulation
 * on one GB300 GPU (sm_103a), the data-parallel hot path of arXiv 2304.13398
 * ("Acceleration for Timing-Aware Gate-Level Logic Simulation with One-Pass
 * GPU Parallelism").
 *
 * Problem (Sec. 2.1): given a combinational netlist of library cells, their
 * 4-value functions (Sec. 2.2, Table 1) and pin-to-pin delays (Sec. 2.3), and
 * the waveforms of the primary inputs over a duration, compute the waveform of
 * every other net.  A waveform is a strictly time-ordered list of transitions
 * (time in ps, value in {0, 1, X, Z}); a net is X before its first transition.
 *
 * Semantics of one gate (Algorithm 2, Eq. 1): the fanin waveforms are merged
 * by time and all transitions at one time are applied together; when the cell
 * value changes, a transition is scheduled at t + min over the pins with a
 * transition at t of that pin's delay toward the new value (rise for 1, fall
 * for 0, the smaller of both for X); a new scheduled transition denies every
 * earlier-determined one that would appear at the same time or later, and a
 * transition equal to the value before it is dropped.  Z is read as X on
 * inputs; cells never output Z.
 *
 * Conventions for every call:
 *   - Return value: GLS_OK (0) or a negative gls_status; no exception, abort
 *     or signal crosses this boundary.  gls_last_error() describes the last
 *     failure on the calling thread.
 *   - Ownership: arrays passed in are read during the call only (the library
 *     copies what it keeps); all device memory is owned by the context and
 *     freed by gls_release / gls_destroy.  Output arrays are caller-owned.
 *   - Pointers are host pointers unless a parameter says "device".
 *   - Net ids: 0..n_pi-1 are the primary inputs, n_pi+g is the output of
 *     gate g (in the caller's gate order).
 *   - Times are int32 ps; every time that can occur in a run (input times plus
 *     the largest path delay) must stay below 2^30 (else GLS_ERANGE), because
 *     the device stores a transition as one 32-bit word (time << 2 | value).
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef GLS_H
#define GLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gls_ctx gls_ctx;

typedef enum gls_status {
    GLS_OK = 0,
    GLS_EINVAL = -1,     /* bad argument, unknown id, malformed netlist            */
    GLS_ECYCLE = -2,     /* the netlist is not a DAG                               */
    GLS_ESTIM = -3,      /* malformed stimulus (order, value range, repeats)       */
    GLS_ERANGE = -4,     /* a time would reach 2^30, or a cell's delay spread is    */
                         /* beyond the device limit GLS_MAX_DELAY_SPREAD            */
    GLS_ENOMEM = -5,     /* device or host allocation failed / budget exceeded     */
    GLS_EOVERFLOW = -6,  /* output larger than the given capacity or run arena     */
    GLS_ETIMEOUT = -7,   /* a bounded device wait gave up                          */
    GLS_ECUDA = -8,      /* CUDA runtime error                                     */
    GLS_EAGAIN = -9      /* gls_run_query: the run is still in progress            */
} gls_status;

/* Cell library (Sec. 2.1 "cells derived from basic gates"); pins a, b, c. */
typedef enum gls_cell {
    GLS_INV = 0,   /* !a             */
    GLS_BUF,       /* a              */
    GLS_AND2,      /* a & b          */
    GLS_OR2,       /* a | b          */
    GLS_NAND2,     /* !(a & b)       */
    GLS_NOR2,      /* !(a | b)       */
    GLS_XOR2,      /* a ^ b          */
    GLS_XNOR2,     /* !(a ^ b)       */
    GLS_MUX2,      /* c ? b : a      */
    GLS_AOI21,     /* !((a & b) | c) */
    GLS_OAI21,     /* !((a | b) & c) */
    GLS_NCELLS
} gls_cell;

/* Largest (max - min) over one cell's rise/fall delays that the device
   pending-transition buffer supports; larger spreads give GLS_ERANGE. */
#define GLS_MAX_DELAY_SPREAD 255

/* Library version (major * 10000 + minor * 100 + patch). */
int gls_version(void);

/* Pin count of a cell, or GLS_EINVAL. */
int gls_cell_arity(int cell);

/*
 * Host-only validation and levelization of a netlist (no GPU needed).
 *   type[n_gates], fanin_off[n_gates+1] (fanin_off[0] = 0), fanin_net[A],
 *   d_rise[A], d_fall[A] with A = fanin_off[n_gates]: gate g reads nets
 *   fanin_net[fanin_off[g] .. fanin_off[g+1]) as pins a, b, c; arc delays in
 *   ps, each in [1, 2^29).
 * Checks: pin count matches the cell, net ids in range, delays in range,
 * delay spread per cell <= GLS_MAX_DELAY_SPREAD (GLS_ERANGE), no cycle
 * (GLS_ECYCLE).  On success *depth_out is the longest path in gates and, when
 * level_out is non-NULL, level_out[g] is gate g's level (1 + max fanin level,
 * primary inputs at level 0).
 */
int gls_check_netlist(int32_t n_pi, int32_t n_gates, const uint8_t *type, const int32_t *fanin_off,
                      const int32_t *fanin_net, const int32_t *d_rise, const int32_t *d_fall,
                      int32_t *depth_out, int32_t *level_out);

/*
 * Host-only validation of a stimulus (the given waveforms, Sec. 2.1).
 *   off[n_pi+1] int64 with off[0] = 0 and non-decreasing; PI i owns
 *   transitions [off[i], off[i+1]) of t (int32 ps) and v (0, 1, 2 = X, 3 = Z).
 * Rules: 0 <= t < 2^30 strictly increasing per PI, v <= 3, no value equal to
 * the one before it in the same PI.  Returns GLS_OK or GLS_ESTIM.
 */
int gls_check_stimulus(int32_t n_pi, const int64_t *off, const int32_t *t, const uint8_t *v);

/*
 * Create a context on CUDA device 'device'.  hbm_budget_bytes caps the device
 * memory the context may hold (0 = 90% of the free memory at creation).
 */
int gls_create(gls_ctx **out, int device, uint64_t hbm_budget_bytes);

/* Free every object of the context and the context itself (NULL is a no-op). */
void gls_destroy(gls_ctx *ctx);

/* Message of the last failure on the calling thread ("" if none). */
const char *gls_last_error(gls_ctx *ctx);

/*
 * Validate (as gls_check_netlist), levelize and copy a netlist to the device:
 * gates are reordered by level, one 64-byte record per gate (fanin net ids,
 * delays, the cell's 4-value table); the device copy is immutable.
 * *netlist_id receives a handle.
 * Paper: the netlist and its cells of Sec. 2.1 (objective statement), each
 * cell's 4-value function of Sec. 2.2 / Table 1 built per Sec. 3.3 (module
 * function), and the pin-to-pin delays of Sec. 2.3 kept as the delay matrix
 * of Sec. 3.2 (rise/fall per arc for both input edges in this classic form).
 */
int gls_load_netlist(gls_ctx *ctx, int32_t n_pi, int32_t n_gates, const uint8_t *type,
                     const int32_t *fanin_off, const int32_t *fanin_net, const int32_t *d_rise,
                     const int32_t *d_fall, int32_t *netlist_id);

/*
 * Copy primary-input waveforms (layout of gls_check_stimulus) to the device
 * in one host-to-device transfer, validate them there and pack each
 * transition into one 32-bit word.  Synchronous.  GLS_ESTIM on a rule
 * violation.  *stim_id receives a handle usable with any netlist of the same
 * n_pi.
 * Paper: the given waveforms of Sec. 2.1, moved to the device in the single
 * transfer before the one-pass evaluation (Sec. 3, Sec. 1.4 algorithmic flow).
 * The stimulus is a handle of its own (n_pi, not a netlist id): one stimulus
 * serves every netlist with that many primary inputs.
 */
int gls_load_stimulus(gls_ctx *ctx, int32_t n_pi, const int64_t *off, const int32_t *t,
                      const uint8_t *v, int32_t *stim_id);

/*
 * Overwrite an existing stimulus in place with new waveforms of the same n_pi
 * and at most the event count it was created with (GLS_EOVERFLOW otherwise).
 * Runs created on it see the new waveforms at their next gls_rerun.
 * Synchronous like gls_load_stimulus.
 */
int gls_update_stimulus(gls_ctx *ctx, int32_t stim_id, const int64_t *off, const int32_t *t,
                        const uint8_t *v);

/*
 * Paper: the one-pass evaluation of Sec. 4 -- Algorithm 1 (every cell is
 * processed once its input waveforms are known; here as one persistent
 * launch in a topological order, or one launch per level) and Algorithm 2 per
 * gate (merge of the fanin waveforms, 4-value function, minimum delay over the
 * changed pins of Sec. 2.3, "glitch eaten" cancellation of Eq. 1), each output
 * reserving its Eq. 2 bound in the device store (Sec. 3.1).  arena_events is
 * the one parameter beyond the paper: the size of that store, which the
 * paper's CSRP allocates up front as well (Eq. 4).
 *
 * Simulate a netlist under a stimulus: allocate the run's waveform store
 * (net descriptors plus an event arena of arena_events 32-bit words; 0 means
 * 256 words per stimulus transition plus 2^20, capped at half of the unused
 * budget) and enqueue the whole evaluation (one persistent launch with the
 * dependency schedule, one launch per level with the level schedule) as one
 * CUDA graph on cuda_stream (a cudaStream_t; NULL = the context's stream).
 * Stream-ordered: returns once the work is enqueued.  The result stays on the
 * device until gls_release.  GLS_ERANGE if a time could reach 2^30.
 */
int gls_simulate(gls_ctx *ctx, int32_t netlist_id, int32_t stim_id, int64_t arena_events,
                 void *cuda_stream, int32_t *run_id);

/*
 * Batched simulation: n_items (netlist, stimulus) pairs -- the same netlist
 * with many stimulus sets, distinct netlists, or both -- evaluated by one
 * graph launch as one disjoint union: their gates are interleaved by level
 * into one work order, so the dependency schedule's single persistent launch
 * (or one launch per level) covers every item and the long gates of one item
 * overlap with the work of the others.  netlist_ids[n_items] and
 * stim_ids[n_items] are loaded handles; items that all name one netlist are
 * evaluated from that netlist's records without a copy.  t_limits[n_items]
 * (NULL = none) keeps only the stimulus transitions before t_limits[i] in
 * item i, i.e. simulates the first t_limits[i] ps of the given waveforms
 * (a request window over a resident stimulus).  arena_events as in
 * gls_simulate (0 = 256 words per stimulus transition of all items plus 2^20,
 * capped at half the unused budget).  Read items back with gls_read_item;
 * gls_run_stats reports all items together.  No counterpart in the paper
 * (Sec. 4 simulates one netlist at a time); each item's waveforms equal a
 * gls_simulate of it (with its stimulus cut at its time limit).
 */
int gls_simulate_batch(gls_ctx *ctx, int32_t n_items, const int32_t *netlist_ids, const int32_t *stim_ids,
                       const int32_t *t_limits, int64_t arena_events, void *cuda_stream, int32_t *run_id);

/* Enqueue the same run again (same buffers, current stimulus contents). */
int gls_rerun(gls_ctx *ctx, int32_t run_id, void *cuda_stream);

/* Non-blocking: GLS_OK when the run's last enqueued evaluation has finished,
   GLS_EAGAIN while it is still in progress. */
int gls_run_query(gls_ctx *ctx, int32_t run_id);

/*
 * Wait for a run and report it: *total_events = output transitions of all
 * gates, *kernel_ms = device time of the last enqueued evaluation (CUDA
 * events around the gate kernels).  Either pointer may be NULL.
 * GLS_EOVERFLOW when the event arena was too small: then *total_events is the
 * arena demand of the gates that were evaluated, a lower bound of the full
 * demand because gates that did not fit leave their readers fewer inputs
 * (retry with at least that much), GLS_ERANGE when a cell's pending transitions
 * exceeded the device buffer, GLS_ETIMEOUT when a device wait for a fanin
 * gate gave up (dependency schedule).
 */
int gls_run_stats(gls_ctx *ctx, int32_t run_id, int64_t *total_events, double *kernel_ms);

/* Wait for a run and report its event arena: *arena_demand = words claimed
   from it, *arena_capacity = the run's arena size; either pointer may be
   NULL.  The warps of a run claim the arena in blocks; each gate reserves its
   Eq. 2 bound inside its warp's block while it runs and keeps only its
   waveform (both padded to 128-byte lines), so the demand is the output
   (padded) plus the unused ends of the blocks (up to a quarter of the arena,
   at most 1 MiB per warp), and it varies with the order in which the warps
   take the gates.  The demand sizes later runs of similar inputs (the
   serving admission model). */
int gls_run_info(gls_ctx *ctx, int32_t run_id, int64_t *arena_demand, int64_t *arena_capacity);

/*
 * Plan the order in which the dependency schedule hands out the gates of a
 * netlist (Algorithm 1: a gate runs once its fanin gates are done, so any
 * topological order gives the same waveforms; the order only decides which
 * ready work the device starts first).  Reads the per-net transition counts
 * of item `item` of the finished run `run_id`, which must be an instance of
 * `netlist_id` that completed without error; weighs each gate by 64 + the
 * transitions on its fanin pins (its evaluation cost); and orders the gates
 * by decreasing weighted longest path to a netlist output, critical path
 * first.  A calibration run over a short window or another stimulus of the
 * same design is enough: only the relative activity of the nets matters.
 * Runs created afterwards with the dependency schedule on this netlist
 * (alone or replicated in a batch) use the order; existing runs keep theirs.
 * run_id = -1 restores level order.  Device memory: 48 bytes per gate.
 * GLS_EINVAL for unknown ids or an item of another netlist; the run's own
 * error when it failed.
 */
int gls_plan_order(gls_ctx *ctx, int32_t netlist_id, int32_t run_id, int32_t item);

/*
 * Paper: a waveform of the device store (Sec. 3.1, CSR rows), copied out.
 *
 * Copy one net's waveform to the host (item 0 of a batch): times into
 * t[cap], values into v[cap].  *n_out always receives the length; GLS_EOVERFLOW if cap < length
 * (nothing copied).  Synchronises with the run.
 */
int gls_read_waveform(gls_ctx *ctx, int32_t run_id, int32_t net, int32_t *t, uint8_t *v,
                      int64_t cap, int64_t *n_out);

/*
 * Paper: the whole store as one CSR (Sec. 3.1) in the single transfer back to
 * the host after the one-pass evaluation (Sec. 3).
 *
 * Copy every net's waveform to the host as one CSR: off[n_nets+1] (int64,
 * caller-allocated) and packed[cap] transitions, each (time << 2) | value,
 * nets in id order.  The device gathers the store into net order first so the
 * result comes back in a single device-to-host transfer.  GLS_EOVERFLOW if
 * cap is smaller than the total (off is still filled).  Synchronous.
 */
int gls_read_all(gls_ctx *ctx, int32_t run_id, int64_t *off, uint32_t *packed, int64_t cap);

/*
 * ---- General cells: full delay matrix, several outputs, user tables -------
 *
 * Sec. 3 keeps delays in a five-dimensional matrix [cell][input pin][output
 * pin][input edge][output value], an entry without an arc being infinite,
 * and builds every cell, user-defined primitives (UDP) included, from one
 * logic function per output.  A netlist of general cells: cell c reads
 * fanin_net[fanin_off[c]..fanin_off[c+1]) (pins a, b, c in order) and drives
 * one net per output; nets are numbered 0..n_pi-1 for the primary inputs,
 * then the outputs of cell 0, cell 1, ... in order.  delays holds, cell after
 * cell, n_in * n_out * 4 entries: delays[((p * n_out + o) * 2 + edge) * 2 +
 * value] with edge 0 for a rising and 1 for a falling input transition and
 * value 0 when the output falls to 0, 1 when it rises to 1, in ps; all four
 * entries of (p, o) are -1 when pin p has no arc to output o, else in
 * [1, 2^29).
 * Semantics (in addition to gls_simulate's): the edge of an input transition
 * follows Verilog's posedge/negedge classes (rising: 0->1, 0->X, 0->Z, X->1,
 * Z->1; falling: the mirror images); an X<->Z transition takes the smaller
 * delay of both edges; an output changing to X the smaller of both values;
 * an output whose change involves no pin with an arc takes its fastest arc
 * toward the new value; an output is X before its first transition
 * whatever its table gives for all-X inputs; each output is scheduled and
 * cancelled (Eq. 1) on its own.
 */
#define GLS_USER_CELL_BASE 16    /* first cell type id of gls_define_cell */
#define GLS_MAX_CELL_OUTPUTS 8

/* The 4^k-entry table of built-in cell `cell` (entry sum v_p 4^p over its k
   pins, values 0, 1, 2 = X), as the library evaluates it: the common value
   of the Boolean function over every 0/1 completion of X/Z inputs. */
int gls_cell_table(int32_t cell, uint8_t *table);

/* Define a cell (a UDP or a multi-output library cell) for this context:
   n_inputs in 1..3, n_outputs in 1..GLS_MAX_CELL_OUTPUTS, tables[o * 4^n_inputs
   + sum v_p 4^p] in {0, 1, 2 = X} for inputs v_p in {0, 1, 2 = X, 3 = Z}.
   *cell_type = GLS_USER_CELL_BASE + (cells defined before).  GLS_EINVAL for
   bad sizes or values. */
int gls_define_cell(gls_ctx *ctx, int32_t n_inputs, int32_t n_outputs, const uint8_t *tables,
                    int32_t *cell_type);

/* Load a netlist of general cells (built-in ids 0..GLS_NCELLS-1 with one
   output, or gls_define_cell ids); layout and delays as described above.
   The same checks and errors as gls_load_netlist, plus GLS_EINVAL for an
   output without any arc.  Netlists with edge-dependent delays, pins without
   arcs or an output that is not X for all-X inputs run on the windowed
   kernels only (GLS_EINVAL at run creation with GLS_KERNEL_SEGMENTED). */
int gls_load_netlist_cells(gls_ctx *ctx, int32_t n_pi, int32_t n_cells, const int32_t *cell_type,
                           const int32_t *fanin_off, const int32_t *fanin_net, const int32_t *delays,
                           int32_t *netlist_id);

/*
 * ---- Task division over time and 64-bit times ----------------------------
 *
 * A stimulus may run longer than the 2^30 - 1 ps a device transition holds
 * (Table 2's longest re-simulation runs to about 3e9 ps), and its waveforms
 * need not fit in HBM at once: a sliced run cuts the stimulus at
 * T_k = k * slice_ps and evaluates the slices in order, each in its own local
 * time, carrying every gate's state across each boundary (its input pin
 * values, its last output value, and the transitions it has scheduled at or
 * after the boundary, which later inputs may still cancel by Eq. 1).  A
 * transition scheduled before a boundary is final then, so the slices'
 * outputs, concatenated, are exactly the unsliced waveforms.  Under the
 * dependency schedule one launch evaluates up to 64 consecutive slices
 * (GLS_OPT_SLICE_GROUP): once a gate's fanins are done for all of them, one
 * warp takes the gate through them in turn, carrying its state from each
 * slice to the next, so the per-gate costs (work claim, record, fanin waits,
 * completion flag) are paid once per launch.  Under the level schedule each
 * slice is one set of level launches.  The waveforms of a launch's slices are
 * copied to host memory once the launch completes; device memory holds one
 * launch's transitions, the stimulus, 12 bytes of descriptors per net and
 * slice of a launch, and 3 * (4 + 4 * 256) bytes of gate state per net.
 */

/* Load a stimulus with 64-bit times: like gls_load_stimulus, with
   0 <= t < 2^62 (checked on the host, GLS_ESTIM).  Usable by sliced runs
   only (other runs give GLS_EINVAL). */
int gls_load_stimulus64(gls_ctx *ctx, int32_t n_pi, const int64_t *off, const int64_t *t,
                        const uint8_t *v, int32_t *stim_id);

/*
 * Simulate netlist_id under stim_id (32- or 64-bit times) in time slices of
 * slice_ps picoseconds; synchronous: returns once every slice is evaluated and
 * copied to host memory (into the context's pinned host pool while it has
 * room, GLS_OPT_HOST_POOL_BYTES).  The last slice runs to the end of all
 * activity.
 * The windowed kernels only (GLS_EINVAL with GLS_KERNEL_SEGMENTED); either
 * schedule and a planned order apply.  arena_events sizes the event arena of
 * one launch (0: about 256 words per stimulus transition of the slices of a
 * launch); a launch that overflows it is evaluated again, from the same
 * input state, with a larger arena.
 * GLS_ERANGE when slice_ps + the longest path delay reaches 2^30 - 1, or when a
 * gate carries more than 256 scheduled transitions across a boundary;
 * GLS_EINVAL for more than 2^20 slices.  gls_run_stats reports the total
 * output transitions and the summed device time of the launches' gate kernels;
 * gls_rerun evaluates every slice again (synchronously); gls_read_all,
 * gls_read_item and gls_read_waveform give GLS_EINVAL for sliced runs.
 */
int gls_simulate_sliced(gls_ctx *ctx, int32_t netlist_id, int32_t stim_id, int64_t slice_ps,
                        int64_t arena_events, void *cuda_stream, int32_t *run_id);

/* Number of slices a sliced run was evaluated in (0 for other runs). */
int gls_run_slices(gls_ctx *ctx, int32_t run_id, int32_t *n_slices);

/* Every net's waveform of a sliced run, in net id order: off[n_nets + 1]
   (always filled), 64-bit times t[cap] and values v[cap].  GLS_EOVERFLOW if
   cap is below the total.  Host memory only; results of more than 4 Mi
   transitions are widened on up to 16 host threads (Sec. 3.1 storage read
   back as one CSR over the whole stimulus). */
int gls_read_all64(gls_ctx *ctx, int32_t run_id, int64_t *off, int64_t *t, uint8_t *v, int64_t cap);

/* One net's waveform of a sliced run: *n_out always receives its length;
   GLS_EOVERFLOW if cap is smaller (nothing copied). */
int gls_read_waveform64(gls_ctx *ctx, int32_t run_id, int32_t net, int64_t *t, uint8_t *v, int64_t cap,
                        int64_t *n_out);

/*
 * Results of a run created with GLS_OPT_HOST_MIRROR, without a device-to-host
 * copy of the waveforms: waits for the run (its error, if it failed), then
 * *arena = the run's pinned host mirror (valid until the run is evaluated
 * again or released), and for every gate g of item `item` in caller order
 * (net n_pi + g) its waveform is (*arena)[gate_off[g] .. gate_off[g] +
 * gate_len[g]), packed (time << 2) | value as in gls_read_all.  Primary
 * inputs are the caller's stimulus and are not listed.  gate_off and
 * gate_len hold n_gates entries (host arrays).  GLS_EINVAL for a run without
 * a mirror.
 */
int gls_read_host(gls_ctx *ctx, int32_t run_id, int32_t item, const uint32_t **arena, int64_t *gate_off,
                  uint32_t *gate_len);

/* Context options (gls_set_option); they apply to runs created afterwards. */
typedef enum gls_option {
    GLS_OPT_SCHEDULE = 1,       /* GLS_SCHEDULE_LEVELS or GLS_SCHEDULE_DEPENDENCY (default)  */
    GLS_OPT_WARPS_PER_CTA = 2,  /* warps per CTA of the gate kernels, 1..32 (default 4)        */
    GLS_OPT_WAIT_LIMIT_MS = 3,  /* bound on one device wait for a fanin gate (default 10000)    */
    GLS_OPT_TEST_WITHHOLD_GATE = 4, /* test hook for the bounded wait: the gate at this level-order
                                       position never signals completion, so its readers wait out
                                       the limit and the run reports GLS_ETIMEOUT (-1 = off)     */
    GLS_OPT_KERNEL = 5,         /* GLS_KERNEL_WINDOWED_WIDE (default), _WINDOWED or _SEGMENTED  */
    GLS_OPT_SEGMENT = 6,        /* segmented kernel: input transitions per lane segment, >= 1
                                   (default 32); a gate uses min(32, ceil(inputs / this)) lanes */
    GLS_OPT_HOST_MIRROR = 8,    /* 1: runs created afterwards (not sliced, windowed kernels)
                                   also copy every gate's waveform into a pinned host mirror of
                                   their event arena as soon as the gate is done (aligned 16-byte
                                   stores), so the results reach host memory while the
                                   simulation runs (gls_read_host);
                                   0 (default): results stay on the device until read */
    GLS_OPT_POOL_BYTES = 7,     /* > 0: allocate one device region of this size now and carve
                                   every later netlist, stimulus and run buffer from it (first
                                   fit, no cudaMalloc/cudaFree per run, so creating and freeing
                                   runs does not synchronise the device); 0: free the pool.
                                   Only when no pool block is in use. */
    GLS_OPT_HOST_POOL_BYTES = 9, /* > 0: allocate one pinned, device-mapped host region of this
                                   size now and carve the host mirrors of later runs
                                   (GLS_OPT_HOST_MIRROR) from it, first fit, instead of pinning
                                   new host memory per run; GLS_ENOMEM at run creation when no
                                   block is large enough.  Sliced runs also keep their slices'
                                   waveforms in it while it has room (the copies from the
                                   device then run at the link's rate), else in ordinary host
                                   memory.  0: free it.  Only when no block is in use. */
    GLS_OPT_SLICE_GROUP = 10    /* sliced runs under the dependency schedule: most time slices
                                   one launch evaluates, 1..64 (default 64) */
} gls_option;

/* Gate kernel variants; all compute the same waveforms.
   SEGMENTED: each lane of a warp evaluates one time segment of the gate
   sequentially and the segments are reconciled once per gate.
   WINDOWED / WINDOWED_WIDE: the warp streams shared-memory windows of 128 /
   352 transitions per pin of 3-input cells (1.5x for 2-input, 3x for
   1-input cells) and merges, evaluates and filters each window
   cooperatively. */
enum { GLS_KERNEL_SEGMENTED = 0, GLS_KERNEL_WINDOWED = 1, GLS_KERNEL_WINDOWED_WIDE = 2 };

/* Schedules of the gate evaluation (Sec. 4.1).
   LEVELS: one kernel launch per DAG level (the topological-layer partition
   the paper criticises, kept as the reference form), all in one CUDA graph.
   DEPENDENCY: one persistent launch; each warp takes the next gate in level
   order (or the netlist's planned order, gls_plan_order) and starts it as
   soon as its fanin gates are done (Algorithm 1's
   readiness test, without layer barriers); a wait longer than
   GLS_OPT_WAIT_LIMIT_MS ends the run with GLS_ETIMEOUT. */
enum { GLS_SCHEDULE_LEVELS = 0, GLS_SCHEDULE_DEPENDENCY = 1 };

/* Set a context option; GLS_EINVAL for an unknown option or value. */
int gls_set_option(gls_ctx *ctx, int option, int64_t value);

/*
 * Simulation that allocates no device memory.  The paper has no counterpart:
 * this entry point serves callers that cannot call cudaMalloc / cudaFree at
 * the time they simulate -- code being captured into a CUDA graph (allocation
 * is not a stream operation), frameworks that own all device memory through
 * their own pool or a fixed budget, and tight loops where an allocation would
 * synchronise the device.  The netlist and stimulus must already be loaded
 * (loading allocates, once, at set-up); the caller passes the output store in
 * device memory:
 *   d_net_ptr[n_nets]    device u64: address of each net's first transition
 *   d_net_len[n_nets]    device u32: transition count of each net
 *   d_arena[arena_words] device u32, 16-byte aligned: gate output
 *                        transitions, each (time << 2) | value;
 *                        arena_words >= 64, and the last 64 words are kept
 *                        free as read padding
 *   d_report[4]          device u32, written at the end of the run:
 *                        [0] status bits (1 = arena too small, 2 = carried
 *                        transitions beyond GLS_MAX_DELAY_SPREAD, 4 = a time
 *                        reached 2^30 - 1), [1] and [2] low and high words of
 *                        the arena demand in words, [3] 0
 * Nets are indexed in the netlist's device order: primary inputs first, then
 * gates sorted by level (level_out of gls_check_netlist), equal levels in
 * gate-id order; primary-input entries point into the loaded stimulus.  The
 * gates run with the level schedule and the context's kernel variant.
 * The run's scratch (per-level work counters, the arena bump pointer, the
 * status word) lives in one statically allocated device array of
 * GLS_NOALLOC_SCRATCH_WORDS 32-bit words (16 KiB) that every GPU which loads
 * the library holds until the process exits; a netlist deeper than
 * GLS_NOALLOC_MAX_LEVELS levels is rejected with GLS_ERANGE.  Each call resets
 * that scratch, and every call on a device shares it: calls whose work
 * overlaps on the GPU (other streams, other contexts on the same device) race
 * and must be serialised by the caller.  The first call on each device looks
 * up the array's device address; make that first call before any stream
 * capture.  Stream-ordered on cuda_stream (NULL = the context's stream), no
 * synchronisation; host-side errors (ids, sizes, GLS_ERANGE) are returned
 * before anything is enqueued.
 */
#define GLS_NOALLOC_MAX_LEVELS 4000
#define GLS_NOALLOC_SCRATCH_WORDS 4096
int gls_simulate_noalloc(gls_ctx *ctx, int32_t netlist_id, int32_t stim_id, uint64_t *d_net_ptr,
                         uint32_t *d_net_len, uint32_t *d_arena, int64_t arena_words, uint32_t *d_report,
                         void *cuda_stream);

/*
 * gls_read_all for item 'item' of a run (0 for runs made by gls_simulate,
 * whose read calls refer to their only item): off[n_nets(item) + 1] and
 * packed[cap] as in gls_read_all, nets in the item's caller order.
 */
int gls_read_item(gls_ctx *ctx, int32_t run_id, int32_t item, int64_t *off, uint32_t *packed, int64_t cap);

/* Free a netlist, stimulus or run handle (ids are unique per context). */
int gls_release(gls_ctx *ctx, int32_t id);

#ifdef __cplusplus
}
#endif
#endif /* GLS_H */
