/*
 * coral.h — C ABI of the GB300 (sm_103a) substrate-step library.
 *
 * The library steps the toroidal substrate of Coralai (Barbieux & Canaan, arXiv 2406.09654):
 * every cell senses a rotation-ordered 3x3 Moore neighbourhood (the "Kernel") of six sensor
 * channels, runs the dense network selected by its GenomeIndex (weights generated by the
 * genome's CPPN, HyperNEAT), and the physics turns the ten actuator outputs into the next
 * substrate (Section "System Design", Section "Experiment", Fig. 1).
 *
 * Conventions shared by every entry point
 *  - Every call returns a coral_status (0 = OK, negative = error). No C++ exception crosses
 *    the ABI. After an error, coral_last_error(s) returns a message (valid until the next call
 *    on the same substrate from the same thread).
 *  - The library owns all device memory of a substrate; it allocates it in
 *    coral_substrate_create and frees it in coral_substrate_destroy. Caller buffers are never
 *    retained or freed by the library: they are copied in or out during the call (calls that
 *    read host buffers wait for their copies; device-to-device copies are stream-ordered).
 *  - Work is enqueued on the CUDA stream given at creation (NULL = the legacy default stream).
 *    coral_step returns after enqueueing; errors that happen on the device (e.g. genome
 *    capacity exhaustion) are latched in a device status word and returned by the next
 *    synchronising call (coral_sync, coral_read_*).
 *  - Grid layout: cell j = y * width + x, row y = 0 is "north"; the torus wraps in x and y.
 *    Channel planes are float32 row-major [height][width]; C is [4][height][width].
 *  - `*_on_device` flags: nonzero = the pointer is a CUDA device pointer on the substrate's
 *    device (for example a torch tensor's data_ptr()), zero = host memory (pinned or pageable).
 *  - Threads: calls on different substrates and batches may run concurrently from different
 *    host threads (they share no mutable state; error messages are per handle, or per thread
 *    for calls without one). Calls on one handle, and on a batch and the substrates it holds,
 *    must not overlap. coral_bucket_noalloc is the exception: its calls share one scratch
 *    array and must not overlap at all (see there).
 */
#ifndef CORAL_H
#define CORAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct coral_substrate coral_substrate;   /* opaque */

typedef enum {
  CORAL_OK = 0,
  CORAL_E_INVALID = -1,   /* bad argument (NULL pointer, size out of range, bad params) */
  CORAL_E_OOM = -2,       /* device allocation failed */
  CORAL_E_CUDA = -3,      /* a CUDA runtime call or kernel launch failed */
  CORAL_E_CAPACITY = -4,  /* a buffer given by the caller is too small */
  CORAL_E_TIMEOUT = -5,   /* a bounded device-side wait gave up */
  CORAL_E_STATE = -6      /* call out of order (e.g. step before any genome table load) */
} coral_status;

typedef enum {
  CORAL_NET_FP32_PERCELL = 0,  /* plain FP32 CUDA-core network, one thread per cell */
  CORAL_NET_BF16_GROUPED = 1   /* BF16 tcgen05 tensor-core network grouped by genome per tile,
                                  FP32 TMEM accumulation, FP32 state */
} coral_path;

/* Channel bits for coral_read_channels / coral_state_load masks. */
enum {
  CORAL_CH_E = 1u << 0, CORAL_CH_I = 1u << 1,
  CORAL_CH_C0 = 1u << 2, CORAL_CH_C1 = 1u << 3, CORAL_CH_C2 = 1u << 4, CORAL_CH_C3 = 1u << 5,
  CORAL_CH_G = 1u << 6,   /* int32 GenomeIndex plane */
  CORAL_CH_R = 1u << 7,   /* uint8 rotation plane, values 0=N 1=E 2=S 3=W */
  CORAL_CH_ALL = 0xFFu
};

/*
 * Method constants. The paper names these mechanisms but prints no values; the defaults
 * returned by coral_params_default are the readings the library and its tests use.
 */
typedef struct coral_params {
  int32_t hidden;          /* H: 0 = one layer 54->10; else 54->H->10 with H in {16,32,48,64} */
  int32_t path;            /* coral_path */
  float k_inv;             /* invest rate: i = k_inv * max(a4, 0)            (default 0.1) */
  float k_liq;             /* liquidate rate: l = k_liq * max(a5, 0)         (default 0.1) */
  float k_exp;             /* explore amount x = k_exp * m * I1              (default 0.5) */
  float k_flow;            /* fraction of energy a cell sends along infrastructure (0.2) */
  float e_day;             /* energy added per cell per step by day          (0.005) */
  float e_night;           /* fraction of energy removed per step by night   (0.005) */
  int32_t day_period;      /* day/night period T in steps; day = first half  (200) */
  int32_t rotation;        /* 1 = kernel ordered by each cell's rotation, 0 = always north */
  int32_t radiation_every; /* M: radiation after step t when (t+1) % M == 0; 0 = off */
  double p_mut;            /* mutation probability per cell and radiation event, in [0, 1]; a
                              cell is hit iff its Philox word < min(floor(p_mut * 2^32), 2^32 - 1) */
  double p_merge;          /* merge probability per cell and radiation event, in [0, 1] (same rule) */
  float sigma_mut;         /* std of the Gaussian added to every gene by a mutation (0.05) */
  uint32_t world;          /* Philox counter word 3 (distinguishes independent worlds) */
  uint64_t seed;           /* Philox key */
} coral_params;

/* Per-step record kept in a device ring (read with coral_read_stats). */
typedef struct coral_stats {
  int64_t step;            /* step index t this record describes (state after step t) */
  double sum_E;            /* FP64 total energy after the step */
  double sum_I;            /* FP64 total infrastructure */
  double sum_C[4];         /* FP64 totals of the communication channels */
  int64_t n_explore;       /* cells that explored */
  int64_t n_takeover;      /* cells taken over */
  int64_t n_live;          /* live genome slots after radiation (-1 when no radiation ran) */
  int64_t n_mut;           /* radiation: mutation hits */
  int64_t n_merge;         /* radiation: merge hits with a different partner genome */
  int64_t n_born;          /* radiation: children given a slot */
  int64_t n_skipped;       /* radiation: hits dropped because no slot was free */
} coral_stats;

/* Fills *p with the default constants above (hidden = 0, FP32 path, seed 0). */
int coral_params_default(coral_params* p);

/*
 * Creates a width x height torus with room for genome_capacity genome slots on the current
 * CUDA device. Substrate: Section "System Design" (a tensor with width, height and named
 * channels). width, height >= 3 (a 2-wide torus makes the north and south neighbours the
 * same cell) and width * height < 2^31; genome_capacity in [1, 2^24].
 * cuda_stream: a cudaStream_t (NULL = legacy default stream). Errors: E_INVALID, E_OOM, E_CUDA.
 */
int coral_substrate_create(const coral_params* p, int32_t width, int32_t height,
                           int32_t genome_capacity, void* cuda_stream, coral_substrate** out);

/* Frees every device buffer of s (synchronises its stream first). NULL is a no-op. */
int coral_substrate_destroy(coral_substrate* s);

/*
 * Copies a full state in: E, I [N], C [4][N] float32; G [N] int32 (each in
 * [0, genome_capacity)); R [N] uint8 (each in 0..3). Any of the five pointers may be NULL
 * to leave that channel unchanged. Values of G and R are checked on the device; a bad
 * value is reported by the next synchronising call as E_INVALID. Steps enqueued before that
 * stay within the library's buffers: a cell whose G is out of range runs slot 0's net and is
 * never a parent or partner at radiation; an R above 3 gives an unspecified rotation. Also resets the step counter to 0 unless coral_set_step is
 * called afterwards.
 */
int coral_state_load(coral_substrate* s, const float* E, const float* I, const float* C,
                     const int32_t* G, const uint8_t* R, int src_on_device);

/*
 * Genome table (Section "System Design": GenomeIndex locates the network parameters).
 * Loads n genomes into slots 0..n-1 and marks slots n..capacity-1 free.
 * cppn_genes: [n][18] float32 CPPN genes, or NULL for direct nets (then radiation must be
 *   off). Gene layout: w[k][i] for hidden node k in (sin, gauss, tanh) and input i in
 *   (x1, y1, x2, y2, bias), k-major (15 floats), then v[k], hidden->output (3 floats).
 * dense_or_null: [n][net_floats] float32 direct nets, used when cppn_genes is NULL:
 *   hidden = 0: W[10][54] row-major then b[10];
 *   hidden = H: W1[H][54], b1[H], W2[10][H], b2[10].
 * Input index i of W/W1 is 6 * rank + channel (rank 0 = centre, then the kernel order;
 * channel order E, I, C0, C1, C2, C3); output order com0..3, invest, liquidate, explore0..3.
 * With CPPN genes, call coral_cppn_generate_weights afterwards.
 */
int coral_genome_table_load(coral_substrate* s, int32_t n, const float* cppn_genes,
                            const float* dense_or_null, int src_on_device);

/*
 * HyperNEAT (Section "System Design"; Fig. 1 C): queries each listed slot's CPPN at every
 * connection (x1, y1, x2, y2) of its dense net and writes the FP32 net and its BF16
 * tensor-core copy. Inputs sit at y = -1, hidden nodes at y = 0, outputs at y = +1, the n
 * nodes of a layer at x = -1 + 2i/(n-1); biases are queried at (0, 0, x2, y2); weights are
 * scaled by 1/sqrt(fan_in). slots_or_null: host int32 slot ids, or NULL = slots 0..n-1.
 */
int coral_cppn_generate_weights(coral_substrate* s, const int32_t* slots_or_null, int32_t n);

/*
 * Enqueues n_steps synchronous updates (Section "System Design": in discrete time steps each
 * cell is updated) on the stream, each: sense + network + actuators (pass 1), exploration,
 * energy flow and day/night (pass 2), FP64 totals into the stats ring, and radiation with
 * CPPN regeneration after steps with (t+1) % M == 0 (Fig. 1 C). Returns after enqueueing.
 * Errors: E_STATE before a genome table is loaded; E_CUDA on launch failure.
 */
int coral_step(coral_substrate* s, int32_t n_steps);

/*
 * Small-genome path of the BF16 tensor-core network (Section "System Design": each cell runs
 * the net its GenomeIndex selects). A 128-cell tile whose cells hold several genomes runs one
 * tensor-core round per genome; with cells > 0, a later round whose genome owns at most `cells`
 * cells of the tile runs on the CUDA cores instead: each of those cells' warps evaluates the
 * net lane by lane (hidden units spread over the lanes, BF16 operands and FP32 sums as on the
 * tensor cores, the weights read from the genome's BF16 blob through L1, the ten outputs
 * reduced over the warp), which saves the tile that round's staging, MMAs and barriers.
 * 0 (the default) = off. Results equal the tensor-core path's up to the FP32 summation order.
 * cells in [0, 128], else E_INVALID. No effect on the FP32 path.
 */
int coral_set_fma_cutoff(coral_substrate* s, int32_t cells);

/*
 * coral_step with CUDA-event timing (tracing): same work, same stream, plus events recorded
 * around each stage. step_ms: [n_steps] device time of each step; stage_ms: [n_steps][3]
 * time of pass 1 (sense + network + actuators), pass 2 (exploration, flow, day/night) and the
 * rest (totals, radiation). Host arrays, either may be NULL. Synchronises.
 */
int coral_step_timed(coral_substrate* s, int32_t n_steps, float* step_ms, float* stage_ms);

/*
 * Copies the planes selected by channel_mask (CORAL_CH_*) of the current state into dst,
 * packed plane after plane in increasing bit order: E, I, C0..C3 as float32 [N], G as int32
 * [N], R as uint8 [N]. dst_bytes must cover them all (else E_CAPACITY). Synchronises.
 */
int coral_read_channels(coral_substrate* s, uint32_t channel_mask, void* dst, size_t dst_bytes,
                        int dst_on_device);

/*
 * Steps a sequence of independent states ("jobs") of this substrate's world from host memory
 * to host memory. Job k's state is read from host_in[k], loaded, validated like
 * coral_state_load, stepped n_steps times starting at step index t0 (so every job sees the same
 * day/night phase and radiation schedule), and the resulting state is written to host_out[k].
 * A state is packed like coral_read_channels with CORAL_CH_ALL: E, I, C0..C3 as float32 [N],
 * G as int32 [N], R as uint8 [N] (29 bytes per cell). An input buffer must not overlap an
 * output buffer; all host_in[k] may be one shared read-only buffer and all host_out[k] one
 * shared buffer (written in job order). The copy in of job k+1, the steps of
 * job k and the copy out of job k-1 run concurrently on separate CUDA streams through two pairs
 * of device staging buffers (allocated at the first call, 4 x 29 bytes per cell, kept until
 * destroy); page-locked host buffers let the copies overlap. Returns after every result is in
 * host memory; the substrate's own state is then the last job's result and its step counter
 * t0 + n_steps. The genome table is the substrate's: a radiation event inside one job changes
 * it for the jobs after it. Errors: E_INVALID for bad arguments or an invalid G/R in any input (reported
 * after all jobs ran), E_OOM, E_CUDA. The paper has no counterpart: this is the library's
 * host-to-host stepping path, used for the end-to-end throughput.
 */
int coral_step_jobs(coral_substrate* s, int32_t n_jobs, const void* const* host_in, void* const* host_out,
                    int32_t n_steps, int64_t t0);

/* Copies up to n stats records starting at step step_from (steps older than the ring's
 * 4096-step window are gone: E_INVALID). Host memory. Synchronises. */
int coral_read_stats(coral_substrate* s, int64_t step_from, int32_t n, coral_stats* out);

/*
 * Bucketing of cells by GenomeIndex: a stable counting sort of the current G (implemented
 * as least-significant-digit passes of stable 8-bit counting sorts). dst_counts:
 * [capacity] int32 cells per slot; dst_perm: [N] int32 cell ids, slot 0's cells in
 * increasing order, then slot 1's, ... Either may be NULL. Host memory. Synchronises.
 */
int coral_read_perm(coral_substrate* s, int32_t* dst_counts, int32_t* dst_perm);

/* Reads the genome table: genes [capacity][18] float32, parent [capacity] int32 (-1 for
 * loaded genomes and never-used slots). Either may be NULL. Host memory. Synchronises. */
int coral_read_genomes(coral_substrate* s, float* genes, int32_t* parent);

/* Reads slot's FP32 dense net in the dense_or_null layout of coral_genome_table_load. */
int coral_read_weights(coral_substrate* s, int32_t slot, float* dst, size_t dst_floats);

/*
 * Genetic similarity (Section "Discussion and Future Work": NEAT's measure of genetic
 * similarity). NEAT's compatibility distance is c1 E/N + c2 D/N + c3 W, W the mean weight
 * difference of matching genes; the CPPNs here share one topology (no excess or disjoint
 * genes), so the distance is c3 * mean_k |g_a[k] - g_b[k]| over the 18 genes, c3 = 0.4.
 * slots: host int32 [n] genome slots; out: host float32 [n][n]. n in [1, 4096]. Synchronises.
 * Phylogeny: the parent column of coral_read_genomes links every born genome to its parent.
 */
int coral_genome_distances(coral_substrate* s, const int32_t* slots, int32_t n, float* out);

/* Step index of the next coral_step (for checkpoint/resume; Philox is keyed by it). */
int coral_set_step(coral_substrate* s, int64_t t);
int coral_get_step(const coral_substrate* s, int64_t* t);

/* Launch configuration chosen at creation (tracing): CTAs of pass 1 and pass 2 and the SM
 * count of the device. Any pointer may be NULL. */
int coral_launch_config(const coral_substrate* s, int32_t* grid_pass1, int32_t* grid_pass2,
                        int32_t* sms);

/*
 * Batched stepping of many independent worlds (many substrates in one launch per pass, the
 * per-step launch sequence replayed as a CUDA graph). All worlds: BF16 path, the same hidden
 * size, a genome table loaded (CPPN genes where radiation is on), whole worlds (no row slabs),
 * the current CUDA device. Each world keeps its own radiation schedule: after a step that ends
 * one of its epochs, its radiation (Section "System Design", Fig. 1 C) runs on the batch stream
 * before the next step's graph, as coral_step runs it. The CTAs of each launch
 * are divided among the worlds in proportion to their sizes, at least one each (each CTA works
 * on one world; a launch asks for 32 times the CTAs of its launch shape, so that the block
 * scheduler evens out small and large worlds), and a world's cells are bit-identical to
 * stepping it alone. The batch has its own stream; before
 * each coral_batch_step it waits for work already enqueued on the worlds' streams, and the
 * worlds' streams wait for the batch's steps, so per-world calls (reads, loads) stay ordered.
 * The substrates stay owned by the caller and must outlive the batch.
 * Errors: E_INVALID (mixed hidden sizes / paths / devices, a row slab), E_STATE (no genome
 * table, radiation with direct nets), E_OOM, E_CUDA.
 */
typedef struct coral_batch coral_batch;
int coral_batch_create(coral_substrate* const* worlds, int32_t n, coral_batch** out);
int coral_batch_destroy(coral_batch* b);
/* Enqueues n_steps steps of every world (each a replay of one captured CUDA graph). */
int coral_batch_step(coral_batch* b, int32_t n_steps);
/* Same, with a CUDA event pair around every step: step_ms[n_steps] (host). Synchronises. */
int coral_batch_step_timed(coral_batch* b, int32_t n_steps, float* step_ms);
/*
 * Autotuner: times trial_steps steps (after one warm-up; graphs only, no radiation, so that
 * the genome tables stay as they are) for each candidate launch shape —
 * pass-1 CTAs per SM in {3, 4, 5, 6} x pass-2 CTAs per SM in {1, 2, 3}, each times 32 as
 * above — then, at the fastest shape, the small-genome cutoff (coral_set_fma_cutoff) in
 * {0, 1, 2, 4, 8}; keeps the fastest and
 * restores every world's state, step index and stats ring afterwards (also after an error,
 * which leaves the launch shape the batch had before the call; a failed save or restore copy
 * returns E_CUDA). choice: [4] = {pass-1 CTAs per SM,
 * pass-2 CTAs per SM, best step time in microseconds, small-genome cutoff} (may be NULL).
 * Synchronises.
 */
int coral_batch_tune(coral_batch* b, int32_t trial_steps, int32_t* choice);
/* The small-genome cutoff of every world in the batch (as coral_set_fma_cutoff; the batch's
 * own setting, not the substrates'), until the next tune. Recaptures the batch's graphs. */
int coral_batch_set_fma_cutoff(coral_batch* b, int32_t cells);

/*
 * Failure-detection self-test (library infrastructure; the paper has no counterpart): launches
 * one CTA that allocates tensor memory and waits, with the same bounded wait the tensor-core
 * kernel uses, on an mbarrier that nothing arrives on, for about wait_us microseconds of SM
 * clock (1 .. 1,000,000). The wait runs out, the kernel records CORAL_E_TIMEOUT, frees its
 * tensor memory and returns; *status_out receives the recorded status. Nothing faults or hangs
 * and the context stays usable. cuda_stream: NULL = legacy default stream. Synchronises.
 */
int coral_selftest_wait_timeout(void* cuda_stream, int32_t wait_us, int32_t* status_out);

/*
 * Known-answer test hook of the radiation's random numbers (reading R2: Philox4x32-10 of
 * Salmon et al., SC'11, keyed by the run seed): evaluates, on the current device, the same
 * Philox4x32-10 function the radiation kernels draw from. ctr: host uint32 [n][4] counters;
 * key: host uint32 [n][2] keys; out: host uint32 [n][4] results. n in [1, 65536], else
 * E_INVALID. Uses the legacy default stream; allocates a temporary device buffer; synchronises.
 */
int coral_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int32_t n);

/*
 * Measurement hook (library infrastructure; the paper has no counterpart): the throughput of
 * the special-function unit for tanh.approx.f32, the instruction the BF16 path's hidden and
 * output activations run on, measured on the current device with eight independent chains
 * per thread over 8 CTAs of 256 threads per SM. *evals_per_s receives evaluations per second.
 * cuda_stream: NULL = legacy default stream. Allocates a small device buffer; synchronises.
 */
int coral_measure_sfu_rate(void* cuda_stream, double* evals_per_s);

/*
 * Row slabs: one world split into horizontal slabs of rows, one substrate per slab (a logical
 * rank; on several GPUs one rank per device). Section "System Design" updates every cell of the
 * substrate synchronously from its neighbourhood, so a slab with copies of its neighbours' rows
 * steps its own rows exactly as the whole world would. A slab substrate is width x (own rows +
 * 6): 3 ghost rows above and below the own rows, refreshed from the neighbouring slabs' own rows
 * before every step (coral_copy_rows). A step's new state depends on the old state within two
 * rows, and radiation's merge partner is one row away, whose post-step state the third ghost
 * row gives exactly. The library keeps no list of slabs: the caller exchanges the rows and runs
 * the radiation protocol (scan every slab, combine, apply every slab), so that the slabs may
 * live in different processes. The results (state, genome table, radiation decisions) are
 * bit-identical to stepping the whole world in one substrate.
 *
 * coral_slab_set: rows [row_lo, row_hi) of s are its own rows (1 <= row_lo < row_hi <=
 * height - 1), the global id of cell (row_lo, 0) is global_cell0 (the Philox counter and the
 * order of radiation hits use global ids; ids stay below 2^32). From then on coral_step runs no
 * radiation on s, and coral_slab_totals / the radiation calls act on the own rows only.
 */
int coral_slab_set(coral_substrate* s, int32_t row_lo, int32_t row_hi, int64_t global_cell0);

/*
 * Copies rows [src_row, src_row + n_rows) of every plane (E, I, C0..C3, G, R) of src's current
 * state into rows [dst_row, dst_row + n_rows) of dst's current state (device to device, same
 * width and device; src == dst allowed for disjoint ranges: a single slab's ghost rows). The
 * copy is ordered after the work enqueued on src's stream, and src's later work after the copy.
 * Returns after enqueueing. Errors: E_INVALID (widths, devices, row ranges), E_CUDA.
 */
int coral_copy_rows(coral_substrate* dst, int32_t dst_row, coral_substrate* src, int32_t src_row, int32_t n_rows);

/* FP64 totals (E, I, C0..C3) over the own rows of a slab (all rows otherwise), fixed summation
 * order: out[6] host. Synchronises. (A slab's stats ring counts its ghost rows too.) */
int coral_slab_totals(coral_substrate* s, double* out);

/*
 * Radiation of a slab, first half (Fig. 1 C; readings R10-R12), for the step that just ran
 * (step index coral_get_step - 1): which genome slots own a cell among the own rows, and the own
 * rows' hits in increasing global cell order. live: host uint8 [capacity] (1 = the slot owns an
 * own cell); hits: host int32 [max_hits][5] = (global cell id, parent slot, merge partner slot
 * or -1, flags: 1 mutation | 2 merge, crossover bits); counts: host int32 [4] = (hits, mutation
 * hits, merge hits, hits listed = min(hits, capacity, max_hits)). Synchronises.
 * Errors: E_STATE (not a slab, no CPPN genomes, no step yet), E_INVALID.
 */
int coral_slab_radiation_scan(coral_substrate* s, uint8_t* live, int32_t* hits, int32_t max_hits, int32_t* counts);

/*
 * Radiation of a slab, second half: live_all = the OR of every slab's live flags; hits_all =
 * every slab's listed hits concatenated in slab order (the global cell order), n_listed rows;
 * counts_all = the sums over the slabs of counts[0..2]. Assigns the lowest free slots to the hits
 * in order (hits beyond the free slots are skipped and counted), writes every child genome into
 * this slab's genome table (each slab holds the whole table), sets G of the own cells among the
 * hits, regenerates the new slots' nets and writes the event counts into the stats record of the
 * step. Every slab must be given the same arguments. Synchronises. Errors: E_STATE, E_INVALID.
 */
int coral_slab_radiation_apply(coral_substrate* s, const uint8_t* live_all, const int32_t* hits_all,
                               int32_t n_listed, const int32_t* counts_all);

/* Waits for the stream and returns the first latched device-side error, if any. */
int coral_sync(coral_substrate* s);

/* Message for the last error on s (or a generic one when s is NULL). Never NULL. */
const char* coral_last_error(const coral_substrate* s);

/*
 * Allocation-free bucketing. The paper has no counterpart: this is a library convenience for
 * callers that cannot allocate device memory when they need the sort — code running inside a
 * stream capture they do not own, real-time loops where an allocator call may synchronise the
 * device or fail under memory pressure, hosts that give the library a fixed memory budget.
 * Same result as coral_read_perm (stable counting sort of cell ids by genome slot), on
 * caller-owned device buffers: G [n_cells] int32 in [0, capacity), counts [capacity] int32 and
 * perm [n_cells] int32 (outputs). Work is enqueued on cuda_stream (NULL = legacy default
 * stream); the call returns after enqueueing and allocates nothing. G is not validated (the
 * call returns before the device reads it): a key outside [0, capacity) is left out of counts
 * (the counts of valid slots stay exact) and perm is still a permutation of the cells, but its
 * order is then unspecified.
 * Limits: n_cells <= 1,048,576 and capacity <= 65,536, else CORAL_E_INVALID with a message in
 * coral_bucket_noalloc_last_error(). The scratch is one fixed 12.3 MiB device array per GPU
 * that loads the library, kept until the process exits, shared by every call: calls that
 * overlap on the GPU (different streams, no ordering) race on it and corrupt each other's
 * results. The first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture.
 */
int coral_bucket_noalloc(const int32_t* G, int64_t n_cells, int32_t capacity, int32_t* counts,
                         int32_t* perm, void* cuda_stream);
const char* coral_bucket_noalloc_last_error(void);

/* Floats in one dense net for a given hidden size (the dense_or_null row length). */
int32_t coral_net_floats(int32_t hidden);

#ifdef __cplusplus
}
#endif

#endif /* CORAL_H */
