/*
 * sqa.h -- C ABI of the GB300 (sm_103a) library for the simulated quantum
 * annealing (SQA) and parallel tempering (PT) hot path of
 *   T. Albash, W. Vinci, D. A. Lidar, "Simulated Quantum Annealing Comparison
 *   between All-to-All Connectivity Schemes", arXiv:1603.03755.
 *
 * What the library computes
 *   A fully connected logical Ising problem H_P = sum_{i<j} J_ij s_i s_j
 *   (Eq. 1, h = 0 as in Sec. III) is embedded into a physical problem, either
 *   by minor embedding on a Chimera graph (Sec. II A: chains of ceil(N/4)+1
 *   spins coupled with -penalty) or by the LHZ scheme (Sec. II B, Eq. 2:
 *   one spin per logical pair with local field J_ij and C(N-1,2) plaquette
 *   constraints of strength penalty).  SQA runs single-spin Metropolis sweeps
 *   over the L Trotter slices of the path-integral representation of
 *   H(t) = A(t) H_X + B(t) H_P (Eq. 3, App. B); PT runs the same sweep at zero
 *   transverse field on P temperature slots with neighbour swaps accepted with
 *   probability min{1, exp[(E_{i+1}-E_i)(beta_{i+1}-beta_i)]} (Eq. 9).  SQA
 *   can also run time-like cluster (Wolff) moves, the paper's own SQA update
 *   (Sec. III).  Readouts are decoded by majority vote (Eqs. 4-5), LHZ
 *   spanning trees (App. A, Eqs. 10-11), LHZ minimum-weight decoding
 *   (Sec. IV A) or LHZ belief propagation (Sec. IV, App. C).  Batches of
 *   jobs run in one persistent launch (replayable from a CUDA graph), and a
 *   server serves a stream of jobs with continuous batching.
 *
 * Conventions
 *   - Every call returns an sqa_status and never aborts the process.
 *   - Spins are bits: bit 0 <-> sigma = +1, bit 1 <-> sigma = -1.  Replica r
 *     of a (site, slice) lives in bit (r % 32) of word (r / 32).
 *   - Physical sites use the canonical numbering of the embedding:
 *     ME site ((r*Lc + c)*2 + u)*4 + k on an Lc x Lc Chimera (Lc = ceil(N/4),
 *     u = 0 vertical shore, u = 1 horizontal shore); LHZ spin (i,j), i<j, at
 *     i*N - i(i+1)/2 + (j-i-1).  Sites the embedding does not use read 0.
 *   - Inputs are copied; output buffers belong to the caller.  "Device"
 *     pointers are CUDA device addresses (e.g. from torch tensors); streams
 *     are cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - A handle is used by one host thread at a time.
 *   - Results are bit-reproducible: they depend only on the descriptor (J,
 *     seed, ...) and never on batch composition, launch shape or device.
 */
#ifndef SQA_GB300_H
#define SQA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SQA_OK = 0,
    SQA_ERR_INVALID = -1,     /* bad argument; nothing was changed */
    SQA_ERR_UNSUPPORTED = -2, /* valid but outside what this build supports */
    SQA_ERR_NOMEM = -3,       /* device or host allocation failed */
    SQA_ERR_CUDA = -4,        /* a CUDA call failed; see sqa_last_error() */
    SQA_ERR_TIMEOUT = -5,     /* a bounded wait ran out */
    SQA_ERR_NO_DEVICE = -6,   /* no CUDA device is visible */
    SQA_ERR_BUSY = -7,        /* resource in use (server full, job pending) */
    SQA_ERR_BOUNDS = -8       /* a bounds-checked build recorded an out-of-range access */
} sqa_status;

typedef enum { SQA_EMB_ME_CHIMERA = 0, SQA_EMB_LHZ = 1 } sqa_embedding;
typedef enum { SQA_KIND_SQA = 0, SQA_KIND_PT = 1 } sqa_kind;
/* SQA update move.  METROPOLIS: single-spin Metropolis sweeps over every
 * (site, slice).  WOLFF: one time-like cluster move per (site, replica) per
 * sweep (Sec. III, App. B): bonds between equal neighbouring slices join with
 * probability 1 - e^(-2 Jperp), the cluster grown from a random slice is
 * flipped with the Metropolis test on its problem-energy change. */
typedef enum { SQA_MOVE_METROPOLIS = 0, SQA_MOVE_WOLFF = 1 } sqa_move;
typedef enum {
    SQA_DECODE_ME_MV = 0,     /* ME majority vote per chain (Eq. 4); ties -> hub spin */
    SQA_DECODE_LHZ_TREES = 1, /* LHZ majority vote over n_trees random trees (Eq. 5) */
    SQA_DECODE_LHZ_STAR = 2,  /* LHZ star tree q_i = q_{0,i} (Eq. 11) */
    SQA_DECODE_LHZ_CHAIN = 3, /* LHZ chain tree q_i = prod_{m<i} q_{m,m+1} (Eq. 10) */
    SQA_DECODE_LHZ_MWD = 4,   /* LHZ minimum-weight decoding (Sec. IV A), exact by enumeration, N <= 24:
                                 the logical state whose pair products disagree with the fewest pair
                                 spins; q_{N-1} = +1, ties to the first state in binary order.  N > 24
                                 (2^23 states per replica and more) -> SQA_ERR_UNSUPPORTED: larger LHZ
                                 problems (the serving stream draws N up to 40) decode with the tree,
                                 vote or belief-propagation methods */
    SQA_DECODE_LHZ_BP = 5     /* LHZ belief propagation (Sec. IV, App. C), N <= 32, error rate 0.2 and
                                 10 iterations (sqa_decode_bp for others), read out by random tree 0 */
} sqa_decode_method;

/* Problem and program description.  All pointers are host pointers; the
 * arrays are copied by sqa_create. */
typedef struct {
    int32_t kind;          /* sqa_kind */
    int32_t embedding;     /* sqa_embedding */
    int32_t n_logical;     /* N >= 2 (ME: N <= 64, LHZ: N <= 64) */
    int32_t n_instances;   /* I >= 1 instances sharing every parameter but J */
    const int32_t *J;      /* [I][N(N-1)/2], row-major upper triangle (i<j) */
    const int32_t *h;      /* NULL, or [I][N] logical fields; non-zero -> UNSUPPORTED */
    int32_t penalty;       /* > 0: ME chain coupling -penalty; LHZ constraint strength */
    int32_t n_sweeps;      /* S >= 1 */
    int32_t n_replicas;    /* R >= 1 independent chains per instance */
    uint64_t seed;         /* keys every random stream */
    /* SQA (kind == SQA_KIND_SQA) */
    int32_t n_slices;      /* L, even, 2 <= L <= 1024 */
    double beta;           /* > 0 */
    const double *A;       /* [S] transverse-field schedule >= 0, or NULL for A = 1 - s */
    const double *B;       /* [S] problem schedule >= 0, or NULL for B = s; s_t = (t+1/2)/S */
    /* PT (kind == SQA_KIND_PT) */
    int32_t n_temps;       /* P >= 1 */
    const double *betas;   /* [P] strictly decreasing (coldest first), > 0 */
    int32_t swap_every;    /* >= 1 sweeps between swap events */
    /* SQA move (sqa_move; 0 = METROPOLIS).  WOLFF needs L <= 128. */
    int32_t move;
} sqa_desc;

typedef struct sqa_handle sqa_handle;

/* Sizes of a created handle. */
typedef struct {
    int32_t n_phys;        /* canonical physical sites (readout row length) */
    int32_t n_used;        /* sites the embedding uses */
    int32_t n_terms;       /* physical terms (couplers, fields, constraints) */
    int32_t z;             /* L for SQA, P for PT */
    int32_t words;         /* W = ceil(R / 32) */
    int32_t delta_min, delta_max; /* range of single-flip energy changes */
    int64_t attempts_per_sweep;   /* I * n_used * Z * R */
    int64_t device_bytes;  /* device memory held by the handle */
    int64_t h2d_bytes;     /* bytes sqa_create copied host -> device */
    int32_t launches_per_run; /* kernel launches of one sqa_run */
    int32_t pad_;
} sqa_info;

/* Builds the embedding (Sec. II A/B), the acceptance tables (uint32
 * thresholds floor(2^32 e^-x), computed on the host in double) and the
 * device state; draws the initial spins.  Synchronous.  On error *out is
 * NULL. */
sqa_status sqa_create(const sqa_desc *desc, sqa_handle **out);
/* Waits for the device, then frees everything the handle holds (a library
 * service, as are the info, tuning and error calls).  NULL is a no-op. */
void sqa_destroy(sqa_handle *h);
/* Sizes of a created handle into *out (caller-owned). */
sqa_status sqa_get_info(const sqa_handle *h, sqa_info *out);

/* Launch shape of the sweep kernel (the autotuner's knobs; results do not
 * depend on them).  words_per_unit: 32-replica words one unit holds
 * (0 = automatic).  use_table: SQA threshold lookup through per-site code
 * tables (1), byte-wise index windows (0), or automatic (-1); PT always uses
 * windows.  cluster: blocks per unit, 1, 2, 4, 8 or 16 (0 = automatic); with
 * C > 1 a thread-block cluster sweeps one unit, each block holding Z/C
 * consecutive slices (SQA, C must divide L/2) or slots (PT, C must divide
 * P).  Fails with SQA_ERR_UNSUPPORTED, leaving the shape unchanged, when the
 * request does not fit.  Synchronizes the device. */
sqa_status sqa_tune(sqa_handle *h, int32_t words_per_unit, int32_t use_table, int32_t cluster);
sqa_status sqa_get_launch(const sqa_handle *h, int32_t *words_per_unit, int32_t *use_table,
                          int32_t *smem_bytes, int32_t *cluster);
/* Slices per thread of the single-spin sweep (another autotuner knob; results
 * do not depend on it): each thread's task covers 1..4 consecutive slices
 * (SQA: slices of one parity) or slots of one (site, word), so that the site's
 * record and the word's hoisted random values are read once for several
 * items.  0 (the default) lets the kernel choose per colour phase the count
 * whose longest thread runs the fewest items.  slices outside 0..4 ->
 * SQA_ERR_INVALID.  Takes effect at the next launch; the cluster moves ignore
 * it. */
sqa_status sqa_tune_slices(sqa_handle *h, int32_t slices);
sqa_status sqa_get_task_slices(const sqa_handle *h, int32_t *slices);

/* Runs the whole program: fresh initial spins, then sweeps 0..S-1 (SQA
 * anneal: Metropolis on the Trotterised H(t) of Eq. 3, App. B, Sec. III; or
 * PT with swaps every swap_every sweeps: App. B, Eq. 9), as one persistent
 * launch over all instances.  Asynchronous on stream; a launch error is
 * returned as SQA_ERR_CUDA. */
sqa_status sqa_run(sqa_handle *h, void *stream);

/* Sweeps t0..t1-1 of the same program (Eq. 3, App. B) continuing from the
 * current state (t0 == 0 draws fresh initial spins first).  Runs split at
 * any t give the same bits as one run (checkpoint/resume).  t outside
 * 0 <= t0 <= t1 <= S -> SQA_ERR_INVALID. */
sqa_status sqa_run_sweeps(sqa_handle *h, int32_t t0, int32_t t1, void *stream);

/* The plain path kept for comparison: the same sweeps as sqa_run, but one
 * kernel launch per instance, in sequence on stream.  Same bits. */
sqa_status sqa_run_per_instance(sqa_handle *h, void *stream);

/* Parallel tempering on the handle's problem (App. B): switches the handle to
 * PT with the given ladder (betas strictly decreasing, coldest first), draws
 * fresh spins and runs n_sweeps sweeps with swaps every swap_every sweeps.
 * Synchronises stream, then replaces the handle's device program; when the
 * new one cannot be set up (SQA_ERR_UNSUPPORTED: couplings and penalty too
 * large for PT's byte-wise windows; SQA_ERR_NOMEM) the handle is left with
 * none, and every later call on it but sqa_destroy returns SQA_ERR_INVALID. */
sqa_status pt_run(sqa_handle *h, const double *betas, int32_t n_temps, int32_t n_sweeps,
                  int32_t swap_every, void *stream);

/* One persistent launch over the units of several handles of any shapes
 * (ragged batching); each handle runs its whole program as in sqa_run
 * (Eq. 3 / App. B, Eq. 9), with the same bits.  hs: n caller-owned handles. */
sqa_status sqa_batch_run(sqa_handle *const *hs, int32_t n, void *stream);

/* Readout of the final state (App. B: one Trotter slice, here slice 0; PT:
 * the coldest slot): out [I][n_phys][W] uint32, bit b of word w = replica
 * 32w + b, 1 <-> sigma = -1, canonical site order; out is caller-owned,
 * host (synchronous) or device (out_is_device, asynchronous on stream). */
sqa_status sqa_readout(sqa_handle *h, uint32_t *out, int32_t out_is_device, void *stream);
/* Whole state, every slice or slot; out [I][Z][n_phys][W] as sqa_readout. */
sqa_status sqa_state(sqa_handle *h, uint32_t *out, int32_t out_is_device, void *stream);
/* Physical energy E_P (Eq. 1 through the embedding; Eq. 2 for LHZ) of every
 * slice/slot and replica; out [I][Z][R] int32, as sqa_readout. */
sqa_status sqa_energies(sqa_handle *h, int32_t *out, int32_t out_is_device, void *stream);

/* Decodes the readout of every replica to a logical state and its logical
 * energy (Eq. 1).  method: sqa_decode_method (ME handles take ME_MV, LHZ
 * handles the LHZ methods).  n_trees: votes for LHZ_TREES (odd; 0 ->
 * ceil(N/4)+1 made odd).  logical_out [I][R][N] int8 (+-1; LHZ fixes
 * logical spin 0 to +1), energy_out [I][R].  If e_ground (host, [I]) is not
 * NULL, success_out [I] counts replicas whose decoded energy equals it.
 * Any output may be NULL. */
sqa_status sqa_decode(sqa_handle *h, int32_t method, int32_t n_trees, int8_t *logical_out,
                      int64_t *energy_out, const int64_t *e_ground, int32_t *success_out,
                      int32_t out_is_device, void *stream);

/* Exact logical ground-state energies of Eq. 1 (h = 0; success means
 * reaching it, Sec. III) by exhaustive search over the 2^(N-1) states with
 * s_{N-1} = +1, on the GPU.  J host [I][N(N-1)/2]; e_out host [I].  N <= 40.
 * One call enumerates at most 2^40 states in all: I * 2^(N-1) > 2^40 (e.g.
 * N = 40 with I > 2, N = 32 with I > 512) -> SQA_ERR_UNSUPPORTED, so that no
 * call holds the device for more than a few seconds.  Synchronous. */
sqa_status sqa_ground_energy(int32_t N, int32_t n_instances, const int32_t *J, int64_t *e_out);

/* Exhaustive ground-state energies for callers that cannot allocate device
 * memory (e.g. a serving process that reserved its whole device budget up
 * front, or code under a memory manager that forbids ad-hoc cudaMalloc).  The
 * paper has no counterpart: this is a service entry point of the library.
 * Same search and result as sqa_ground_energy, but J_dev ([I][N(N-1)/2]
 * int32) and e_dev ([I] int64) are caller-owned device buffers, the call is
 * asynchronous on stream, and nothing is allocated: the per-instance running
 * minima live in a fixed device array of 4096 entries (32 KiB held on every
 * device that loads the library, until exit).  I > 4096 or N outside 2..40
 * -> SQA_ERR_INVALID; I * 2^(N-1) > 2^40 -> SQA_ERR_UNSUPPORTED (the same
 * work bound as sqa_ground_energy).  J_dev and e_dev must be device (or
 * managed) memory of the current device, checked with
 * cudaPointerGetAttributes (SQA_ERR_INVALID otherwise); their lengths cannot
 * be checked from raw pointers and are the caller's to get right.  The first
 * call on a device looks up that array's address (cudaGetSymbolAddress) and
 * caches it with the current CUDA context; a call that finds another context
 * current (after cudaDeviceReset, say) looks it up again.  Make the first
 * call on a device, and the first after a reset, before any stream capture.
 * All calls share the array and reset it at the start, so calls that overlap
 * on the GPU race with each other; calls queued one after another on one
 * stream do not. */
sqa_status sqa_ground_energy_noalloc(int32_t N, int32_t n_instances, const int32_t *J_dev,
                                     int64_t *e_dev, void *stream);

/* Belief-propagation decoding of an LHZ handle's readouts (Sec. IV, App. C):
 * pair values start at the readout's pair spins s and are updated
 * `iterations` times, all pairs at once, p_ij <- sign(L0 s_ij + L2 sum_l
 * p_il p_lj) over the N-2 third spins l (ties keep p_ij), with
 * L0 = ln((1-e)/e) and L2 = ln(((1-e)^2 + e^2) / (2 e (1-e))) for error rate
 * e in (0, 1/2]; random tree 0 of the instance then reads the logical
 * state.  N <= 32.  Outputs and streams as sqa_decode. */
sqa_status sqa_decode_bp(sqa_handle *h, double error_rate, int32_t iterations, int8_t *logical_out,
                         int64_t *energy_out, const int64_t *e_ground, int32_t *success_out,
                         int32_t out_is_device, void *stream);

/* ---- reusable batches (CUDA graph) and the launch-shape autotuner ---- */

typedef struct sqa_batch sqa_batch;
/* Batches, the autotuner and the server are library services: the paper's
 * instances and runs are independent jobs, and these only schedule them
 * (each job's results are those of sqa_run).
 *
 * Plans the handles (SQA or PT, any sizes) once for one persistent launch of
 * the multi-job sweep kernel: every job's units in one list, longest first.
 * The handles must outlive the batch and must not be tuned, switched to PT
 * (pt_run) or destroyed while it exists. */
sqa_status sqa_batch_create(sqa_handle *const *hs, int32_t n, sqa_batch **out);
/* Asynchronous on stream: fresh initial spins for every job, then all their
 * sweeps.  The first call captures this sequence into a CUDA graph; every
 * call replays the graph (the same anneal, bit for bit, as sqa_batch_run). */
sqa_status sqa_batch_launch(sqa_batch *b, void *stream);
/* Times the batch with 0 (the planner's words per unit for each job) and
 * 1, 2, 4, ... words per unit for every job (each job takes the largest of
 * W, ceil(W/2), ... not above it), n_trial sweeps each, keeps the fastest,
 * then with it times slices per task 0 (each job's own setting) and 1..4 for
 * every job (see sqa_tune_slices), then the SQA threshold lookup of every
 * job (its own plan, code tables, byte windows; a job that a form does not
 * fit keeps its own), keeping the fastest at each step.  Synchronous; leaves the handles' spins at the end of a trial (a
 * launch starts from fresh initial spins).  words_per_unit and
 * attempts_per_s (either may be NULL) receive the choice and its trial
 * rate. */
sqa_status sqa_batch_autotune(sqa_batch *b, int32_t n_trial, void *stream, int32_t *words_per_unit,
                              double *attempts_per_s);
/* Waits for the device (a replay may still be in flight on any stream) and
 * frees the batch; the handles stay the caller's.  NULL is a no-op. */
void sqa_batch_destroy(sqa_batch *b);
/* Times h's sweep kernel in every launch shape that fits (cluster size 1, 2,
 * 4, 8, 16; table or window lookup; words per unit W, ceil(W/2), ..., 1) on
 * n_trial sweeps from sweep 0 and keeps the fastest (as sqa_tune), then with
 * that shape slices per task 0..4 (as sqa_tune_slices; not for cluster
 * moves).  h's
 * spins are saved and restored.  Synchronous; the out pointers (may be
 * NULL) receive the choice and its trial rate in attempts/s. */
sqa_status sqa_autotune(sqa_handle *h, int32_t n_trial, void *stream, int32_t *words_per_unit,
                        int32_t *use_table, int32_t *cluster, double *attempts_per_s);

/* ---- serving: continuous batching of SQA and PT jobs ---- */

typedef struct sqa_server sqa_server;
typedef enum { SQA_JOB_QUEUED = 0, SQA_JOB_RUNNING = 1, SQA_JOB_DONE = 2, SQA_JOB_FAILED = 3 } sqa_job_state;
typedef struct {
    int32_t state;         /* sqa_job_state */
    int32_t status;        /* sqa_status of a failed job */
    double t_submit, t_start, t_done; /* seconds on the server's clock */
    int64_t device_bytes;  /* device memory the job held while resident */
} sqa_job_info;
typedef struct {
    int64_t jobs_submitted, jobs_done, jobs_failed, chunks, attempts;
    int64_t resident, queued, max_resident, bytes_in_use, max_bytes;
    /* worker wall time: admitting jobs, launching chunks and retiring jobs,
     * waiting for the GPU */
    double admit_s, advance_s, idle_s;
    int32_t worker_status, pad_;
    /* packed launches of small jobs' chunks (multi-job kernels), and the
     * worker time spent building and launching them and retiring jobs (parts
     * of advance_s) */
    int64_t packs;
    double pack_s, retire_s;
    double create_s;  /* part of admit_s: creating handles (planning, tables, uploads) */
    double pad2_;
} sqa_server_stats;

/* A server owns a worker thread that serves jobs on the current device.  It
 * admits queued jobs in arrival order while their device memory fits
 * mem_budget_bytes (a job larger than the budget fails with SQA_ERR_NOMEM)
 * and runs each resident job as a chain of chunks of its sweeps, about
 * unit_attempts_per_chunk attempts per work unit each (0 picks 1e7).  Jobs
 * whose work units fit one block each are packed: whenever jobs are ready for
 * their next chunk, the chunks of all of them on one path (PT, SQA tables,
 * SQA windows, ...) go into one launch of that path's multi-job kernel, and
 * several packs run at once on different streams; jobs that need thread-block
 * clusters run their chunks as launches of their own sweep kernel on
 * higher-priority streams.  Admission never waits on the GPU: a job's tables
 * are uploaded from pinned memory on a stream of their own and its initial
 * spins are drawn just before its first chunk.  A finished job's energies and
 * state are copied to pinned host memory behind its final chunk, and the job
 * is retired (results kept on the host, device memory freed in stream order)
 * once those copies have landed.  Results are
 * bit-identical to sqa_run of the same descriptor, whatever else was
 * resident.  The server keeps up to mem_budget_bytes of freed memory in the
 * device's default stream-ordered memory pool for reuse. */
sqa_status sqa_server_create(int64_t mem_budget_bytes, int64_t unit_attempts_per_chunk, sqa_server **out);
/* Copies desc (kind SQA or PT) and queues it; thread-safe. */
sqa_status sqa_server_submit(sqa_server *s, const sqa_desc *desc, uint64_t *job_id);
sqa_status sqa_server_poll(sqa_server *s, uint64_t job_id, sqa_job_info *info);
/* Blocks until the job is done or failed; SQA_ERR_TIMEOUT after timeout_s. */
sqa_status sqa_server_wait(sqa_server *s, uint64_t job_id, double timeout_s);
/* Host outputs of a done job: state [I][Z][n_phys][W], energies [I][Z][R]
 * (either may be NULL).  SQA_ERR_BUSY while the job is pending. */
sqa_status sqa_server_result(sqa_server *s, uint64_t job_id, uint32_t *state_out, int32_t *energies_out);
/* Forgets a done or failed job. */
sqa_status sqa_server_release(sqa_server *s, uint64_t job_id);
sqa_status sqa_server_get_stats(sqa_server *s, sqa_server_stats *out);
/* Stops the worker, waits for the chunks in flight and frees every job. */
void sqa_server_destroy(sqa_server *s);

/* ---- host-only views of the library's planning (no device needed) ---- */

/* The physical problem the library builds for one instance (Sec. II A/B):
 * terms w * prod(sigma) in canonical site numbering.  term_mem is
 * [cap_terms][4] (-1 pads), colour [n_phys] (-1 for unused sites).  J is
 * [N(N-1)/2].  Fails with SQA_ERR_INVALID if cap_terms is too small. */
sqa_status sqa_plan_terms(int32_t embedding, int32_t N, const int32_t *J, int32_t penalty,
                          int32_t cap_terms, int32_t *n_phys, int32_t *n_terms,
                          int32_t *term_size, int32_t *term_mem, int32_t *term_w,
                          int32_t *colour);

/* Device bytes sqa_create allocates for desc (the admission estimate of the
 * serving loop): exact except the work-unit list, counted as one unit per
 * 32-replica word, so an upper bound.  Host only; 0 on an invalid desc. */
int64_t sqa_plan_device_bytes(const sqa_desc *desc);

/* The acceptance thresholds (Eq. 3, App. B) sqa_create would upload for desc: SQA
 * [S][nd][3] indexed by ((delta - dmin)/2, (m + 2)/2), PT [P][nd] indexed
 * by (delta - dmin)/2, nd = (dmax - dmin)/2 + 1.  cap is the length of T. */
sqa_status sqa_plan_tables(const sqa_desc *desc, uint32_t *T, int64_t cap, int32_t *dmin,
                           int32_t *dmax);

/* The cluster-move tables (Sec. III, Sec. V) sqa_create would upload for an
 * SQA desc with move = SQA_MOVE_WOLFF: Tb [S] bond thresholds; acc_off, acc_len [S] and
 * Tacc (cap entries) the acceptance thresholds T(alpha_t D) of sweep t for
 * D = 2, 4, ..., 2 acc_len[t] at Tacc[acc_off[t] + D/2 - 1]; *n_acc gets the
 * total.  Any output may be NULL to query sizes. */
sqa_status sqa_plan_wolff_tables(const sqa_desc *desc, uint32_t *Tb, int32_t *acc_off, int32_t *acc_len,
                                 uint32_t *Tacc, int64_t cap, int64_t *n_acc);

/* PT swap thresholds of slots (pair, pair+1) (Eq. 9): out[dE-1] for
 * dE = 1..*len, zero beyond. */
sqa_status sqa_plan_swap_table(const double *betas, int32_t n_temps, int32_t pair, uint32_t *out,
                               int32_t cap, int32_t *len);

/* The random spanning tree (App. A) number `tree` of instance `inst` used
 * by SQA_DECODE_LHZ_TREES: parent[v], parent[0] = -1. */
sqa_status sqa_plan_tree(int32_t N, uint64_t seed, int32_t inst, int32_t tree, int32_t *parent);

/* Diagnostic for the roofline (no paper counterpart): sustained integer
 * instructions per SM clock (all lanes) of one
 * instruction kind on the current device, from a dependency-free
 * microbenchmark timed with the SM clock counter.  kind: 0 LOP3, 1 IADD3,
 * 2 IMAD, 3 IMAD.WIDE, 4 IMAD.HI, 5 LOP3/IMAD alternating, 6 Philox4x32-10
 * blocks (result in blocks, not instructions), 7 the same with one
 * 32x32->64 multiply per product.  Synchronous. */
sqa_status sqa_int_peak(int32_t kind, double *lane_ops_per_clk_per_sm);

/* Bounds-checked builds (no paper counterpart; a debugging aid).  A build
 * compiled with -DSQA_BOUNDS_CHECK tests, before each access of the sweep,
 * energy and decode kernels, every shared-memory address against the
 * block's dynamic window and every state, threshold-row, tie-array,
 * tie-list, PT swap and cluster-move ring index against its buffer.  An
 * access out of range is skipped (a load reads 0) and recorded in a device
 * status word; no kernel traps, so the context stays usable.
 * sqa_bounds_checked() returns 1 in such a build, 0 otherwise.
 * sqa_check_status() synchronises the device, copies the record into
 * record[4] and clears it: record[0] = violations since the last call,
 * record[1] = the check site of the first (1 shared memory, 2 state word,
 * 3 threshold row, 4 tie array, 5 tie list, 6 decoded tie item, 7 a
 * neighbouring block's slice, 8 PT swap, 9 cluster-move ring), record[2] =
 * its index (for shared memory: its shared-window byte address),
 * record[3] = the bound it broke.  Returns SQA_OK when nothing was
 * recorded, SQA_ERR_BOUNDS otherwise (detail in sqa_last_error()); in an
 * unchecked build SQA_OK with a zero record.  record NULL -> SQA_ERR_INVALID. */
int32_t sqa_bounds_checked(void);
sqa_status sqa_check_status(uint32_t record[4]);

const char *sqa_strerror(sqa_status s);
/* Detail of the last error on this thread (CUDA message, bad field). */
const char *sqa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
