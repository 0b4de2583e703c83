// The handle behind the C ABI's opaque sqa_handle, and the internal entry
// points shared by the C ABI (capi.cu) and the serving loop (server.cu).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "sqa_internal.h"

// A named NVTX range over a scope, so that a profiler's host timeline shows
// the library's calls (create, run, decode, batch launches, serving chunks);
// with no profiler attached a push and a pop cost a few nanoseconds.
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

struct sqa_handle {
    // copied description
    int kind = 0, emb = 0, N = 0, I = 0, penalty = 0, S = 0, R = 0, L = 0, P = 0, swap_every = 1;
    int move = 0;  // SQA: sqa_move
    uint64_t seed = 0;
    double beta = 0;
    std::vector<int32_t> J;
    std::vector<double> A, B, betas;
    sqa::Plan plan;
    int smax = 0, dmin = 0, dmax = 0, nd = 0;
    bool window_limit_exceeded = false;
    int force_wc = 0, force_mode = -1, force_cluster = 0;  // sqa_tune overrides (0 / -1: automatic)
    int force_slices = 0;  // sqa_tune_slices override (0: automatic)
    // device
    sqa::JobDev job{};
    uint32_t *d_state = nullptr;
    sqa::SiteRec *d_sites = nullptr;
    uint32_t *d_T = nullptr;
    sqa::ETerm *d_eterms = nullptr;
    sqa::EClass *d_ecls = nullptr;
    uint32_t *d_Tsw = nullptr;
    uint32_t *d_Tb = nullptr, *d_Tacc = nullptr;
    int *d_accoff = nullptr, *d_acclen = nullptr;
    int *d_swoff = nullptr, *d_swlen = nullptr;
    int *d_canon = nullptr, *d_compact = nullptr;
    int32_t *d_J = nullptr;
    int *d_chain = nullptr, *d_pair = nullptr;
    int *d_parents = nullptr, *d_orders = nullptr;
    int cur_trees = -1, cur_tree_kind = -1;
    sqa::JobDev *d_job = nullptr;
    sqa::Unit *d_units = nullptr;
    int n_units = 0;
    int *d_counter = nullptr;
    uint2 *d_tieq = nullptr;  // tie queue of the single-spin sweep (JobDev::tieq)
    size_t tieq_cap = 0;      // its entries
    std::vector<sqa::Unit> units;
    int64_t device_bytes = 0;
    int64_t h2d_bytes = 0;
    std::vector<void *> allocs;
    bool ready = false;  // a complete device program is resident (set by its setup)
    bool lazy_tieq = false;  // setup leaves the tie queue to ensure_tieq (served jobs)
    bool units_staged = false;  // d_units lies inside the setup's one upload (not freed alone)
    // served jobs: the setup's allocations and its one upload go on
    // setup_stream without a host wait; the upload's bytes wait in pending
    // until the server copies them to pinned memory and queues the copy to
    // pending_dst, then records setup_ev
    cudaStream_t setup_stream = nullptr;
    std::vector<unsigned char> pending;
    void *pending_dst = nullptr;
    cudaEvent_t setup_ev = nullptr;
};


namespace sqa {

constexpr int kThreads = 256;  // threads per block of every kernel here

sqa_status device_ready();
// SMs of the device (after device_ready).
int num_sms();
// SQA_OK when h holds a complete device program (else SQA_ERR_INVALID: NULL,
// or its last setup failed part way, e.g. a rejected pt_run).
sqa_status usable(const sqa_handle *h);
void set_error(const std::string &msg);
sqa_status cuda_fail(cudaError_t e, const char *where);
// Draws fresh initial spins for every instance of h on stream s.
sqa_status launch_init(sqa_handle *h, cudaStream_t s);
// Blocks for one launch of kernel over n_units units (at most one wave).
int grid_for(const void *kernel, int smem_bytes, int n_units, int threads = kThreads);
// The sweep kernels' paths (kernels.cu): 0 PT, 1 SQA windows, 2 SQA tables,
// 3 / 4 SQA cluster moves (L <= 64 / L <= 128), 5 SQA tables of two-spin
// terms, 6 PT of two-spin terms; each path has a single-job and a multi-job
// kernel, and its own block size.
constexpr int kMaxModes = 7;
int sweep_mode(const JobDev &J);
int sweep_mode_threads(int mode);
const void *sweep_one_entry_mode(int mode);
const void *sweep_multi_entry(int mode);
// One persistent launch of the multi-job kernel of a path over n_units units
// (each names its job in jobs), pulling units from *counter.
cudaError_t launch_sweep_multi(int mode, int grid, int smem, const JobDev *jobs, const Unit *units, int n_units,
                               int *counter, cudaStream_t s);
// The units of a mixed batch, one run per path: units[u0, u0 + n) run in one
// launch of that path's multi-job kernel with grid blocks of smem bytes.
// The launches run concurrently, so each has its own rows of the tie queue
// (JobDev::tieq), from row row0.
struct MultiGroup {
    int mode, u0, n, smem, grid, row0, threads;
};
// Sorts units by path (longest first within a path) into groups, sizes their
// launches and orders them by work; returns the tie-queue rows of all groups.
int group_units(const std::vector<JobDev> &jobs, std::vector<Unit> &units, std::vector<MultiGroup> &groups);
// Points every job's tie queue at its group's rows of d_tieq (stride entries a row).
void assign_tieq(std::vector<JobDev> &jobs, const std::vector<MultiGroup> &groups, uint2 *d_tieq, int stride);
// Zeroes the kMaxModes counters and launches every group on s: with fork,
// each on its own stream of this host thread's pool, all joined back into s
// (the groups run concurrently); otherwise one after another on s.
cudaError_t launch_groups(const std::vector<MultiGroup> &groups, const JobDev *d_jobs, const Unit *d_units,
                          int *d_counters, cudaStream_t s, bool fork = true);
// Device bytes sqa_create would allocate for desc (host-only estimate, exact
// for the state and tables).
int64_t estimate_device_bytes(const sqa_desc *d);
// Frees h in stream order on s, without a device-wide synchronization.
void destroy_on_stream(sqa_handle *h, cudaStream_t s);
// Blocks of a launch of a job's own sweep kernel over n_units units.
int launch_grid(const JobDev &J, int n_units);
// One launch of a job's own sweep kernel over all its units.
cudaError_t launch_job_sweeps(const JobDev &J, const Unit *units, int n_units, int *counter, cudaStream_t s);
// sqa_create; with init false nothing waits on the host: the initial spins
// are not drawn (the caller launches launch_init on its own stream before
// the first sweep), allocations are queued on setup_stream and the upload is
// left in h->pending for the caller to queue from pinned memory, so that
// creation never waits behind work already on a busy GPU.
// With init false the tie queue of the handle's own sweep kernel is not
// allocated either (a served job packed into multi-job launches never uses
// it; ensure_tieq allocates it before the handle's own first launch).
sqa_status create_handle(const sqa_desc *d, sqa_handle **out, bool init, cudaStream_t setup_stream);
sqa_status ensure_tieq(sqa_handle *h);
// Enqueues on s the energy of every (instance, slice or slot, replica) of h
// into dev_out (device, [I][Z][R] int32), as sqa_energies computes them.
cudaError_t enqueue_energies(const sqa_handle *h, int32_t *dev_out, cudaStream_t s);
// Plans h's launch (J, units) for the multi-job kernel of batches, with
// c_forced blocks per cluster (0: any) and force_wc words per unit (0: the
// planner's choice), without changing h.
sqa_status plan_job(sqa_handle *h, int c_forced, int force_wc, JobDev &J, std::vector<Unit> &units);
// Sweeps [t0, t1) of every unit of h with its current launch shape, on s.
sqa_status run_sweeps(sqa_handle *h, int t0, int t1, cudaStream_t s);

}  // namespace sqa
