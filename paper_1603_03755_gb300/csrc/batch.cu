// Reusable ragged batches replayed from a CUDA graph, and the launch-shape
// autotuner (for one handle and for a batch).
//
// A batch fixes a set of handles (SQA or PT jobs of any sizes) and plans
// them once for the multi-job persistent kernels: every job's units (one
// instance's run of words) in one list, grouped by the job's path (PT, SQA
// windows, SQA tables, ...) and longest first within a path.  Its first
// launch captures, on a private stream, the initial-spin kernel of every job,
// the reset of the work counters and one persistent sweep launch per path
// into a CUDA graph; every launch replays that graph on the caller's stream.  An anneal
// always starts from its initial spins, so a replay repeats the same anneal
// bit for bit.
//
// The autotuner times candidate launch shapes on a short trial and keeps the
// fastest.  Results never depend on the launch shape (every random number is
// keyed by sweep, site, slice, replica and instance), so tuning changes speed
// only.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "handle.h"
#include "layout.cuh"

using namespace sqa;

#define SQA_TRY(call)                                       \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

struct sqa_batch {
    std::vector<sqa_handle *> hs;
    int policy = 0;  // words per unit for every job (0: the planner's choice per job)
    int slices = 0;  // slices per task for every job (0: each job's own setting)
    int lookup = -1; // SQA threshold lookup for every job: 1 tables, 0 windows, -1 each job's own plan
    std::vector<JobDev> jobs;
    std::vector<Unit> units;
    std::vector<MultiGroup> groups;  // one persistent launch per path
    JobDev *d_jobs = nullptr;
    Unit *d_units = nullptr;
    int *d_counter = nullptr;
    uint2 *d_tieq = nullptr;  // tie queue of the persistent blocks (JobDev::tieq)
    size_t cap_jobs = 0, cap_units = 0, cap_tieq = 0;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void drop_graph(sqa_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// Plans every job for one block per unit with the batch's words-per-unit
// policy, sweeps [0, min(trial, S)) (trial 0: all), and uploads the lists.
sqa_status plan_batch(sqa_batch *b, int trial)
{
    b->jobs.clear();
    b->units.clear();
    for (size_t k = 0; k < b->hs.size(); k++) {
        sqa_handle *h = b->hs[k];
        JobDev J;
        std::vector<Unit> ju;
        // the job's own words per unit: the largest of W, ceil(W/2), ... <= policy
        int f = 0;
        if (b->policy > 0) {
            f = h->job.W;
            while (f > b->policy && f > 1) f = (f + 1) / 2;
        }
        const int keep_mode = h->force_mode;
        if (b->lookup >= 0 && h->kind == SQA_KIND_SQA && !(b->lookup == 0 && h->window_limit_exceeded))
            h->force_mode = b->lookup;
        sqa_status st = plan_job(h, 1, f, J, ju);
        if (st != SQA_OK && h->force_mode != keep_mode) {  // that lookup does not fit this job: its own plan
            h->force_mode = keep_mode;
            st = plan_job(h, 1, f, J, ju);
        }
        h->force_mode = keep_mode;
        if (st != SQA_OK) return st;
        J.t0 = 0;
        J.t1 = trial > 0 ? std::min(trial, h->S) : h->S;
        if (b->slices > 0) J.task_slices = b->slices;
        b->jobs.push_back(J);
        for (Unit u : ju) {
            u.job = (int)k;
            b->units.push_back(u);
        }
    }
    const int rows = group_units(b->jobs, b->units, b->groups);
    if (b->jobs.size() > b->cap_jobs) {
        if (b->d_jobs) cudaFree(b->d_jobs);
        b->d_jobs = nullptr;
        SQA_TRY(cudaMalloc((void **)&b->d_jobs, b->jobs.size() * sizeof(JobDev)));
        b->cap_jobs = b->jobs.size();
    }
    if (b->units.size() > b->cap_units) {
        if (b->d_units) cudaFree(b->d_units);
        b->d_units = nullptr;
        SQA_TRY(cudaMalloc((void **)&b->d_units, b->units.size() * sizeof(Unit)));
        b->cap_units = b->units.size();
    }
    // one tie queue for the persistent blocks of every path's launch: a row
    // of the largest phase of any job per block
    int stride = 1;
    for (const JobDev &J : b->jobs) stride = std::max(stride, tie_items(J, J.wc));
    const size_t need = (size_t)rows * (size_t)stride;
    if (need > b->cap_tieq) {
        if (b->d_tieq) cudaFree(b->d_tieq);
        b->d_tieq = nullptr;
        b->cap_tieq = 0;
        SQA_TRY(cudaMalloc((void **)&b->d_tieq, need * sizeof(uint2)));
        b->cap_tieq = need;
    }
    assign_tieq(b->jobs, b->groups, b->d_tieq, stride);
    SQA_TRY(cudaMemcpy(b->d_jobs, b->jobs.data(), b->jobs.size() * sizeof(JobDev), cudaMemcpyHostToDevice));
    SQA_TRY(cudaMemcpy(b->d_units, b->units.data(), b->units.size() * sizeof(Unit), cudaMemcpyHostToDevice));
    drop_graph(b);
    return SQA_OK;
}

// Initial spins of every job, then one persistent sweep launch per path, on s.
sqa_status launch_plain(sqa_batch *b, cudaStream_t s)
{
    sqa_status st;
    for (sqa_handle *h : b->hs)
        if ((st = launch_init(h, s)) != SQA_OK) return st;
    SQA_TRY(launch_groups(b->groups, b->d_jobs, b->d_units, b->d_counter, s));
    return SQA_OK;
}

sqa_status build_graph(sqa_batch *b)
{
    cudaStream_t cs = nullptr;
    SQA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    sqa_status st = e == cudaSuccess ? launch_plain(b, cs) : cuda_fail(e, "cudaStreamBeginCapture");
    if (e == cudaSuccess) {
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (st == SQA_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
    }
    if (st == SQA_OK) {
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            st = cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return st;
}

int64_t batch_attempts(const sqa_batch *b)
{
    int64_t a = 0;
    for (size_t k = 0; k < b->hs.size(); k++) {
        const JobDev &J = b->jobs[k];
        a += (int64_t)J.n * J.Z * b->hs[k]->R * b->hs[k]->I * (J.t1 - J.t0);
    }
    return a;
}

// Seconds of fn() on s, timed with events after one untimed run.
template <class F>
sqa_status time_on(cudaStream_t s, F fn, double *sec)
{
    sqa_status st = fn();
    if (st != SQA_OK) return st;
    cudaEvent_t e0, e1;
    SQA_TRY(cudaEventCreate(&e0));
    const cudaError_t ec = cudaEventCreate(&e1);
    if (ec != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ec, "cudaEventCreate");
    }
    cudaEventRecord(e0, s);
    st = fn();
    cudaEventRecord(e1, s);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (st == SQA_OK && e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SQA_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "autotune trial");
    *sec = ms * 1e-3;
    return SQA_OK;
}

}  // namespace

extern "C" {

sqa_status sqa_batch_create(sqa_handle *const *hs, int32_t n, sqa_batch **out)
{
    NvtxScope nvtx_("sqa_batch_create");
    if (!hs || n < 1 || !out) return set_error("batch arguments"), SQA_ERR_INVALID;
    *out = nullptr;
    for (int k = 0; k < n; k++) {
        const sqa_status us = usable(hs[k]);
        if (us != SQA_OK) return us;
    }
    sqa_batch *b = new (std::nothrow) sqa_batch();
    if (!b) return SQA_ERR_NOMEM;
    b->hs.assign(hs, hs + n);
    cudaError_t e = cudaMalloc((void **)&b->d_counter, kMaxModes * sizeof(int));
    sqa_status st = e == cudaSuccess ? plan_batch(b, 0) : cuda_fail(e, "sqa_batch_create");
    if (st != SQA_OK) {
        sqa_batch_destroy(b);
        return st;
    }
    *out = b;
    return SQA_OK;
}

sqa_status sqa_batch_launch(sqa_batch *b, void *stream)
{
    NvtxScope nvtx_("sqa_batch_launch");
    if (!b) return set_error("NULL batch"), SQA_ERR_INVALID;
    if (!b->exec) {
        const sqa_status st = build_graph(b);
        if (st != SQA_OK) return st;
    }
    SQA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return SQA_OK;
}

sqa_status sqa_batch_autotune(sqa_batch *b, int32_t n_trial, void *stream, int32_t *words_per_unit,
                              double *attempts_per_s)
{
    NvtxScope nvtx_("sqa_batch_autotune");
    if (!b || n_trial < 1) return set_error("autotune arguments"), SQA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int wmax = 1;
    for (sqa_handle *h : b->hs) wmax = std::max(wmax, h->job.W);
    const int keep = b->policy;
    int best = -1;
    double best_t = 0, best_rate = 0;
    for (int pol : {0, 1, 2, 4, 8, 16, 32}) {
        if (pol > wmax) break;
        b->policy = pol;
        if (plan_batch(b, n_trial) != SQA_OK) continue;
        double t = 0;
        const sqa_status st = time_on(s, [&] { return launch_plain(b, s); }, &t);
        if (st != SQA_OK) {
            b->policy = keep;
            plan_batch(b, 0);
            return st;
        }
        if (best < 0 || t < best_t) {
            best = pol;
            best_t = t;
            best_rate = (double)batch_attempts(b) / t;
        }
    }
    b->policy = best < 0 ? keep : best;
    // then slices per task, with that policy (0: each job's own setting)
    const int keep_slices = b->slices;
    int best_s = keep_slices;
    if (best >= 0)
        for (int sl = 0; sl <= kTaskSlices; sl++) {
            b->slices = sl;
            if (plan_batch(b, n_trial) != SQA_OK) continue;
            double t = 0;
            const sqa_status st = time_on(s, [&] { return launch_plain(b, s); }, &t);
            if (st != SQA_OK) {
                b->slices = keep_slices;
                plan_batch(b, 0);
                return st;
            }
            if (t < best_t) {
                best_t = t;
                best_s = sl;
                best_rate = (double)batch_attempts(b) / t;
            }
        }
    b->slices = best_s;
    // then the SQA threshold lookup for every job (tables or windows; -1 each
    // job's own plan), with those settings
    const int keep_lookup = b->lookup;
    int best_l = keep_lookup;
    if (best >= 0)
        for (int lk : {-1, 1, 0}) {
            b->lookup = lk;
            if (plan_batch(b, n_trial) != SQA_OK) continue;
            double t = 0;
            const sqa_status st = time_on(s, [&] { return launch_plain(b, s); }, &t);
            if (st != SQA_OK) {
                b->lookup = keep_lookup;
                plan_batch(b, 0);
                return st;
            }
            if (t < best_t) {
                best_t = t;
                best_l = lk;
                best_rate = (double)batch_attempts(b) / t;
            }
        }
    b->lookup = best_l;
    const sqa_status st = plan_batch(b, 0);
    if (st != SQA_OK) return st;
    if (words_per_unit) *words_per_unit = b->policy;
    if (attempts_per_s) *attempts_per_s = best_rate;
    return SQA_OK;
}

void sqa_batch_destroy(sqa_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    drop_graph(b);
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_units) cudaFree(b->d_units);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_tieq) cudaFree(b->d_tieq);
    delete b;
}

sqa_status sqa_autotune(sqa_handle *h, int32_t n_trial, void *stream, int32_t *words_per_unit,
                        int32_t *use_table, int32_t *cluster, double *attempts_per_s)
{
    NvtxScope nvtx_("sqa_autotune");
    const sqa_status us = usable(h);
    if (us != SQA_OK) return us;
    if (n_trial < 1) return set_error("autotune arguments"), SQA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const int trial = std::min<int>(n_trial, h->S);
    const size_t bytes = (size_t)h->I * h->job.Z * h->job.n * h->job.W * sizeof(uint32_t);
    uint32_t *saved = nullptr;
    SQA_TRY(cudaMallocAsync((void **)&saved, bytes, s));
    const cudaError_t ecp = cudaMemcpyAsync(saved, h->d_state, bytes, cudaMemcpyDeviceToDevice, s);
    if (ecp != cudaSuccess) {
        cudaFreeAsync(saved, s);
        return cuda_fail(ecp, "sqa_autotune save");
    }
    const int keep_wc = h->force_wc, keep_mode = h->force_mode, keep_c = h->force_cluster, keep_s = h->force_slices;
    const int64_t attempts = (int64_t)h->job.n * h->job.Z * h->R * h->I * trial;
    struct Choice {
        int wc, lut, C;
        double t;
    } best{0, -1, 0, -1};
    sqa_status st = SQA_OK;
    for (int C = 1; C <= 16 && st == SQA_OK; C *= 2)
        for (int lut : {1, 0}) {
            if (h->kind == SQA_KIND_PT && lut == 0) continue;  // PT has one lookup form
            const int mode = h->kind == SQA_KIND_PT ? -1 : lut;
            for (int wc = h->job.W; wc >= 1; wc = wc > 1 ? (wc + 1) / 2 : 0) {
                if (sqa_tune(h, wc, mode, C) == SQA_OK) {
                    double t = 0;
                    st = time_on(s, [&] { return run_sweeps(h, 0, trial, s); }, &t);
                    if (st != SQA_OK) break;
                    if (best.t < 0 || t < best.t) best = Choice{wc, mode, C, t};
                }
                if (wc == 1) break;
            }
            if (st != SQA_OK) break;
        }
    sqa_status rs = best.t > 0 ? sqa_tune(h, best.wc, best.lut, best.C) : sqa_tune(h, keep_wc, keep_mode, keep_c);
    // then slices per task with the chosen shape (0: the kernel's own choice)
    int best_s = keep_s;
    if (rs == SQA_OK && st == SQA_OK && best.t > 0 && h->move != SQA_MOVE_WOLFF)
        for (int sl = 0; sl <= kTaskSlices && st == SQA_OK; sl++) {
            sqa_tune_slices(h, sl);
            double t = 0;
            st = time_on(s, [&] { return run_sweeps(h, 0, trial, s); }, &t);
            if (st == SQA_OK && t < best.t) {
                best.t = t;
                best_s = sl;
            }
        }
    if (rs == SQA_OK) sqa_tune_slices(h, best_s);
    cudaMemcpyAsync(h->d_state, saved, bytes, cudaMemcpyDeviceToDevice, s);
    cudaFreeAsync(saved, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (st != SQA_OK) return st;
    if (rs != SQA_OK) return rs;
    if (e != cudaSuccess) return cuda_fail(e, "sqa_autotune");
    if (best.t <= 0) return set_error("no launch shape fits"), SQA_ERR_UNSUPPORTED;
    if (words_per_unit) *words_per_unit = h->job.wc;
    if (use_table) *use_table = h->job.use_lut;
    if (cluster) *cluster = h->job.csize;
    if (attempts_per_s) *attempts_per_s = (double)attempts / best.t;
    return SQA_OK;
}

}  // extern "C"
