// Serving loop: continuous batching of SQA and PT jobs on one GPU.
//
// Jobs are submitted from any host thread.  One worker thread owns the GPU
// work.  It admits queued jobs in arrival order while their device memory
// fits the budget (planning them on the host and uploading their resident
// state), gives each a stream from a pool, and keeps one chunk of each
// resident job's sweeps in flight: one launch of the job's own sweep kernel
// (its own launch shape, a thread-block cluster per unit when planned so)
// worth about `unit_attempts` attempts per unit.  When a chunk finishes the
// worker launches the job's next one, so the kernels of all resident jobs
// share the GPU, a job's blocks go back to the scheduler between chunks, and
// no job waits for another at a global barrier.  A finished job's state and
// energies are copied to the host and its memory is freed in stream order.
//
// A job's random numbers depend only on its own descriptor and sweep
// indices, so its result is the same whether it ran alone or among other
// jobs, and however its sweeps were cut into chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "handle.h"

using namespace sqa;

namespace {

constexpr int kPoolStreams = 64;

struct Job {
    uint64_t id = 0;
    sqa_desc desc{};
    std::vector<int32_t> J;
    std::vector<double> A, B, betas;
    sqa_job_info info{};
    sqa_handle *h = nullptr;
    int stream = -1;                // index into the stream pool
    int t_next = 0;                 // first sweep of the chunk in flight
    int t_chunk_end = 0;            // end of the chunk in flight
    cudaEvent_t done = nullptr;     // recorded after the chunk in flight
    std::vector<uint32_t> state;    // [I][Z][n_phys][W] once done
    std::vector<int32_t> energies;  // [I][Z][R] once done
};

double now_s(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct sqa_server {
    int64_t budget = 0;
    int64_t unit_target = 0;  // attempts per unit per chunk
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<uint64_t, Job *> jobs;
    std::deque<Job *> queue;
    std::vector<Job *> active;
    uint64_t next_id = 1;
    bool stop = false;
    int64_t used = 0;
    sqa_server_stats stats{};
    int device = 0;
    cudaStream_t pool[kPoolStreams] = {};
    int pool_load[kPoolStreams] = {};
    std::thread worker;
    sqa_status worker_status = SQA_OK;
};

namespace {

// Marks j failed with status st (caller holds s->mu).
void fail_job(sqa_server *s, Job *j, sqa_status st)
{
    j->info.state = SQA_JOB_FAILED;
    j->info.status = st;
    j->info.t_done = now_s(s->t0);
    s->stats.jobs_failed++;
    s->cv_done.notify_all();
}

// Launches the chunk of j's sweeps that starts at j->t_next, on j's stream
// (the caller counts it in the stats under s->mu).
sqa_status launch_chunk(sqa_server *s, Job *j)
{
    NvtxScope nvtx_("server_chunk");
    sqa_handle *h = j->h;
    JobDev J = h->job;
    const int64_t unit_attempts = (int64_t)J.n * J.zr * J.wc * 32;
    int64_t sweeps = std::max<int64_t>(1, s->unit_target / std::max<int64_t>(unit_attempts, 1));
    sweeps = std::min<int64_t>(sweeps, h->S - j->t_next);
    J.t0 = j->t_next;
    J.t1 = J.t0 + (int)sweeps;
    cudaStream_t st = s->pool[j->stream];
    cudaError_t e = launch_job_sweeps(J, h->d_units, h->n_units, h->d_counter, st);
    if (e == cudaSuccess) e = cudaEventRecord(j->done, st);
    if (e != cudaSuccess) return cuda_fail(e, "server chunk");
    j->t_chunk_end = J.t1;
    return SQA_OK;
}

// Releases j's device resources in stream order (caller holds s->mu).
void drop_device(sqa_server *s, Job *j)
{
    if (j->h) {
        s->used -= j->h->device_bytes;
        destroy_on_stream(j->h, s->pool[j->stream]);
        j->h = nullptr;
    }
    if (j->done) cudaEventDestroy(j->done);
    j->done = nullptr;
    if (j->stream >= 0) s->pool_load[j->stream]--;
    j->stream = -1;
}

// Admits queued jobs in arrival order while they fit the memory budget and
// starts their first chunks.
void admit(sqa_server *s)
{
    NvtxScope nvtx_("server_admit");
    for (;;) {
        Job *j = nullptr;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->queue.empty()) return;
            j = s->queue.front();
            const int64_t need = estimate_device_bytes(&j->desc);
            if (need > s->budget) {
                s->queue.pop_front();
                fail_job(s, j, SQA_ERR_NOMEM);
                continue;
            }
            if (s->used + need > s->budget && !s->active.empty()) return;  // wait for memory
            s->queue.pop_front();
        }
        sqa_handle *h = nullptr;
        sqa_status st = sqa_create(&j->desc, &h);
        cudaEvent_t ev = nullptr;
        if (st == SQA_OK) {
            const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) {
                sqa_destroy(h);
                st = cuda_fail(e, "server event");
            }
        }
        std::lock_guard<std::mutex> lock(s->mu);
        if (st != SQA_OK) {
            fail_job(s, j, st);
            continue;
        }
        int q = 0;
        for (int k = 1; k < kPoolStreams; k++)
            if (s->pool_load[k] < s->pool_load[q]) q = k;
        s->pool_load[q]++;
        j->stream = q;
        j->h = h;
        j->done = ev;
        j->t_next = 0;
        j->info.state = SQA_JOB_RUNNING;
        j->info.t_start = now_s(s->t0);
        j->info.device_bytes = h->device_bytes;
        s->used += h->device_bytes;
        st = launch_chunk(s, j);
        if (st != SQA_OK) {
            cudaStreamSynchronize(s->pool[q]);
            drop_device(s, j);
            fail_job(s, j, st);
            continue;
        }
        s->stats.chunks++;
        s->active.push_back(j);
        s->stats.max_resident = std::max<int64_t>(s->stats.max_resident, (int64_t)s->active.size());
        s->stats.max_bytes = std::max(s->stats.max_bytes, s->used);
    }
}

// Copies a finished job's state and energies to the host and frees its memory.
void retire(sqa_server *s, Job *j)
{
    sqa_handle *h = j->h;
    cudaStream_t st = s->pool[j->stream];
    j->state.resize((size_t)h->I * h->job.Z * h->job.n_phys * h->job.W);
    j->energies.resize((size_t)h->I * h->job.Z * h->R);
    sqa_status rs = sqa_state(h, j->state.data(), 0, st);
    if (rs == SQA_OK) rs = sqa_energies(h, j->energies.data(), 0, st);
    std::lock_guard<std::mutex> lock(s->mu);
    drop_device(s, j);
    if (rs == SQA_OK) {
        j->info.state = SQA_JOB_DONE;
        j->info.status = SQA_OK;
        j->info.t_done = now_s(s->t0);
        s->stats.jobs_done++;
        s->cv_done.notify_all();
    } else {
        fail_job(s, j, rs);
    }
}

// Accounts every chunk that has finished, then launches the job's next chunk
// or retires the job.
sqa_status advance(sqa_server *s, bool *progressed)
{
    std::vector<Job *> keep;
    keep.reserve(s->active.size());
    sqa_status status = SQA_OK;
    for (Job *j : s->active) {
        const cudaError_t q = status == SQA_OK ? cudaEventQuery(j->done) : cudaErrorNotReady;
        if (q == cudaErrorNotReady) {
            keep.push_back(j);
            continue;
        }
        if (q != cudaSuccess) {
            status = cuda_fail(q, "server chunk");
            keep.push_back(j);
            continue;
        }
        *progressed = true;
        sqa_handle *h = j->h;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stats.attempts += (int64_t)(j->t_chunk_end - j->t_next) * h->plan.n * h->job.Z * h->R * h->I;
        }
        j->t_next = j->t_chunk_end;
        if (j->t_next < h->S) {
            status = launch_chunk(s, j);
            if (status == SQA_OK) {
                std::lock_guard<std::mutex> lock(s->mu);
                s->stats.chunks++;
            }
            keep.push_back(j);
        } else {
            retire(s, j);
        }
    }
    std::lock_guard<std::mutex> lock(s->mu);
    s->active.swap(keep);
    return status;
}

void worker_loop(sqa_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->active.empty())
                s->cv_work.wait_for(lock, std::chrono::milliseconds(20),
                                    [&] { return s->stop || !s->queue.empty(); });
            if (s->stop) return;
        }
        const auto c0 = std::chrono::steady_clock::now();
        admit(s);
        const auto c1 = std::chrono::steady_clock::now();
        bool progressed = false;
        const sqa_status st = advance(s, &progressed);
        const auto c2 = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stats.admit_s += std::chrono::duration<double>(c1 - c0).count();
            s->stats.advance_s += std::chrono::duration<double>(c2 - c1).count();
        }
        if (st != SQA_OK) {
            // a launch or a chunk failed: fail every resident job
            for (int q = 0; q < kPoolStreams; q++) cudaStreamSynchronize(s->pool[q]);
            std::lock_guard<std::mutex> lock(s->mu);
            s->worker_status = st;
            for (Job *j : s->active) {
                drop_device(s, j);
                fail_job(s, j, st);
            }
            s->active.clear();
            continue;
        }
        if (!progressed) {
            // no chunk finished: wait briefly for the GPU or for a new job
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait_for(lock, std::chrono::microseconds(100),
                                [&] { return s->stop || !s->queue.empty(); });
            s->stats.idle_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - c2).count();
        }
    }
}

}  // namespace

extern "C" {

sqa_status sqa_server_create(int64_t mem_budget_bytes, int64_t unit_attempts_per_chunk, sqa_server **out)
{
    if (!out || mem_budget_bytes <= 0 || unit_attempts_per_chunk < 0) return set_error("server arguments"), SQA_ERR_INVALID;
    *out = nullptr;
    sqa_status st = device_ready();
    if (st != SQA_OK) return st;
    sqa_server *s = new (std::nothrow) sqa_server();
    if (!s) return SQA_ERR_NOMEM;
    s->budget = mem_budget_bytes;
    s->unit_target = unit_attempts_per_chunk > 0 ? unit_attempts_per_chunk : (int64_t)4e7;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    cudaError_t e = cudaSuccess;
    // keep freed job memory in the device's stream-ordered pool for reuse by
    // the next jobs instead of handing it back to the driver at each sync
    cudaMemPool_t mp;
    if (cudaDeviceGetDefaultMemPool(&mp, s->device) == cudaSuccess) {
        uint64_t keep = (uint64_t)mem_budget_bytes;
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (int q = 0; q < kPoolStreams && e == cudaSuccess; q++) e = cudaStreamCreateWithFlags(&s->pool[q], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (int q = 0; q < kPoolStreams; q++)
            if (s->pool[q]) cudaStreamDestroy(s->pool[q]);
        delete s;
        return cuda_fail(e, "sqa_server_create");
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return SQA_OK;
}

sqa_status sqa_server_submit(sqa_server *s, const sqa_desc *d, uint64_t *job_id)
{
    NvtxScope nvtx_("sqa_server_submit");
    if (!s || !d || !job_id) return set_error("submit arguments"), SQA_ERR_INVALID;
    Job *j = new (std::nothrow) Job();
    if (!j) return SQA_ERR_NOMEM;
    j->desc = *d;
    const int npair = d->n_logical * (d->n_logical - 1) / 2;
    if (d->J && d->n_instances > 0 && d->n_logical >= 2) {
        j->J.assign(d->J, d->J + (size_t)d->n_instances * npair);
        j->desc.J = j->J.data();
    }
    if (d->kind == SQA_KIND_SQA && d->A && d->B && d->n_sweeps > 0) {
        j->A.assign(d->A, d->A + d->n_sweeps);
        j->B.assign(d->B, d->B + d->n_sweeps);
        j->desc.A = j->A.data();
        j->desc.B = j->B.data();
    }
    if (d->kind == SQA_KIND_PT && d->betas && d->n_temps > 0) {
        j->betas.assign(d->betas, d->betas + d->n_temps);
        j->desc.betas = j->betas.data();
    }
    j->desc.h = nullptr;
    if (d->h)
        for (int64_t i = 0; i < (int64_t)d->n_instances * d->n_logical; i++)
            if (d->h[i] != 0) {
                delete j;
                return set_error("non-zero logical fields need an ancilla"), SQA_ERR_UNSUPPORTED;
            }
    std::lock_guard<std::mutex> lock(s->mu);
    j->id = s->next_id++;
    j->info.state = SQA_JOB_QUEUED;
    j->info.t_submit = now_s(s->t0);
    s->jobs[j->id] = j;
    s->queue.push_back(j);
    s->stats.jobs_submitted++;
    *job_id = j->id;
    s->cv_work.notify_one();
    return SQA_OK;
}

sqa_status sqa_server_poll(sqa_server *s, uint64_t job_id, sqa_job_info *info)
{
    if (!s || !info) return set_error("poll arguments"), SQA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error("unknown job"), SQA_ERR_INVALID;
    *info = it->second->info;
    return SQA_OK;
}

sqa_status sqa_server_wait(sqa_server *s, uint64_t job_id, double timeout_s)
{
    if (!s) return set_error("wait arguments"), SQA_ERR_INVALID;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error("unknown job"), SQA_ERR_INVALID;
    Job *j = it->second;
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [&] {
        return j->info.state == SQA_JOB_DONE || j->info.state == SQA_JOB_FAILED;
    });
    return ok ? SQA_OK : SQA_ERR_TIMEOUT;
}

sqa_status sqa_server_result(sqa_server *s, uint64_t job_id, uint32_t *state_out, int32_t *energies_out)
{
    if (!s) return set_error("result arguments"), SQA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error("unknown job"), SQA_ERR_INVALID;
    Job *j = it->second;
    if (j->info.state == SQA_JOB_FAILED) return (sqa_status)j->info.status;
    if (j->info.state != SQA_JOB_DONE) return set_error("job not finished"), SQA_ERR_BUSY;
    if (state_out) std::copy(j->state.begin(), j->state.end(), state_out);
    if (energies_out) std::copy(j->energies.begin(), j->energies.end(), energies_out);
    return SQA_OK;
}

sqa_status sqa_server_release(sqa_server *s, uint64_t job_id)
{
    if (!s) return set_error("release arguments"), SQA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error("unknown job"), SQA_ERR_INVALID;
    Job *j = it->second;
    if (j->info.state != SQA_JOB_DONE && j->info.state != SQA_JOB_FAILED) return set_error("job still pending"), SQA_ERR_BUSY;
    s->jobs.erase(it);
    delete j;
    return SQA_OK;
}

sqa_status sqa_server_get_stats(sqa_server *s, sqa_server_stats *out)
{
    if (!s || !out) return set_error("stats arguments"), SQA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->resident = (int64_t)s->active.size();
    out->queued = (int64_t)s->queue.size();
    out->bytes_in_use = s->used;
    out->worker_status = s->worker_status;
    return SQA_OK;
}

void sqa_server_destroy(sqa_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (int q = 0; q < kPoolStreams; q++)
        if (s->pool[q]) cudaStreamSynchronize(s->pool[q]);
    for (Job *j : s->active) drop_device(s, j);
    s->active.clear();
    for (auto &kv : s->jobs) delete kv.second;
    for (int q = 0; q < kPoolStreams; q++)
        if (s->pool[q]) {
            cudaStreamSynchronize(s->pool[q]);
            cudaStreamDestroy(s->pool[q]);
        }
    delete s;
}

}  // extern "C"
