// Serving loop: continuous batching of SQA and PT jobs on one GPU.
//
// Jobs are submitted from any host thread.  One worker thread owns the GPU
// work: at every epoch boundary it admits queued jobs in arrival order while
// their device memory fits the budget (creating their resident state), runs
// one launch of the multi-job sweep kernel in which every resident job
// advances its own range of sweeps, and retires the jobs that reached their
// last sweep (state and energies copied to host, device memory freed).  A
// job's random numbers depend only on its own descriptor and sweep indices,
// so its result is the same whether it ran alone or among other jobs, and
// however its sweeps were cut into epochs.
//
// Sweeps per epoch are chosen per job so that each of its units does about the
// same work, which bounds the epoch length by the work target rather than by
// the largest job.  Each resident job runs its own sweep kernel (with its own
// launch shape, a thread-block cluster per unit when planned so), on a pool of
// streams so the kernels of all resident jobs share the GPU; new jobs are
// planned and uploaded on the host while the epoch runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "handle.h"

namespace sqa {
void set_error(const std::string &msg);
// One launch of a job's own sweep kernel over all its units (capi.cu).
cudaError_t launch_job_sweeps(const JobDev &J, const Unit *units, int n_units, int *counter, cudaStream_t s);
}

constexpr int kPoolStreams = 16;

using namespace sqa;

namespace {

struct Job {
    uint64_t id = 0;
    sqa_desc desc{};
    std::vector<int32_t> J;
    std::vector<double> A, B, betas;
    sqa_job_info info{};
    sqa_handle *h = nullptr;
    int t_next = 0;                 // next sweep to run
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
    int64_t unit_target = 0;  // attempts per unit per epoch
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
    cudaStream_t stream = nullptr;
    // epoch launch resources
    JobDev *h_jobs = nullptr;  // pinned
    JobDev *d_jobs = nullptr;
    Unit *d_units = nullptr;
    int *d_counter = nullptr;
    int cap_jobs = 0, cap_units = 0;
    cudaStream_t pool[16] = {};
    cudaEvent_t ev_start = nullptr, ev_pool[16] = {};
    std::thread worker;
    sqa_status worker_status = SQA_OK;
};

namespace {

sqa_status ensure_capacity(sqa_server *s, int nj, int nu)
{
    if (nj > s->cap_jobs) {
        const int cap = std::max(nj, 2 * s->cap_jobs);
        if (s->h_jobs) cudaFreeHost(s->h_jobs);
        if (s->d_jobs) cudaFree(s->d_jobs);
        s->h_jobs = nullptr;
        s->d_jobs = nullptr;
        cudaError_t e = cudaMallocHost((void **)&s->h_jobs, sizeof(JobDev) * cap);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_jobs, sizeof(JobDev) * cap);
        if (e != cudaSuccess) return cuda_fail(e, "server job buffers");
        s->cap_jobs = cap;
    }
    if (nu > s->cap_units) {
        const int cap = std::max(nu, 2 * s->cap_units);
        if (s->d_units) cudaFree(s->d_units);
        s->d_units = nullptr;
        cudaError_t e = cudaMalloc((void **)&s->d_units, sizeof(Unit) * cap);
        if (e != cudaSuccess) return cuda_fail(e, "server unit buffer");
        s->cap_units = cap;
    }
    return SQA_OK;
}

// Admit queued jobs in arrival order while they fit the memory budget; the
// new jobs go to *into (the resident list, or the list that joins it after
// the running epoch).
void admit(sqa_server *s, std::vector<Job *> *into)
{
    for (;;) {
        Job *j = nullptr;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            if (s->queue.empty()) return;
            j = s->queue.front();
            const int64_t need = estimate_device_bytes(&j->desc);
            if (need > s->budget) {
                s->queue.pop_front();
                j->info.state = SQA_JOB_FAILED;
                j->info.status = SQA_ERR_NOMEM;
                j->info.t_done = now_s(s->t0);
                s->stats.jobs_failed++;
                s->cv_done.notify_all();
                continue;
            }
            if (s->used + need > s->budget && !(s->active.empty() && into->empty())) return;  // wait for memory
            s->queue.pop_front();
        }
        sqa_handle *h = nullptr;
        const sqa_status st = sqa_create(&j->desc, &h);
        std::lock_guard<std::mutex> lock(s->mu);
        if (st != SQA_OK) {
            j->info.state = SQA_JOB_FAILED;
            j->info.status = st;
            j->info.t_done = now_s(s->t0);
            s->stats.jobs_failed++;
            s->cv_done.notify_all();
            continue;
        }
        j->h = h;
        j->t_next = 0;
        j->info.state = SQA_JOB_RUNNING;
        j->info.t_start = now_s(s->t0);
        j->info.device_bytes = h->device_bytes;
        s->used += h->device_bytes;
        into->push_back(j);
        s->stats.max_resident = std::max<int64_t>(s->stats.max_resident, (int64_t)(s->active.size() + into->size()));
        s->stats.max_bytes = std::max(s->stats.max_bytes, s->used);
    }
}

// Launch one epoch over the resident jobs (asynchronous): each job's own
// sweep kernel (a cluster launch when its units span several blocks) for its
// next range of sweeps, the jobs spread over a pool of streams so their
// kernels run side by side.
sqa_status epoch(sqa_server *s)
{
    const int nj = (int)s->active.size();
    sqa_status st = ensure_capacity(s, nj, 0);
    if (st != SQA_OK) return st;
    cudaError_t e = cudaEventRecord(s->ev_start, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "server epoch start");
    for (int k = 0; k < nj; k++) {
        sqa_handle *h = s->active[k]->h;
        JobDev J = h->job;
        const int64_t unit_attempts = (int64_t)J.n * J.zr * J.wc * 32;
        int64_t sweeps = std::max<int64_t>(1, s->unit_target / std::max<int64_t>(unit_attempts, 1));
        sweeps = std::min<int64_t>(sweeps, h->S - s->active[k]->t_next);
        J.t0 = s->active[k]->t_next;
        J.t1 = J.t0 + (int)sweeps;
        s->h_jobs[k] = J;
        cudaStream_t ps = s->pool[k % kPoolStreams];
        e = cudaStreamWaitEvent(ps, s->ev_start, 0);
        if (e == cudaSuccess) e = launch_job_sweeps(J, h->d_units, h->n_units, h->d_counter, ps);
        if (e != cudaSuccess) return cuda_fail(e, "server epoch launch");
    }
    for (int q = 0; q < std::min(nj, kPoolStreams); q++) {
        e = cudaEventRecord(s->ev_pool[q], s->pool[q]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_pool[q], 0);
        if (e != cudaSuccess) return cuda_fail(e, "server epoch join");
    }
    return SQA_OK;
}

// Wait for the epoch launched by epoch() and advance its jobs.
sqa_status finish_epoch(sqa_server *s)
{
    const int nj = (int)s->active.size();
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "server epoch");
    for (int k = 0; k < nj; k++) {
        Job *j = s->active[k];
        const int ran = s->h_jobs[k].t1 - s->h_jobs[k].t0;
        j->t_next += ran;
        s->stats.attempts += (int64_t)ran * (int64_t)j->h->plan.n * j->h->job.Z * j->h->R * j->h->I;
    }
    s->stats.epochs++;
    return SQA_OK;
}

// Copy finished jobs' results to the host and free their device memory.
sqa_status retire(sqa_server *s)
{
    std::vector<Job *> keep;
    for (Job *j : s->active) {
        sqa_handle *h = j->h;
        if (j->t_next < h->S) {
            keep.push_back(j);
            continue;
        }
        j->state.resize((size_t)h->I * h->job.Z * h->job.n_phys * h->job.W);
        j->energies.resize((size_t)h->I * h->job.Z * h->R);
        sqa_status st = sqa_state(h, j->state.data(), 0, s->stream);
        if (st == SQA_OK) st = sqa_energies(h, j->energies.data(), 0, s->stream);
        const int64_t bytes = h->device_bytes;
        sqa_destroy(h);
        std::lock_guard<std::mutex> lock(s->mu);
        j->h = nullptr;
        s->used -= bytes;
        j->info.state = st == SQA_OK ? SQA_JOB_DONE : SQA_JOB_FAILED;
        j->info.status = st;
        j->info.t_done = now_s(s->t0);
        if (st == SQA_OK)
            s->stats.jobs_done++;
        else
            s->stats.jobs_failed++;
        s->cv_done.notify_all();
    }
    s->active = keep;
    return SQA_OK;
}

void worker_loop(sqa_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait_for(lock, std::chrono::milliseconds(20),
                                [&] { return s->stop || !s->queue.empty() || !s->active.empty(); });
            if (s->stop) return;
        }
        std::vector<Job *> incoming;
        auto c0 = std::chrono::steady_clock::now();
        admit(s, &s->active);
        auto c1 = std::chrono::steady_clock::now();
        s->stats.admit_s += std::chrono::duration<double>(c1 - c0).count();
        if (s->active.empty()) continue;
        sqa_status st = epoch(s);
        // while the GPU runs the epoch: plan and upload the next jobs
        auto c2 = std::chrono::steady_clock::now();
        if (st == SQA_OK) admit(s, &incoming);
        auto c3 = std::chrono::steady_clock::now();
        if (st == SQA_OK) st = finish_epoch(s);
        auto c4 = std::chrono::steady_clock::now();
        if (st == SQA_OK) st = retire(s);
        auto c5 = std::chrono::steady_clock::now();
        s->stats.admit_s += std::chrono::duration<double>(c3 - c2).count();
        s->stats.epoch_s += std::chrono::duration<double>((c2 - c1) + (c4 - c3)).count();
        s->stats.retire_s += std::chrono::duration<double>(c5 - c4).count();
        s->active.insert(s->active.end(), incoming.begin(), incoming.end());
        if (st != SQA_OK) {
            std::lock_guard<std::mutex> lock(s->mu);
            s->worker_status = st;
            for (Job *j : s->active) {
                j->info.state = SQA_JOB_FAILED;
                j->info.status = st;
                if (j->h) {
                    s->used -= j->h->device_bytes;
                    sqa_destroy(j->h);
                    j->h = nullptr;
                }
            }
            s->active.clear();
            s->cv_done.notify_all();
        }
    }
}

}  // namespace

extern "C" {

sqa_status sqa_server_create(int64_t mem_budget_bytes, int64_t unit_attempts_per_epoch, sqa_server **out)
{
    if (!out || mem_budget_bytes <= 0 || unit_attempts_per_epoch < 0) return set_error("server arguments"), SQA_ERR_INVALID;
    *out = nullptr;
    sqa_status st = device_ready();
    if (st != SQA_OK) return st;
    sqa_server *s = new (std::nothrow) sqa_server();
    if (!s) return SQA_ERR_NOMEM;
    s->budget = mem_budget_bytes;
    s->unit_target = unit_attempts_per_epoch > 0 ? unit_attempts_per_epoch : (int64_t)4e7;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_counter, sizeof(int));
    for (int q = 0; q < kPoolStreams && e == cudaSuccess; q++) {
        e = cudaStreamCreateWithFlags(&s->pool[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_pool[q], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return cuda_fail(e, "sqa_server_create");
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return SQA_OK;
}

sqa_status sqa_server_submit(sqa_server *s, const sqa_desc *d, uint64_t *job_id)
{
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
    for (Job *j : s->active)
        if (j->h) sqa_destroy(j->h);
    for (auto &kv : s->jobs) delete kv.second;
    if (s->h_jobs) cudaFreeHost(s->h_jobs);
    if (s->d_jobs) cudaFree(s->d_jobs);
    if (s->d_units) cudaFree(s->d_units);
    if (s->d_counter) cudaFree(s->d_counter);
    for (int q = 0; q < kPoolStreams; q++) {
        if (s->pool[q]) cudaStreamDestroy(s->pool[q]);
        if (s->ev_pool[q]) cudaEventDestroy(s->ev_pool[q]);
    }
    if (s->ev_start) cudaEventDestroy(s->ev_start);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
