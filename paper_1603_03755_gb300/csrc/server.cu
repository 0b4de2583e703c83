// Serving loop: continuous batching of SQA and PT jobs on one GPU.
//
// Jobs are submitted from any host thread.  One worker thread owns the GPU
// work.  It admits queued jobs in arrival order while their device memory
// fits the budget (planning them on the host and uploading their resident
// state) and keeps one chunk of each resident job's sweeps in flight, worth
// about `unit_attempts` attempts per unit (one instance's run of words).
//
// Packing.  Jobs whose units fit one block each (most of them: a job of a few
// hundred replicas has at most eight words) are packed: whenever jobs are
// ready for their next chunk, the worker puts the chunks of all of them that
// share a path (PT, SQA tables, SQA windows, cluster moves) into one launch
// of that path's multi-job sweep kernel, on a stream of the pool, so that
// many small jobs fill the GPU together instead of each occupying a handful
// of blocks.  Several packs are in flight at once on different streams, so
// a pack's tail overlaps the others' work; when a pack finishes, its jobs
// are ready again and go into the next pack with whatever else is ready.
// Jobs whose units need a thread-block cluster run their chunks as launches
// of their own sweep kernel on higher-priority streams.
//
// Nothing the worker does waits on the GPU.  A new job's tables go up in one
// copy from pinned memory on an upload stream (its initial spins are drawn
// on the stream of its first chunk, after that copy); a finished job's
// energies and state are copied into pinned memory behind its final chunk,
// and the job is retired when those copies have landed.  Scratch of packs
// comes from a memory pool of its own that reuses memory only once freed
// work has completed, so that no allocation waits for a pack in flight.
//
// A job's random numbers depend only on its own descriptor and sweep
// indices, so its result is the same whether it ran alone or among other
// jobs, and however its sweeps were cut into chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "handle.h"
#include "layout.cuh"

using namespace sqa;

namespace {

constexpr int kPoolStreams = 64;
constexpr int kOwnStreams = 32;  // pool streams 0..31: jobs with their own launches, high priority
constexpr int kPackSplit = 2;    // packs a set of ready jobs is cut into (their tails overlap)
constexpr int kAdmitBatch = 16;  // jobs admitted per pass of the worker
// Ready jobs are packed only when the resident jobs hold at least this many
// units per SM (more than a wave of the sweep kernels' blocks); below it each
// runs its own chunk launch.  On the serving benchmark's stream (with 32
// hardware connections): packing always gave the highest saturated capacity
// (3.79e11 attempts/s) but p99 latencies of 6.2-8.2 s under Poisson load;
// 4 gave 3.03e11 and 4.6-5.3 s, 2 gave 2.88e11 and 4.6-5.2 s.
constexpr int kPackMinUnitsPerSM = 4;
// Default attempts per unit per chunk: on the serving benchmark's job stream
// (200 jobs, all at once) 1e7 finished in 14.9 s, against 15.4 s (5e6),
// 18.3 s (2e6), 18.3 s (4e7 with 16-block clusters for long jobs) and 16.3 s
// (1.6e8); launching a long cluster job's sweeps in one launch instead of
// chunks doubled it (32 s: its wide clusters held SMs the packs waited for).
constexpr int64_t kUnitTarget = 10'000'000;
constexpr size_t kArenaBytes = (size_t)256 << 20;  // pinned arena of result copies

struct Pack;

struct Job {
    uint64_t id = 0;
    sqa_desc desc{};
    std::vector<int32_t> J;
    std::vector<double> A, B, betas;
    sqa_job_info info{};
    sqa_handle *h = nullptr;
    bool packed = false;            // chunks run in packs of the multi-job kernels
    JobDev pj{};                    // packed: the job planned for one block per unit
    std::vector<Unit> pu;           // packed: its units
    Pack *pack = nullptr;           // packed: the pack holding the chunk in flight
    bool own_inflight = false;      // packed: a chunk of its own kernel in flight instead
    int stream = -1;                // own chunks: index into the stream pool
    int t_next = 0;                 // first sweep of the chunk in flight
    int t_chunk_end = 0;            // end of the chunk in flight
    cudaEvent_t done = nullptr;     // own chunks: recorded after the chunk in flight
    cudaEvent_t out_ev = nullptr;   // recorded after the final chunk's result copies
    void *pin = nullptr;            // pinned host buffer of those copies: state, then energies
    size_t pin_bytes = 0;
    void *up_pin = nullptr;         // pinned source of the setup's upload (until the first chunk is done)
    size_t up_bytes = 0;
    std::vector<uint32_t> state;    // [I][Z][n_phys][W] once done
    std::vector<int32_t> energies;  // [I][Z][R] once done
};

// One launch of the multi-job kernels over chunks of several jobs.
struct Pack {
    int stream = -1;
    cudaEvent_t done = nullptr;
    std::vector<Job *> jobs;
    void *pin = nullptr;  // pinned copy of the pack's job descriptors and unit list
    size_t pin_bytes = 0;
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
    std::vector<Job *> active;   // resident jobs (packed or not)
    std::vector<Job *> ready;    // packed jobs waiting for their next pack
    std::vector<Pack *> packs;   // packs in flight
    std::vector<Job *> retiring; // final chunk done or in flight, result copies pending
    // pinned host memory for result copies: one arena allocated up front
    // (a page-locked allocation while kernels run would serialize the
    // device), its free ranges by offset; buffers allocated beyond it are
    // kept for reuse
    char *arena = nullptr;
    std::map<size_t, size_t> arena_free;
    std::vector<std::pair<void *, size_t>> pinned_free;
    uint64_t next_id = 1;
    bool stop = false;
    int64_t used = 0;
    sqa_server_stats stats{};
    int device = 0;
    cudaStream_t pool[kPoolStreams] = {};
    int pool_load[kPoolStreams] = {};
    int next_pack_stream = 0;
    cudaStream_t retire_stream = nullptr;  // frees of finished jobs
    cudaStream_t upload_stream = nullptr;  // new jobs' allocations and uploads
    // scratch of packs and result copies (descriptors, unit lists, tie
    // queues, energies): its own pool, reused only once a free has completed,
    // so that no allocation waits for a pack in flight on another stream
    cudaMemPool_t scratch = nullptr;
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

// Sweeps of j's next chunk: about unit_target attempts per unit.
int chunk_sweeps(const sqa_server *s, const Job *j, const JobDev &J)
{
    const int64_t unit_attempts = (int64_t)J.n * J.zr * J.wc * 32;
    int64_t sweeps = std::max<int64_t>(1, s->unit_target / std::max<int64_t>(unit_attempts, 1));
    return (int)std::min<int64_t>(sweeps, j->h->S - j->t_next);
}

void pinned_release(sqa_server *s, void *p, size_t bytes);

// A pinned host buffer of at least `bytes` (from the server's free list, else new).
cudaError_t pinned_get(sqa_server *s, size_t bytes, void **p, size_t *got)
{
    const size_t need = (bytes + 4095) & ~(size_t)4095;
    for (auto it = s->arena_free.begin(); it != s->arena_free.end(); ++it)
        if (it->second >= need) {
            const size_t off = it->first, len = it->second;
            s->arena_free.erase(it);
            if (len > need) s->arena_free[off + need] = len - need;
            *p = s->arena + off;
            *got = need;
            return cudaSuccess;
        }
    size_t best = (size_t)-1;
    for (size_t k = 0; k < s->pinned_free.size(); k++)
        if (s->pinned_free[k].second >= bytes && (best == (size_t)-1 || s->pinned_free[k].second < s->pinned_free[best].second))
            best = k;
    if (best != (size_t)-1) {
        *p = s->pinned_free[best].first;
        *got = s->pinned_free[best].second;
        s->pinned_free.erase(s->pinned_free.begin() + (long)best);
        return cudaSuccess;
    }
    const size_t sz = std::max<size_t>((bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1), 1u << 20);
    *got = sz;
    return cudaMallocHost(p, sz);
}

// After j's final chunk, in stream order on st: the energies of every slice
// or slot (energy kernel into a stream-ordered scratch array), then the
// state (compact site order) and the energies copied into a pinned host
// buffer, and an event.  The worker retires j once the event has completed,
// without waiting on the GPU: the result kernels and copies queue behind the
// chunk instead of behind whatever else holds the SMs.
sqa_status enqueue_outputs(sqa_server *s, Job *j, cudaStream_t st)
{
    sqa_handle *h = j->h;
    const size_t state_bytes = (size_t)h->I * h->job.Z * h->job.n * h->job.W * 4;
    const size_t en_bytes = (size_t)h->I * h->job.Z * h->R * 4;
    cudaError_t e = pinned_get(s, state_bytes + en_bytes, &j->pin, &j->pin_bytes);
    int32_t *d_en = nullptr;
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&d_en, std::max<size_t>(en_bytes, 4), s->scratch, st);
    if (e == cudaSuccess) e = enqueue_energies(h, d_en, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync((char *)j->pin + state_bytes, d_en, en_bytes, cudaMemcpyDeviceToHost, st);
    if (d_en) cudaFreeAsync(d_en, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(j->pin, h->d_state, state_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->out_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(j->out_ev, st);
    if (e != cudaSuccess) return cuda_fail(e, "server result copies");
    return SQA_OK;
}

// Launches the chunk of j's sweeps that starts at j->t_next with j's own
// sweep kernel, on j's stream (the caller counts it in the stats under s->mu).
sqa_status launch_chunk(sqa_server *s, Job *j)
{
    NvtxScope nvtx_("server_chunk");
    sqa_handle *h = j->h;
    JobDev J = h->job;
    J.t0 = j->t_next;
    J.t1 = J.t0 + chunk_sweeps(s, j, J);
    cudaStream_t st = s->pool[j->stream];
    if (j->t_next == 0) {
        if (h->setup_ev && cudaStreamWaitEvent(st, h->setup_ev, 0) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "server chunk");
        const sqa_status si = launch_init(h, st);
        if (si != SQA_OK) return si;
    }
    cudaError_t e = launch_job_sweeps(J, h->d_units, h->n_units, h->d_counter, st);
    if (e != cudaSuccess) return cuda_fail(e, "server chunk");
    j->t_chunk_end = J.t1;
    if (J.t1 >= h->S) {
        const sqa_status so = enqueue_outputs(s, j, st);
        if (so != SQA_OK) return so;
    }
    e = cudaEventRecord(j->done, st);
    if (e != cudaSuccess) return cuda_fail(e, "server chunk");
    return SQA_OK;
}

// One pack: the next chunk of every job of js (one path) in one launch of
// that path's multi-job kernel, on the next stream of the pool.  Its job
// descriptors, unit list, counters and tie queue live in stream-ordered
// allocations freed behind the launch.
sqa_status launch_pack(sqa_server *s, const std::vector<Job *> &js)
{
    NvtxScope nvtx_("server_pack");
    const auto c0 = std::chrono::steady_clock::now();
    Pack *pk = new (std::nothrow) Pack();
    if (!pk) return SQA_ERR_NOMEM;
    std::vector<JobDev> jobs;
    std::vector<Unit> units;
    for (size_t k = 0; k < js.size(); k++) {
        Job *j = js[k];
        JobDev J = j->pj;
        J.t0 = j->t_next;
        J.t1 = J.t0 + chunk_sweeps(s, j, J);
        j->t_chunk_end = J.t1;
        jobs.push_back(J);
        for (Unit u : j->pu) {
            u.job = (int)k;
            units.push_back(u);
        }
    }
    std::vector<MultiGroup> groups;
    const int rows = group_units(jobs, units, groups);
    int stride = 1;
    for (const JobDev &J : jobs) stride = std::max(stride, tie_items(J, J.wc));
    pk->stream = kOwnStreams + s->next_pack_stream;
    s->next_pack_stream = (s->next_pack_stream + 1) % (kPoolStreams - kOwnStreams);
    cudaStream_t st = s->pool[pk->stream];
    JobDev *d_jobs = nullptr;
    Unit *d_units = nullptr;
    int *d_counter = nullptr;
    uint2 *d_tieq = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&pk->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&d_tieq, (size_t)rows * stride * sizeof(uint2), s->scratch, st);
    assign_tieq(jobs, groups, d_tieq, stride);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&d_jobs, jobs.size() * sizeof(JobDev), s->scratch, st);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&d_units, units.size() * sizeof(Unit), s->scratch, st);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void **)&d_counter, kMaxModes * sizeof(int), s->scratch, st);
    // the descriptors go through pinned memory: a pageable source would hold
    // a driver staging buffer until this stream reaches the copy, and other
    // copies (a new job's upload) would wait for it
    const size_t jb = jobs.size() * sizeof(JobDev), ub = units.size() * sizeof(Unit);
    if (e == cudaSuccess) e = pinned_get(s, jb + ub, &pk->pin, &pk->pin_bytes);
    if (e == cudaSuccess) {
        memcpy(pk->pin, jobs.data(), jb);
        memcpy((char *)pk->pin + jb, units.data(), ub);
        e = cudaMemcpyAsync(d_jobs, pk->pin, jb, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_units, (char *)pk->pin + jb, ub, cudaMemcpyHostToDevice, st);
    for (Job *j : js)
        if (e == cudaSuccess && j->t_next == 0) {
            if (j->h->setup_ev) e = cudaStreamWaitEvent(st, j->h->setup_ev, 0);
            if (e == cudaSuccess && launch_init(j->h, st) != SQA_OK) e = cudaErrorLaunchFailure;
        }
    if (e == cudaSuccess) e = launch_groups(groups, d_jobs, d_units, d_counter, st, false);
    if (d_tieq) cudaFreeAsync(d_tieq, st);
    if (d_jobs) cudaFreeAsync(d_jobs, st);
    if (d_units) cudaFreeAsync(d_units, st);
    if (d_counter) cudaFreeAsync(d_counter, st);
    for (Job *j : js)
        if (e == cudaSuccess && j->t_chunk_end >= j->h->S && enqueue_outputs(s, j, st) != SQA_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaEventRecord(pk->done, st);
    if (e != cudaSuccess) {
        if (pk->done) cudaEventDestroy(pk->done);
        cudaStreamSynchronize(st);
        pinned_release(s, pk->pin, pk->pin_bytes);
        delete pk;
        return cuda_fail(e, "server pack");
    }
    pk->jobs = js;
    for (Job *j : js) j->pack = pk;
    std::lock_guard<std::mutex> lock(s->mu);
    s->packs.push_back(pk);
    s->stats.chunks += (int64_t)js.size();
    s->stats.packs++;
    s->stats.pack_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - c0).count();
    return SQA_OK;
}

// Packs every ready job: one pack per path (PT, SQA tables, SQA windows,
// ...), each one launch of that path's multi-job kernel on its own stream,
// so that the paths run side by side; a path with units enough to fill the
// GPU more than once is cut into kPackSplit packs, whose tails overlap.
sqa_status launch_ready(sqa_server *s)
{
    std::vector<Job *> ready;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        ready.swap(s->ready);
    }
    if (ready.empty()) return SQA_OK;
    size_t resident_units = 0;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (Job *a : s->active) resident_units += a->packed ? a->pu.size() : (size_t)a->h->n_units;
    }
    if (resident_units < (size_t)num_sms() * kPackMinUnitsPerSM) {
        // few units resident: the GPU has room for every job's own launch,
        // and a job then keeps its own pace instead of a pack's slowest unit
        for (Job *j : ready) {
            const sqa_status st = launch_chunk(s, j);
            if (st != SQA_OK) return st;
            j->own_inflight = true;
            std::lock_guard<std::mutex> lock(s->mu);
            s->stats.chunks++;
        }
        return SQA_OK;
    }
    std::vector<std::vector<Job *>> by_mode(kMaxModes);
    for (Job *j : ready) by_mode[sweep_mode(j->pj)].push_back(j);
    for (auto &js : by_mode) {
        if (js.empty()) continue;
        size_t n_units = 0;
        for (Job *j : js) n_units += j->pu.size();
        const int parts = n_units >= (size_t)num_sms() * 4 && js.size() >= 2 ? kPackSplit : 1;
        std::vector<std::vector<Job *>> cut(parts);
        for (size_t k = 0; k < js.size(); k++) cut[k % parts].push_back(js[k]);
        for (auto &c : cut) {
            if (c.empty()) continue;
            const sqa_status st = launch_pack(s, c);
            if (st != SQA_OK) return st;
        }
    }
    return SQA_OK;
}

// Releases j's device resources in stream order (caller holds s->mu).
void drop_device(sqa_server *s, Job *j)
{
    if (j->h) {
        s->used -= j->h->device_bytes;
        // on the retire stream, which holds only short work: a later
        // allocation that reuses this memory waits on nothing long
        destroy_on_stream(j->h, s->retire_stream);
        j->h = nullptr;
    }
    if (j->done) cudaEventDestroy(j->done);
    j->done = nullptr;
    if (j->stream >= 0) s->pool_load[j->stream]--;
    j->stream = -1;
}

// Admits queued jobs in arrival order while they fit the memory budget, at
// most kAdmitBatch per call (so that packs of the jobs admitted so far start
// while a long queue is still being planned): packed jobs join the ready
// list, the others start their first chunks.
void admit(sqa_server *s)
{
    NvtxScope nvtx_("server_admit");
    for (int n_admitted = 0; n_admitted < kAdmitBatch; n_admitted++) {
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
            if (s->used + need > s->budget && (!s->active.empty() || !s->retiring.empty()))
                return;  // wait for memory
            s->queue.pop_front();
        }
        sqa_handle *h = nullptr;
        const auto c0 = std::chrono::steady_clock::now();
        sqa_status st = create_handle(&j->desc, &h, false, s->upload_stream);  // spins: before the first chunk
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stats.create_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - c0).count();
        }
        // one block per unit (no cluster) in the job's own plan: packed
        bool packed = false;
        if (st == SQA_OK && h->job.csize == 1) packed = plan_job(h, 1, 0, j->pj, j->pu) == SQA_OK && j->pj.csize == 1;
        if (st == SQA_OK) st = ensure_tieq(h);  // its own sweep kernel's (a packed job too runs it when the GPU is quiet)
        if (st == SQA_OK) {
            // the setup's one upload, from pinned memory, then the event the
            // job's first launch waits for
            cudaError_t e = cudaSuccess;
            if (!h->pending.empty()) {
                e = pinned_get(s, h->pending.size(), &j->up_pin, &j->up_bytes);
                if (e == cudaSuccess) {
                    memcpy(j->up_pin, h->pending.data(), h->pending.size());
                    e = cudaMemcpyAsync(h->pending_dst, j->up_pin, h->pending.size(), cudaMemcpyHostToDevice,
                                        s->upload_stream);
                }
                std::vector<unsigned char>().swap(h->pending);
            }
            if (e == cudaSuccess) e = cudaEventRecord(h->setup_ev, s->upload_stream);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "server upload");
                cudaStreamSynchronize(s->upload_stream);
                std::lock_guard<std::mutex> lock(s->mu);
                pinned_release(s, j->up_pin, j->up_bytes);
                j->up_pin = nullptr;
                sqa_destroy(h);
                h = nullptr;
            }
        }
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
        j->h = h;
        j->packed = packed;
        j->t_next = 0;
        j->info.state = SQA_JOB_RUNNING;
        j->info.t_start = now_s(s->t0);
        j->info.device_bytes = h->device_bytes;
        s->used += h->device_bytes;
        int q = 0;
        for (int k = 1; k < kOwnStreams; k++)
            if (s->pool_load[k] < s->pool_load[q]) q = k;
        s->pool_load[q]++;
        j->stream = q;
        j->done = ev;
        if (packed) {
            s->ready.push_back(j);
        } else {
            st = launch_chunk(s, j);
            if (st != SQA_OK) {
                cudaStreamSynchronize(s->pool[q]);
                drop_device(s, j);
                fail_job(s, j, st);
                continue;
            }
            s->stats.chunks++;
        }
        s->active.push_back(j);
        s->stats.max_resident = std::max<int64_t>(s->stats.max_resident, (int64_t)s->active.size());
        s->stats.max_bytes = std::max(s->stats.max_bytes, s->used);
    }
}

// Returns a pinned buffer to the arena (merged with free neighbours) or to
// the list of buffers beyond it.
void pinned_release(sqa_server *s, void *p, size_t bytes)
{
    char *c = (char *)p;
    if (c && s->arena && c >= s->arena && c < s->arena + kArenaBytes) {
        size_t off = (size_t)(c - s->arena), len = bytes;
        auto next = s->arena_free.lower_bound(off);
        if (next != s->arena_free.end() && next->first == off + len) {
            len += next->second;
            next = s->arena_free.erase(next);
        }
        if (next != s->arena_free.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                len += prev->second;
                s->arena_free.erase(prev);
            }
        }
        s->arena_free[off] = len;
    } else if (c) {
        s->pinned_free.emplace_back(p, bytes);
    }
}

// Returns j's pinned buffers (caller holds s->mu).
void pinned_put(sqa_server *s, Job *j)
{
    pinned_release(s, j->up_pin, j->up_bytes);
    j->up_pin = nullptr;
    j->up_bytes = 0;
    pinned_release(s, j->pin, j->pin_bytes);
    j->pin = nullptr;
    j->pin_bytes = 0;
    if (j->out_ev) cudaEventDestroy(j->out_ev);
    j->out_ev = nullptr;
}

// A retiring job whose result copies have completed: its state in canonical
// site order (unused sites 0) and its energies from the pinned buffer, then
// its device memory freed in stream order.
void finish_retire(sqa_server *s, Job *j)
{
    const auto c0 = std::chrono::steady_clock::now();
    sqa_handle *h = j->h;
    const int I = h->I, Z = h->job.Z, n = h->job.n, np = h->job.n_phys, W = h->job.W;
    const uint32_t *cs = (const uint32_t *)j->pin;
    j->state.assign((size_t)I * Z * np * W, 0u);
    for (int iz = 0; iz < I * Z; iz++)
        for (int ph = 0; ph < np; ph++) {
            const int si = h->plan.compact[ph];
            if (si < 0) continue;
            std::copy(cs + ((size_t)iz * n + si) * W, cs + ((size_t)iz * n + si + 1) * W,
                      j->state.begin() + ((size_t)iz * np + ph) * W);
        }
    const int32_t *en = (const int32_t *)((const char *)j->pin + (size_t)I * Z * n * W * 4);
    j->energies.assign(en, en + (size_t)I * Z * h->R);
    std::lock_guard<std::mutex> lock(s->mu);
    pinned_put(s, j);
    drop_device(s, j);
    s->stats.retire_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - c0).count();
    j->info.state = SQA_JOB_DONE;
    j->info.status = SQA_OK;
    j->info.t_done = now_s(s->t0);
    s->stats.jobs_done++;
    s->cv_done.notify_all();
}

// A chunk of j finished: account it, then retire j or make it ready for its
// next chunk (packed: the next pack; own: a launch now).  Returns the jobs
// that stay resident in keep.
sqa_status chunk_done(sqa_server *s, Job *j, std::vector<Job *> &keep)
{
    sqa_handle *h = j->h;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stats.attempts += (int64_t)(j->t_chunk_end - j->t_next) * h->plan.n * h->job.Z * h->R * h->I;
    }
    j->t_next = j->t_chunk_end;
    j->pack = nullptr;
    if (j->up_pin) {  // the chunk waited for the setup's upload: its source is free
        std::lock_guard<std::mutex> lock(s->mu);
        pinned_release(s, j->up_pin, j->up_bytes);
        j->up_pin = nullptr;
        j->up_bytes = 0;
    }
    if (j->t_next >= h->S) {
        // its result copies were queued behind the final chunk
        std::lock_guard<std::mutex> lock(s->mu);
        s->retiring.push_back(j);
        return SQA_OK;
    }
    keep.push_back(j);
    if (j->packed) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->ready.push_back(j);
        return SQA_OK;
    }
    const sqa_status st = launch_chunk(s, j);
    if (st == SQA_OK) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stats.chunks++;
    }
    return st;
}

// Accounts every pack and own chunk that has finished, retires finished
// jobs, launches own next chunks and packs every ready job.
sqa_status advance(sqa_server *s, bool *progressed)
{
    sqa_status status = SQA_OK;
    std::vector<Job *> keep;
    keep.reserve(s->active.size());
    // packs: a finished pack hands all its jobs on
    std::vector<Pack *> packs;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        packs.swap(s->packs);
    }
    std::vector<Pack *> live;
    std::vector<Job *> finished;  // jobs of finished packs
    for (Pack *pk : packs) {
        const cudaError_t q = status == SQA_OK ? cudaEventQuery(pk->done) : cudaErrorNotReady;
        if (q == cudaErrorNotReady) {
            live.push_back(pk);
            continue;
        }
        if (q != cudaSuccess) {
            status = cuda_fail(q, "server pack");
            live.push_back(pk);
            continue;
        }
        *progressed = true;
        for (Job *j : pk->jobs) finished.push_back(j);
        cudaEventDestroy(pk->done);
        {
            std::lock_guard<std::mutex> lock(s->mu);
            pinned_release(s, pk->pin, pk->pin_bytes);
        }
        delete pk;
    }
    for (Job *j : s->active) {
        if (j->packed && !j->own_inflight) {
            if (j->pack == nullptr || std::find(finished.begin(), finished.end(), j) != finished.end()) {
                if (j->pack == nullptr) {
                    keep.push_back(j);  // ready, waiting for its pack
                } else if (status == SQA_OK) {
                    status = chunk_done(s, j, keep);
                } else {
                    keep.push_back(j);
                }
            } else {
                keep.push_back(j);
            }
            continue;
        }
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
        j->own_inflight = false;
        if (status == SQA_OK) status = chunk_done(s, j, keep);
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->active.swap(keep);
        for (Pack *pk : live) s->packs.push_back(pk);
    }
    // retiring jobs whose result copies have landed
    std::vector<Job *> ret, still;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        ret.swap(s->retiring);
    }
    for (Job *j : ret) {
        const cudaError_t q = status == SQA_OK ? cudaEventQuery(j->out_ev) : cudaErrorNotReady;
        if (q == cudaErrorNotReady) {
            still.push_back(j);
        } else if (q != cudaSuccess) {
            status = cuda_fail(q, "server result copies");
            still.push_back(j);
        } else {
            *progressed = true;
            finish_retire(s, j);
        }
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (Job *j : still) s->retiring.push_back(j);
    }
    if (status == SQA_OK) status = launch_ready(s);
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
            cudaStreamSynchronize(s->retire_stream);
            std::lock_guard<std::mutex> lock(s->mu);
            s->worker_status = st;
            for (Pack *pk : s->packs) {
                cudaEventDestroy(pk->done);
                pinned_release(s, pk->pin, pk->pin_bytes);
                delete pk;
            }
            s->packs.clear();
            s->ready.clear();
            for (Job *j : s->active) {
                drop_device(s, j);
                fail_job(s, j, st);
            }
            s->active.clear();
            for (Job *j : s->retiring) {
                pinned_put(s, j);
                drop_device(s, j);
                fail_job(s, j, st);
            }
            s->retiring.clear();
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
    s->unit_target = unit_attempts_per_chunk > 0 ? unit_attempts_per_chunk : kUnitTarget;
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
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    e = cudaMemPoolCreate(&s->scratch, &props);
    if (e == cudaSuccess) {
        uint64_t keep = (uint64_t)mem_budget_bytes;
        int no = 0;
        cudaMemPoolSetAttribute(s->scratch, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaMemPoolSetAttribute(s->scratch, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    // jobs with their own launches (the long, wide ones) before packs of small ones
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    for (int q = 0; q < kPoolStreams && e == cudaSuccess; q++)
        e = cudaStreamCreateWithPriority(&s->pool[q], cudaStreamNonBlocking, q < kOwnStreams ? prio_high : prio_low);
    // result copies at the highest priority: their small kernels take the
    // first free block slots instead of queueing behind persistent packs
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->retire_stream, cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->upload_stream, cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess && cudaMallocHost((void **)&s->arena, kArenaBytes) == cudaSuccess)
        s->arena_free[0] = kArenaBytes;
    else
        cudaGetLastError();  // no arena: result buffers are allocated as jobs finish
    if (e != cudaSuccess) {
        for (int q = 0; q < kPoolStreams; q++)
            if (s->pool[q]) cudaStreamDestroy(s->pool[q]);
        if (s->retire_stream) cudaStreamDestroy(s->retire_stream);
        if (s->upload_stream) cudaStreamDestroy(s->upload_stream);
        if (s->scratch) cudaMemPoolDestroy(s->scratch);
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
    for (Pack *pk : s->packs) {
        cudaEventDestroy(pk->done);
        pinned_release(s, pk->pin, pk->pin_bytes);
        delete pk;
    }
    s->packs.clear();
    s->ready.clear();
    if (s->retire_stream) cudaStreamSynchronize(s->retire_stream);
    for (Job *j : s->active) drop_device(s, j);
    s->active.clear();
    for (Job *j : s->retiring) {
        pinned_put(s, j);
        drop_device(s, j);
    }
    s->retiring.clear();
    for (auto &kv : s->jobs) delete kv.second;
    for (int q = 0; q < kPoolStreams; q++)
        if (s->pool[q]) {
            cudaStreamSynchronize(s->pool[q]);
            cudaStreamDestroy(s->pool[q]);
        }
    if (s->retire_stream) {
        cudaStreamSynchronize(s->retire_stream);
        cudaStreamDestroy(s->retire_stream);
    }
    if (s->upload_stream) {
        cudaStreamSynchronize(s->upload_stream);
        cudaStreamDestroy(s->upload_stream);
    }
    for (auto &pb : s->pinned_free) cudaFreeHost(pb.first);
    if (s->arena) cudaFreeHost(s->arena);
    if (s->scratch) cudaMemPoolDestroy(s->scratch);
    delete s;
}

}  // extern "C"
