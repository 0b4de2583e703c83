// C ABI of the SQA / PT library (include/sqa.h): handle lifecycle, launch
// planning and the host side of every entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "handle.h"
#include "layout.cuh"
#include "philox.cuh"
#include "sqa_internal.h"

namespace sqa {

__global__ void init_kernel(JobDev J, const int *canon);
// The single-job sweep kernel (kernels.cu), one instantiation per path.
const void *sweep_one_entry(const JobDev &J);

// Threads per block of the single-job kernel on a job's path.
int sweep_one_threads(const JobDev &J);
cudaError_t launch_sweep_one(const JobDev &J, const Unit *units, int n_units, int *counter, int grid,
                             cudaStream_t s);
int max_active_clusters(const JobDev &J);
static const void *one_kernel(const JobDev &J) { return sweep_one_entry(J); }
__global__ void energy_kernel(JobDev J, int32_t *out);
__global__ void canon_kernel(JobDev J, const int *compact_of, int z0, int zcount, uint32_t *out);
__global__ void decode_kernel(JobDev J, DecodeArgs D);
__global__ void ground_kernel(int N, const int32_t *J, int chunk_bits, int64_t n_chunks,
                              unsigned long long *best);

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

sqa_status cuda_fail(cudaError_t e, const char *where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return SQA_ERR_CUDA;
}

#define SQA_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

static int g_num_sms = 0;

int num_sms() { return g_num_sms; }
static int g_smem_limit = 0;  // dynamic shared memory one sweep block may use

sqa_status device_ready()
{
    int dev = 0, n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        g_err = "no CUDA device";
        return SQA_ERR_NO_DEVICE;
    }
    SQA_CUDA(cudaGetDevice(&dev));
    if (g_num_sms == 0) {
        cudaDeviceProp prop;
        SQA_CUDA(cudaGetDeviceProperties(&prop, dev));
        const void *ks[14];
        for (int m = 0; m < kMaxModes; m++) {
            ks[m] = sweep_one_entry_mode(m);
            ks[kMaxModes + m] = sweep_multi_entry(m);
        }
        int limit = (int)prop.sharedMemPerBlockOptin;
        for (const void *k : ks) {
            cudaFuncAttributes fk;
            SQA_CUDA(cudaFuncGetAttributes(&fk, k));
            limit = std::min(limit, (int)prop.sharedMemPerBlockOptin - (int)fk.sharedSizeBytes);
        }
        for (const void *k : ks) SQA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
        // single-job kernels may run 16-block clusters (one unit over 16 SMs'
        // worth of blocks); where the device refuses, clusters stop at 8
        for (int m = 0; m < kMaxModes; m++)
            if (cudaFuncSetAttribute(sweep_one_entry_mode(m), cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess)
                cudaGetLastError();
        g_num_sms = prop.multiProcessorCount;
        g_smem_limit = limit;
    }
    return SQA_OK;
}

sqa_status usable(const sqa_handle *h)
{
    if (!h) return set_error("NULL handle"), SQA_ERR_INVALID;
    if (!h->ready) return set_error("the handle has no device program (its last setup failed)"), SQA_ERR_INVALID;
    return SQA_OK;
}

}  // namespace sqa

using namespace sqa;


namespace {

template <typename T>
sqa_status dalloc(sqa_handle *h, T **p, size_t count)
{
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    // stream-ordered: freeing later needs no device-wide synchronization
    cudaError_t e = cudaMallocAsync(&q, bytes, h->setup_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return SQA_ERR_NOMEM;
    }
    h->allocs.push_back(q);
    h->device_bytes += (int64_t)bytes;
    *p = (T *)q;
    return SQA_OK;
}

template <typename T>
sqa_status upload(sqa_handle *h, T **p, const std::vector<T> &v)
{
    sqa_status st = dalloc(h, p, v.size());
    if (st != SQA_OK) return st;
    if (!v.empty()) SQA_CUDA(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    h->h2d_bytes += (int64_t)(v.size() * sizeof(T));
    return SQA_OK;
}

// Host arrays gathered for one upload: every array at a 256-byte aligned
// offset of one staging buffer, copied by one cudaMemcpy into one device
// allocation (a synchronous copy can wait behind work other streams queued
// on the same hardware queue, so a handle's setup makes as few as it can).
struct Staging {
    std::vector<unsigned char> host;
    std::vector<std::pair<void **, size_t>> fix;  // where each array's device address goes, its offset
    int64_t counted = 0, bytes = 0;               // device bytes as separate allocations would count, payload
};

template <typename T>
void stage(Staging &sg, T **p, const std::vector<T> &v)
{
    const size_t off = (sg.host.size() + 255) & ~(size_t)255;
    const size_t b = v.size() * sizeof(T);
    sg.host.resize(off + std::max<size_t>(b, sizeof(T)));
    if (b) memcpy(sg.host.data() + off, v.data(), b);
    sg.fix.emplace_back((void **)p, off);
    sg.counted += (int64_t)(std::max<size_t>(v.size(), 1) * sizeof(T));
    sg.bytes += (int64_t)b;
}

sqa_status commit(sqa_handle *h, Staging &sg)
{
    unsigned char *q = nullptr;
    const cudaError_t e = cudaMallocAsync((void **)&q, std::max<size_t>(sg.host.size(), 1), h->setup_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return SQA_ERR_NOMEM;
    }
    h->allocs.push_back(q);
    h->device_bytes += sg.counted;
    for (auto &f : sg.fix) *f.first = q + f.second;
    h->h2d_bytes += sg.bytes;
    if (h->lazy_tieq) {
        // served job: the caller queues the copy (pending_upload)
        h->pending.swap(sg.host);
        h->pending_dst = q;
        return SQA_OK;
    }
    if (!sg.host.empty()) SQA_CUDA(cudaMemcpy(q, sg.host.data(), sg.host.size(), cudaMemcpyHostToDevice));
    return SQA_OK;
}

// Frees every device buffer of h in stream order on s and forgets them: h
// runs nothing until a setup completes again.
void free_all(sqa_handle *h, cudaStream_t s = 0)
{
    for (void *p : h->allocs)
        if (p) cudaFreeAsync(p, s);
    h->allocs.clear();
    h->device_bytes = 0;
    h->h2d_bytes = 0;
    h->ready = false;
    h->d_state = nullptr;
    h->d_sites = nullptr;
    h->d_T = nullptr;
    h->d_eterms = nullptr;
    h->d_ecls = nullptr;
    h->d_Tsw = h->d_Tb = h->d_Tacc = nullptr;
    h->d_accoff = h->d_acclen = h->d_swoff = h->d_swlen = nullptr;
    h->d_canon = h->d_compact = nullptr;
    h->d_J = nullptr;
    h->d_chain = h->d_pair = nullptr;
    h->d_parents = h->d_orders = nullptr;
    h->cur_trees = h->cur_tree_kind = -1;
    h->d_job = nullptr;
    h->d_units = nullptr;
    h->n_units = 0;
    h->d_counter = nullptr;
    h->d_tieq = nullptr;
    h->tieq_cap = 0;
}


// Row stride (words) of the shared state for units of wc words: consecutive
// lanes take consecutive words, then the next z step (two slices for SQA, one
// slot for PT); pad the row so those lanes fall on distinct banks.
int zstride_for(const JobDev &J, int wc)
{
    // the n used sites and a zero slot (site n) that absent term members read
    int zs = (J.n + 1) * wc;
    if (J.kind == SQA_KIND_SQA && J.move == SQA_MOVE_WOLFF) {
        // cluster moves: a warp reads 32 consecutive rows, on distinct banks
        // when the row stride is odd
        if (zs % 2 == 0) zs++;
    } else if (J.kind == SQA_KIND_SQA) {
        if (wc % 2 == 0) {
            while ((2 * zs) % 32 != wc % 32) zs++;
        } else {
            while (zs % 2 == 0) zs++;
        }
    } else {
        while (zs % 32 != wc % 32) zs++;
    }
    return zs;
}

int unit_smem(const JobDev &J, int wc, int *zstride_out)
{
    const int zs = zstride_for(J, wc);
    *zstride_out = zs;
    return (int)smem_layout(J, wc, zs).total;
}

int blocks_per_sm(const void *kernel, int smem, int threads = kThreads)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

// Choose the launch shape of a job: blocks per unit (a cluster of C blocks
// splitting the slices or slots), words per unit and, for SQA, table or
// window mode.  Objective: the most blocks busy at once, counting a cluster's
// blocks at 90 % (barriers and remote reads); then smaller C, table mode,
// more words per unit.  c_forced > 0 restricts C.  Writes J's shape fields
// and the unit list.
// Relative costs behind the planner's choice between per-site code tables
// and byte-wise windows, in units of one table-mode item (32 attempts):
// measured, a window-mode item costs about 1.25 of them, and rebuilding one
// table entry (once per sweep in every block) about 0.15.  On the 1024 x 256
// ME K_8 workload (12288 items per block per sweep, ~1200 entries) tables
// run 1.4x faster; on 8-block clusters of single-instance jobs, with few
// items per block, windows ran 6-70 % faster in every case measured.
constexpr double kWindowItem = 1.25;
constexpr double kTableEntry = 0.15;

// table_cost: weigh table rebuilds against window lookups (single-job
// kernels); the multi-job kernel of batches keeps preferring tables, which
// measured faster there.
sqa_status plan_shape(sqa_handle *h, int c_forced, JobDev &J, std::vector<Unit> &units, bool table_cost = true)
{
    struct Best {
        double score = -1;
        int C = 0, wc = 0, lut = 0;
    } best;
    // automatic plans stop at 8-block clusters: wider ones are hard to place
    // beside other work (16 is available through sqa_tune)
    const int cmax = c_forced > 0 ? c_forced : 8;
    const bool wolff = J.kind == SQA_KIND_SQA && J.move == SQA_MOVE_WOLFF;
    for (int C = c_forced > 0 ? c_forced : 1; C <= cmax; C *= 2) {
        if (J.kind == SQA_KIND_SQA ? (J.Z % (2 * C)) : (J.Z % C)) continue;
        if (wolff && C > 1) continue;  // a cluster move needs the whole ring in one block
        J.csize = C;
        J.zr = J.Z / C;
        const int modes = J.kind == SQA_KIND_SQA && !wolff ? 2 : 1;
        for (int m = modes - 1; m >= 0; m--) {
            J.use_lut = J.kind == SQA_KIND_SQA ? m : 0;
            if (!J.use_lut && h->window_limit_exceeded) continue;
            if (h->force_mode >= 0 && J.kind == SQA_KIND_SQA && J.use_lut != h->force_mode) continue;
            for (int wc = J.W; wc >= 1; wc = wc > 1 ? (wc + 1) / 2 : 0) {
                const bool take = h->force_wc <= 0 || wc == std::min(h->force_wc, J.W);
                if (take) {
                    int zs = 0;
                    const int smem = unit_smem(J, wc, &zs);
                    if (smem <= g_smem_limit) {
                        J.smem_bytes = smem;
                        J.wc = wc;
                        J.zstride = zs;
                        const int active = C == 1 ? blocks_per_sm(one_kernel(J), smem, sweep_one_threads(J)) * g_num_sms
                                                  : max_active_clusters(J);
                        const int64_t n_units = (int64_t)h->I * ((J.W + wc - 1) / wc);
                        // PT clusters exchange boundary slots every swap event:
                        // only when one block cannot hold the unit
                        double eff = C == 1 ? 1.0 : (J.kind == SQA_KIND_PT ? 0.05 : 0.9);
                        if (table_cost && J.kind == SQA_KIND_SQA && !wolff) {
                            // a block's sweep in item units: table lookups cost 1 per
                            // item plus the per-sweep rebuild of every site's table;
                            // byte windows cost kWindowItem per item and no rebuild
                            const double items = (double)J.n * J.zr * wc;
                            const double cost = J.use_lut ? items + kTableEntry * J.lut_entries
                                                          : kWindowItem * items;
                            eff *= items / cost;
                        }
                        const double busy = (double)std::min<int64_t>(n_units, active) * C * eff;
                        const bool better = busy > best.score * 1.0001 ||
                                            (busy >= best.score * 0.9999 && C == best.C &&
                                             (J.use_lut > best.lut || (J.use_lut == best.lut && wc > best.wc)));
                        if (active > 0 && better) best = Best{busy, C, wc, J.use_lut};
                    }
                }
                if (wc == 1) break;
            }
        }
    }
    if (best.score <= 0) {
        set_error("the requested unit does not fit in shared memory");
        return SQA_ERR_UNSUPPORTED;
    }
    J.csize = best.C;
    J.zr = J.Z / best.C;
    J.use_lut = best.lut;
    J.wc = best.wc;
    J.smem_bytes = unit_smem(J, best.wc, &J.zstride);
    units.clear();
    for (int i = 0; i < h->I; i++)
        for (int w0 = 0; w0 < J.W; w0 += J.wc) units.push_back(Unit{0, i, w0, std::min(J.wc, J.W - w0)});
    return SQA_OK;
}

sqa_status plan_units(sqa_handle *h) { return plan_shape(h, h->force_cluster, h->job, h->units); }

// Entries of a job's tie queue: every item of one colour phase of every
// unit, for any launch shape (grid x items per block phase <= units x words x
// phase items per word, and words per unit round the W words up to at most
// 2W).  Host-only, so the admission estimate is exact.
int64_t tieq_entries(const Plan &pl, int kind, int move, int64_t I, int64_t Z, int64_t W)
{
    if (kind == SQA_KIND_SQA && move == SQA_MOVE_WOLFF) return 0;
    int nq = 0;
    for (int c = 0; c < pl.ncol; c++) nq = std::max(nq, pl.col_ptr[c + 1] - pl.col_ptr[c]);
    const int64_t zn = kind == SQA_KIND_SQA ? (Z + 1) / 2 : Z;
    return (int64_t)nq * zn * I * 2 * W;
}

// Points the job at the handle's tie queue with the current shape's stride
// (allocated once at setup: tieq_entries covers every shape).
void set_tieq(sqa_handle *h)
{
    JobDev &J = h->job;
    J.tieq = h->d_tieq;
    J.tieq_stride = h->d_tieq ? tie_items(J, J.wc) : 0;
}

sqa_status validate(const sqa_desc *d)
{
    if (!d) return set_error("desc is NULL"), SQA_ERR_INVALID;
    if (d->kind != SQA_KIND_SQA && d->kind != SQA_KIND_PT) return set_error("kind"), SQA_ERR_INVALID;
    if (d->embedding != SQA_EMB_ME_CHIMERA && d->embedding != SQA_EMB_LHZ)
        return set_error("embedding"), SQA_ERR_INVALID;
    if (d->n_logical < 2 || d->n_logical > kMaxN) return set_error("n_logical out of range"), SQA_ERR_INVALID;
    if (d->n_instances < 1 || !d->J) return set_error("n_instances / J"), SQA_ERR_INVALID;
    if (d->penalty <= 0) return set_error("penalty must be > 0"), SQA_ERR_INVALID;
    if (d->n_sweeps < 1 || d->n_replicas < 1) return set_error("n_sweeps / n_replicas"), SQA_ERR_INVALID;
    {
        // bound the magnitudes before any per-site sum is formed (the exact
        // limit, a site's weight sum within the int16 records, comes later)
        const int32_t lim = 1 << 24;
        if (d->penalty > lim) return set_error("penalty too large"), SQA_ERR_UNSUPPORTED;
        const int64_t npair = (int64_t)d->n_logical * (d->n_logical - 1) / 2;
        for (int64_t i = 0; i < (int64_t)d->n_instances * npair; i++)
            if (d->J[i] > lim || d->J[i] < -lim) return set_error("couplings too large"), SQA_ERR_UNSUPPORTED;
    }
    if (d->h) {
        for (int64_t i = 0; i < (int64_t)d->n_instances * d->n_logical; i++)
            if (d->h[i] != 0) return set_error("non-zero logical fields need an ancilla"), SQA_ERR_UNSUPPORTED;
    }
    if (d->move != SQA_MOVE_METROPOLIS && d->move != SQA_MOVE_WOLFF) return set_error("move"), SQA_ERR_INVALID;
    if (d->kind == SQA_KIND_SQA && d->move == SQA_MOVE_WOLFF && d->n_slices > 128)
        return set_error("cluster moves need n_slices <= 128"), SQA_ERR_UNSUPPORTED;
    if (d->kind == SQA_KIND_SQA) {
        if (d->n_slices < 2 || (d->n_slices & 1) || d->n_slices > 1024)
            return set_error("n_slices must be even, 2..1024"), SQA_ERR_INVALID;
        if (!(d->beta > 0) || !isfinite(d->beta)) return set_error("beta"), SQA_ERR_INVALID;
        if ((d->A == nullptr) != (d->B == nullptr)) return set_error("give both A and B or neither"), SQA_ERR_INVALID;
        if (d->A)
            for (int t = 0; t < d->n_sweeps; t++)
                if (!(d->A[t] >= 0) || !(d->B[t] >= 0) || !isfinite(d->A[t]) || !isfinite(d->B[t]))
                    return set_error("schedule values must be finite and >= 0"), SQA_ERR_INVALID;
    } else {
        if (d->n_temps < 1 || !d->betas || d->swap_every < 1) return set_error("PT ladder"), SQA_ERR_INVALID;
        for (int p = 0; p < d->n_temps; p++)
            if (!(d->betas[p] > 0) || !isfinite(d->betas[p])) return set_error("betas must be > 0"), SQA_ERR_INVALID;
        for (int p = 0; p + 1 < d->n_temps; p++)
            if (!(d->betas[p] > d->betas[p + 1])) return set_error("betas must decrease"), SQA_ERR_INVALID;
    }
    return SQA_OK;
}

// (Re)build the program-dependent part: tables, site records, state.
sqa_status setup_program(sqa_handle *h)
{
    free_all(h);
    const Plan &pl = h->plan;
    const int N = h->N, npair = N * (N - 1) / 2;
    h->smax = 0;
    for (int i = 0; i < h->I; i++)
        h->smax = std::max(h->smax, site_weight_sum_max(pl, h->J.data() + (size_t)i * npair, h->penalty));
    const int K = h->kind == SQA_KIND_SQA ? 6 : 2;
    // byte-wise windows hold K*S_i (+2 for SQA) per site; the SQA table mode
    // has no such limit
    const bool wolff = h->kind == SQA_KIND_SQA && h->move == SQA_MOVE_WOLFF;
    h->window_limit_exceeded = !wolff && K * h->smax + 2 > kMaxByteWindow;
    if (h->window_limit_exceeded && h->kind == SQA_KIND_PT) {
        set_error("penalty/couplings too large for the byte-wise threshold window");
        return SQA_ERR_UNSUPPORTED;
    }
    if (3 * h->smax + 8 > 32767) {
        set_error("penalty/couplings too large");
        return SQA_ERR_UNSUPPORTED;
    }
    h->dmin = -2 * h->smax;
    h->dmax = 2 * h->smax;
    h->nd = (h->dmax - h->dmin) / 2 + 1;
    JobDev &J = h->job;
    J = JobDev{};
    J.kind = h->kind;
    J.n = pl.n;
    J.n_phys = pl.n_phys;
    J.Z = h->kind == SQA_KIND_SQA ? h->L : h->P;
    J.W = (h->R + 31) / 32;
    J.R = h->R;
    J.n_inst = h->I;
    J.ncol = pl.ncol;
    for (int c = 0; c <= kMaxColours; c++) J.col_ptr[c] = pl.col_ptr[c];
    J.nrow = h->kind == SQA_KIND_SQA ? 3 * h->nd : h->nd;
    J.n_eterms = (int)pl.terms.size();
    J.swap_every = h->swap_every;
    J.csize = 1;
    J.zr = J.Z;
    J.task_slices = h->force_slices;
    J.t0 = 0;
    J.t1 = h->S;
    J.seed_lo = (uint32_t)h->seed;
    const uint32_t shi = (uint32_t)(h->seed >> 32);
    J.key_hi = shi ^ kDomSweepHi;
    J.key_lo = shi ^ kDomSweepLo;
    J.key_swap = shi ^ kDomSwap;
    for (int r = 0; r < 10; r++) {
        J.rk0[r] = J.seed_lo + (uint32_t)r * 0x9E3779B9u;
        J.rk_hi[r] = J.key_hi + (uint32_t)r * 0xBB67AE85u;
        J.rk_lo[r] = J.key_lo + (uint32_t)r * 0xBB67AE85u;
    }
    J.move = wolff ? SQA_MOVE_WOLFF : SQA_MOVE_METROPOLIS;
    J.pairs = 1;
    for (const PlanTerm &t : pl.terms) J.pairs = J.pairs && t.size == 2;
    J.key_wstart = shi ^ kDomWStart;
    J.key_wbond = shi ^ kDomWBond;
    J.key_wacc = shi ^ kDomWAcc;

    std::vector<SiteRec> sites, all_sites;
    std::vector<ETerm> et, all_et;
    std::vector<EClass> ec, all_ec;
    int n_ecls = 0;
    bool ecls_ok = true;
    J.lut_entries = 0;
    for (int i = 0; i < pl.n; i++) J.lut_entries += 1 << ((int)pl.site_terms[i].size() + 2);
    for (int i = 0; i < h->I; i++) {
        const int32_t *Ji = h->J.data() + (size_t)i * npair;
        build_sites(pl, Ji, h->penalty, K, h->smax, sites);
        all_sites.insert(all_sites.end(), sites.begin(), sites.end());
        const int nc = build_eterms(pl, Ji, h->penalty, et, ec);
        if (nc == 0) ecls_ok = false;
        n_ecls = std::max(n_ecls, nc);
        all_et.insert(all_et.end(), et.begin(), et.end());
        all_ec.insert(all_ec.end(), ec.begin(), ec.end());
    }
    h->d_T = h->d_Tsw = h->d_Tb = h->d_Tacc = nullptr;
    h->d_swoff = h->d_swlen = h->d_accoff = h->d_acclen = nullptr;
    std::vector<uint32_t> T, Tsw, Tb, Tacc;
    std::vector<int> swoff, swlen, accoff, acclen;
    if (wolff) {
        wolff_tables(h->A.data(), h->B.data(), h->beta, h->L, h->S, h->dmax, Tb, Tacc, accoff, acclen);
    } else if (h->kind == SQA_KIND_SQA) {
        sqa_tables(h->A.data(), h->B.data(), h->beta, h->L, h->S, h->dmin, h->dmax, T);
    } else {
        pt_tables(h->betas.data(), h->P, h->dmin, h->dmax, T);
        swap_tables(h->betas.data(), h->P, Tsw, swoff, swlen);
    }
    sqa_status st;
    if ((st = dalloc(h, &h->d_state, (size_t)h->I * J.Z * J.n * J.W)) != SQA_OK) return st;
    Staging sg;
    stage(sg, &h->d_sites, all_sites);
    stage(sg, &h->d_eterms, all_et);
    stage(sg, &h->d_ecls, all_ec);
    J.n_ecls = ecls_ok ? n_ecls : 0;
    if (wolff) {
        stage(sg, &h->d_Tb, Tb);
        stage(sg, &h->d_Tacc, Tacc);
        stage(sg, &h->d_accoff, accoff);
        stage(sg, &h->d_acclen, acclen);
    } else {
        stage(sg, &h->d_T, T);
    }
    if (h->kind == SQA_KIND_PT) {
        stage(sg, &h->d_Tsw, Tsw);
        stage(sg, &h->d_swoff, swoff);
        stage(sg, &h->d_swlen, swlen);
    }
    stage(sg, &h->d_canon, pl.canon);
    stage(sg, &h->d_compact, pl.compact);
    stage(sg, &h->d_J, h->J);
    if (h->emb == SQA_EMB_ME_CHIMERA)
        stage(sg, &h->d_chain, pl.chain);
    else
        stage(sg, &h->d_pair, pl.pair);
    if ((st = plan_units(h)) != SQA_OK) return st;
    stage(sg, &h->d_units, h->units);
    h->units_staged = true;
    if ((st = commit(h, sg)) != SQA_OK) return st;
    h->cur_trees = -1;
    J.state = h->d_state;
    J.sites = h->d_sites;
    J.T = h->d_T;
    J.eterms = h->d_eterms;
    J.ecls = h->d_ecls;
    J.Tsw = h->d_Tsw;
    J.sw_off = h->d_swoff;
    J.sw_len = h->d_swlen;
    J.Tb = h->d_Tb;
    J.Tacc = h->d_Tacc;
    J.acc_off = h->d_accoff;
    J.acc_len = h->d_acclen;
    if (!h->lazy_tieq && (st = ensure_tieq(h)) != SQA_OK) return st;
    if ((st = dalloc(h, &h->d_job, 1)) != SQA_OK) return st;
    h->n_units = (int)h->units.size();
    if ((st = dalloc(h, &h->d_counter, 1)) != SQA_OK) return st;
    h->ready = true;
    return SQA_OK;
}

sqa_status launch_sweeps(sqa_handle *h, int t0, int t1, int u0, int nu, cudaStream_t s)
{
    const sqa_status sq = ensure_tieq(h);  // a served handle allocates it on its first own launch
    if (sq != SQA_OK) return sq;
    if (!h->d_units || u0 < 0 || nu < 0 || u0 + nu > h->n_units)
        return set_error("no unit list on the device (a failed sqa_tune)"), SQA_ERR_INVALID;
    h->job.t0 = t0;
    h->job.t1 = t1;
    SQA_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(int), s));
    const int grid = launch_grid(h->job, nu);
    SQA_CUDA(launch_sweep_one(h->job, h->d_units + u0, nu, h->d_counter, grid, s));
    return SQA_OK;
}

sqa_status decode_trees(sqa_handle *h, int method, int n_trees)
{
    if (h->cur_trees == n_trees && h->cur_tree_kind == method) return SQA_OK;
    const int N = h->N;
    std::vector<int> par((size_t)h->I * n_trees * N), ord((size_t)h->I * n_trees * N);
    for (int i = 0; i < h->I; i++)
        for (int t = 0; t < n_trees; t++) {
            int *p = par.data() + ((size_t)i * n_trees + t) * N;
            int *o = ord.data() + ((size_t)i * n_trees + t) * N;
            if (method == SQA_DECODE_LHZ_TREES)
                prufer_tree(N, h->seed, i, t, p, o);
            else if (method == SQA_DECODE_LHZ_STAR)
                star_tree(N, p, o);
            else
                chain_tree(N, p, o);
        }
    sqa_status st;
    if ((st = upload(h, &h->d_parents, par)) != SQA_OK) return st;
    if ((st = upload(h, &h->d_orders, ord)) != SQA_OK) return st;
    h->cur_trees = n_trees;
    h->cur_tree_kind = method;
    return SQA_OK;
}

}  // namespace

namespace sqa {

sqa_status launch_init(sqa_handle *h, cudaStream_t s)
{
    const int64_t total = (int64_t)h->I * h->job.Z * h->job.n * h->job.W;
    const int blocks = (int)std::min<int64_t>((total + kThreads - 1) / kThreads, 4 * 1024);
    init_kernel<<<std::max(blocks, 1), kThreads, 0, s>>>(h->job, h->d_canon);
    SQA_CUDA(cudaGetLastError());
    return SQA_OK;
}

int grid_for(const void *kernel, int smem_bytes, int n_units, int threads)
{
    int per_sm = std::max(blocks_per_sm(kernel, smem_bytes, threads), 1);
    return std::max(1, std::min(n_units, per_sm * g_num_sms));
}

// Threads per block of a path's multi-job launch: the path's own width,
// except that SQA single-spin units so small that a 256-thread block would
// hold under kSmallItems items per thread per colour phase (weighted by the
// units' work) run 128-thread blocks, twice as many per SM; the kernels size
// themselves from blockDim.  Measured (2000 sweeps, one session): 256
// one-instance ME K_12 jobs 9.02e11 -> 1.10e12 attempts/s; the ragged LHZ/ME
// mix, whose units mostly stay at 256, 8.91e11 -> 8.84e11; forcing 128 on
// every group took the mix to 7.68e11.
constexpr double kSmallItems = 4.0;

static int multi_threads(const std::vector<JobDev> &jobs, const std::vector<Unit> &units, int mode, size_t i, size_t j)
{
    const int full = sweep_mode_threads(mode);
    if (mode != 1 && mode != 2 && mode != 5) return full;
    double items = 0, work = 0;
    for (size_t u = i; u < j; u++) {
        const JobDev &x = jobs[units[u].job];
        if (2 * units[u].wc > 128) return full;  // a block stages the hoisted values of 2 x wc words
        const double w = (double)x.n * x.zr * units[u].wc;  // items per sweep
        items += w / (2.0 * x.ncol * full) * w;            // per thread and phase, weighted by work
        work += w;
    }
    return work > 0 && items / work < kSmallItems ? 128 : full;
}

int group_units(const std::vector<JobDev> &jobs, std::vector<Unit> &units, std::vector<MultiGroup> &groups)
{
    // by path, then longest units first so the tail of each launch is short
    std::stable_sort(units.begin(), units.end(), [&](const Unit &a, const Unit &b) {
        const JobDev &x = jobs[a.job], &y = jobs[b.job];
        const int ma = sweep_mode(x), mb = sweep_mode(y);
        if (ma != mb) return ma < mb;
        const double ca = (double)x.n * x.Z * a.wc * (x.t1 - x.t0);
        const double cb = (double)y.n * y.Z * b.wc * (y.t1 - y.t0);
        return ca > cb;
    });
    groups.clear();
    for (size_t i = 0; i < units.size();) {
        const int mode = sweep_mode(jobs[units[i].job]);
        size_t j = i;
        int smem = 0;
        while (j < units.size() && sweep_mode(jobs[units[j].job]) == mode) smem = std::max(smem, jobs[units[j++].job].smem_bytes);
        MultiGroup g;
        g.mode = mode;
        g.u0 = (int)i;
        g.n = (int)(j - i);
        g.smem = smem;
        g.threads = multi_threads(jobs, units, mode, i, j);
        g.grid = grid_for(sweep_multi_entry(mode), smem, g.n, g.threads);
        g.row0 = 0;
        groups.push_back(g);
        i = j;
    }
    // the path with the most work starts first; the others fill its tail
    std::vector<double> work(groups.size(), 0.0);
    for (size_t k = 0; k < groups.size(); k++)
        for (int u = groups[k].u0; u < groups[k].u0 + groups[k].n; u++) {
            const JobDev &x = jobs[units[u].job];
            work[k] += (double)x.n * x.Z * units[u].wc * (x.t1 - x.t0);
        }
    std::vector<size_t> order(groups.size());
    for (size_t k = 0; k < order.size(); k++) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
    std::vector<MultiGroup> sorted;
    int rows = 0;  // concurrent launches: each path's blocks get their own tie-queue rows
    for (size_t k : order) {
        sorted.push_back(groups[k]);
        sorted.back().row0 = rows;
        rows += groups[k].grid;
    }
    groups.swap(sorted);
    return rows;
}

namespace {
// Streams and events of this host thread for forking a batch's path launches
// off the caller's stream (one set per device).
struct ForkPool {
    cudaStream_t st[kMaxModes] = {};
    cudaEvent_t fork = nullptr, join[kMaxModes] = {};
};

cudaError_t fork_pool(ForkPool **out)
{
    thread_local std::vector<ForkPool> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((int)pools.size() <= dev) pools.resize(dev + 1);
    ForkPool &p = pools[dev];
    if (!p.fork) {
        for (int k = 0; k < kMaxModes && e == cudaSuccess; k++) {
            e = cudaStreamCreateWithFlags(&p.st[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.join[k], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    *out = &p;
    return cudaSuccess;
}
}  // namespace

void assign_tieq(std::vector<JobDev> &jobs, const std::vector<MultiGroup> &groups, uint2 *d_tieq, int stride)
{
    for (JobDev &J : jobs) {
        J.tieq = d_tieq;
        J.tieq_stride = stride;
        for (const MultiGroup &g : groups)
            if (g.mode == sweep_mode(J)) J.tieq = d_tieq + (size_t)g.row0 * (size_t)stride;
    }
}

// One group's persistent launch, at its block width.
static cudaError_t launch_group(const MultiGroup &g, const JobDev *d_jobs, const Unit *d_units, int *d_counters,
                                cudaStream_t s)
{
    const Unit *units = d_units + g.u0;
    int n = g.n;
    int *counter = d_counters + g.mode;
    void *args[] = {(void *)&d_jobs, (void *)&units, (void *)&n, (void *)&counter};
    return cudaLaunchKernel(sweep_multi_entry(g.mode), dim3((unsigned)g.grid), dim3((unsigned)g.threads), args,
                            (size_t)g.smem, s);
}

cudaError_t launch_groups(const std::vector<MultiGroup> &groups, const JobDev *d_jobs, const Unit *d_units,
                          int *d_counters, cudaStream_t s, bool fork)
{
    cudaError_t e = cudaMemsetAsync(d_counters, 0, kMaxModes * sizeof(int), s);
    if (e != cudaSuccess || groups.empty()) return e;
    if (groups.size() == 1 || !fork) {
        for (size_t k = 0; k < groups.size() && e == cudaSuccess; k++) {
            const MultiGroup &g = groups[k];
            e = launch_group(g, d_jobs, d_units, d_counters, s);
        }
        return e;
    }
    // several paths: each persistent launch on its own stream after the
    // caller's stream, all joined back into it, so that blocks of the next
    // path take the SMs the previous path's blocks leave at the end of its
    // work (the paths' tails overlap instead of running one after another)
    ForkPool *p = nullptr;
    if ((e = fork_pool(&p)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(p->fork, s)) != cudaSuccess) return e;
    for (size_t k = 0; k < groups.size() && e == cudaSuccess; k++) {
        const MultiGroup &g = groups[k];
        e = cudaStreamWaitEvent(p->st[k], p->fork, 0);
        if (e == cudaSuccess)
            e = launch_group(g, d_jobs, d_units, d_counters, p->st[k]);
        if (e == cudaSuccess) e = cudaEventRecord(p->join[k], p->st[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->join[k], 0);
    }
    return e;
}

int launch_grid(const JobDev &J, int n_units)
{
    if (J.csize == 1) return grid_for(sweep_one_entry(J), J.smem_bytes, n_units, sweep_one_threads(J));
    return std::max(1, std::min(n_units, max_active_clusters(J))) * J.csize;
}

int64_t estimate_device_bytes(const sqa_desc *d)
{
    if (validate(d) != SQA_OK) return 0;
    Plan pl;
    std::string err;
    if (!build_plan(d->embedding, d->n_logical, pl, err)) return 0;
    const int N = d->n_logical, I = d->n_instances, npair = N * (N - 1) / 2;
    int smax = 0;
    for (int i = 0; i < I; i++) smax = std::max(smax, site_weight_sum_max(pl, d->J + (size_t)i * npair, d->penalty));
    const int64_t nd = 2 * smax + 1;
    const int64_t Z = d->kind == SQA_KIND_SQA ? d->n_slices : d->n_temps;
    const int64_t W = (d->n_replicas + 31) / 32;
    const auto al = [](int64_t b) { return std::max<int64_t>(b, 1); };
    int64_t b = 0;
    b += al((int64_t)I * Z * pl.n * W * 4);                          // state
    b += al((int64_t)I * pl.n * (int64_t)sizeof(SiteRec));           // site records
    b += al((int64_t)I * (int64_t)pl.terms.size() * (int64_t)sizeof(ETerm));
    b += al((int64_t)I * kMaxEClasses * (int64_t)sizeof(EClass));
    if (d->kind == SQA_KIND_SQA && d->move == SQA_MOVE_WOLFF) {
        std::vector<double> A(d->n_sweeps), B(d->n_sweeps);
        for (int t = 0; t < d->n_sweeps; t++) {
            const double s = ((double)t + 0.5) / (double)d->n_sweeps;
            A[t] = d->A ? d->A[t] : 1.0 - s;
            B[t] = d->B ? d->B[t] : s;
        }
        std::vector<uint32_t> Tb, Tacc;
        std::vector<int> off, len;
        wolff_tables(A.data(), B.data(), d->beta, d->n_slices, d->n_sweeps, 2 * smax, Tb, Tacc, off, len);
        b += al((int64_t)Tb.size() * 4) + al((int64_t)Tacc.size() * 4) + 2 * al((int64_t)off.size() * 4);
    } else if (d->kind == SQA_KIND_SQA) {
        b += al((int64_t)d->n_sweeps * 3 * nd * 4);                  // thresholds
    } else {
        b += al((int64_t)d->n_temps * nd * 4);
        std::vector<uint32_t> T;
        std::vector<int> off, len;
        swap_tables(d->betas, d->n_temps, T, off, len);
        b += al((int64_t)T.size() * 4) + 2 * al((int64_t)off.size() * 4);
    }
    b += al((int64_t)pl.canon.size() * 4) + al((int64_t)pl.compact.size() * 4) + al((int64_t)I * npair * 4);
    b += d->embedding == SQA_EMB_ME_CHIMERA ? al((int64_t)pl.chain.size() * 4) : al((int64_t)pl.pair.size() * 4);
    b += al((int64_t)sizeof(JobDev)) + al((int64_t)I * W * (int64_t)sizeof(Unit)) + al(4);
    const int64_t ne = tieq_entries(pl, d->kind, d->move, I, Z, W);
    if (ne > 0) b += ne * (int64_t)sizeof(uint2);
    return b;
}

sqa_status plan_job(sqa_handle *h, int c_forced, int force_wc, JobDev &J, std::vector<Unit> &units)
{
    const int keep = h->force_wc;
    h->force_wc = force_wc;
    J = h->job;
    const sqa_status st = plan_shape(h, c_forced, J, units, false);
    h->force_wc = keep;
    return st;
}

sqa_status run_sweeps(sqa_handle *h, int t0, int t1, cudaStream_t s)
{
    return launch_sweeps(h, t0, t1, 0, h->n_units, s);
}

cudaError_t launch_job_sweeps(const JobDev &J, const Unit *units, int n_units, int *counter, cudaStream_t s)
{
    return launch_sweep_one(J, units, n_units, counter, launch_grid(J, n_units), s);
}

}  // namespace sqa

extern "C" {

const char *sqa_strerror(sqa_status s)
{
    switch (s) {
    case SQA_OK: return "ok";
    case SQA_ERR_INVALID: return "invalid argument";
    case SQA_ERR_UNSUPPORTED: return "unsupported";
    case SQA_ERR_NOMEM: return "out of memory";
    case SQA_ERR_CUDA: return "CUDA error";
    case SQA_ERR_TIMEOUT: return "timeout";
    case SQA_ERR_NO_DEVICE: return "no CUDA device";
    case SQA_ERR_BUSY: return "busy";
    case SQA_ERR_BOUNDS: return "bounds check";
    }
    return "unknown status";
}

const char *sqa_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace sqa {
sqa_status ensure_tieq(sqa_handle *h)
{
    if (h->d_tieq || h->tieq_cap) return SQA_OK;
    const int64_t ne = tieq_entries(h->plan, h->kind, h->move, h->I, h->job.Z, h->job.W);
    sqa_status st;
    if (ne > 0 && (st = dalloc(h, &h->d_tieq, (size_t)ne)) != SQA_OK) return st;
    h->tieq_cap = (size_t)ne;
    set_tieq(h);
    return SQA_OK;
}

sqa_status create_handle(const sqa_desc *d, sqa_handle **out, bool init, cudaStream_t setup_stream)
{
    if (!out) return set_error("out is NULL"), SQA_ERR_INVALID;
    *out = nullptr;
    sqa_status st = validate(d);
    if (st != SQA_OK) return st;
    if ((st = device_ready()) != SQA_OK) return st;
    sqa_handle *h = new (std::nothrow) sqa_handle();
    if (!h) return SQA_ERR_NOMEM;
    h->kind = d->kind;
    h->lazy_tieq = !init;
    h->setup_stream = init ? (cudaStream_t)0 : setup_stream;
    h->emb = d->embedding;
    h->N = d->n_logical;
    h->I = d->n_instances;
    h->penalty = d->penalty;
    h->S = d->n_sweeps;
    h->R = d->n_replicas;
    h->seed = d->seed;
    const int npair = h->N * (h->N - 1) / 2;
    h->J.assign(d->J, d->J + (size_t)h->I * npair);
    if (d->kind == SQA_KIND_SQA) {
        h->move = d->move;
        h->L = d->n_slices;
        h->beta = d->beta;
        h->A.resize(h->S);
        h->B.resize(h->S);
        for (int t = 0; t < h->S; t++) {
            if (d->A) {
                h->A[t] = d->A[t];
                h->B[t] = d->B[t];
            } else {
                const double s = ((double)t + 0.5) / (double)h->S;
                h->A[t] = 1.0 - s;
                h->B[t] = s;
            }
        }
    } else {
        h->P = d->n_temps;
        h->betas.assign(d->betas, d->betas + h->P);
        h->swap_every = d->swap_every;
    }
    std::string err;
    if (!build_plan(h->emb, h->N, h->plan, err)) {
        delete h;
        return set_error(err), SQA_ERR_UNSUPPORTED;
    }
    st = setup_program(h);
    if (st == SQA_OK && init) st = launch_init(h, 0);
    if (st == SQA_OK && init) {
        // the legacy stream: waits for this handle's work only, not for work
        // on non-blocking streams (the serving loop's chunks in flight)
        cudaError_t e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) st = cuda_fail(e, "sqa_create");
    } else if (st == SQA_OK) {
        // no wait on the host: the caller queues the upload on setup_stream
        // (pending_upload) and its first user's stream waits for setup_ev
        const cudaError_t e = cudaEventCreateWithFlags(&h->setup_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) st = cuda_fail(e, "sqa_create");
    }
    if (st != SQA_OK) {
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return SQA_OK;
}

}  // namespace sqa

extern "C" {

sqa_status sqa_create(const sqa_desc *d, sqa_handle **out)
{
    NvtxScope nvtx_("sqa_create");
    return create_handle(d, out, true, 0);
}

void sqa_destroy(sqa_handle *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->setup_ev) cudaEventDestroy(h->setup_ev);
    free_all(h);
    cudaStreamSynchronize(0);
    delete h;
}

}  // extern "C"

namespace sqa {
// Frees a handle whose work is known to be complete once stream s reaches
// this point (the serving loop): no device-wide synchronization.
void destroy_on_stream(sqa_handle *h, cudaStream_t s)
{
    if (!h) return;
    if (h->setup_ev) cudaEventDestroy(h->setup_ev);
    free_all(h, s);
    delete h;
}

cudaError_t enqueue_energies(const sqa_handle *h, int32_t *dev_out, cudaStream_t s)
{
    const size_t count = (size_t)h->I * h->job.Z * h->R;
    const int blocks = (int)std::min<size_t>((count + kThreads - 1) / kThreads, 8192);
    energy_kernel<<<std::max(blocks, 1), kThreads, 0, s>>>(h->job, dev_out);
    return cudaGetLastError();
}

}  // namespace sqa

extern "C" {

sqa_status sqa_get_info(const sqa_handle *h, sqa_info *o)
{
    if (!h || !o) return set_error("NULL argument"), SQA_ERR_INVALID;
    o->n_phys = h->plan.n_phys;
    o->n_used = h->plan.n;
    o->n_terms = (int32_t)h->plan.terms.size();
    o->z = h->job.Z;
    o->words = h->job.W;
    o->delta_min = h->dmin;
    o->delta_max = h->dmax;
    o->attempts_per_sweep = (int64_t)h->I * h->plan.n * h->job.Z * h->R;
    o->device_bytes = h->device_bytes;
    o->h2d_bytes = h->h2d_bytes;
    o->launches_per_run = 2;  // init_kernel + sweep_kernel
    o->pad_ = 0;
    return SQA_OK;
}


sqa_status sqa_tune(sqa_handle *h, int32_t words_per_unit, int32_t use_table, int32_t cluster)
{
    sqa_status us = usable(h);
    if (us != SQA_OK) return us;
    if (words_per_unit < 0 || use_table < -1 || use_table > 1 || cluster < 0 || cluster > 16 ||
        (cluster & (cluster - 1)))
        return set_error("tune arguments"), SQA_ERR_INVALID;
    if (use_table == 0 && h->window_limit_exceeded) return set_error("window mode cannot hold this problem"), SQA_ERR_UNSUPPORTED;
    const int old_wc = h->force_wc, old_mode = h->force_mode, old_c = h->force_cluster;
    h->force_wc = words_per_unit;
    h->force_mode = use_table;
    h->force_cluster = cluster;
    const JobDev keep = h->job;
    const std::vector<Unit> keep_units = h->units;
    sqa_status st = plan_units(h);
    if (st != SQA_OK) {
        h->force_wc = old_wc;
        h->force_mode = old_mode;
        h->force_cluster = old_c;
        h->job = keep;
        h->units = keep_units;
        return st;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "sqa_tune");
    if (!h->units_staged) {  // a list inside the setup's one upload stays until the handle goes
        SQA_CUDA(cudaFreeAsync(h->d_units, 0));
        for (auto &p : h->allocs)
            if (p == (void *)h->d_units) p = nullptr;
    }
    h->units_staged = false;
    h->device_bytes -= (int64_t)(std::max<size_t>(keep_units.size(), 1) * sizeof(Unit));
    h->d_units = nullptr;
    h->n_units = 0;  // the handle runs nothing until a unit list is on the device again
    if ((st = upload(h, &h->d_units, h->units)) != SQA_OK) {
        h->d_units = nullptr;
        return st;
    }
    h->n_units = (int)h->units.size();
    set_tieq(h);
    return SQA_OK;
}

sqa_status sqa_get_launch(const sqa_handle *h, int32_t *words_per_unit, int32_t *use_table, int32_t *smem_bytes,
                          int32_t *cluster)
{
    if (!h) return set_error("NULL handle"), SQA_ERR_INVALID;
    if (words_per_unit) *words_per_unit = h->job.wc;
    if (use_table) *use_table = h->job.use_lut;
    if (smem_bytes) *smem_bytes = h->job.smem_bytes;
    if (cluster) *cluster = h->job.csize;
    return SQA_OK;
}

sqa_status sqa_tune_slices(sqa_handle *h, int32_t slices)
{
    const sqa_status us = usable(h);
    if (us != SQA_OK) return us;
    if (slices < 0 || slices > kTaskSlices) return set_error("slices per task: 0..4"), SQA_ERR_INVALID;
    h->force_slices = slices;
    h->job.task_slices = slices;
    return SQA_OK;
}

sqa_status sqa_get_task_slices(const sqa_handle *h, int32_t *slices)
{
    if (!h || !slices) return set_error("NULL argument"), SQA_ERR_INVALID;
    *slices = h->job.task_slices;
    return SQA_OK;
}

sqa_status sqa_run_sweeps(sqa_handle *h, int32_t t0, int32_t t1, void *stream)
{
    NvtxScope nvtx_("sqa_run_sweeps");
    sqa_status us = usable(h);
    if (us != SQA_OK) return us;
    if (t0 < 0 || t1 < t0 || t1 > h->S) return set_error("sweep range"), SQA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    sqa_status st;
    if (t0 == 0 && (st = launch_init(h, s)) != SQA_OK) return st;
    if (t1 > t0) return launch_sweeps(h, t0, t1, 0, h->n_units, s);
    return SQA_OK;
}

sqa_status sqa_run(sqa_handle *h, void *stream)
{
    if (!h) return set_error("NULL handle"), SQA_ERR_INVALID;
    return sqa_run_sweeps(h, 0, h->S, stream);
}

sqa_status sqa_run_per_instance(sqa_handle *h, void *stream)
{
    NvtxScope nvtx_("sqa_run_per_instance");
    sqa_status us = usable(h);
    if (us != SQA_OK) return us;
    cudaStream_t s = (cudaStream_t)stream;
    sqa_status st;
    if ((st = launch_init(h, s)) != SQA_OK) return st;
    int u = 0;
    while (u < h->n_units) {
        int v = u;
        while (v < h->n_units && h->units[v].inst == h->units[u].inst) v++;
        if ((st = launch_sweeps(h, 0, h->S, u, v - u, s)) != SQA_OK) return st;
        u = v;
    }
    return SQA_OK;
}

sqa_status pt_run(sqa_handle *h, const double *betas, int32_t n_temps, int32_t n_sweeps,
                  int32_t swap_every, void *stream)
{
    NvtxScope nvtx_("pt_run");
    if (!h || !betas || n_temps < 1 || n_sweeps < 1 || swap_every < 1)
        return set_error("pt_run arguments"), SQA_ERR_INVALID;
    for (int p = 0; p < n_temps; p++)
        if (!(betas[p] > 0) || !isfinite(betas[p])) return set_error("betas must be > 0"), SQA_ERR_INVALID;
    for (int p = 0; p + 1 < n_temps; p++)
        if (!(betas[p] > betas[p + 1])) return set_error("betas must decrease"), SQA_ERR_INVALID;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "pt_run");
    h->kind = SQA_KIND_PT;
    h->P = n_temps;
    h->betas.assign(betas, betas + n_temps);
    h->S = n_sweeps;
    h->swap_every = swap_every;
    sqa_status st = setup_program(h);
    if (st != SQA_OK) return st;
    return sqa_run(h, stream);
}

sqa_status sqa_batch_run(sqa_handle *const *hs, int32_t n, void *stream)
{
    NvtxScope nvtx_("sqa_batch_run");
    if (!hs || n < 1) return set_error("batch arguments"), SQA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<JobDev> jobs;
    std::vector<Unit> units;
    sqa_status st;
    for (int k = 0; k < n; k++) {
        sqa_handle *h = hs[k];
        if ((st = usable(h)) != SQA_OK) return st;
        if ((st = launch_init(h, s)) != SQA_OK) return st;
        // the multi-job kernel runs every unit in one block: plan each job
        // for a single block per unit
        JobDev J = h->job;
        std::vector<Unit> ju;
        if ((st = plan_shape(h, 1, J, ju, false)) != SQA_OK) return st;
        J.t0 = 0;
        J.t1 = h->S;
        jobs.push_back(J);
        for (Unit u : ju) {
            u.job = k;
            units.push_back(u);
        }
    }
    std::vector<MultiGroup> groups;
    const int rows = group_units(jobs, units, groups);
    JobDev *d_jobs = nullptr;
    Unit *d_units = nullptr;
    int *d_counter = nullptr;
    uint2 *d_tieq = nullptr;
    int stride = 1;
    for (const JobDev &J : jobs) stride = std::max(stride, tie_items(J, J.wc));
    cudaError_t e = cudaMallocAsync((void **)&d_tieq, (size_t)rows * stride * sizeof(uint2), s);
    assign_tieq(jobs, groups, d_tieq, stride);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_jobs, jobs.size() * sizeof(JobDev), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_units, units.size() * sizeof(Unit), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_counter, kMaxModes * sizeof(int), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(JobDev), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_groups(groups, d_jobs, d_units, d_counter, s);
    // freed in stream order after the launch (or at once on an error); host
    // vectors are consumed: pageable copies are staged before return
    if (d_tieq) cudaFreeAsync(d_tieq, s);
    if (d_jobs) cudaFreeAsync(d_jobs, s);
    if (d_units) cudaFreeAsync(d_units, s);
    if (d_counter) cudaFreeAsync(d_counter, s);
    if (e != cudaSuccess) return cuda_fail(e, "sqa_batch_run");
    return SQA_OK;
}

static sqa_status to_out(void *dst, const void *dev_src, size_t bytes, int out_is_device, cudaStream_t s)
{
    SQA_CUDA(cudaMemcpyAsync(dst, dev_src, bytes, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!out_is_device) SQA_CUDA(cudaStreamSynchronize(s));
    return SQA_OK;
}

static sqa_status canon_out(sqa_handle *h, int z0, int zc, uint32_t *out, int out_is_device, void *stream)
{
    sqa_status us = usable(h);
    if (us != SQA_OK) return us;
    if (!out) return set_error("NULL argument"), SQA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t count = (size_t)h->I * zc * h->job.n_phys * h->job.W;
    uint32_t *dst = out;
    if (!out_is_device) SQA_CUDA(cudaMallocAsync((void **)&dst, count * 4, s));
    const int blocks = (int)std::min<size_t>((count + kThreads - 1) / kThreads, 8192);
    canon_kernel<<<std::max(blocks, 1), kThreads, 0, s>>>(h->job, h->d_compact, z0, zc, dst);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        if (!out_is_device) cudaFreeAsync(dst, s);
        return cuda_fail(e, "canon_kernel");
    }
    if (!out_is_device) {
        sqa_status st = to_out(out, dst, count * 4, 0, s);
        cudaFreeAsync(dst, s);
        return st;
    }
    return SQA_OK;
}

sqa_status sqa_readout(sqa_handle *h, uint32_t *out, int32_t out_is_device, void *stream)
{
    NvtxScope nvtx_("sqa_readout");
    return canon_out(h, 0, 1, out, out_is_device, stream);
}

sqa_status sqa_state(sqa_handle *h, uint32_t *out, int32_t out_is_device, void *stream)
{
    if (!h) return set_error("NULL handle"), SQA_ERR_INVALID;
    return canon_out(h, 0, h->job.Z, out, out_is_device, stream);
}

sqa_status sqa_energies(sqa_handle *h, int32_t *out, int32_t out_is_device, void *stream)
{
    NvtxScope nvtx_("sqa_energies");
    sqa_status us = usable(h);
    if (us != SQA_OK) return us;
    if (!out) return set_error("NULL argument"), SQA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t count = (size_t)h->I * h->job.Z * h->R;
    int32_t *dst = out;
    if (!out_is_device) SQA_CUDA(cudaMallocAsync((void **)&dst, count * 4, s));
    const int blocks = (int)std::min<size_t>((count + kThreads - 1) / kThreads, 8192);
    energy_kernel<<<std::max(blocks, 1), kThreads, 0, s>>>(h->job, dst);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        if (!out_is_device) cudaFreeAsync(dst, s);
        return cuda_fail(e, "energy_kernel");
    }
    if (!out_is_device) {
        sqa_status st = to_out(out, dst, count * 4, 0, s);
        cudaFreeAsync(dst, s);
        return st;
    }
    return SQA_OK;
}

static sqa_status decode_impl(sqa_handle *h, int32_t method, int32_t n_trees, double bp_error, int32_t bp_iters,
                              int8_t *logical_out, int64_t *energy_out, const int64_t *e_ground,
                              int32_t *success_out, int32_t out_is_device, void *stream);

sqa_status sqa_decode(sqa_handle *h, int32_t method, int32_t n_trees, int8_t *logical_out,
                      int64_t *energy_out, const int64_t *e_ground, int32_t *success_out,
                      int32_t out_is_device, void *stream)
{
    return decode_impl(h, method, n_trees, 0.2, 10, logical_out, energy_out, e_ground, success_out, out_is_device,
                       stream);
}

sqa_status sqa_decode_bp(sqa_handle *h, double error_rate, int32_t iterations, int8_t *logical_out,
                         int64_t *energy_out, const int64_t *e_ground, int32_t *success_out,
                         int32_t out_is_device, void *stream)
{
    if (!(error_rate > 0.0 && error_rate <= 0.5) || iterations < 0)
        return set_error("error_rate in (0, 1/2], iterations >= 0"), SQA_ERR_INVALID;
    return decode_impl(h, SQA_DECODE_LHZ_BP, 1, error_rate, iterations, logical_out, energy_out, e_ground,
                       success_out, out_is_device, stream);
}

static sqa_status decode_impl(sqa_handle *h, int32_t method, int32_t n_trees, double bp_error, int32_t bp_iters,
                              int8_t *logical_out, int64_t *energy_out, const int64_t *e_ground,
                              int32_t *success_out, int32_t out_is_device, void *stream)
{
    NvtxScope nvtx_("sqa_decode");
    const sqa_status us = usable(h);
    if (us != SQA_OK) return us;
    const bool me = h->emb == SQA_EMB_ME_CHIMERA;
    if (me != (method == SQA_DECODE_ME_MV) ||
        (method < SQA_DECODE_ME_MV || method > SQA_DECODE_LHZ_BP))
        return set_error("decode method does not match the embedding"), SQA_ERR_INVALID;
    if (method == SQA_DECODE_LHZ_BP && h->N > 32)
        return set_error("belief-propagation decoding keeps pair rows as 32-bit masks: N <= 32"),
               SQA_ERR_UNSUPPORTED;
    if (method == SQA_DECODE_LHZ_MWD && h->N > 24)
        return set_error("minimum-weight decoding enumerates 2^(N-1) states: N <= 24"), SQA_ERR_UNSUPPORTED;
    if (method == SQA_DECODE_LHZ_TREES) {
        if (n_trees == 0) {
            n_trees = (h->N + 3) / 4 + 1;
            if (n_trees % 2 == 0) n_trees++;
        }
        if (n_trees < 1 || n_trees > 1024) return set_error("n_trees"), SQA_ERR_INVALID;
    } else {
        n_trees = 1;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sqa_status st;
    // belief propagation reads out with random tree 0
    const int tree_method = method == SQA_DECODE_LHZ_BP ? SQA_DECODE_LHZ_TREES : method;
    if (method == SQA_DECODE_LHZ_BP) n_trees = 1;
    if (!me && method != SQA_DECODE_LHZ_MWD && (st = decode_trees(h, tree_method, n_trees)) != SQA_OK) return st;
    const size_t nrep = (size_t)h->I * h->R;
    DecodeArgs D{};
    D.method = method;
    D.N = h->N;
    D.n_trees = n_trees;
    D.Lc = h->plan.Lc;
    D.chain = h->d_chain;
    D.pair = h->d_pair;
    D.parents = h->d_parents;
    D.orders = h->d_orders;
    D.J = h->d_J;
    D.bp_iters = bp_iters;
    if (method == SQA_DECODE_LHZ_BP) {
        // decisions of sign(L0 s + L2 S) for s = +-1, S = -(N-2) .. N-2,
        // evaluated in double on the host: 0 on an exact tie (keep the value)
        const double e = bp_error;
        const double L0 = log((1.0 - e) / e);
        const double L2 = log(((1.0 - e) * (1.0 - e) + e * e) / (2.0 * e * (1.0 - e)));
        for (int neg = 0; neg < 2; neg++)
            for (int S = -(h->N - 2); S <= h->N - 2; S++) {
                const double d = L0 * (double)(neg ? -1 : 1) + L2 * (double)S;
                D.bp_dec[neg][S + h->N - 2] = (int8_t)(d > 0.0 ? 1 : (d < 0.0 ? -1 : 0));
            }
    }
    // temporaries, freed in stream order on every return
    struct Temps {
        cudaStream_t s;
        void *p[4];
        int n;
        ~Temps()
        {
            for (int i = 0; i < n; i++) cudaFreeAsync(p[i], s);
        }
    } tmp{s, {}, 0};
    auto temp = [&](void **ptr, size_t bytes) {
        const cudaError_t e = cudaMallocAsync(ptr, bytes, s);
        if (e == cudaSuccess) tmp.p[tmp.n++] = *ptr;
        return e;
    };
    int8_t *d_log = logical_out;
    int64_t *d_en = energy_out, *d_eg = nullptr;
    int32_t *d_succ = success_out;
    if (!out_is_device) {
        if (logical_out) SQA_CUDA(temp((void **)&d_log, nrep * h->N));
        if (energy_out) SQA_CUDA(temp((void **)&d_en, nrep * 8));
        if (success_out) SQA_CUDA(temp((void **)&d_succ, (size_t)h->I * 4));
    }
    if (e_ground) {
        SQA_CUDA(temp((void **)&d_eg, (size_t)h->I * 8));
        SQA_CUDA(cudaMemcpyAsync(d_eg, e_ground, (size_t)h->I * 8, cudaMemcpyHostToDevice, s));
    }
    if (d_succ) SQA_CUDA(cudaMemsetAsync(d_succ, 0, (size_t)h->I * 4, s));
    D.logical = d_log;
    D.energy = d_en;
    D.e_ground = d_eg;
    D.success = e_ground ? d_succ : nullptr;
    const int blocks = (int)std::min<size_t>((nrep + 127) / 128, 8192);
    decode_kernel<<<std::max(blocks, 1), 128, 0, s>>>(h->job, D);
    SQA_CUDA(cudaGetLastError());
    if (!out_is_device) {
        if (logical_out) SQA_CUDA(cudaMemcpyAsync(logical_out, d_log, nrep * h->N, cudaMemcpyDeviceToHost, s));
        if (energy_out) SQA_CUDA(cudaMemcpyAsync(energy_out, d_en, nrep * 8, cudaMemcpyDeviceToHost, s));
        if (success_out) SQA_CUDA(cudaMemcpyAsync(success_out, d_succ, (size_t)h->I * 4, cudaMemcpyDeviceToHost, s));
        SQA_CUDA(cudaStreamSynchronize(s));
    }
    return SQA_OK;
}

sqa_status sqa_ground_energy(int32_t N, int32_t n_instances, const int32_t *J, int64_t *e_out)
{
    NvtxScope nvtx_("sqa_ground_energy");
    if (N < 2 || N > 40 || n_instances < 1 || !J || !e_out) return set_error("ground arguments"), SQA_ERR_INVALID;
    // a bound on the search's work: one call enumerates at most 2^40 states
    // in all (a few seconds), so no call can hold the device for hours
    if ((double)n_instances * std::ldexp(1.0, N - 1) > std::ldexp(1.0, 40))
        return set_error("sqa_ground_energy: n_instances * 2^(N-1) exceeds the search budget of 2^40 states"),
               SQA_ERR_UNSUPPORTED;
    sqa_status st = device_ready();
    if (st != SQA_OK) return st;
    const size_t npair = (size_t)N * (N - 1) / 2;
    int32_t *dJ = nullptr;
    unsigned long long *dbest = nullptr;
    SQA_CUDA(cudaMalloc(&dJ, npair * n_instances * 4));
    cudaError_t e = cudaMalloc(&dbest, (size_t)n_instances * 8);
    if (e != cudaSuccess) {
        cudaFree(dJ);
        return cuda_fail(e, "cudaMalloc");
    }
    e = cudaMemcpy(dJ, J, npair * n_instances * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dbest, 0xFF, (size_t)n_instances * 8);
    const int total_bits = N - 1;
    const int chunk_bits = std::max(0, std::min(total_bits, total_bits - 17));
    const int64_t n_chunks = (int64_t)1 << (total_bits - chunk_bits);
    const int bx = (int)std::min<int64_t>((n_chunks + 127) / 128, 2048);
    if (e == cudaSuccess) {
        ground_kernel<<<dim3(std::max(bx, 1), n_instances), 128>>>(N, dJ, chunk_bits, n_chunks, dbest);
        e = cudaGetLastError();
    }
    std::vector<unsigned long long> best(n_instances);
    if (e == cudaSuccess) e = cudaMemcpy(best.data(), dbest, (size_t)n_instances * 8, cudaMemcpyDeviceToHost);
    cudaFree(dJ);
    cudaFree(dbest);
    if (e != cudaSuccess) return cuda_fail(e, "ground_kernel");
    for (int i = 0; i < n_instances; i++) e_out[i] = (int64_t)(best[i] ^ 0x8000000000000000ull);
    return SQA_OK;
}

sqa_status sqa_plan_terms(int32_t embedding, int32_t N, const int32_t *J, int32_t penalty,
                          int32_t cap_terms, int32_t *n_phys, int32_t *n_terms,
                          int32_t *term_size, int32_t *term_mem, int32_t *term_w,
                          int32_t *colour)
{
    if (N < 2 || N > kMaxN || !J || !n_phys || !n_terms) return set_error("plan_terms arguments"), SQA_ERR_INVALID;
    Plan pl;
    std::string err;
    if (!build_plan(embedding, N, pl, err)) return set_error(err), SQA_ERR_INVALID;
    *n_phys = pl.n_phys;
    *n_terms = (int32_t)pl.terms.size();
    if ((int)pl.terms.size() > cap_terms) return set_error("cap_terms too small"), SQA_ERR_INVALID;
    for (size_t t = 0; t < pl.terms.size(); t++) {
        const PlanTerm &x = pl.terms[t];
        if (term_size) term_size[t] = x.size;
        if (term_mem)
            for (int k = 0; k < 4; k++) term_mem[t * 4 + k] = k < x.size ? x.mem[k] : -1;
        if (term_w) term_w[t] = x.jidx >= 0 ? J[x.jidx] : -penalty;
    }
    if (colour) {
        for (int s = 0; s < pl.n_phys; s++) colour[s] = -1;
        for (int c = 0; c < pl.ncol; c++)
            for (int i = pl.col_ptr[c]; i < pl.col_ptr[c + 1]; i++) colour[pl.canon[i]] = c;
    }
    return SQA_OK;
}

int64_t sqa_plan_device_bytes(const sqa_desc *d) { return estimate_device_bytes(d); }

sqa_status sqa_plan_tables(const sqa_desc *d, uint32_t *T, int64_t cap, int32_t *dmin_out,
                           int32_t *dmax_out)
{
    sqa_status st = validate(d);
    if (st != SQA_OK) return st;
    Plan pl;
    std::string err;
    if (!build_plan(d->embedding, d->n_logical, pl, err)) return set_error(err), SQA_ERR_INVALID;
    const int npair = d->n_logical * (d->n_logical - 1) / 2;
    int smax = 0;
    for (int i = 0; i < d->n_instances; i++)
        smax = std::max(smax, site_weight_sum_max(pl, d->J + (size_t)i * npair, d->penalty));
    const int dmin = -2 * smax, dmax = 2 * smax;
    std::vector<uint32_t> tab;
    if (d->kind == SQA_KIND_SQA) {
        std::vector<double> A(d->n_sweeps), B(d->n_sweeps);
        for (int t = 0; t < d->n_sweeps; t++) {
            const double s = ((double)t + 0.5) / (double)d->n_sweeps;
            A[t] = d->A ? d->A[t] : 1.0 - s;
            B[t] = d->B ? d->B[t] : s;
        }
        sqa_tables(A.data(), B.data(), d->beta, d->n_slices, d->n_sweeps, dmin, dmax, tab);
    } else {
        pt_tables(d->betas, d->n_temps, dmin, dmax, tab);
    }
    if (dmin_out) *dmin_out = dmin;
    if (dmax_out) *dmax_out = dmax;
    if (!T) return SQA_OK;
    if ((int64_t)tab.size() > cap) return set_error("cap too small"), SQA_ERR_INVALID;
    memcpy(T, tab.data(), tab.size() * 4);
    return SQA_OK;
}

sqa_status sqa_plan_wolff_tables(const sqa_desc *d, uint32_t *Tb, int32_t *acc_off, int32_t *acc_len,
                                 uint32_t *Tacc, int64_t cap, int64_t *n_acc)
{
    sqa_status st = validate(d);
    if (st != SQA_OK) return st;
    if (d->kind != SQA_KIND_SQA) return set_error("cluster moves are SQA only"), SQA_ERR_INVALID;
    Plan pl;
    std::string err;
    if (!build_plan(d->embedding, d->n_logical, pl, err)) return set_error(err), SQA_ERR_INVALID;
    const int npair = d->n_logical * (d->n_logical - 1) / 2;
    int smax = 0;
    for (int i = 0; i < d->n_instances; i++)
        smax = std::max(smax, site_weight_sum_max(pl, d->J + (size_t)i * npair, d->penalty));
    std::vector<double> A(d->n_sweeps), B(d->n_sweeps);
    for (int t = 0; t < d->n_sweeps; t++) {
        const double s = ((double)t + 0.5) / (double)d->n_sweeps;
        A[t] = d->A ? d->A[t] : 1.0 - s;
        B[t] = d->B ? d->B[t] : s;
    }
    std::vector<uint32_t> tb, tacc;
    std::vector<int> off, len;
    wolff_tables(A.data(), B.data(), d->beta, d->n_slices, d->n_sweeps, 2 * smax, tb, tacc, off, len);
    int64_t total = 0;
    for (int x : len) total += x;
    if (n_acc) *n_acc = total;
    if (Tb) memcpy(Tb, tb.data(), tb.size() * 4);
    if (acc_off) memcpy(acc_off, off.data(), off.size() * 4);
    if (acc_len) memcpy(acc_len, len.data(), len.size() * 4);
    if (Tacc) {
        if (total > cap) return set_error("cap too small"), SQA_ERR_INVALID;
        memcpy(Tacc, tacc.data(), (size_t)total * 4);
    }
    return SQA_OK;
}

sqa_status sqa_plan_swap_table(const double *betas, int32_t n_temps, int32_t pair, uint32_t *out,
                               int32_t cap, int32_t *len)
{
    if (!betas || n_temps < 2 || pair < 0 || pair + 1 >= n_temps || !len) return set_error("swap table arguments"), SQA_ERR_INVALID;
    std::vector<uint32_t> T;
    std::vector<int> off, ln;
    swap_tables(betas, n_temps, T, off, ln);
    *len = ln[pair];
    if (!out) return SQA_OK;
    if (ln[pair] > cap) return set_error("cap too small"), SQA_ERR_INVALID;
    memcpy(out, T.data() + off[pair], (size_t)ln[pair] * 4);
    return SQA_OK;
}

sqa_status sqa_plan_tree(int32_t N, uint64_t seed, int32_t inst, int32_t tree, int32_t *parent)
{
    if (N < 2 || N > kMaxN || !parent || inst < 0 || tree < 0) return set_error("tree arguments"), SQA_ERR_INVALID;
    std::vector<int> order(N), par(N);
    prufer_tree(N, seed, inst, tree, par.data(), order.data());
    for (int v = 0; v < N; v++) parent[v] = par[v];
    return SQA_OK;
}

}  // extern "C"
