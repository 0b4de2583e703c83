// Kernels of the SQA / PT hot path (arXiv:1603.03755), sm_103a.
//
// Data layout.  Spins are bits (1 <-> sigma = -1); one 32-bit word holds 32
// independent replicas of one (site, slice).  Global state is
// [instance][z][site][word] with sites in compact order (used sites sorted by
// graph colour), z the Trotter slice (SQA) or temperature slot (PT).
//
// Work.  A unit is a run of words of one instance; replicas in different
// words never interact, so a unit is an independent system.  The persistent
// sweep kernel pulls units from a global counter, stages the unit's state,
// its site records and its threshold rows in shared memory, runs every sweep
// of the launch there and writes the state back.  Within a sweep the colour
// classes (SQA: colour x slice parity; PT: colour) run in order with a block
// barrier between them; all items of a class are independent.
//
// Per item (site, z, word) the kernel forms, for each term of the site, the
// word of replicas whose term value is negative (XOR of the members' words,
// inverted for negative weights).  Four replicas at a time (bits j, j+8,
// j+16, j+24) it then sums the weighted term bits and the temporal
// disagreements byte-wise into the site's window of the threshold row,
// loads the four thresholds and compares them with the high 16 bits of the
// replicas' uniforms; only when those bits tie with the threshold's high
// half is the low half drawn (probability 2^-16).
#include <cuda_runtime.h>
#include <stdint.h>

#include "philox.cuh"
#include "sqa_internal.h"

namespace sqa {

__device__ __forceinline__ uint32_t valid_bits(int R, int gw)
{
    const int left = R - 32 * gw;
    return left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
}

__device__ __forceinline__ uint32_t bytes4(uint32_t v, int j) { return (v >> j) & 0x01010101u; }

__device__ __forceinline__ U4 pick4(const U4 &a, const U4 &b, const U4 &c, const U4 &d, int r)
{
    return r == 0 ? a : (r == 1 ? b : (r == 2 ? c : d));
}

// ---------------------------------------------------------------------------
// Initial spins: bit (r % 32) of word (r/32) % 4 of the INIT stream at
// counter (canonical site, z, r/128, instance).
// ---------------------------------------------------------------------------
__global__ void init_kernel(JobDev J, const int *canon)
{
    const int64_t total = (int64_t)J.n_inst * J.Z * J.n * J.W;
    const uint32_t k1 = J.key_hi ^ kDomSweepHi ^ kDomInit;  // seed_hi ^ kDomInit
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int gw = (int)(i % J.W);
        int64_t r = i / J.W;
        const int si = (int)(r % J.n);
        r /= J.n;
        const int z = (int)(r % J.Z);
        const int inst = (int)(r / J.Z);
        const U4 v = philox((uint32_t)canon[si], (uint32_t)z, (uint32_t)(gw >> 2), (uint32_t)inst,
                            J.seed_lo, k1);
        J.state[i] = word_of(v, gw & 3) & valid_bits(J.R, gw);
    }
}

// ---------------------------------------------------------------------------
// The persistent sweep kernel.
// ---------------------------------------------------------------------------
struct Smem {
    uint32_t *S;      // [Z][zstride]
    uint32_t *T;      // SQA: one row; PT: P rows
    SiteRec *sites;   // [n]
    int32_t *E;       // PT: [P][wc*32]
    uint32_t *M;      // PT: swap masks [P/2+1][wc]
};

__device__ __forceinline__ Smem carve(const JobDev &J, unsigned char *base)
{
    Smem m;
    size_t off = 0;
    m.S = (uint32_t *)(base + off);
    off += (size_t)J.Z * J.zstride * 4;
    m.T = (uint32_t *)(base + off);
    off += (size_t)(J.kind == SQA_KIND_SQA ? J.nrow : J.Z * J.nrow) * 4;
    off = (off + 15) & ~(size_t)15;
    m.sites = (SiteRec *)(base + off);
    off += (size_t)J.n * sizeof(SiteRec);
    m.E = (int32_t *)(base + off);
    m.M = nullptr;
    if (J.kind == SQA_KIND_PT) {
        off += (size_t)J.Z * J.wc * 32 * 4;
        m.M = (uint32_t *)(base + off);
    }
    return m;
}

// Term planes of one item: pl[k] has bit b set when term k's value is
// negative for replica b; kw[k] is K * |w_k|.
__device__ __forceinline__ void term_planes(const SiteRec &sr, const uint32_t *row, int wc, int w,
                                            uint32_t s, uint32_t (&pl)[kMaxTerms],
                                            uint32_t (&kw)[kMaxTerms])
{
#pragma unroll
    for (int k = 0; k < kMaxTerms; k++) {
        pl[k] = 0u;
        kw[k] = 0u;
        if (k < sr.nterm) {
            const TermRec tr = sr.t[k];
            uint32_t p = s;
            if (tr.p[0] >= 0) p ^= row[tr.p[0] * wc + w];
            if (tr.p[1] >= 0) p ^= row[tr.p[1] * wc + w];
            if (tr.p[2] >= 0) p ^= row[tr.p[2] * wc + w];
            const int wv = tr.w;
            // value w * prod(sigma) is negative iff (product is -1) xor (w < 0)
            const uint32_t neg = (uint32_t)(wv >> 31);
            pl[k] = p ^ neg;
            kw[k] = (uint32_t)(wv < 0 ? -wv : wv);
        }
    }
}

// Byte-wise window offsets of replicas (j, j+8, j+16, j+24).  A term whose
// value is negative turns positive on a flip: it raises delta by 2|w|, which
// is K*|w|/... in row units; see build_sites.
template <int KIND>
__device__ __forceinline__ uint32_t window4(const uint32_t (&pl)[kMaxTerms],
                                            const uint32_t (&kw)[kMaxTerms], uint32_t d1,
                                            uint32_t d2, int j)
{
    uint32_t a = KIND == SQA_KIND_SQA ? 0x02020202u : 0u;
#pragma unroll
    for (int k = 0; k < kMaxTerms; k++) a += kw[k] * bytes4(pl[k], j);
    if (KIND == SQA_KIND_SQA) a -= bytes4(d1, j) + bytes4(d2, j);
    return a;
}

template <int KIND>
__device__ __forceinline__ void sweep_item(const JobDev &J, const Smem &sm, int inst, int w0, int wc,
                                           int t, int si, int z, int w)
{
    const SiteRec &sr = sm.sites[si];
    uint32_t *row = sm.S + (size_t)z * J.zstride;
    const uint32_t s = row[si * wc + w];
    uint32_t d1 = 0u, d2 = 0u;
    const int Z = J.Z;
    if (KIND == SQA_KIND_SQA) {
        const int zu = z == 0 ? Z - 1 : z - 1;
        const int zd = z == Z - 1 ? 0 : z + 1;
        // a temporal neighbour that disagrees lowers m by 2: m = 2 - 2*tc
        d1 = s ^ sm.S[(size_t)zu * J.zstride + si * wc + w];
        d2 = s ^ sm.S[(size_t)zd * J.zstride + si * wc + w];
    }
    uint32_t pl[kMaxTerms], kw[kMaxTerms];
    term_planes(sr, row, wc, w, s, pl, kw);

    const int gw = w0 + w;
    const uint32_t slot = (uint32_t)(sr.canon * Z + z);
    const uint32_t g0 = (uint32_t)gw * 4u;
    const U4 A0 = philox((uint32_t)t, slot, g0 + 0u, (uint32_t)inst, J.seed_lo, J.key_hi);
    const U4 A1 = philox((uint32_t)t, slot, g0 + 1u, (uint32_t)inst, J.seed_lo, J.key_hi);
    const U4 A2 = philox((uint32_t)t, slot, g0 + 2u, (uint32_t)inst, J.seed_lo, J.key_hi);
    const U4 A3 = philox((uint32_t)t, slot, g0 + 3u, (uint32_t)inst, J.seed_lo, J.key_hi);
    const uint32_t *Trow = KIND == SQA_KIND_SQA ? sm.T : sm.T + (size_t)z * J.nrow;
    const int base = sr.base;

    uint32_t acc = 0u, tie = 0u;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t a = window4<KIND>(pl, kw, d1, d2, j);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const uint32_t T = Trow[base + ((a >> (8 * r)) & 0xFFu)];
            const U4 &Ar = r == 0 ? A0 : (r == 1 ? A1 : (r == 2 ? A2 : A3));
            const uint32_t aw = word_of(Ar, j >> 1);
            const uint32_t uh = (j & 1) ? (aw & 0xFFFF0000u) : (aw << 16);
            const uint32_t bit = 1u << (j + 8 * r);
            if ((uh | 0xFFFFu) < T) acc |= bit;           // high half decides: accept
            if ((uh ^ T) < 0x10000u) tie |= bit;          // high halves equal: undecided
        }
    }
    while (tie) {
        const int b = __ffs(tie) - 1;
        tie &= tie - 1u;
        const int j = b & 7, r = b >> 3;
        const U4 Br = philox((uint32_t)t, slot, g0 + (uint32_t)r, (uint32_t)inst, J.seed_lo, J.key_lo);
        const U4 Ar = pick4(A0, A1, A2, A3, r);
        const uint32_t sh = 16u * (uint32_t)(j & 1);
        uint32_t u = (((word_of(Ar, j >> 1) >> sh) & 0xFFFFu) << 16) | ((word_of(Br, j >> 1) >> sh) & 0xFFFFu);
        u = u < 0xFFFFFFFEu ? u : 0xFFFFFFFEu;
        const uint32_t a = window4<KIND>(pl, kw, d1, d2, j);
        const uint32_t T = Trow[base + ((a >> (8 * r)) & 0xFFu)];
        if (u < T)
            acc |= 1u << b;
        else
            acc &= ~(1u << b);
    }
    row[si * wc + w] = s ^ (acc & valid_bits(J.R, gw));
}

// PT: energies of every (slot, replica) of the unit, then the swap event.
__device__ void pt_swap(const JobDev &J, const Smem &sm, int inst, int w0, int wc, int e)
{
    const int P = J.Z, n = J.n;
    const ETerm *et = J.eterms + (size_t)inst * J.n_eterms;
    const int nthr = blockDim.x;
    __syncthreads();
    for (int it = threadIdx.x; it < P * wc * 32; it += nthr) {
        const int b = it & 31, r = it >> 5, w = r % wc, p = r / wc;
        const uint32_t *row = sm.S + (size_t)p * J.zstride;
        int32_t E = 0;
        for (int q = 0; q < J.n_eterms; q++) {
            const ETerm x = et[q];
            uint32_t v = row[x.m[0] * wc + w];
            if (x.size > 1) v ^= row[x.m[1] * wc + w];
            if (x.size > 2) v ^= row[x.m[2] * wc + w];
            if (x.size > 3) v ^= row[x.m[3] * wc + w];
            E += ((v >> b) & 1u) ? -x.w : x.w;
        }
        sm.E[(p * wc + w) * 32 + b] = E;
    }
    __syncthreads();
    const int p0 = e & 1;
    const int npairs = p0 + 1 < P ? (P - 1 - p0 + 1) / 2 : 0;
    for (int it = threadIdx.x; it < npairs * wc * 32; it += nthr) {
        const int b = it & 31, r = it >> 5, w = r % wc, k = r / wc;
        const int p = p0 + 2 * k;
        const int gw = w0 + w;
        const int rho = gw * 32 + b;
        const int dE = sm.E[((p + 1) * wc + w) * 32 + b] - sm.E[(p * wc + w) * 32 + b];
        bool accept = dE <= 0;
        if (!accept && dE <= J.sw_len[p]) {
            const U4 v = philox((uint32_t)e, (uint32_t)p, (uint32_t)(rho >> 2), (uint32_t)inst, J.seed_lo,
                                J.key_swap);
            accept = word_of(v, rho & 3) < J.Tsw[J.sw_off[p] + dE - 1];
        }
        const uint32_t M = __ballot_sync(0xFFFFFFFFu, accept) & valid_bits(J.R, gw);
        if (b == 0) sm.M[k * wc + w] = M;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < npairs * n * wc; it += nthr) {
        const int w = it % wc, r = it / wc, si = r % n, k = r / n;
        const int p = p0 + 2 * k;
        uint32_t *a = sm.S + (size_t)p * J.zstride + si * wc + w;
        uint32_t *c = sm.S + (size_t)(p + 1) * J.zstride + si * wc + w;
        const uint32_t d = (*a ^ *c) & sm.M[k * wc + w];
        *a ^= d;
        *c ^= d;
    }
    __syncthreads();
}

template <int KIND>
__device__ void run_unit(const JobDev &J, const Smem &sm, const Unit &u)
{
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int Z = J.Z, n = J.n, wc = u.wc, inst = u.inst, w0 = u.w0;
    // stage state and site records
    for (int i = tid; i < Z * n * wc; i += nthr) {
        const int w = i % wc, r = i / wc, si = r % n, z = r / n;
        sm.S[(size_t)z * J.zstride + si * wc + w] = J.state[(((size_t)inst * Z + z) * n + si) * J.W + w0 + w];
    }
    {
        const uint32_t *src = (const uint32_t *)(J.sites + (size_t)inst * n);
        uint32_t *dst = (uint32_t *)sm.sites;
        for (int i = tid; i < n * (int)(sizeof(SiteRec) / 4); i += nthr) dst[i] = src[i];
    }
    if (KIND == SQA_KIND_PT)
        for (int i = tid; i < Z * J.nrow; i += nthr) sm.T[i] = J.T[i];
    __syncthreads();

    for (int t = J.t0; t < J.t1; t++) {
        if (KIND == SQA_KIND_SQA) {
            for (int i = tid; i < J.nrow; i += nthr) sm.T[i] = __ldg(J.T + (size_t)t * J.nrow + i);
            __syncthreads();
            const int half = Z >> 1;
            for (int cls = 0; cls < 2 * J.ncol; cls++) {
                const int chi = cls >> 1, par = cls & 1;
                const int c0 = J.col_ptr[chi];
                const int nitems = (J.col_ptr[chi + 1] - c0) * half * wc;
                for (int it = tid; it < nitems; it += nthr) {
                    const int w = it % wc, r = it / wc, zh = r % half, si = c0 + r / half;
                    sweep_item<SQA_KIND_SQA>(J, sm, inst, w0, wc, t, si, 2 * zh + par, w);
                }
                __syncthreads();
            }
        } else {
            for (int chi = 0; chi < J.ncol; chi++) {
                const int c0 = J.col_ptr[chi];
                const int nitems = (J.col_ptr[chi + 1] - c0) * Z * wc;
                for (int it = tid; it < nitems; it += nthr) {
                    const int w = it % wc, r = it / wc, p = r % Z, si = c0 + r / Z;
                    sweep_item<SQA_KIND_PT>(J, sm, inst, w0, wc, t, si, p, w);
                }
                __syncthreads();
            }
            if (Z > 1 && (t + 1) % J.swap_every == 0) pt_swap(J, sm, inst, w0, wc, (t + 1) / J.swap_every - 1);
        }
    }
    for (int i = tid; i < Z * n * wc; i += nthr) {
        const int w = i % wc, r = i / wc, si = r % n, z = r / n;
        J.state[(((size_t)inst * Z + z) * n + si) * J.W + w0 + w] = sm.S[(size_t)z * J.zstride + si * wc + w];
    }
}

__global__ void __launch_bounds__(256) sweep_kernel(const JobDev *jobs, const Unit *units, int n_units,
                                                    int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_unit;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int ui = s_unit;
        __syncthreads();
        if (ui >= n_units) break;
        const Unit u = units[ui];
        const JobDev &J = jobs[u.job];
        const Smem sm = carve(J, smem_raw);
        if (J.kind == SQA_KIND_SQA)
            run_unit<SQA_KIND_SQA>(J, sm, u);
        else
            run_unit<SQA_KIND_PT>(J, sm, u);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Energies E_P of every (instance, z, replica): sum of w * prod(sigma).
// ---------------------------------------------------------------------------
__global__ void energy_kernel(JobDev J, int32_t *out)
{
    const int64_t total = (int64_t)J.n_inst * J.Z * J.R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int rho = (int)(i % J.R);
        const int64_t r = i / J.R;
        const int z = (int)(r % J.Z), inst = (int)(r / J.Z);
        const int gw = rho >> 5, b = rho & 31;
        const uint32_t *st = J.state + ((size_t)inst * J.Z + z) * J.n * J.W;
        const ETerm *et = J.eterms + (size_t)inst * J.n_eterms;
        int32_t E = 0;
        for (int q = 0; q < J.n_eterms; q++) {
            const ETerm x = et[q];
            uint32_t v = 0u;
            for (int k = 0; k < x.size; k++) v ^= st[(size_t)x.m[k] * J.W + gw];
            E += ((v >> b) & 1u) ? -x.w : x.w;
        }
        out[i] = E;
    }
}

// State in canonical site order: out [I][zcount][n_phys][W] from slices
// z0 .. z0+zcount-1; unused sites read 0.
__global__ void canon_kernel(JobDev J, const int *compact_of, int z0, int zcount, uint32_t *out)
{
    const int64_t total = (int64_t)J.n_inst * zcount * J.n_phys * J.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int gw = (int)(i % J.W);
        int64_t r = i / J.W;
        const int ph = (int)(r % J.n_phys);
        r /= J.n_phys;
        const int zz = (int)(r % zcount), inst = (int)(r / zcount);
        const int si = compact_of[ph];
        out[i] = si < 0 ? 0u : J.state[(((size_t)inst * J.Z + z0 + zz) * J.n + si) * J.W + gw];
    }
}

// ---------------------------------------------------------------------------
// Decoding of the readout slice (z = 0) of every (instance, replica).
// ---------------------------------------------------------------------------
__global__ void decode_kernel(JobDev J, DecodeArgs D)
{
    const int64_t total = (int64_t)J.n_inst * J.R;
    const int N = D.N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int rho = (int)(i % J.R), inst = (int)(i / J.R);
        const int gw = rho >> 5, b = rho & 31;
        const uint32_t *st = J.state + (size_t)inst * J.Z * J.n * J.W;  // z = 0
        auto sig = [&](int si) -> int { return ((st[(size_t)si * J.W + gw] >> b) & 1u) ? -1 : 1; };
        int8_t q[kMaxN];
        if (D.method == SQA_DECODE_ME_MV) {
            const int len = D.Lc + 1;
            for (int l = 0; l < N; l++) {
                int sum = 0;
                for (int k = 0; k < len; k++) sum += sig(D.chain[l * len + k]);
                q[l] = (int8_t)(sum > 0 ? 1 : (sum < 0 ? -1 : sig(D.chain[l * len])));
            }
        } else {
            int votes[kMaxN];
            int8_t first[kMaxN];
            for (int l = 0; l < N; l++) votes[l] = 0;
            for (int tr = 0; tr < D.n_trees; tr++) {
                const int *par = D.parents + ((size_t)inst * D.n_trees + tr) * N;
                const int *ord = D.orders + ((size_t)inst * D.n_trees + tr) * N;
                int8_t v[kMaxN];
                v[0] = 1;
                for (int k = 1; k < N; k++) {
                    const int x = ord[k], p = par[x];
                    v[x] = (int8_t)(v[p] * sig(D.pair[p * N + x]));
                }
                for (int l = 0; l < N; l++) {
                    votes[l] += v[l];
                    if (tr == 0) first[l] = v[l];
                }
            }
            for (int l = 0; l < N; l++) q[l] = (int8_t)(votes[l] > 0 ? 1 : (votes[l] < 0 ? -1 : first[l]));
        }
        const int32_t *Ji = D.J + (size_t)inst * (N * (N - 1) / 2);
        int64_t E = 0;
        int k = 0;
        for (int a = 0; a < N; a++)
            for (int c = a + 1; c < N; c++) E += (int64_t)Ji[k++] * q[a] * q[c];
        if (D.logical)
            for (int l = 0; l < N; l++) D.logical[i * N + l] = q[l];
        if (D.energy) D.energy[i] = E;
        if (D.success && D.e_ground && E == D.e_ground[inst]) atomicAdd(D.success + inst, 1);
    }
}

// ---------------------------------------------------------------------------
// Exhaustive ground state: 2^(N-1) states with s_{N-1} = +1, walked in Gray
// code order in chunks of 2^chunk_bits, energy updated with local fields.
// ---------------------------------------------------------------------------
__global__ void ground_kernel(int N, const int32_t *J, int chunk_bits, int64_t n_chunks,
                              unsigned long long *best)
{
    __shared__ int32_t Jm[40 * 40];
    const int inst = blockIdx.y;
    const int32_t *Ji = J + (size_t)inst * (N * (N - 1) / 2);
    for (int x = threadIdx.x; x < N * N; x += blockDim.x) {
        const int a = x / N, c = x % N;
        int v = 0;
        if (a != c) {
            const int i = a < c ? a : c, j = a < c ? c : a;
            v = Ji[i * N - i * (i + 1) / 2 + (j - i - 1)];
        }
        Jm[x] = v;
    }
    __syncthreads();
    long long local_best = LLONG_MAX;
    for (int64_t ch = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ch < n_chunks;
         ch += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x0 = (uint64_t)ch << chunk_bits;
        const uint64_t g0 = x0 ^ (x0 >> 1);
        int s[40];
        for (int i = 0; i < N - 1; i++) s[i] = ((g0 >> i) & 1) ? -1 : 1;
        s[N - 1] = 1;
        int h[40];
        long long E = 0;
        for (int i = 0; i < N; i++) {
            int f = 0;
            for (int j = 0; j < N; j++) f += Jm[i * N + j] * s[j];
            h[i] = f;
            E += (long long)s[i] * f;
        }
        E /= 2;
        long long m = E;
        const uint64_t steps = (uint64_t)1 << chunk_bits;
        for (uint64_t k = 1; k < steps; k++) {
            const int f = __ffsll((long long)(x0 + k)) - 1;  // bit that changes in the Gray code
            E += -2LL * s[f] * h[f];
            const int sf = s[f];
            for (int j = 0; j < N; j++) h[j] -= 2 * sf * Jm[j * N + f];
            s[f] = -sf;
            m = E < m ? E : m;
        }
        local_best = m < local_best ? m : local_best;
    }
    // order-preserving map of signed to unsigned for atomicMin
    const unsigned long long key = (unsigned long long)local_best ^ 0x8000000000000000ull;
    atomicMin(best + inst, key);
}

}  // namespace sqa
