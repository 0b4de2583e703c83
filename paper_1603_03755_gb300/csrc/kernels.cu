// Kernels of the SQA / PT hot path (arXiv:1603.03755), sm_103a.
//
// Data layout.  Spins are bits (1 <-> sigma = -1); one 32-bit word holds 32
// independent replicas of one (site, slice).  Global state is
// [instance][z][site][word] with sites in compact order (used sites sorted by
// graph colour), z the Trotter slice (SQA) or temperature slot (PT).
//
// Work.  A unit is a run of words of one instance; replicas in different
// words never interact, so a unit is an independent system.  The single-job
// sweep kernel gives units to blocks (or thread-block clusters, which split a
// unit's slices or slots) in turn; the multi-job kernel of ragged batches
// and the serving loop pulls them from a counter.  A block stages its
// unit's state, site records and threshold rows in shared memory, runs every
// sweep of the launch there and writes the state back.  Within a sweep the
// colour classes (SQA: colour x slice parity; PT: colour) run in order with a
// barrier between them; all items of a class are independent.
//
// Per item (site, z, word) the single-spin sweep draws the item's two
// SWEEP_HI Philox blocks (one byte per replica, of which the uniform's 7-bit
// high part), forms for each term of the site the word of replicas whose
// term value is negative (the two-spin-term table path: whose spin product
// is -1, its tables folding in the weight's sign) and, for SQA, the two
// temporal disagreement words, turns them into one threshold byte per
// replica (a per-site code table of the thresholds' top 7 bits after an 8x8
// bit-matrix transpose, or byte-wise sums into the site's window of the
// threshold row) and compares four replicas per instruction through the
// borrow-free byte subtraction of a guard-bit word; a tie of the high parts
// (probability 2^-7) goes to the block's tie array and is resolved after the
// phase from the SWEEP_LO stream's low 25 bits.  PT recounts energies for
// its swaps in bit-sliced form.  The time-like cluster moves work one warp
// per (site, word) on the site's whole imaginary-time ring.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "check.cuh"
#include "layout.cuh"
#include "handle.h"
#include "philox.cuh"
#include "sqa_internal.h"

namespace sqa {


__device__ __forceinline__ uint32_t valid_bits(int R, int gw)
{
    const int left = R - 32 * gw;
    return left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
}

__device__ __forceinline__ uint32_t bytes4(uint32_t v, int j) { return (v >> j) & 0x01010101u; }

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
//
// A unit (one instance's run of words) is swept by a cluster of C blocks
// (C = 1, 2, 4 or 8).  Block rank r owns the contiguous slices (SQA) or
// temperature slots (PT) [r*zr, (r+1)*zr), zr = Z/C, in its shared memory.
// SQA reads the temporal neighbours of its first and last slice from the
// neighbouring blocks' shared memory and separates colour phases with a
// cluster barrier; PT slots never interact within a sweep, and swap events
// exchange the boundary slots' energies and words across blocks.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

struct Smem {
    uint32_t *S;      // [zr][zstride]
    uint32_t *T;      // full thresholds: SQA one row, PT zr rows
    uint8_t *Tb;      // T >> 25: PT zr rows, SQA window mode one row
    uint32_t lut;     // SQA table mode: shared address of the per-site byte tables (256-byte aligned)
    SiteRec *sites;   // [n]
    int32_t *E;       // PT: [zr][wc*32]
    uint32_t *M;      // PT: swap masks [zr/2+1][wc]
    uint32_t *qdiv;   // per colour: the task decode's divisor {m, sh} (FastDiv)
    uint32_t *tq;     // this block's tie array: one tie mask per item of a phase (global memory)
    uint32_t tq_words;  // its length in words
    uint4 *ph;        // per word of the unit and SWEEP_HI block: the sweep's hoisted Philox values
    uint4 *rec;       // per site: the tie record (two uint4)
    uint2 *rq;        // per warp: kRequeue entries of items with ties left after a tie pass
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ Smem carve(const JobDev &J, unsigned char *base)
{
    const SmemOffsets o = smem_layout(J, J.wc, J.zstride);
    Smem m;
    m.S = (uint32_t *)(base + o.S);
    m.T = (uint32_t *)(base + o.T);
    m.Tb = (uint8_t *)(base + o.Tb);
    m.lut = (saddr(base + o.lut) + (kLutSlot - 1)) & ~(uint32_t)(kLutSlot - 1);
    m.sites = (SiteRec *)(base + o.sites);
    m.E = (int32_t *)(base + o.E);
    m.M = (uint32_t *)(base + o.M);
    m.qdiv = (uint32_t *)(base + o.Q + 16);
    m.tq = (uint32_t *)(J.tieq + (size_t)blockIdx.x * (size_t)J.tieq_stride);
    m.tq_words = 2u * (uint32_t)J.tieq_stride;
    m.ph = (uint4 *)(base + o.P);
    m.rec = (uint4 *)(base + o.R);
    m.rq = (uint2 *)(base + o.RQ);
    return m;
}

// The block's place in its cluster, and the neighbouring blocks' slices
// next to its own (SQA temporal neighbours across the block boundary).
struct Part {
    int C, rank, z0, zr;
    const uint32_t *up;  // slice z0 - 1 (the previous block's last slice)
    const uint32_t *dn;  // slice z0 + zr (the next block's first slice)
};

__device__ __forceinline__ void cluster_barrier(int C)
{
    if (C > 1)
        cg::this_cluster().sync();
    else
        __syncthreads();
}

// Division by a runtime divisor d >= 1 for numerators x < 2^31:
// floor(x/d) = umulhi(x, m) >> sh with m = ceil(2^(31+l)/d), l = ceil(log2 d),
// sh = l - 1; d = 1 is m = 0 (quotient x).
struct FastDiv {
    uint32_t m, sh;
};

__device__ __forceinline__ FastDiv make_div(uint32_t d)
{
    FastDiv f;
    if (d <= 1) {
        f.m = 0;
        f.sh = 0;
        return f;
    }
    const uint32_t l = 32u - __clz(d - 1u);  // ceil(log2 d)
    const unsigned long long num = 1ull << (31 + l);
    f.m = (uint32_t)((num + d - 1) / d);
    f.sh = l - 1u;
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, FastDiv f) { return f.m == 0 ? x : (__umulhi(x, f.m) >> f.sh); }

// Shared memory by 32-bit shared-window address (the sweep's hot loads).
__device__ __forceinline__ uint32_t lds32(uint32_t a)
{
    uint32_t v = 0u;
    if (SQA_SHARED_OK(a, 4u)) asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ uint32_t lds8(uint32_t a)
{
    uint32_t v = 0u;
    if (SQA_SHARED_OK(a, 1u)) asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts32(uint32_t a, uint32_t v)
{
    if (SQA_SHARED_OK(a, 4u)) asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ void sts8(uint32_t a, uint32_t v)
{
    if (SQA_SHARED_OK(a, 1u)) asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Term planes of one item: bit b of pl[k] is set when term k's value is
// negative for replica b (it turns positive on a flip); without SIGN, when
// the product of the term's spins is -1 (the per-site tables of minor
// embedding fold the weight's sign in, so its items never load weights).
// kw[k] is K*|w_k|.  PAIRS: every term has exactly one other member (minor
// embedding); otherwise absent members read the zero word of site n.
template <bool PAIRS, bool SIGN = true>
__device__ __forceinline__ void term_planes(const SiteRec &sr, uint32_t row, int n, int wc, int w, uint32_t s,
                                            uint32_t (&pl)[kMaxTerms], uint32_t (&kw)[kMaxTerms])
{
#pragma unroll
    for (int k = 0; k < kMaxTerms; k++) {
        pl[k] = 0u;
        kw[k] = 0u;
        if (k < sr.nterm) {
            const TermRec tr = sr.t[k];
            uint32_t p = s;
            if (PAIRS) {
                p ^= lds32(row + 4u * (uint32_t)(tr.p[0] * wc + w));
            } else {
                // an absent member (-1) reads the row's zero slot at site n
                const uint32_t z = (uint32_t)n;
                p ^= lds32(row + 4u * (min((uint32_t)(int)tr.p[0], z) * wc + w));
                p ^= lds32(row + 4u * (min((uint32_t)(int)tr.p[1], z) * wc + w));
                p ^= lds32(row + 4u * (min((uint32_t)(int)tr.p[2], z) * wc + w));
            }
            if (SIGN) {
                const int wv = tr.w;
                // w * prod(sigma) is negative iff (product is -1) xor (w < 0)
                pl[k] = p ^ (uint32_t)(wv >> 31);
                kw[k] = (uint32_t)(wv < 0 ? -wv : wv);
            } else {
                pl[k] = p;
            }
        }
    }
}

// Threshold index bytes of replicas (j, j+8, j+16, j+24): sum of K*|w| over
// the terms that turn positive, added byte-wise.
__device__ __forceinline__ uint32_t window4(const uint32_t (&pl)[kMaxTerms],
                                            const uint32_t (&kw)[kMaxTerms], int j)
{
    uint32_t a = 0u;
#pragma unroll
    for (int k = 0; k < kMaxTerms; k++) a += kw[k] * bytes4(pl[k], j);
    return a;
}

// Bit-matrix transpose of four 8x8 blocks held in eight words: afterwards byte
// b of P[j] holds bit (8b + j) of every input word, input word i at bit i.
__device__ __forceinline__ void transpose8(uint32_t (&P)[8])
{
#define SQA_SWAP(a, b, d, m)                                   \
    {                                                          \
        const uint32_t t_ = ((P[a] >> (d)) ^ P[b]) & (m);      \
        P[b] ^= t_;                                            \
        P[a] ^= t_ << (d);                                     \
    }
    SQA_SWAP(0, 4, 4, 0x0F0F0F0Fu) SQA_SWAP(1, 5, 4, 0x0F0F0F0Fu)
    SQA_SWAP(2, 6, 4, 0x0F0F0F0Fu) SQA_SWAP(3, 7, 4, 0x0F0F0F0Fu)
    SQA_SWAP(0, 2, 2, 0x33333333u) SQA_SWAP(1, 3, 2, 0x33333333u)
    SQA_SWAP(4, 6, 2, 0x33333333u) SQA_SWAP(5, 7, 2, 0x33333333u)
    SQA_SWAP(0, 1, 1, 0x55555555u) SQA_SWAP(2, 3, 1, 0x55555555u)
    SQA_SWAP(4, 5, 1, 0x55555555u) SQA_SWAP(6, 7, 1, 0x55555555u)
#undef SQA_SWAP
}

// The SWEEP_HI blocks of one sweep and unit, counter (t, slot, c2, inst)
// with t and inst fixed: c2 = 2*word + h enters through B*c2 in round 0, t
// through A*t; the slot is XOR-ed in by round 0 and first multiplied in
// round 1.  So per (word, h) three values fix rounds 0-2 apart from the
// slot (P0 = hi(B c2) ^ ka0; Q2, O3 = hi(A m0) ^ kb2, lo(A m0) with m0 the
// round-1 word that does not depend on the slot), and two values are the
// same for the whole sweep (U2 = lo(A t) ^ kb1, U3 = lo(B n2) ^ ka2).  A
// block then costs 16 wide multiplies instead of 20, with the same bits.
struct PhiloxSweep {
    uint32_t U2, U3, n2;
};

__device__ __forceinline__ PhiloxSweep philox_sweep(const JobDev &J, uint32_t t, uint32_t inst)
{
    uint32_t hiA, loA, hiB2, loB2;
    mul_wide(0xD2511F53u, t, hiA, loA);
    PhiloxSweep p;
    p.n2 = hiA ^ inst ^ J.rk_hi[0];
    mul_wide(0xCD9E8D57u, p.n2, hiB2, loB2);
    p.U2 = loA ^ J.rk_hi[1];
    p.U3 = loB2 ^ J.rk0[2];
    return p;
}

// {P0, Q2, O3} of (word gw, block h) for the sweep (ps from philox_sweep).
__device__ __forceinline__ uint4 philox_word(const JobDev &J, const PhiloxSweep &ps, uint32_t gw, uint32_t h)
{
    uint32_t hiB, loB, hiB2, loB2, hiA3, loA3;
    mul_wide(0xCD9E8D57u, 2u * gw + h, hiB, loB);
    mul_wide(0xCD9E8D57u, ps.n2, hiB2, loB2);
    const uint32_t m0 = hiB2 ^ loB ^ J.rk0[1];
    mul_wide(0xD2511F53u, m0, hiA3, loA3);
    return make_uint4(hiB ^ J.rk0[0], hiA3 ^ J.rk_hi[2], loA3, 0u);
}

// The SWEEP_HI block of the item's slot from its word's hoisted values.
__device__ __forceinline__ U4 philox_hi(const JobDev &J, const PhiloxSweep &ps, const uint4 &pw, uint32_t slot)
{
    uint32_t hiA2, loA2, hiB3, loB3;
    mul_wide(0xD2511F53u, pw.x ^ slot, hiA2, loA2);           // round 1: A * n0
    const uint32_t m2 = hiA2 ^ ps.U2, m3 = loA2;
    mul_wide(0xCD9E8D57u, m2, hiB3, loB3);                    // round 2: B * m2
    uint32_t c0 = hiB3 ^ ps.U3, c1 = loB3, c2 = pw.y ^ m3, c3 = pw.z;
#pragma unroll
    for (int r = 3; r < 10; r++) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_wide(0xD2511F53u, c0, hi0, lo0);
        mul_wide(0xCD9E8D57u, c2, hi1, lo1);
        const uint32_t n0 = hi1 ^ c1 ^ J.rk0[r], n2 = hi0 ^ c3 ^ J.rk_hi[r];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// The keys of the two sweep streams.
struct Keys {
    uint32_t k0, khi, klo;
};

// Full threshold index of a replica from its code (SQA: bit 0, 1 = the two
// temporal disagreements, bit 2+k = term k negative; FOLD: bit 2+k = the
// product of term k's spins is -1, so term k is negative when that bit
// differs from the weight's sign bit; PT: bit k = term k negative).
template <int KIND, bool FOLD = false>
__device__ __forceinline__ int full_index(const SiteRec &sr, uint32_t code)
{
    int U = KIND == SQA_KIND_SQA ? 2 - (int)(code & 1u) - (int)((code >> 1) & 1u) : 0;
    const int sh = KIND == SQA_KIND_SQA ? 2 : 0;
#pragma unroll
    for (int k = 0; k < kMaxTerms; k++) {
        if (k < sr.nterm) {
            const int wv = sr.t[k].w;
            const uint32_t neg = FOLD ? (((code >> (k + sh)) & 1u) ^ (uint32_t)(wv < 0)) : ((code >> (k + sh)) & 1u);
            if (neg) U += wv < 0 ? -wv : wv;
        }
    }
    return sr.base + U;
}

// The compare of one item, four replicas per word: X_j holds the 7-bit high
// parts h of replicas (j, j+8, j+16, j+24) under a guard bit in its four
// bytes, Q_j the top 7 bits of their thresholds (T >> 25).  Per byte,
// D = (128 + h) - (T >> 25) never borrows, and its bit 7 is set iff
// h >= T >> 25; D - 1 has bit 7 set iff h > T >> 25.  Gathered over the
// eight words (bit 8b + j for replica j + 8b), ge marks the replicas whose
// high part decides reject or is tied, gt those that reject outright; ties
// (ge and not gt, probability 2^-7) are resolved from the low 25 bits.
__device__ __forceinline__ void swar_compare(const U4 &A0, const U4 &A1, const uint32_t (&Q)[8], uint32_t &ge,
                                             uint32_t &gt)
{
    const uint32_t H = 0x80808080u;
    ge = 0u;
    gt = 0u;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t x = word_of(j < 4 ? A0 : A1, j & 3) | H;
        const uint32_t d1 = x - Q[j];
        const uint32_t d2 = d1 - 0x01010101u;
        ge = (ge >> 1) | (d1 & H);
        gt = (gt >> 1) | (d2 & H);
    }
}

// Four table bytes gathered into one word: byte b from the entry at the
// shared address formed by code byte b under the slot's aligned base.
__device__ __forceinline__ uint32_t gather_lut(uint32_t code, uint32_t slot)
{
    const uint32_t t0 = lds8(__byte_perm(code, slot, 0x7650u));
    const uint32_t t1 = lds8(__byte_perm(code, slot, 0x7651u));
    const uint32_t t2 = lds8(__byte_perm(code, slot, 0x7652u));
    const uint32_t t3 = lds8(__byte_perm(code, slot, 0x7653u));
    return (t3 * 256u + t2) * 65536u + (t1 * 256u + t0);
}

// Four threshold bytes of a window: byte b from base + byte b of the index word.
__device__ __forceinline__ uint32_t gather_window(uint32_t idx, uint32_t base)
{
    const uint32_t t0 = lds8(base + (idx & 0xFFu));
    const uint32_t t1 = lds8(base + __byte_perm(idx, 0u, 0x4441u));
    const uint32_t t2 = lds8(base + __byte_perm(idx, 0u, 0x4442u));
    const uint32_t t3 = lds8(base + (idx >> 24));
    return (t3 * 256u + t2) * 65536u + (t1 * 256u + t0);
}

// Everything an item of one task needs besides its slice or slot.
struct Task {
    int si, w, gw, wc;     // site, word in the unit, global word, words of the unit
    uint32_t own;          // byte offset of the item's word in a row
    uint32_t nb[kMaxTerms];  // PAIRS: byte offsets of the neighbours' words (absent: own, a zero plane)
    uint32_t slot0;        // canonical site * Z (random-number counter)
    uint32_t lut;          // SQA table mode: shared address of the site's table
    uint32_t swz;          // SQA table mode: the site's code swizzle (lut_swizzle)
    uint32_t valid;        // replicas of the word that exist
    uint4 ph0, ph1;        // the word's hoisted SWEEP_HI values (blocks 0 and 1)
};

// The planes of an item and, for SQA, its temporal disagreement words.  NB:
// the task holds the neighbours' offsets (minor embedding with sign-folded
// tables); otherwise they come from the site record.
template <int KIND, bool PAIRS, bool SIGN, bool NB>
__device__ __forceinline__ void item_planes(const JobDev &J, const Smem &sm, const Part &pt, const Task &tk,
                                            const SiteRec &sr, int zl, uint32_t &s, uint32_t (&pl)[kMaxTerms],
                                            uint32_t (&kw)[kMaxTerms], uint32_t &d1, uint32_t &d2)
{
    const uint32_t S0 = saddr(sm.S), zs4 = 4u * (uint32_t)J.zstride;
    const uint32_t row = S0 + (uint32_t)zl * zs4;
    s = lds32(row + tk.own);
    if (NB) {
        // minor embedding, sign-folded tables: the task's neighbour offsets
#pragma unroll
        for (int k = 0; k < kMaxTerms; k++) {
            pl[k] = s ^ lds32(row + tk.nb[k]);
            kw[k] = 0u;
        }
    } else {
        term_planes<PAIRS, SIGN>(sr, row, J.n, tk.wc, tk.w, s, pl, kw);
    }
    d1 = d2 = 0u;
    if (KIND == SQA_KIND_SQA) {
        // temporal disagreements: m = sigma (sigma_up + sigma_dn) = 2 - 2 (d1 + d2)
        uint32_t up, dn;
        if (pt.C == 1) {
            // one block holds the whole ring: the rows wrap around (selects, no branches)
            const uint32_t ur = zl > 0 ? row - zs4 : S0 + (uint32_t)(pt.zr - 1) * zs4;
            const uint32_t dr = zl < pt.zr - 1 ? row + zs4 : S0;
            up = lds32(ur + tk.own);
            dn = lds32(dr + tk.own);
        } else {
            if (zl > 0)
                up = lds32(row - zs4 + tk.own);
            else
                up = SQA_IN(kChkNeighbour, tk.own >> 2, J.zstride) ? pt.up[tk.own >> 2] : 0u;
            if (zl < pt.zr - 1)
                dn = lds32(row + zs4 + tk.own);
            else
                dn = SQA_IN(kChkNeighbour, tk.own >> 2, J.zstride) ? pt.dn[tk.own >> 2] : 0u;
        }
        d1 = s ^ up;
        d2 = s ^ dn;
    }
}

// The SWEEP_LO round keys, held in registers for a tie pass.
struct LoKeys {
    uint32_t a[10], b[10];
};

// A site's tie record (kTieRec bytes in shared memory): the threshold index
// of a replica is U0 + sum_k sw_k * (bit of term plane k) minus its two
// temporal bits (SQA).  With FOLD a plane bit is the spin product and term k
// turns positive when it differs from the weight's sign, so a negative
// weight counts |w| when the bit is 0: U0 takes |w| and sw_k = -|w|.  For
// minor embedding (FOLD) the record also keeps each term's other member
// (absent terms: the site itself, a zero plane).
template <bool FOLD>
__device__ __forceinline__ void tie_record(const SiteRec &sr, int si, int sqa, uint32_t *rec)
{
    int U0 = sr.base + (sqa ? 2 : 0), sw[kMaxTerms], p0[kMaxTerms];
#pragma unroll
    for (int k = 0; k < kMaxTerms; k++) {
        const int wv = k < sr.nterm ? (int)sr.t[k].w : 0, aw = wv < 0 ? -wv : wv;
        const bool f = FOLD && wv < 0;
        U0 += f ? aw : 0;
        sw[k] = f ? -aw : aw;
        p0[k] = k < sr.nterm ? (int)sr.t[k].p[0] : si;
    }
    rec[0] = (uint32_t)U0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        rec[1 + k] = ((uint32_t)sw[2 * k] & 0xFFFFu) | ((uint32_t)sw[2 * k + 1] << 16);
        rec[4 + k] = ((uint32_t)p0[2 * k] & 0xFFFFu) | ((uint32_t)p0[2 * k + 1] << 16);
    }
    rec[7] = 0u;
}

// Resolves ties of the item at slice or slot zl (site si, word w): the
// lowest one of tm, or all of them when ALL.  A tied replica's high part
// equals its threshold's top 7 bits, so it accepts iff its low 25 bits
// (SWEEP_LO stream) are below the threshold's low 25 bits, or the threshold
// stands for x <= 0.  The item's planes are recomputed from the state (the
// phase changes no neighbour of it, and its tied bits are still unflipped).
// Returns the ties left.
template <int KIND, bool LUT, bool PAIRS, bool ALL>
__device__ __forceinline__ uint32_t resolve_ties(const JobDev &J, const Smem &sm, const Part &pt, const LoKeys &lk,
                                                 int inst, int w0, int wc, int t, int si, int zl, int w, uint32_t tm)
{
    constexpr bool FOLD = KIND == SQA_KIND_SQA && LUT && PAIRS;
    const SiteRec &sr = sm.sites[si];
    const uint4 ra = sm.rec[2 * si], rb = sm.rec[2 * si + 1];
    Task tk;
    tk.si = si;
    tk.w = w;
    tk.wc = wc;
    tk.own = 4u * (uint32_t)(si * wc + w);
    if (FOLD) {
        const uint32_t pp[3] = {rb.x, rb.y, rb.z};
#pragma unroll
        for (int k = 0; k < kMaxTerms; k++)
            tk.nb[k] = 4u * ((uint32_t)(pp[k >> 1] >> (16 * (k & 1)) & 0xFFFFu) * (uint32_t)wc + (uint32_t)w);
    }
    uint32_t s, pl[kMaxTerms], kw[kMaxTerms], d1, d2;
    item_planes<KIND, PAIRS, !FOLD, FOLD>(J, sm, pt, tk, sr, zl, s, pl, kw, d1, d2);
    const uint32_t gw = (uint32_t)(w0 + w);
    const uint32_t slot = (uint32_t)sr.canon * (uint32_t)J.Z + (uint32_t)(pt.z0 + zl);
    const uint32_t *Trow = KIND == SQA_KIND_SQA ? sm.T : sm.T + (size_t)zl * J.nrow;
    const int U0 = (int)ra.x;
    const uint32_t swp[3] = {ra.y, ra.z, ra.w};
    uint32_t flip = 0u;
    do {
        const int b = __ffs(tm) - 1;
        tm &= tm - 1u;
        int U = U0;
        if (KIND == SQA_KIND_SQA) U -= (int)((d1 >> b) & 1u) + (int)((d2 >> b) & 1u);
#pragma unroll
        for (int k = 0; k < kMaxTerms; k++)
            U += (int)((pl[k] >> b) & 1u) * (int)(int16_t)(swp[k >> 1] >> (16 * (k & 1)));
        const uint32_t T = SQA_IN(kChkThreshold, U, J.nrow) ? Trow[U] : 0u;
        const uint32_t rho = gw * 32u + (uint32_t)b;
        const U4 B = philox_rk((uint32_t)t, slot, rho >> 2, (uint32_t)inst, lk.a, lk.b);
        const uint32_t r = rho & 3u;
        const uint32_t l = (r == 0 ? B.x : r == 1 ? B.y : r == 2 ? B.z : B.w) >> 7;
        if (T == 0xFFFFFFFFu || l < (T & 0x1FFFFFFu)) flip |= 1u << b;
    } while (ALL && tm);
    const uint32_t a = saddr(sm.S) + (uint32_t)zl * 4u * (uint32_t)J.zstride + tk.own;
    sts32(a, lds32(a) ^ flip);
    return tm;
}

// One item: the word of 32 replicas of the task's site at local slice or
// slot zl.  Draws the two SWEEP_HI blocks of the word, forms per replica the
// threshold index (a per-site table entry by code, or a window index), and
// compares four replicas per instruction; flips the replicas whose high
// parts accept, and returns the tie mask (ties are left unflipped).
template <int KIND, bool LUT, bool PAIRS>
__device__ __forceinline__ uint32_t metro_item(const JobDev &J, const PhiloxSweep &ps, const Smem &sm, const Part &pt,
                                               const Task &tk, const SiteRec &sr, int zl)
{
    constexpr bool FOLD = KIND == SQA_KIND_SQA && LUT && PAIRS;
    uint32_t s, pl[kMaxTerms], kw[kMaxTerms], d1, d2;
    item_planes<KIND, PAIRS, !FOLD, FOLD>(J, sm, pt, tk, sr, zl, s, pl, kw, d1, d2);
    const uint32_t slot = tk.slot0 + (uint32_t)(pt.z0 + zl);
    // the word's two SWEEP_HI blocks: 16 bytes each, one per replica
    const U4 A0 = philox_hi(J, ps, tk.ph0, slot);
    const U4 A1 = philox_hi(J, ps, tk.ph1, slot);
    uint32_t Q[8];
    if (KIND == SQA_KIND_SQA && LUT) {
        uint32_t code[8];
        code[0] = d1;
        code[1] = d2;
#pragma unroll
        for (int k = 0; k < kMaxTerms; k++) code[k + 2] = pl[k];
        // code bits 4-6 swizzled by the site (the table stores entry c at c ^ swz)
        code[4] ^= 0u - (tk.swz >> 4 & 1u);
        code[5] ^= 0u - (tk.swz >> 5 & 1u);
        code[6] ^= 0u - (tk.swz >> 6 & 1u);
        transpose8(code);
#pragma unroll
        for (int j = 0; j < 8; j++) Q[j] = gather_lut(code[j], tk.lut);
    } else {
        const uint32_t wb = saddr(KIND == SQA_KIND_SQA ? sm.Tb : sm.Tb + (size_t)zl * J.nrow) + (uint32_t)sr.base;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            uint32_t a = window4(pl, kw, j);
            if (KIND == SQA_KIND_SQA) a += 0x02020202u - bytes4(d1, j) - bytes4(d2, j);
            Q[j] = gather_window(a, wb);
        }
    }
    uint32_t ge, gt;
    swar_compare(A0, A1, Q, ge, gt);
    const uint32_t S0 = saddr(sm.S);
    sts32(S0 + (uint32_t)zl * 4u * (uint32_t)J.zstride + tk.own, s ^ (~ge & tk.valid));
    return ge & ~gt & tk.valid;
}

// Stores a task's tie masks in the block's tie array: word tau * czc + i
// for slice or slot i of task tau (0 where the item does not exist or did
// not tie), every word of the phase written, so the array needs no counter.
__device__ __forceinline__ void store_task_ties(const Smem &sm, int tau, int czc, const uint32_t (&tm)[kTaskSlices])
{
    uint32_t *a = sm.tq + (size_t)tau * czc;
#pragma unroll
    for (int i = 0; i < kTaskSlices; i++)
        if (i < czc && SQA_IN(kChkTieArray, (size_t)tau * czc + i, sm.tq_words)) a[i] = tm[i];
}

// Where a site's table keeps the entry of code c: at byte c ^ swz of its
// slot.  The slots are 256-byte aligned, so without it the same code of
// different sites would fall on the same shared-memory bank; the lanes of a
// warp work on up to eight sites (consecutive lanes take consecutive words
// of one site), and XOR-ing code bits 4-6 with the site's low three bits
// moves each site's entries by 4 (site % 8) banks.
__device__ __forceinline__ uint32_t lut_swizzle(int si) { return ((uint32_t)si & 7u) << 4; }

// SQA: per-site byte tables for sweep t from the staged threshold row:
// entry c is the top 7 bits (T >> 25) of T[base + 2 + sum of K|w_k| over
// the negative terms - the two temporal bits], term k negative when code
// bit 2+k is set (FOLD: when it, the spin product being -1, differs from
// the sign of w_k).  Only the 2^(nterm+2) codes a site can produce are
// written.
template <bool FOLD>
__device__ void build_luts(const JobDev &J, const Smem &sm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int si = warp; si < J.n; si += nw) {
        const SiteRec &sr = sm.sites[si];
        const int nt = sr.nterm, base = sr.base;
        // the site's weights once, in registers (entries are independent)
        int aw[kMaxTerms];
        uint32_t flip[kMaxTerms];
#pragma unroll
        for (int k = 0; k < kMaxTerms; k++) {
            const int wv = k < nt ? (int)sr.t[k].w : 0;
            aw[k] = wv < 0 ? -wv : wv;
            flip[k] = FOLD ? (uint32_t)(wv < 0) : 0u;
        }
        const int ne = 1 << (nt + 2);
        const uint32_t slot = sm.lut + (uint32_t)si * kLutSlot, swz = lut_swizzle(si);
        for (int c = lane; c < ne; c += 32) {
            // as full_index: bits of terms k >= nt are 0 and their weights 0
            int U = 2 - (c & 1) - ((c >> 1) & 1);
#pragma unroll
            for (int k = 0; k < kMaxTerms; k++)
                if ((((uint32_t)c >> (k + 2)) & 1u) ^ flip[k]) U += aw[k];
            sts8(slot + ((uint32_t)c ^ swz), SQA_IN(kChkThreshold, base + U, J.nrow) ? sm.T[base + U] >> 25 : 0u);
        }
    }
}

// Carry-save adder on bit vectors: a + b + c = l + 2 h in every bit position.
__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c)
{
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// Value bits of energy term q for the 32 replicas of word w of a slot's row:
// bit b set when the product of the term's spins is -1 for replica b.
__device__ __forceinline__ uint32_t eterm_bits(const ETerm &x, const uint32_t *row, int wc, int w)
{
    uint32_t v = row[x.m[0] * wc + w];
    if (x.size > 1) v ^= row[x.m[1] * wc + w];
    if (x.size > 2) v ^= row[x.m[2] * wc + w];
    if (x.size > 3) v ^= row[x.m[3] * wc + w];
    return v;
}

// Bit-sliced count, for each of the 32 replicas, of the n terms (all of SZ
// spins) at et whose value is negative: P[k] = bit k of every replica's
// count.  A carry-save adder tree folds 16 terms into ones/twos/fours/eights
// planes; a ripple adder takes the sixteens (12 planes, counts below 4096).
// A term's spin indices are read as one 8-byte load.
template <int SZ>
__device__ __forceinline__ void count_terms(const ETerm *et, int n, const uint32_t *row, int wc, int w,
                                            uint32_t (&P)[12])
{
    uint32_t ones = 0u, twos = 0u, fours = 0u, eights = 0u;
#pragma unroll
    for (int q2 = 4; q2 < 12; q2++) P[q2] = 0u;
    for (int q = 0; q < n; q += 16) {
        uint32_t v[16];
#pragma unroll
        for (int i = 0; i < 16; i++) {
            v[i] = 0u;
            if (q + i < n) {
                const uint2 mm = __ldg(reinterpret_cast<const uint2 *>(et + q + i));
                uint32_t x = row[(int)(mm.x & 0xFFFFu) * wc + w];
                if (SZ > 1) x ^= row[(int)(mm.x >> 16) * wc + w];
                if (SZ > 2) x ^= row[(int)(mm.y & 0xFFFFu) * wc + w];
                if (SZ > 3) x ^= row[(int)(mm.y >> 16) * wc + w];
                v[i] = x;
            }
        }
        uint32_t tA, tB, fA, fB, eA, eB, s16;
        csa(tA, ones, ones, v[0], v[1]);
        csa(tB, ones, ones, v[2], v[3]);
        csa(fA, twos, twos, tA, tB);
        csa(tA, ones, ones, v[4], v[5]);
        csa(tB, ones, ones, v[6], v[7]);
        csa(fB, twos, twos, tA, tB);
        csa(eA, fours, fours, fA, fB);
        csa(tA, ones, ones, v[8], v[9]);
        csa(tB, ones, ones, v[10], v[11]);
        csa(fA, twos, twos, tA, tB);
        csa(tA, ones, ones, v[12], v[13]);
        csa(tB, ones, ones, v[14], v[15]);
        csa(fB, twos, twos, tA, tB);
        csa(eB, fours, fours, fA, fB);
        csa(s16, eights, eights, eA, eB);
#pragma unroll
        for (int q2 = 4; q2 < 12; q2++) {
            const uint32_t carry = P[q2] & s16;
            P[q2] ^= s16;
            s16 = carry;
        }
    }
    P[0] = ones;
    P[1] = twos;
    P[2] = fours;
    P[3] = eights;
}

// PT: energies of the block's slots.  E_b = sum_t w_t - 2 sum_c w_c n_c(b),
// where n_c(b) counts the terms of class c (a run of terms of one weight)
// whose value is negative for replica b.  One thread per (slot, word, class)
// counts for all 32 replicas at once in bit-sliced form (count_terms); two
// 8x8 bit-matrix transposes turn the planes into per-replica counts, added
// into E.
// Instances with too many distinct weights fall back to a per-replica loop.
__device__ void pt_energies(const JobDev &J, const Smem &sm, int inst, int wc, int zr)
{
    const ETerm *et = J.eterms + (size_t)inst * J.n_eterms;
    const int nthr = blockDim.x;
    if (J.n_ecls == 0) {
        for (int it = threadIdx.x; it < zr * wc * 32; it += nthr) {
            const int b = it & 31, r = it >> 5, w = r % wc, p = r / wc;
            const uint32_t *row = sm.S + (size_t)p * J.zstride;
            int32_t E = 0;
            for (int q = 0; q < J.n_eterms; q++) {
                const ETerm x = et[q];
                E += ((eterm_bits(x, row, wc, w) >> b) & 1u) ? -x.w : x.w;
            }
            sm.E[(p * wc + w) * 32 + b] = E;
        }
        return;
    }
    const EClass *cls = J.ecls + (size_t)inst * kMaxEClasses;
    const int total = cls[0].total;
    for (int it = threadIdx.x; it < zr * wc * 32; it += nthr) sm.E[it] = total;
    __syncthreads();
    const int nc = J.n_ecls;
    for (int it = threadIdx.x; it < zr * wc * nc; it += nthr) {
        // consecutive threads take consecutive slots (distinct banks)
        const int p = it % zr, r = it / zr, w = r % wc, c = r / wc;
        const EClass k = cls[c];
        if (k.count == 0) continue;
        const uint32_t *row = sm.S + (size_t)p * J.zstride;
        uint32_t P[12];
        switch (k.size) {
        case 1: count_terms<1>(et + k.start, k.count, row, wc, w, P); break;
        case 2: count_terms<2>(et + k.start, k.count, row, wc, w, P); break;
        case 3: count_terms<3>(et + k.start, k.count, row, wc, w, P); break;
        default: count_terms<4>(et + k.start, k.count, row, wc, w, P); break;
        }
        // planes -> per-replica counts: byte b of lo[j] / up[j] holds bits
        // 0-7 / 8-11 of the count of replica 8b + j
        uint32_t lo[8] = {P[0], P[1], P[2], P[3], P[4], P[5], P[6], P[7]};
        uint32_t up[8] = {P[8], P[9], P[10], P[11], 0u, 0u, 0u, 0u};
        transpose8(lo);
        transpose8(up);
        int32_t *Ew = sm.E + (p * wc + w) * 32;
        const int m2w = -2 * k.w;
#pragma unroll
        for (int j = 0; j < 8; j++)
#pragma unroll
            for (int b8 = 0; b8 < 4; b8++) {
                // start at a slot-dependent replica so that lanes of a warp
                // hit distinct banks
                const int bb = (b8 + (p >> 3)) & 3;
                const int n = (int)(__byte_perm(lo[j], 0u, 0x4440u + (uint32_t)bb) |
                                    (__byte_perm(up[j], 0u, 0x4440u + (uint32_t)bb) << 8));
                if (n) atomicAdd(Ew + 8 * bb + j, m2w * n);
            }
    }
}

// PT swap event e: slots (p, p+1) with p = e%2, e%2 + 2, ... exchange
// configurations replica by replica (Eq. 9).  The block handles the pairs
// whose lower slot it owns; a pair straddling two blocks reads the upper
// slot's energies and words from the next block and writes its words there.
__device__ void pt_swap(const JobDev &J, const Smem &sm, const Part &pt, int inst, int w0, int wc, int e)
{
    const int P = J.Z, n = J.n, zr = pt.zr, z0 = pt.z0;
    const int nthr = blockDim.x;
    __syncthreads();
    pt_energies(J, sm, inst, wc, zr);
    cluster_barrier(pt.C);  // every block's energies are final
    const int32_t *E_next = sm.E;
    uint32_t *S_next = sm.S;
    if (pt.C > 1) {
        cg::cluster_group cl = cg::this_cluster();
        const int nr = (pt.rank + 1) % pt.C;
        E_next = cl.map_shared_rank(sm.E, nr);
        S_next = cl.map_shared_rank(sm.S, nr);
    }
    // pairs with the lower slot in [z0, z0+zr) and the upper slot < P
    const int first = z0 + ((((e & 1) - z0) % 2) + 2) % 2;
    const int last = min(z0 + zr - 1, P - 2);
    const int npairs = last >= first ? (last - first) / 2 + 1 : 0;
    for (int it = threadIdx.x; it < npairs * wc * 32; it += nthr) {
        const int b = it & 31, r = it >> 5, w = r % wc, k = r / wc;
        const int p = first + 2 * k, pl = p - z0;
        const int gw = w0 + w;
        const int rho = gw * 32 + b;
        // (the ballot below stays convergent: a failed check only clears accept)
        const bool ok = SQA_IN(kChkSwap, pl, zr);
        const int32_t Eu = !ok ? 0 : pl + 1 < zr ? sm.E[((pl + 1) * wc + w) * 32 + b] : E_next[(0 * wc + w) * 32 + b];
        const int dE = !ok ? 0 : Eu - sm.E[(pl * wc + w) * 32 + b];
        bool accept = ok && dE <= 0;
        if (ok && !accept && dE <= J.sw_len[p]) {
            const U4 v = philox((uint32_t)e, (uint32_t)p, (uint32_t)(rho >> 2), (uint32_t)inst, J.seed_lo,
                                J.key_swap);
            accept = word_of(v, rho & 3) < J.Tsw[J.sw_off[p] + dE - 1];
        }
        const uint32_t M = __ballot_sync(0xFFFFFFFFu, accept) & valid_bits(J.R, gw);
        if (b == 0 && SQA_IN(kChkSwap, k * wc + w, (zr / 2 + 1) * wc)) sm.M[k * wc + w] = M;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < npairs * n * wc; it += nthr) {
        const int w = it % wc, r = it / wc, si = r % n, k = r / n;
        const int pl = first + 2 * k - z0;
        uint32_t *a = sm.S + (size_t)pl * J.zstride + si * wc + w;
        uint32_t *c = pl + 1 < zr ? sm.S + (size_t)(pl + 1) * J.zstride + si * wc + w : S_next + si * wc + w;
        if (!(SQA_IN(kChkSwap, k * wc + w, (zr / 2 + 1) * wc) && SQA_IN(kChkSwap, pl, zr))) continue;
        const uint32_t va = *a, vc = *c;
        const uint32_t d = (va ^ vc) & sm.M[k * wc + w];
        *a = va ^ d;
        *c = vc ^ d;
    }
    cluster_barrier(pt.C);  // swapped words are visible before the next sweep
}

// ---------------------------------------------------------------------------
// Time-like cluster (Wolff) moves.  One warp moves one (site, word): lane l
// holds slices l*SPL .. l*SPL+SPL-1 of the site's imaginary-time ring, and
// after the energy transpose lane l also stands for replica l of the word.
// ---------------------------------------------------------------------------

// 32 x 32 bit transpose across the warp: afterwards bit j of lane i's word is
// bit i of lane j's input word (five butterfly stages of block swaps).
__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const uint32_t m = d == 16 ? 0x0000FFFFu : d == 8 ? 0x00FF00FFu : d == 4 ? 0x0F0F0F0Fu : d == 2 ? 0x33333333u
                                                                                                   : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, d);
        x = (lane & d) ? ((x & ~m) | ((y >> d) & m)) : ((x & m) | ((y & m) << d));
    }
    return x;
}

// Replicas of und whose bond uniform is below T, compared bit-serially from
// the most significant bit: bit 31-k of replica b's uniform is bit b of
// plane k, plane k being word k%4 of the bond stream at counter
// (t, slot, g8 + k/4, inst).  Planes are drawn only while some replica of
// und is undecided.
__device__ __forceinline__ uint32_t bond_below(uint32_t und, uint32_t T, uint32_t t, uint32_t slot, uint32_t g8,
                                               uint32_t inst, uint32_t k0, uint32_t kb)
{
    uint32_t lt = 0u;
    for (int q = 0; q < 8 && und; q++) {
        const U4 P = philox(t, slot, g8 + (uint32_t)q, inst, k0, kb);
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            const uint32_t r = word_of(P, kk);
            if ((T >> (31 - (4 * q + kk))) & 1u) {
                lt |= und & ~r;
                und &= r;
            } else {
                und &= ~r;
            }
        }
    }
    return lt;
}

// One cluster move for every replica of word w of site si (one warp).
template <int SPL>
__device__ __forceinline__ void wolff_item(const JobDev &J, const Smem &sm, uint32_t *start, int inst, int w0, int wc,
                                           int t, int si, int w, uint32_t Tb, int aoff, int alen, int lane)
{
    const SiteRec &sr = sm.sites[si];
    const int L = J.Z;
    const int idx = si * wc + w;
    const int gw = w0 + w;
    const uint32_t canon = (uint32_t)sr.canon;
    const uint32_t full = 0xFFFFFFFFu;
    uint32_t s[SPL], A[SPL], St[SPL], C[SPL];
    // spins and bonds of this lane's slices; bond j joins slice tau_j to tau_j + 1
#pragma unroll
    for (int j = 0; j < SPL; j++) {
        const int tau = lane * SPL + j;
        s[j] = 0u;
        A[j] = 0u;
        if (tau < L && SQA_IN(kChkRing, (size_t)tau * J.zstride + idx, (size_t)L * J.zstride)) {
            s[j] = sm.S[(size_t)tau * J.zstride + idx];
            const uint32_t nx = sm.S[(size_t)(tau + 1 == L ? 0 : tau + 1) * J.zstride + idx];
            const uint32_t eq = ~(s[j] ^ nx);
            A[j] = Tb == 0xFFFFFFFFu ? eq
                                     : bond_below(eq, Tb, (uint32_t)t, canon * (uint32_t)L + (uint32_t)tau,
                                                  (uint32_t)gw * 8u, (uint32_t)inst, J.seed_lo, J.key_wbond);
        }
    }
    // start slice of replica `lane`, gathered into per-slice start masks
    {
        const uint32_t rho = (uint32_t)gw * 32u + (uint32_t)lane;
        const U4 P = philox((uint32_t)t, canon, rho >> 2, (uint32_t)inst, J.seed_lo, J.key_wstart);
        const int tau0 = (int)__umulhi(word_of(P, (int)(rho & 3u)), (uint32_t)L);
#pragma unroll
        for (int j = 0; j < SPL; j++) start[lane * SPL + j] = 0u;
        __syncwarp();
        const uint32_t same = __match_any_sync(full, tau0);
        if (lane == __ffs(same) - 1) start[tau0] = same;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < SPL; j++) St[j] = lane * SPL + j < L ? start[lane * SPL + j] : 0u;
    }
    // growth along the ring as two scans of x -> G | (x & P) maps
    const int last_lane = (L - 1) / SPL, last_slot = (L - 1) % SPL;
    uint32_t Awrap = 0u;  // bond (L-1 -> 0), held by the owner of slice L-1
#pragma unroll
    for (int j = 0; j < SPL; j++)
        if (j == last_slot) Awrap = A[j];
    Awrap = __shfl_sync(full, Awrap, last_lane);
    uint32_t Ain0 = __shfl_up_sync(full, A[SPL - 1], 1);  // bond into this lane's first slice
    if (lane == 0) Ain0 = Awrap;
    uint32_t F[SPL];
    {
        // forward: x_tau = St_tau | (x_{tau-1} & A_{tau-1})
        uint32_t P = full, G = 0u;
#pragma unroll
        for (int j = 0; j < SPL; j++)
            if (lane * SPL + j < L) {
                const uint32_t a = j == 0 ? Ain0 : A[j - 1];
                G = St[j] | (G & a);
                P &= a;
            }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t Pu = __shfl_up_sync(full, P, d), Gu = __shfl_up_sync(full, G, d);
            if (lane >= d) {
                G |= Gu & P;
                P &= Pu;
            }
        }
        const uint32_t wrap = __shfl_sync(full, G, 31);  // slice L-1 after one pass from zero
        uint32_t Pex = __shfl_up_sync(full, P, 1), Gex = __shfl_up_sync(full, G, 1);
        if (lane == 0) {
            Pex = full;
            Gex = 0u;
        }
        uint32_t x = Gex | (wrap & Pex);
#pragma unroll
        for (int j = 0; j < SPL; j++) {
            F[j] = 0u;
            if (lane * SPL + j < L) {
                x = St[j] | (x & (j == 0 ? Ain0 : A[j - 1]));
                F[j] = x;
            }
        }
    }
    {
        // backward: x_tau = St_tau | (x_{tau+1} & A_tau)
        uint32_t P = full, G = 0u;
#pragma unroll
        for (int j = SPL - 1; j >= 0; j--)
            if (lane * SPL + j < L) {
                G = St[j] | (G & A[j]);
                P &= A[j];
            }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t Pd = __shfl_down_sync(full, P, d), Gd = __shfl_down_sync(full, G, d);
            if (lane + d < 32) {
                G |= Gd & P;
                P &= Pd;
            }
        }
        const uint32_t wrap = __shfl_sync(full, G, 0);  // slice 0 after one pass from zero
        uint32_t Pex = __shfl_down_sync(full, P, 1), Gex = __shfl_down_sync(full, G, 1);
        if (lane == 31) {
            Pex = full;
            Gex = 0u;
        }
        uint32_t x = Gex | (wrap & Pex);
#pragma unroll
        for (int j = SPL - 1; j >= 0; j--) {
            C[j] = F[j];
            if (lane * SPL + j < L) {
                x = St[j] | (x & A[j]);
                C[j] |= x;
            }
        }
    }
    // problem-energy change of each replica's cluster: lane b counts, over the
    // cluster's slices, the negative terms (per term) and the slices
    int cnt_c = 0, D6 = 0;
    {
#pragma unroll
        for (int j = 0; j < SPL; j++) cnt_c += __popc(warp_transpose(C[j], lane));
        for (int k = 0; k < sr.nterm; k++) {
            const TermRec tr = sr.t[k];
            int cnt = 0;
#pragma unroll
            for (int j = 0; j < SPL; j++) {
                const int tau = lane * SPL + j;
                uint32_t v = 0u;
                if (tau < L) {
                    const uint32_t *row = sm.S + (size_t)tau * J.zstride;
                    // absent members (-1) read the row's zero slot at site n
                    const uint32_t zs = (uint32_t)J.n;
                    v = s[j] ^ row[min((uint32_t)(int)tr.p[0], zs) * wc + w] ^
                        row[min((uint32_t)(int)tr.p[1], zs) * wc + w] ^ row[min((uint32_t)(int)tr.p[2], zs) * wc + w];
                    v = (v ^ (uint32_t)((int)tr.w >> 31)) & C[j];  // term negative, slice in the cluster
                }
                cnt += __popc(warp_transpose(v, lane));
            }
            const int aw = tr.w < 0 ? -tr.w : tr.w;  // 6 |w|
            D6 += aw * (4 * cnt - 2 * cnt_c);
        }
    }
    // Metropolis test on x = alpha * D; the temporal part is in the growth
    const int D = D6 / 6;
    bool acc = D <= 0;
    if (!acc) {
        const int q = D >> 1;
        const uint32_t T = q <= alen ? __ldg(J.Tacc + aoff + q - 1) : 0u;
        const uint32_t rho = (uint32_t)gw * 32u + (uint32_t)lane;
        const U4 P = philox((uint32_t)t, canon, rho >> 2, (uint32_t)inst, J.seed_lo, J.key_wacc);
        acc = T == 0xFFFFFFFFu || word_of(P, (int)(rho & 3u)) < T;
    }
    const uint32_t flip = __ballot_sync(full, acc) & valid_bits(J.R, gw);
#pragma unroll
    for (int j = 0; j < SPL; j++) {
        const int tau = lane * SPL + j;
        if (tau < L && SQA_IN(kChkRing, (size_t)tau * J.zstride + idx, (size_t)L * J.zstride))
            sm.S[(size_t)tau * J.zstride + idx] = s[j] ^ (C[j] & flip);
    }
}

// A unit of time-like cluster sweeps: the whole imaginary-time ring of every
// site stays in this block (no cluster split).
template <int SPL>
__device__ void run_unit_wolff(const JobDev &J, const Smem &sm, const Unit &u)
{
    const int nthr = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int Z = J.Z, n = J.n, wc = u.wc, inst = u.inst, w0 = u.w0;
    const size_t n_state = (size_t)J.n_inst * Z * n * J.W;
    for (int i = tid; i < Z * n * wc; i += nthr) {
        const int w = i % wc, r = i / wc, si = r % n, zl = r / n;
        const size_t g = (((size_t)inst * Z + zl) * n + si) * J.W + w0 + w;
        sm.S[(size_t)zl * J.zstride + si * wc + w] = SQA_IN(kChkState, g, n_state) ? J.state[g] : 0u;
    }
    for (int i = tid; i < Z * wc; i += nthr) sm.S[(size_t)(i / wc) * J.zstride + n * wc + i % wc] = 0u;
    {
        const uint32_t *src = (const uint32_t *)(J.sites + (size_t)inst * n);
        uint32_t *dst = (uint32_t *)sm.sites;
        for (int i = tid; i < n * (int)(sizeof(SiteRec) / 4); i += nthr) dst[i] = src[i];
    }
    __syncthreads();
    uint32_t *start = sm.M + (size_t)warp * SPL * 32;
    for (int t = J.t0; t < J.t1; t++) {
        const uint32_t Tb = __ldg(J.Tb + t);
        const int aoff = __ldg(J.acc_off + t), alen = __ldg(J.acc_len + t);
        for (int chi = 0; chi < J.ncol; chi++) {
            const int c0 = J.col_ptr[chi];
            const int nitems = (J.col_ptr[chi + 1] - c0) * wc;
            for (int it = warp; it < nitems; it += nwarps)
                wolff_item<SPL>(J, sm, start, inst, w0, wc, t, c0 + it / wc, it % wc, Tb, aoff, alen, lane);
            __syncthreads();
        }
    }
    for (int i = tid; i < Z * n * wc; i += nthr) {
        const int w = i % wc, r = i / wc, si = r % n, zl = r / n;
        const size_t g = (((size_t)inst * Z + zl) * n + si) * J.W + w0 + w;
        if (SQA_IN(kChkState, g, n_state)) J.state[g] = sm.S[(size_t)zl * J.zstride + si * wc + w];
    }
    __syncthreads();
}

// Slices (SQA: slice pairs) or slots per task for one colour phase of
// `pairs` (site, word) pairs and zn slice steps: the chunk whose longest
// thread runs the fewest items (ties to the longer chunk, at most
// kTaskSlices, the unrolled task body), so a
// task's site record is read once for several items.
__device__ __forceinline__ int chunk_for(int pairs, int zn, int nthr)
{
    int best_c = 1;
    long long best = -1;
    for (int c = 1; c <= kTaskSlices && c <= zn; c++) {
        const long long tasks = (long long)pairs * ((zn + c - 1) / c);
        const long long cost = (tasks + nthr - 1) / nthr * c;
        if (best < 0 || cost <= best) {
            best = cost;
            best_c = c;
        }
    }
    return best_c;
}

template <int KIND, bool LUT, bool PAIRS>
__device__ void run_unit(const JobDev &J, const Smem &sm, const Unit &u)
{
    constexpr bool FOLD = KIND == SQA_KIND_SQA && LUT && PAIRS;
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int Z = J.Z, n = J.n, wc = u.wc, inst = u.inst, w0 = u.w0;
    const Keys K{J.seed_lo, J.key_hi, J.key_lo};
    Part pt;
    pt.C = J.csize;
    pt.zr = J.zr;
    pt.rank = 0;
    pt.up = pt.dn = nullptr;
    if (pt.C > 1) {
        cg::cluster_group cl = cg::this_cluster();
        pt.rank = (int)cl.block_rank();
        pt.up = cl.map_shared_rank(sm.S, (pt.rank + pt.C - 1) % pt.C) + (size_t)(pt.zr - 1) * J.zstride;
        pt.dn = cl.map_shared_rank(sm.S, (pt.rank + 1) % pt.C);
    }
    pt.z0 = pt.rank * pt.zr;
    const int zr = pt.zr, z0 = pt.z0;
    // stage this block's slices (and each row's zero slot) and the site records
    const size_t n_state = (size_t)J.n_inst * Z * n * J.W;
    for (int i = tid; i < zr * n * wc; i += nthr) {
        const int w = i % wc, r = i / wc, si = r % n, zl = r / n;
        const size_t g = (((size_t)inst * Z + z0 + zl) * n + si) * J.W + w0 + w;
        sm.S[(size_t)zl * J.zstride + si * wc + w] = SQA_IN(kChkState, g, n_state) ? J.state[g] : 0u;
    }
    for (int i = tid; i < zr * wc; i += nthr) sm.S[(size_t)(i / wc) * J.zstride + n * wc + i % wc] = 0u;
    {
        const uint32_t *src = (const uint32_t *)(J.sites + (size_t)inst * n);
        uint32_t *dst = (uint32_t *)sm.sites;
        for (int i = tid; i < n * (int)(sizeof(SiteRec) / 4); i += nthr) dst[i] = src[i];
    }
    if (KIND == SQA_KIND_PT)
        for (int i = tid; i < zr * J.nrow; i += nthr) {
            const uint32_t T = J.T[(size_t)z0 * J.nrow + i];
            sm.T[i] = T;
            sm.Tb[i] = (uint8_t)(T >> 25);
        }
    for (int si = tid; si < n; si += nthr) {
        uint32_t rec[8];
        tie_record<FOLD>(J.sites[(size_t)inst * n + si], si, KIND == SQA_KIND_SQA, rec);
        sm.rec[2 * si] = make_uint4(rec[0], rec[1], rec[2], rec[3]);
        sm.rec[2 * si + 1] = make_uint4(rec[4], rec[5], rec[6], rec[7]);
    }
    if (tid < J.ncol) {
        const FastDiv f = make_div((uint32_t)(J.col_ptr[tid + 1] - J.col_ptr[tid]));
        sm.qdiv[2 * tid] = f.m;
        sm.qdiv[2 * tid + 1] = f.sh;
    }
    const FastDiv div_wc = make_div((uint32_t)wc), div_zs = make_div((uint32_t)J.zstride);
    cluster_barrier(pt.C);
    const int zn = KIND == SQA_KIND_SQA ? (zr >> 1) : zr;
    int cz[kMaxColours];
#pragma unroll
    for (int c = 0; c < kMaxColours; c++)
        cz[c] = c >= J.ncol ? 1
                : J.task_slices > 0 ? min(min(J.task_slices, kTaskSlices), zn)
                                    : chunk_for((J.col_ptr[c + 1] - J.col_ptr[c]) * wc, zn, nthr);
    const int warp = tid >> 5, lane = tid & 31;
    uint2 *rq = sm.rq + (size_t)warp * kRequeue;

    for (int t = J.t0; t < J.t1; t++) {
        const PhiloxSweep ps = philox_sweep(J, (uint32_t)t, (uint32_t)inst);
        if (tid < 2 * wc) sm.ph[tid] = philox_word(J, ps, (uint32_t)(w0 + (tid >> 1)), (uint32_t)(tid & 1));
        if (KIND == SQA_KIND_SQA) {
            for (int i = tid; i < J.nrow; i += nthr) {
                const uint32_t T = __ldg(J.T + (size_t)t * J.nrow + i);
                sm.T[i] = T;
                if (!LUT) sm.Tb[i] = (uint8_t)(T >> 25);
            }
            __syncthreads();
            if (LUT) {
                build_luts<FOLD>(J, sm);
                __syncthreads();
            }
        }
        if (KIND == SQA_KIND_PT) __syncthreads();  // the sweep's hoisted Philox values
        const int nph = KIND == SQA_KIND_SQA ? 2 * J.ncol : J.ncol;
        for (int cls = 0; cls < nph; cls++) {
            const int chi = KIND == SQA_KIND_SQA ? cls >> 1 : cls, par = KIND == SQA_KIND_SQA ? cls & 1 : 0;
            const int c0 = J.col_ptr[chi], nq = J.col_ptr[chi + 1] - c0;
            int czc = cz[0];
#pragma unroll
            for (int c = 1; c < kMaxColours; c++)
                if (chi == c) czc = cz[c];
            const int ntasks = nq * wc * ((zn + czc - 1) / czc);
            const FastDiv div_nq{sm.qdiv[2 * chi], sm.qdiv[2 * chi + 1]};
            for (int tau = tid; tau < ntasks; tau += nthr) {
                const int r = (int)fdiv((uint32_t)tau, div_wc), w = tau - r * wc;
                const int ch = (int)fdiv((uint32_t)r, div_nq), q = r - ch * nq;
                const int si = c0 + q;
                const SiteRec &sr = sm.sites[si];
                Task tk;
                tk.si = si;
                tk.w = w;
                tk.gw = w0 + w;
                tk.wc = wc;
                tk.own = 4u * (uint32_t)(si * wc + w);
                tk.slot0 = (uint32_t)sr.canon * (uint32_t)Z;
                tk.valid = valid_bits(J.R, tk.gw);
                tk.lut = sm.lut + (uint32_t)si * kLutSlot;
                tk.swz = lut_swizzle(si);
                tk.ph0 = sm.ph[2 * w];
                tk.ph1 = sm.ph[2 * w + 1];
                if (FOLD) {
                    const uint4 rb = sm.rec[2 * si + 1];
                    const uint32_t pp[3] = {rb.x, rb.y, rb.z};
#pragma unroll
                    for (int k = 0; k < kMaxTerms; k++)
                        tk.nb[k] = 4u * ((uint32_t)(pp[k >> 1] >> (16 * (k & 1)) & 0xFFFFu) * (uint32_t)wc + (uint32_t)w);
                }
                const int zlo = ch * czc, zhi = min(zn, zlo + czc);
                const int dz = KIND == SQA_KIND_SQA ? 2 : 1, zl0 = KIND == SQA_KIND_SQA ? 2 * zlo + par : zlo;
                uint32_t tm[kTaskSlices];
#pragma unroll
                for (int i = 0; i < kTaskSlices; i++)
                    tm[i] = zlo + i < zhi ? metro_item<KIND, LUT, PAIRS>(J, ps, sm, pt, tk, sr, zl0 + i * dz) : 0u;
                store_task_ties(sm, tau, czc, tm);
            }
            __syncthreads();  // the phase's tie array is complete
            {
                LoKeys lk;
#pragma unroll
                for (int r = 0; r < 10; r++) {
                    lk.a[r] = J.rk0[r];
                    lk.b[r] = J.rk_lo[r];
                }
                // the item of tie-array word p: task p / czc, slice or slot p % czc
                const auto resolve_at = [&](uint32_t p, uint32_t tmv) -> uint32_t {
                    const uint32_t tau = czc == 4 ? p >> 2 : czc == 2 ? p >> 1 : czc == 1 ? p : __umulhi(p, 0xAAAAAAABu) >> 1;
                    const uint32_t i = p - tau * (uint32_t)czc;
                    const uint32_t r = fdiv(tau, div_wc), w = tau - r * (uint32_t)wc;
                    const uint32_t ch = fdiv(r, div_nq), q = r - ch * (uint32_t)nq;
                    const int zz = (int)(ch * (uint32_t)czc + i);
                    const int zl = KIND == SQA_KIND_SQA ? 2 * zz + par : zz;
                    if (!(SQA_IN(kChkItem, q, nq) && SQA_IN(kChkItem, zl, zr) && SQA_IN(kChkItem, w, wc))) return 0u;
                    return resolve_ties<KIND, LUT, PAIRS, false>(J, sm, pt, lk, inst, w0, wc, t, c0 + (int)q, zl, (int)w,
                                                                 tmv);
                };
                // each warp scans its share of the array, gathers the tied
                // items on its list and resolves one tie of 32 of them at a
                // time (every lane busy); items with ties left go back on
                // the list.  The list holds 63 entries at most: rounds run
                // until fewer than 32 are left before a scan step adds at
                // most 32 (a round takes 32 off before it puts at most 32
                // back, and every round resolves 32 ties, so they end).
                const uint32_t lt = (1u << lane) - 1u;
                const auto round = [&](uint32_t nl) -> uint32_t {
                    __syncwarp();
                    const bool mine = (uint32_t)lane < nl, tail = 32u + (uint32_t)lane < nl;
                    const uint2 en = mine ? rq[lane] : make_uint2(0u, 0u);
                    const uint2 tl = tail && SQA_IN(kChkRequeue, 32 + lane, kRequeue) ? rq[32 + lane]
                                                                                       : make_uint2(0u, 0u);
                    __syncwarp();
                    if (tail) rq[lane] = tl;
                    const uint32_t m = nl > 32u ? nl - 32u : 0u;
                    const uint32_t left = mine ? resolve_at(en.x, en.y) : 0u;
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, left != 0u);
                    __syncwarp();
                    const uint32_t slot = m + (uint32_t)__popc(bal & lt);
                    if (left && SQA_IN(kChkRequeue, slot, kRequeue)) rq[slot] = make_uint2(en.x, left);
                    return m + (uint32_t)__popc(bal);
                };
                const uint32_t npos = (uint32_t)(ntasks * czc);
                uint32_t nl = 0u;
                for (uint32_t base = (uint32_t)(tid - lane); base < npos; base += (uint32_t)nthr) {
                    const uint32_t p = base + (uint32_t)lane;
                    const uint32_t tmv = p < npos && SQA_IN(kChkTieArray, p, sm.tq_words) ? sm.tq[p] : 0u;
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, tmv != 0u);
                    __syncwarp();
                    const uint32_t slot = nl + (uint32_t)__popc(bal & lt);
                    if (tmv && SQA_IN(kChkRequeue, slot, kRequeue)) rq[slot] = make_uint2(p, tmv);
                    nl += (uint32_t)__popc(bal);
                    while (nl >= 32u) nl = round(nl);
                }
                while (nl > 0u) nl = round(nl);
            }
            if (KIND == SQA_KIND_SQA)
                cluster_barrier(pt.C);  // neighbouring blocks read this phase's boundary slices
            else
                __syncthreads();
        }
        if (KIND == SQA_KIND_PT && Z > 1 && (t + 1) % J.swap_every == 0)
            pt_swap(J, sm, pt, inst, w0, wc, (t + 1) / J.swap_every - 1);
    }
    for (int i = tid; i < zr * n * wc; i += nthr) {
        const int w = i % wc, r = i / wc, si = r % n, zl = r / n;
        const size_t g = (((size_t)inst * Z + z0 + zl) * n + si) * J.W + w0 + w;
        if (SQA_IN(kChkState, g, n_state)) J.state[g] = sm.S[(size_t)zl * J.zstride + si * wc + w];
    }
    cluster_barrier(pt.C);  // no block restages while another still reads its slices
}

// One job: the descriptor is a kernel parameter, so its fields (the Philox
// keys among them) are uniform across the grid.  One instantiation per path
// (0 / 6 PT, 1 SQA windows, 2 / 5 SQA tables, 3 / 4 SQA cluster moves) so each gets
// its own registers: three blocks of 256 threads per SM (80 registers) for
// the SQA paths but the cluster moves on rings of up to 64 slices, which fit
// four (64 registers, no spills); PT runs two blocks of 384 threads (a PT
// job usually has one unit per ladder, fewer units than block slots, so
// wider blocks give the busy SMs more warps).  Units go to clusters in turn (all units of a job
// cost the same).  The two-spin-term table path (5) folds the weights' signs
// into its code tables (FOLD): the items never load the weights.  Measured
// against term-value codes: +4.7 % on this path, while folding on the
// general-term path ran 0.6 % slower, so that path keeps term-value codes.
// The multi-job kernels below are instantiated per path the same way.
template <int MODE>
__global__ void __launch_bounds__(MODE == 0 || MODE == 6 ? 384 : 256, MODE == 3 ? 4 : (MODE == 0 || MODE == 6 ? 2 : 3))
    sweep_kernel_one(const __grid_constant__ JobDev J, const Unit *units, int n_units, int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem sm = carve(J, smem_raw);
    const int C = J.csize;
    const int cid = (int)blockIdx.x / C, ncl = (int)gridDim.x / C;
    for (int ui = cid; ui < n_units; ui += ncl) {
        const Unit u = units[ui];
        if (MODE == 0)
            run_unit<SQA_KIND_PT, false, false>(J, sm, u);
        else if (MODE == 6)
            run_unit<SQA_KIND_PT, false, true>(J, sm, u);
        else if (MODE == 2)
            run_unit<SQA_KIND_SQA, true, false>(J, sm, u);
        else if (MODE == 5)
            run_unit<SQA_KIND_SQA, true, true>(J, sm, u);
        else if (MODE == 3)
            run_unit_wolff<2>(J, sm, u);
        else if (MODE == 4)
            run_unit_wolff<4>(J, sm, u);
        else
            run_unit<SQA_KIND_SQA, false, false>(J, sm, u);
    }
}

// Host side of the single-job kernel: its entry for a job's path, and the
// launch (a cluster launch when the job's units span several blocks).
// Modes: 0 PT, 1 SQA windows, 2 SQA tables, 3 / 4 SQA cluster moves with
// 2 / 4 slices per lane (L <= 64 / L <= 128), 5 / 6 SQA tables / PT with
// two-spin terms only (minor embedding).
static int one_mode(const JobDev &J)
{
    if (J.kind == SQA_KIND_PT) return J.pairs ? 6 : 0;
    if (J.move == SQA_MOVE_WOLFF) return J.Z <= 64 ? 3 : 4;
    return J.use_lut ? (J.pairs ? 5 : 2) : 1;
}

const void *sweep_one_entry_mode(int mode)
{
    switch (mode) {
    case 0: return (const void *)sweep_kernel_one<0>;
    case 1: return (const void *)sweep_kernel_one<1>;
    case 2: return (const void *)sweep_kernel_one<2>;
    case 3: return (const void *)sweep_kernel_one<3>;
    case 4: return (const void *)sweep_kernel_one<4>;
    case 5: return (const void *)sweep_kernel_one<5>;
    default: return (const void *)sweep_kernel_one<6>;
    }
}

const void *sweep_one_entry(const JobDev &J) { return sweep_one_entry_mode(one_mode(J)); }

int sweep_one_threads(const JobDev &J)
{
    const int m = one_mode(J);
    return m == 0 || m == 6 ? 384 : 256;
}

cudaError_t launch_sweep_one(const JobDev &J, const Unit *units, int n_units, int *counter, int grid,
                             cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)sweep_one_threads(J));
    cfg.dynamicSmemBytes = (size_t)J.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)J.csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (one_mode(J)) {
    case 0: return cudaLaunchKernelEx(&cfg, sweep_kernel_one<0>, J, units, n_units, counter);
    case 1: return cudaLaunchKernelEx(&cfg, sweep_kernel_one<1>, J, units, n_units, counter);
    case 2: return cudaLaunchKernelEx(&cfg, sweep_kernel_one<2>, J, units, n_units, counter);
    case 3: return cudaLaunchKernelEx(&cfg, sweep_kernel_one<3>, J, units, n_units, counter);
    case 4: return cudaLaunchKernelEx(&cfg, sweep_kernel_one<4>, J, units, n_units, counter);
    case 5: return cudaLaunchKernelEx(&cfg, sweep_kernel_one<5>, J, units, n_units, counter);
    default: return cudaLaunchKernelEx(&cfg, sweep_kernel_one<6>, J, units, n_units, counter);
    }
}

// Clusters of C blocks of this job's path that can be resident at once.
int max_active_clusters(const JobDev &J)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)J.csize * 1024u);
    cfg.blockDim = dim3((unsigned)sweep_one_threads(J));
    cfg.dynamicSmemBytes = (size_t)J.smem_bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)J.csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, sweep_one_entry(J), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Several jobs of one path (each unit in one block): each unit names its
// job; the block copies that job's descriptor into shared memory.  One
// instantiation per path, with the registers and blocks per SM of the
// single-job kernel of that path; a batch of mixed paths runs one
// persistent launch per path, one after another.
template <int MODE>
__global__ void __launch_bounds__(MODE == 0 || MODE == 6 ? 384 : 256, MODE == 3 ? 4 : (MODE == 0 || MODE == 6 ? 2 : 3))
    sweep_kernel_multi(const JobDev *jobs, const Unit *units, int n_units, int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_unit;
    __shared__ JobDev s_job;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int ui = s_unit;
        if (ui < n_units && threadIdx.x == 0) s_job = jobs[units[ui].job];
        __syncthreads();
        if (ui >= n_units) break;
        if (s_job.csize != 1) continue;  // units of this kernel live in one block
        const Unit u = units[ui];
        const Smem sm = carve(s_job, smem_raw);
        if (MODE == 0)
            run_unit<SQA_KIND_PT, false, false>(s_job, sm, u);
        else if (MODE == 6)
            run_unit<SQA_KIND_PT, false, true>(s_job, sm, u);
        else if (MODE == 2)
            run_unit<SQA_KIND_SQA, true, false>(s_job, sm, u);
        else if (MODE == 5)
            run_unit<SQA_KIND_SQA, true, true>(s_job, sm, u);
        else if (MODE == 3)
            run_unit_wolff<2>(s_job, sm, u);
        else if (MODE == 4)
            run_unit_wolff<4>(s_job, sm, u);
        else
            run_unit<SQA_KIND_SQA, false, false>(s_job, sm, u);
        __syncthreads();
    }
}

int sweep_mode(const JobDev &J) { return one_mode(J); }

int sweep_mode_threads(int mode) { return mode == 0 || mode == 6 ? 384 : 256; }

const void *sweep_multi_entry(int mode)
{
    switch (mode) {
    case 0: return (const void *)sweep_kernel_multi<0>;
    case 1: return (const void *)sweep_kernel_multi<1>;
    case 2: return (const void *)sweep_kernel_multi<2>;
    case 3: return (const void *)sweep_kernel_multi<3>;
    case 4: return (const void *)sweep_kernel_multi<4>;
    case 5: return (const void *)sweep_kernel_multi<5>;
    default: return (const void *)sweep_kernel_multi<6>;
    }
}

cudaError_t launch_sweep_multi(int mode, int grid, int smem, const JobDev *jobs, const Unit *units, int n_units,
                               int *counter, cudaStream_t s)
{
    const dim3 g((unsigned)grid), b((unsigned)sweep_mode_threads(mode));
    switch (mode) {
    case 0: sweep_kernel_multi<0><<<g, b, smem, s>>>(jobs, units, n_units, counter); break;
    case 1: sweep_kernel_multi<1><<<g, b, smem, s>>>(jobs, units, n_units, counter); break;
    case 2: sweep_kernel_multi<2><<<g, b, smem, s>>>(jobs, units, n_units, counter); break;
    case 3: sweep_kernel_multi<3><<<g, b, smem, s>>>(jobs, units, n_units, counter); break;
    case 4: sweep_kernel_multi<4><<<g, b, smem, s>>>(jobs, units, n_units, counter); break;
    case 5: sweep_kernel_multi<5><<<g, b, smem, s>>>(jobs, units, n_units, counter); break;
    default: sweep_kernel_multi<6><<<g, b, smem, s>>>(jobs, units, n_units, counter); break;
    }
    return cudaGetLastError();
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
            for (int k = 0; k < x.size; k++)
                if (SQA_IN(kChkState, x.m[k], J.n)) v ^= st[(size_t)x.m[k] * J.W + gw];
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
        auto sig = [&](int si) -> int {
            if (!SQA_IN(kChkState, si, J.n)) return 1;
            return ((st[(size_t)si * J.W + gw] >> b) & 1u) ? -1 : 1;
        };
        int8_t q[kMaxN];
        if (D.method == SQA_DECODE_ME_MV) {
            const int len = D.Lc + 1;
            for (int l = 0; l < N; l++) {
                int sum = 0;
                for (int k = 0; k < len; k++) sum += sig(D.chain[l * len + k]);
                q[l] = (int8_t)(sum > 0 ? 1 : (sum < 0 ? -1 : sig(D.chain[l * len])));
            }
        } else if (D.method == SQA_DECODE_LHZ_BP) {
            // belief propagation: rows of pair values as bit masks (bit c of
            // P[a] set <-> p_ac = -1); the N-2 checks of pair (a,c) sum to
            // (N-2) - 2 popc((P[a] ^ P[c]) without bits a, c)
            uint32_t P[32], S0[32], Q[32];
            for (int a = 0; a < N; a++) {
                uint32_t g = 0u;
                for (int c = 0; c < N; c++)
                    if (c != a && sig(D.pair[a * N + c]) < 0) g |= 1u << c;
                P[a] = S0[a] = g;
            }
            const uint32_t all = N == 32 ? 0xFFFFFFFFu : ((1u << N) - 1u);
            for (int it = 0; it < D.bp_iters; it++) {
                for (int a = 0; a < N; a++) Q[a] = 0u;
                for (int a = 0; a < N; a++)
                    for (int c = a + 1; c < N; c++) {
                        const int mis = __popc((P[a] ^ P[c]) & all & ~(1u << a) & ~(1u << c));
                        const int S = (N - 2) - 2 * mis;
                        const int dec = D.bp_dec[(S0[a] >> c) & 1u][S + N - 2];
                        const bool neg = dec == 0 ? ((P[a] >> c) & 1u) != 0 : dec < 0;
                        if (neg) {
                            Q[a] |= 1u << c;
                            Q[c] |= 1u << a;
                        }
                    }
                for (int a = 0; a < N; a++) P[a] = Q[a];
            }
            const int *par = D.parents + (size_t)inst * D.n_trees * N;  // tree 0
            const int *ord = D.orders + (size_t)inst * D.n_trees * N;
            q[0] = 1;
            for (int k = 1; k < N; k++) {
                const int x = ord[k], p = par[x];
                q[x] = (int8_t)(q[p] * (((P[p] >> x) & 1u) ? -1 : 1));
            }
        } else if (D.method == SQA_DECODE_LHZ_MWD) {
            // minimum-weight decoding: walk the 2^(N-1) assignments with
            // q_{N-1} = +1 in Gray-code order; M counts the pair spins that
            // disagree with q_a q_b (bit a of X set <-> q_a = -1, bit b of
            // G[a] set <-> pair spin (a,b) is -1).  Flipping bit k toggles
            // the N-1 pairs at k.
            uint32_t G[24];
            for (int a = 0; a < N; a++) {
                uint32_t g = 0u;
                for (int c = 0; c < N; c++)
                    if (c != a && sig(D.pair[a * N + c]) < 0) g |= 1u << c;
                G[a] = g;
            }
            const uint32_t all = N == 32 ? 0xFFFFFFFFu : ((1u << N) - 1u);
            int M = 0;
            for (int a = 0; a < N; a++) M += __popc(G[a] & ~((2u << a) - 1u));
            uint32_t X = 0u, bestX = 0u;
            int bestM = M;
            const uint32_t steps = 1u << (N - 1);
            for (uint32_t k2 = 1; k2 < steps; k2++) {
                const int k = __ffs(k2) - 1;
                const uint32_t xk = (X >> k) & 1u ? all : 0u;
                const int mis = __popc((G[k] ^ X ^ xk) & all & ~(1u << k));
                M += (N - 1) - 2 * mis;
                X ^= 1u << k;
                if (M < bestM || (M == bestM && X < bestX)) {
                    bestM = M;
                    bestX = X;
                }
            }
            for (int l = 0; l < N; l++) q[l] = (int8_t)((bestX >> l) & 1u ? -1 : 1);
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

extern "C" {

int32_t sqa_bounds_checked(void)
{
#ifdef SQA_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

sqa_status sqa_check_status(uint32_t *record)
{
    if (!record) return sqa::set_error("NULL record"), SQA_ERR_INVALID;
    for (int k = 0; k < 4; k++) record[k] = 0u;
#ifdef SQA_BOUNDS_CHECK
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(record, sqa::g_check, 4 * sizeof(uint32_t));
    const uint32_t zero[4] = {0u, 0u, 0u, 0u};
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(sqa::g_check, zero, sizeof(zero));
    if (e != cudaSuccess) return sqa::cuda_fail(e, "sqa_check_status");
    if (record[0] != 0u) {
        sqa::set_error("bounds check: " + std::to_string(record[0]) + " violation(s), first at check site " +
                       std::to_string(record[1]) + ", index " + std::to_string(record[2]) + " of bound " +
                       std::to_string(record[3]));
        return SQA_ERR_BOUNDS;
    }
#endif
    return SQA_OK;
}

}  // extern "C"
