// Shared-memory layout of one unit of the sweep kernel, computed the same way
// on the host (launch sizing) and on the device (carving).
#pragma once
#include <stddef.h>

#include "sqa_internal.h"

#if defined(__CUDACC__)
#define SQA_LHD __host__ __device__ __forceinline__
#else
#define SQA_LHD inline
#endif

namespace sqa {

// Per-site byte tables of the single-spin sweep: one 256-byte slot per site,
// each starting on a 256-byte boundary of the shared window, so that a
// replica's 8-bit code placed in the low byte of the slot's address is the
// entry's address.
constexpr int kLutSlot = 256;

struct SmemOffsets {
    size_t S;      // state [zr][zstride] words (this block's slices or slots; word n*wc.. of a row: zero slot)
    size_t T;      // full thresholds: SQA one row, PT P rows
    size_t Tb;     // top 7 bits of the thresholds (T >> 25), bytes: PT P rows, SQA window mode one row
    size_t lut;    // SQA table mode: per-site byte tables (n slots of kLutSlot, plus alignment slack)
    size_t sites;  // SiteRec [n]
    size_t E;      // PT: energies [P][wc*32]
    size_t M;      // PT: swap masks [P/2+1][wc]; cluster moves: per-warp start masks [8][64 or 128]
    size_t Q;      // 64 bytes: from byte 16, per colour the divisor of the task decode
    size_t P;      // single-spin sweep: per word of the unit and SWEEP_HI block, the sweep's
                   // slice-independent Philox values {P0, Q2, O3, 0} (4 words)
    size_t R;      // single-spin sweep: per site, the tie record (kTieRec bytes)
    size_t RQ;     // single-spin sweep: per warp, kRequeue tie-queue entries (uint2)
    size_t total;
};

SQA_LHD size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

constexpr int kTieRec = 32;     // per-site tie record: threshold-index base and weights, neighbours
constexpr int kRequeue = 64;    // per-warp list of tied items of a tie pass
constexpr int kTaskSlices = 4;  // slices (SQA: slice pairs) or slots per task of the single-spin sweep
constexpr int kMaxWarps = 12;   // warps per block (384 threads) the layout provides for

// Items of one colour phase of a block (SQA: colour x slice parity; PT:
// colour), at most: every one of them may tie (two equal 7-bit high parts,
// probability 1 - (127/128)^32 = 0.222 for a full word), so this many
// entries of the block's tie queue hold any phase.
SQA_LHD int tie_items(const JobDev &J, int wc)
{
    int nq = 0;
    for (int c = 0; c < J.ncol; c++) nq = J.col_ptr[c + 1] - J.col_ptr[c] > nq ? J.col_ptr[c + 1] - J.col_ptr[c] : nq;
    return nq * (J.kind == SQA_KIND_SQA ? (J.zr + 1) / 2 : J.zr) * wc;
}

SQA_LHD SmemOffsets smem_layout(const JobDev &J, int wc, int zstride)
{
    SmemOffsets o;
    size_t off = 0;
    o.S = off;
    off += (size_t)J.zr * zstride * 4;
    if (J.kind == SQA_KIND_SQA && J.move == SQA_MOVE_WOLFF) {
        // cluster moves: the state, the site records and, per warp, the
        // start masks of one ring (M): no threshold rows, tables or queue
        o.T = o.Tb = o.lut = o.Q = o.P = o.R = o.RQ = off;
        off = align16(off);
        o.sites = off;
        off += (size_t)J.n * sizeof(SiteRec);
        off = align16(off);
        o.E = o.M = off;
        off += (size_t)(256 / 32) * (J.Z <= 64 ? 64 : 128) * 4;
        o.total = align16(off);
        return o;
    }
    o.T = off;
    off += (size_t)(J.kind == SQA_KIND_SQA ? J.nrow : J.zr * J.nrow) * 4;
    o.Tb = off;
    if (J.kind == SQA_KIND_PT)
        off += (size_t)J.zr * J.nrow;
    else if (!J.use_lut)
        off += (size_t)J.nrow;
    off = align16(off);
    o.lut = off;
    if (J.kind == SQA_KIND_SQA && J.use_lut) off += (size_t)(J.n + 1) * kLutSlot;
    off = align16(off);
    o.sites = off;
    off += (size_t)J.n * sizeof(SiteRec);
    o.E = off;
    o.M = off;
    if (J.kind == SQA_KIND_PT) {
        off += (size_t)J.zr * wc * 32 * 4;
        o.M = off;
        off += (size_t)(J.zr / 2 + 1) * wc * 4;
    }
    off = align16(off);
    o.Q = off;
    off += 64;
    o.P = off;
    off += (size_t)wc * 2 * 16;
    o.R = off;
    off += (size_t)J.n * kTieRec;
    o.RQ = off;
    off += (size_t)kMaxWarps * kRequeue * 8;
    o.total = align16(off);
    return o;
}

}  // namespace sqa
