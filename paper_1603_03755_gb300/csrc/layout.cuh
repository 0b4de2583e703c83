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

struct SmemOffsets {
    size_t S;      // state [zr][zstride] words (this block's slices or slots; word n*wc.. of a row: zero slot)
    size_t T;      // full thresholds: SQA one row, PT P rows
    size_t Tq;     // high halves of the thresholds (T & 0xFFFF0000): PT P rows, SQA window mode one row
    size_t lut;    // SQA: per-site tables of threshold high halves
    size_t sites;  // SiteRec [n]
    size_t E;      // PT: energies [P][wc*32]
    size_t M;      // PT: swap masks [P/2+1][wc]; cluster moves: per-warp start masks [8][64 or 128]
    size_t total;
};

SQA_LHD size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

SQA_LHD SmemOffsets smem_layout(const JobDev &J, int wc, int zstride)
{
    SmemOffsets o;
    size_t off = 0;
    o.S = off;
    off += (size_t)J.zr * zstride * 4;
    if (J.kind == SQA_KIND_SQA && J.move == SQA_MOVE_WOLFF) {
        // cluster moves: the state, the site records and, per warp, the
        // start masks of one ring (M): no threshold rows or tables
        o.T = o.Tq = o.lut = off;
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
    o.Tq = off;
    if (J.kind == SQA_KIND_PT)
        off += (size_t)J.zr * J.nrow * 4;
    else if (!J.use_lut)
        off += (size_t)J.nrow * 4;
    o.lut = off;
    if (J.kind == SQA_KIND_SQA && J.use_lut) off += (size_t)J.lut_entries * 4;
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
    o.total = align16(off);
    return o;
}

}  // namespace sqa
