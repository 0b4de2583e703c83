// Bounds checks of the checked build (compiled with -DSQA_BOUNDS_CHECK).
//
// Every check tests an index (or a shared-window byte address) against the
// size of the buffer it selects from, before the access.  An index out of
// range is recorded in a device status word and the access is skipped: a
// load reads 0 and a store does nothing, so the kernel runs to its end and
// the context stays usable.  No check traps.  The host reads and clears the
// record with sqa_check_status().  Without SQA_BOUNDS_CHECK every check is
// the constant true and compiles away.
#pragma once
#include <stdint.h>

namespace sqa {

// Where a violation was found (record[1] of sqa_check_status).
enum CheckSite : uint32_t {
    kChkShared = 1,     // a shared-memory load or store outside the block's dynamic window
    kChkState = 2,      // a global state word index
    kChkThreshold = 3,  // a threshold-row index (threshold index U or its row)
    kChkTieArray = 4,   // a word of the block's tie array
    kChkRequeue = 5,    // an entry of a warp's tie list
    kChkItem = 6,       // a site, slice or word decoded from a tie-array position
    kChkNeighbour = 7,  // a word of a neighbouring block's slices (cluster)
    kChkSwap = 8,       // a PT energy, swap mask or swap-threshold index
    kChkRing = 9,       // a word of a cluster-move ring
};

#ifdef SQA_BOUNDS_CHECK
// record: [0] violations, [1] site of the first, [2] its index, [3] its bound
// (defined here: the one translation unit with kernels includes this header)
__device__ unsigned int g_check[4];

__device__ __noinline__ void check_fail(uint32_t site, uint32_t idx, uint32_t bound)
{
    if (atomicAdd(&g_check[0], 1u) == 0u) {
        g_check[1] = site;
        g_check[2] = idx;
        g_check[3] = bound;
    }
}

// true when 0 <= idx < bound; records the violation otherwise
__device__ __forceinline__ bool in_range(uint32_t site, long long idx, long long bound)
{
    if (idx >= 0 && idx < bound) return true;
    check_fail(site, (uint32_t)idx, (uint32_t)bound);
    return false;
}

// true when [a, a + bytes) lies in this block's dynamic shared memory
__device__ __forceinline__ bool shared_ok(uint32_t a, uint32_t bytes)
{
    extern __shared__ __align__(16) unsigned char sqa_dyn_smem[];
    const uint32_t lo = (uint32_t)__cvta_generic_to_shared(sqa_dyn_smem);
    uint32_t sz;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(sz));
    if (a >= lo && a - lo + bytes <= sz) return true;
    check_fail(kChkShared, a, lo + sz);
    return false;
}
#define SQA_IN(site, idx, bound) ::sqa::in_range((site), (long long)(idx), (long long)(bound))
#define SQA_SHARED_OK(a, bytes) ::sqa::shared_ok((a), (bytes))
#else
#define SQA_IN(site, idx, bound) true
#define SQA_SHARED_OK(a, bytes) true
#endif

}  // namespace sqa
