// Exhaustive logical ground-state search that allocates no device memory.
//
// sqa_ground_energy (capi.cu) copies J to a cudaMalloc'd buffer and keeps the
// per-instance running minimum in a second cudaMalloc'd buffer.  Some callers
// cannot allocate: a serving process that reserved its whole device budget up
// front, or code running under a memory manager that owns every device byte
// and forbids ad-hoc cudaMalloc.  For them, sqa_ground_energy_noalloc takes J
// and the result as caller-owned device buffers and keeps the running minima
// in the fixed array below instead.
//
// The array is a file-scope __device__ variable, so every device that loads
// the library holds kNoAllocMaxInstances * 8 bytes (32 KiB) of it until the
// process exits.  In host code its name is only a stand-in, not a device
// address: the address is fetched with cudaGetSymbolAddress, on the device
// that is current, by the first call there, and cached together with the
// CUDA context it belongs to; a call that finds another context current (the
// device was reset, or its primary context destroyed and created again)
// fetches it again.  The first call on a device should therefore come before
// any stream capture.  All calls share the array (the minima are reset at the
// start of each call), so calls that overlap on the GPU race with each other.
#include <cuda.h>  // CUcontext only: the driver is reached through the runtime's entry-point query
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/sqa.h"

namespace sqa {

__global__ void ground_kernel(int N, const int32_t *J, int chunk_bits, int64_t n_chunks,
                              unsigned long long *best);
void set_error(const std::string &msg);

constexpr int kNoAllocMaxInstances = 4096;
constexpr int kNoAllocMaxDevices = 64;
constexpr int kGroundMaxStatesLog2 = 40;  // n_instances * 2^(N-1) states at most per call

static __device__ __align__(256) unsigned long long g_ground_minima[kNoAllocMaxInstances];

static std::mutex g_minima_mu;
static unsigned long long *g_minima_addr[kNoAllocMaxDevices];
static CUcontext g_minima_ctx[kNoAllocMaxDevices];

// The current CUDA context (null when it cannot be queried), through the
// runtime's driver entry-point query, so that the library needs no link
// against the driver library.
static CUcontext current_context()
{
    typedef CUresult (*get_ctx_fn)(CUcontext *);
    static get_ctx_fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (get_ctx_fn)p;
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

__global__ void noalloc_reset_minima(unsigned long long *best, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) best[i] = ~0ull;
}

// The search stores energies with the sign bit flipped so that unsigned
// atomicMin orders them as signed values; undo that into the caller's buffer.
__global__ void noalloc_write_energies(const unsigned long long *best, int n, int64_t *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int64_t)(best[i] ^ 0x8000000000000000ull);
}

}  // namespace sqa

using namespace sqa;

extern "C" sqa_status sqa_ground_energy_noalloc(int32_t N, int32_t n_instances, const int32_t *J_dev,
                                                int64_t *e_dev, void *stream)
{
    if (N < 2 || N > 40 || !J_dev || !e_dev || n_instances < 1) {
        set_error("sqa_ground_energy_noalloc: need 2 <= N <= 40, n_instances >= 1 and non-NULL buffers");
        return SQA_ERR_INVALID;
    }
    if (n_instances > kNoAllocMaxInstances) {
        set_error("sqa_ground_energy_noalloc: n_instances exceeds the fixed scratch of 4096 instances");
        return SQA_ERR_INVALID;
    }
    if ((double)n_instances * std::ldexp(1.0, N - 1) > std::ldexp(1.0, kGroundMaxStatesLog2)) {
        set_error("sqa_ground_energy_noalloc: n_instances * 2^(N-1) exceeds the search budget of 2^40 states");
        return SQA_ERR_UNSUPPORTED;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        set_error("sqa_ground_energy_noalloc: no usable current device");
        return SQA_ERR_NO_DEVICE;
    }
    // both buffers must be device (or managed) memory of the current device:
    // a host pointer or another device's buffer would be read out of place
    for (const void *p : {(const void *)J_dev, (const void *)e_dev}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            set_error("sqa_ground_energy_noalloc: a buffer is not a CUDA device pointer");
            return SQA_ERR_INVALID;
        }
        const bool on_device = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
        if (!on_device || (a.type == cudaMemoryTypeDevice && a.device != dev)) {
            set_error("sqa_ground_energy_noalloc: J_dev and e_dev must be device memory of the current device");
            return SQA_ERR_INVALID;
        }
    }
    unsigned long long *minima = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_minima_mu);
        const CUcontext ctx = current_context();
        if (!g_minima_addr[dev] || g_minima_ctx[dev] != ctx) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_ground_minima);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                set_error(std::string("sqa_ground_energy_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return SQA_ERR_CUDA;
            }
            g_minima_addr[dev] = (unsigned long long *)p;
            g_minima_ctx[dev] = ctx;
        }
        minima = g_minima_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int total_bits = N - 1;
    const int chunk_bits = total_bits > 17 ? total_bits - 17 : 0;
    const int64_t n_chunks = (int64_t)1 << (total_bits - chunk_bits);
    int64_t bx = (n_chunks + 127) / 128;
    if (bx > 2048) bx = 2048;
    const int nb = (n_instances + 255) / 256;
    noalloc_reset_minima<<<nb, 256, 0, s>>>(minima, n_instances);
    ground_kernel<<<dim3((unsigned)(bx < 1 ? 1 : bx), (unsigned)n_instances), 128, 0, s>>>(N, J_dev, chunk_bits,
                                                                                       n_chunks, minima);
    noalloc_write_energies<<<nb, 256, 0, s>>>(minima, n_instances, e_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("sqa_ground_energy_noalloc: ") + cudaGetErrorString(e));
        return SQA_ERR_CUDA;
    }
    return SQA_OK;
}
