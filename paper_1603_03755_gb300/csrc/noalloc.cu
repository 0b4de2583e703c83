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
// address: the address is fetched with cudaGetSymbolAddress, once per device,
// on that device, by the first call there, and cached.  That first call should
// therefore come before any stream capture.  All calls share the array (the
// minima are reset at the start of each call), so calls that overlap on the
// GPU race with each other.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/sqa.h"

namespace sqa {

__global__ void ground_kernel(int N, const int32_t *J, int chunk_bits, int64_t n_chunks,
                              unsigned long long *best);
void set_error(const std::string &msg);

constexpr int kNoAllocMaxInstances = 4096;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_ground_minima[kNoAllocMaxInstances];

static std::mutex g_minima_mu;
static unsigned long long *g_minima_addr[kNoAllocMaxDevices];

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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        set_error("sqa_ground_energy_noalloc: no usable current device");
        return SQA_ERR_NO_DEVICE;
    }
    unsigned long long *minima = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_minima_mu);
        if (!g_minima_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_ground_minima);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                set_error(std::string("sqa_ground_energy_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return SQA_ERR_CUDA;
            }
            g_minima_addr[dev] = (unsigned long long *)p;
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
