// perch_best_noalloc: the argmin of J = J_o + J_r for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc once they are running: a serving
// process that reserves all of its HBM up front and treats any later
// allocation as a fault (cudaMalloc can synchronise the device and stall the
// streams of every other request), or a host framework whose own allocator owns
// the device memory and must not see allocations it did not make.  Such callers
// cannot create a perch_ctx, whose creation allocates the argmin's scratch.
// This entry point needs no context: the argmin kernel's scratch (one partial
// result per block and a completion ticket) lives in the file-scope device
// array below, which every GPU that loads the library holds until the process
// exits.  The caller passes the inputs and outputs as device pointers.
#include "perch.h"
#include "perch_internal.cuh"

#include <mutex>

namespace {

// The argmin launches at most perch::kBestMaxBlocks blocks; each block leaves
// three 64-bit words, and one more word holds the ticket.
constexpr int kScratchWords = 3 * perch::kBestMaxBlocks + 32;   // 24.8 KB
static_assert(kScratchWords >= 3 * perch::kBestMaxBlocks + 1, "partials plus the ticket");

static __device__ __align__(256) unsigned long long g_best_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_scratch_addr[kMaxDevices] = {};

// Device address of g_best_scratch on the current device, looked up once per
// device.  The host-side symbol is only a stand-in: kernels must be given the
// address that cudaGetSymbolAddress returns.
cudaError_t scratch_on_current_device(unsigned long long** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_best_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// True iff p is device memory of the current device (not host, pinned host
// or managed memory, and not another GPU's): the kernel would fault, or
// silently read host memory, on anything else.
bool on_current_device(const void* p, int dev)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" perch_status perch_best_noalloc(const int32_t* costs, const uint64_t* ids, int64_t n,
                                           int64_t* best_index, int32_t* best_cost,
                                           void* cuda_stream)
{
    if (!costs || !best_index || !best_cost) return PERCH_E_INVALID;
    if (n < 1 || n > 0x7FFFFFFFll) return PERCH_E_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PERCH_E_CUDA;
    }
    if (!on_current_device(costs, dev) || !on_current_device(best_index, dev) ||
        !on_current_device(best_cost, dev) || (ids && !on_current_device(ids, dev)))
        return PERCH_E_INVALID;
    unsigned long long* scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PERCH_E_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    perch::BestArgs a{};
    a.costs = costs;
    a.ids = reinterpret_cast<const unsigned long long*>(ids);
    a.n = n;
    a.best_index = reinterpret_cast<long long*>(best_index);
    a.best_cost = best_cost;
    a.partial = scratch;
    a.ticket = reinterpret_cast<unsigned*>(scratch + 3 * perch::kBestMaxBlocks);
    // the ticket must start at zero; the partials are written before they are read
    e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = perch::launch_best(a, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PERCH_E_CUDA;
    }
    return PERCH_OK;
}
