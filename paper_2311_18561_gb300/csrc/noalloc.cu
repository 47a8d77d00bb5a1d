// noalloc.cu -- pvg_sort_pairs_noalloc: the stable radix sort of
// pvg_sort_pairs for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: code that runs while a CUDA graph
// is being captured, real-time or callback threads where an allocation can
// block on a device-wide synchronisation, and hosts whose memory manager
// forbids allocations outside its own pool.  This entry point runs the same
// kernels as pvg_sort_pairs but keeps all of its scratch (ping-pong key /
// value buffers, digit histograms, the element count) in the fixed arrays
// below, which live in this library's device image.  Every GPU that loads
// the library holds them (about 9.1 MiB: two 4 MiB ping-pong buffers and
// the sort's digit-histogram scratch, sized for up to 1024 sort blocks
// whatever the SM count) until the process exits.
//
// Host code cannot use these array names as device addresses (on the host
// they name host-side stand-ins), so each device's addresses are looked up
// once with cudaGetSymbolAddress while that device is current, and then
// passed to the kernels.
#include <mutex>

#include "../../include/pvg.h"
#include "pvg_internal.cuh"

namespace {

constexpr uint32_t kNoAllocMaxPairs = 1u << 20;               // 1,048,576 pairs
constexpr size_t kNoAllocTempBytes = pvg::kSortTempBytes;  // digit histograms + scan partials
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_noalloc_keys[kNoAllocMaxPairs];
static __device__ __align__(256) uint32_t g_noalloc_vals[kNoAllocMaxPairs];
static __device__ __align__(256) unsigned char g_noalloc_temp[kNoAllocTempBytes];
static __device__ __align__(256) uint32_t g_noalloc_count[4];

struct Scratch {
    uint32_t *keys = nullptr, *vals = nullptr, *count = nullptr;
    void *temp = nullptr;
};

std::mutex g_mutex;
Scratch g_scratch[kMaxDevices];
bool g_ready[kMaxDevices] = {};

// Device addresses of the fixed arrays on device `dev` (current).
pvg_status_t scratch_for(int dev, Scratch *out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_ready[dev]) {
        Scratch s;
        if (cudaGetSymbolAddress((void **)&s.keys, g_noalloc_keys) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&s.vals, g_noalloc_vals) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&s.count, g_noalloc_count) != cudaSuccess ||
            cudaGetSymbolAddress(&s.temp, g_noalloc_temp) != cudaSuccess) {
            cudaGetLastError();
            return PVG_ERR_CUDA;
        }
        g_scratch[dev] = s;
        g_ready[dev] = true;
    }
    *out = g_scratch[dev];
    return PVG_OK;
}

__global__ void k_noalloc_set_count(uint32_t *count, uint32_t n) { *count = n; }

}  // namespace

extern "C" pvg_status_t pvg_sort_pairs_noalloc(uint32_t *keys, uint32_t *vals, int64_t n, int32_t begin_bit,
                                               int32_t end_bit, void *stream) {
    if (n < 0 || n > (int64_t)kNoAllocMaxPairs || begin_bit < 0 || end_bit > 32 || begin_bit >= end_bit)
        return PVG_ERR_INVALID;
    if (n == 0) return PVG_OK;
    if (!keys || !vals) return PVG_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PVG_ERR_CUDA;
    }
    Scratch sc;
    const pvg_status_t st = scratch_for(dev, &sc);
    if (st != PVG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    pvg::note_launch();
    k_noalloc_set_count<<<1, 1, 0, s>>>(sc.count, (uint32_t)n);
    bool in_alt = false;
    pvg::radix_sort_pairs(keys, vals, sc.keys, sc.vals, sc.count, (uint32_t)n, begin_bit, end_bit, sc.temp, s,
                          &in_alt);
    if (in_alt) {
        if (cudaMemcpyAsync(keys, sc.keys, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(vals, sc.vals, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return PVG_ERR_CUDA;
        }
    }
    return cudaGetLastError() == cudaSuccess ? PVG_OK : PVG_ERR_CUDA;
}
