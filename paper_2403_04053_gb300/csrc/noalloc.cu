// Allocation-free far-field cross-section.
//
// Some callers cannot allocate device memory once they are running: a service whose GPU
// memory budget is fixed and fully reserved at start-up, or a latency-critical loop in
// which an allocation (and the device-wide synchronisation cudaFree implies) is not
// acceptable.  pstd_cross_section_noalloc serves them: it is pstd_cross_section with
// device inputs and outputs, whose only scratch -- the per-split partial sums of the
// surface transform -- lives in the file-scope device array below instead of a buffer
// the grid allocates on demand.
//
// The array is kNoAllocScratchElems double2 entries (16 MiB) per device, held until the
// process exits.  Host code cannot use its name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device current)
// and caches it; every later call on the device reuses it.  Under CUDA's lazy module
// loading (the default) that lookup is also what loads the module on the device and
// commits the array, so the first call can fail for lack of memory: callers make it once
// at start-up, before their memory budget is reserved and before any stream capture.  Every call on a device shares the array and it keeps the last
// call's contents; nothing in it needs clearing, because the transform writes every
// entry it later reads.  Calls whose kernels overlap on the GPU (different streams, or
// different grids on one device) race on the array and must be serialised by the caller.
#include <mutex>

#include "pstd_internal.h"

namespace {

constexpr long long kNoAllocScratchElems = 1LL << 20;   // double2 entries = 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double2 g_noalloc_scratch[kNoAllocScratchElems];

std::mutex g_scratch_mutex;
double2* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" pstd_status pstd_cross_section_noalloc(pstd_grid* g, int b, int f, const double* theta, const double* phi,
                                                  long M, double* out_dsdo, void* out_f)
{
    if (!g) return pstd::grid_error(nullptr, PSTD_EINVAL, "null grid");
    if (M < 0 || (M > 0 && (!theta || !phi || !out_dsdo))) return pstd::grid_error(g, PSTD_EINVAL, "null argument or M < 0");
    if (M > kNoAllocScratchElems)
        return pstd::grid_error(g, PSTD_EINVAL, "pstd_cross_section_noalloc: M above the maximum of 1048576 directions");
    const int dev = pstd::grid_device(g);
    if (dev < 0 || dev >= kMaxDevices) return pstd::grid_error(g, PSTD_EINVAL, "device ordinal above 63");
    double2* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            int prev = -1;
            if (cudaGetDevice(&prev) != cudaSuccess) return pstd::grid_error(g, PSTD_ECUDA, "cudaGetDevice failed");
            if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return pstd::grid_error(g, PSTD_ECUDA, "cudaSetDevice failed");
            void* addr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (prev != dev) cudaSetDevice(prev);
            if (e != cudaSuccess || !addr)
                return pstd::grid_error(g, PSTD_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch array failed");
            g_scratch_addr[dev] = static_cast<double2*>(addr);
        }
        scratch = g_scratch_addr[dev];
    }
    if (M == 0) return PSTD_OK;
    // every caller pointer must be device (or managed) memory of the grid's device: a host or
    // other-device pointer would reach the kernels unchecked
    const void* ptrs[4] = {theta, phi, out_dsdo, out_f};
    for (const void* p : ptrs) {
        if (!p) continue;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return pstd::grid_error(g, PSTD_EINVAL, "pstd_cross_section_noalloc: argument is not a CUDA pointer");
        }
        const bool on_dev = (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
        if (!on_dev)
            return pstd::grid_error(g, PSTD_EINVAL, "pstd_cross_section_noalloc: arguments must be device memory of the grid's device");
    }
    return pstd::far_field_into_scratch(g, b, f, theta, phi, M, out_dsdo, static_cast<double2*>(out_f), scratch,
                                        kNoAllocScratchElems);
}
