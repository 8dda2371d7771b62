// launch_cache.cu -- per-process caches of host-side launch preparation: a
// kernel's dynamic shared-memory limit is raised once per (device, kernel)
// to the largest size asked so far, and occupancy queries are answered from
// a table.  Both are host calls costing microseconds, which would otherwise
// run before every launch (and leave the GPU idle behind short kernels).
#include <map>
#include <mutex>
#include <tuple>

#include "mclahe_internal.cuh"

namespace mclahe {

namespace {
std::mutex g_mu;
std::map<std::pair<int, const void *>, size_t> g_smem;
std::map<std::tuple<int, const void *, int, size_t>, int> g_occ;

int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev;
}
}  // namespace

cudaError_t ensure_smem(const void *func, size_t bytes) {
    const auto key = std::make_pair(current_device(), func);
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_smem.find(key);
    if (it != g_smem.end() && it->second >= bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) g_smem[key] = bytes;
    return e;
}

cudaError_t cached_occupancy(const void *func, int threads, size_t smem, int *per_sm) {
    const auto key = std::make_tuple(current_device(), func, threads, smem);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_occ.find(key);
        if (it != g_occ.end()) {
            *per_sm = it->second;
            return cudaSuccess;
        }
    }
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, func, threads, smem);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_mu);
        g_occ[key] = *per_sm;
    }
    return e;
}

}  // namespace mclahe
