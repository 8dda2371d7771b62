// noalloc.cu -- mclahe_forward_noalloc: the forward pass for callers that
// cannot allocate device memory.
//
// mclahe_forward needs a caller-allocated workspace for the per-kernel range
// keys, histograms and mapping tables.  Some callers have no way to provide
// one: a plugin or custom-operator interface that hands over only the input
// and output buffers, code that runs where allocation is forbidden or would
// break a fixed memory budget, or a foreign-language caller without a CUDA
// allocator.  This entry point takes its workspace from a fixed array that is
// part of the library image instead.
//
// The array lives in device global memory; every GPU on which the library is
// used holds MCLAHE_NOALLOC_SCRATCH_BYTES of it until the process exits.  Host
// code cannot use the array's name as a device address, so every call looks
// the address up with cudaGetSymbolAddress on the current device (a host-side
// lookup; the first one on a device may load the library's device code, so
// that first call should come before any stream capture).  Looking it up per
// call keeps the address right even if the device's context was reset and the
// module reloaded.  All calls share the one array, so calls whose work
// overlaps on the GPU (other streams, other threads) race; the forward pass
// clears the parts that must start at zero on every call.  The array's first
// word is the status word of its workspace: mclahe_noalloc_sync_status reads
// and clears it.
#include <mutex>

#include "mclahe_internal.cuh"

namespace mclahe {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MCLAHE_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_setup_mutex;

// Device address of the scratch array on the current device.
cudaError_t scratch_address(unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}
}  // namespace

}  // namespace mclahe

using namespace mclahe;

extern "C" mclahe_status mclahe_forward_noalloc(mclahe_plan_t p, const float *d_in, float *d_out,
                                                const float *d_clip, mclahe_stream_t stream) {
    if (!p) return MCLAHE_ERR_INVALID_ARG;
    // the forward pass uses the workspace up to the start of the backward scratch
    const size_t need = p->ws.scratch;
    if (need > size_t(MCLAHE_NOALLOC_SCRATCH_BYTES)) return MCLAHE_ERR_UNSUPPORTED;
    if (!d_in || !d_out || d_in == d_out) return MCLAHE_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_in) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15))
        return MCLAHE_ERR_INVALID_ARG;
    unsigned char *ws = nullptr;
    if (scratch_address(&ws) != cudaSuccess) return MCLAHE_ERR_CUDA;
    return forward_impl(*p, d_in, d_out, ws, d_clip, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" mclahe_status mclahe_noalloc_sync_status(mclahe_stream_t stream) {
    unsigned char *ws = nullptr;
    if (scratch_address(&ws) != cudaSuccess) return MCLAHE_ERR_CUDA;
    // the status word sits at offset 0 of every plan's workspace layout
    return mclahe_sync_status(ws, stream);
}
