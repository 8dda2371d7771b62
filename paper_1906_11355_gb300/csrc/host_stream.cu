// host_stream.cu -- mclahe_forward_host: many volumes of one plan that live in
// host memory, each copied in, mapped (Algorithm 1) and copied out, with the
// copies of neighbouring volumes overlapping.
//
// Two device slots (input buffer, output buffer, workspace) alternate between
// the volumes.  Volume v uses slot s = v mod 2:
//   copy-in stream   waits until the forward of volume v - 2 has read slot s's
//                    input, copies h_in[v] into it, records in_ready[s];
//   caller's stream  waits for in_ready[s] and for the copy-out of volume
//                    v - 2 (slot s's output is free), runs the forward pass,
//                    records fwd_done[s];
//   copy-out stream  waits for fwd_done[s], copies the output to h_out[v],
//                    records out_free[s].
// So while volume v is mapped, volume v + 1 is copied in and volume v - 1 is
// copied out: both copy directions and the kernels run at once.  The caller's
// stream finally waits for the last copies.  The copy streams and events
// belong to the library (one set per device, kept for the process); one call
// is enqueued at a time.
#include <map>
#include <mutex>

#include "mclahe_internal.cuh"

namespace mclahe {
namespace {

struct HostStreams {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t start = nullptr, in_ready[2] = {}, fwd_done[2] = {}, out_free[2] = {};
    bool ok = false;
};
std::mutex g_host_mutex;
std::map<int, HostStreams> g_host;

HostStreams *host_streams() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    HostStreams &h = g_host[dev];
    if (!h.ok) {
        if (cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming) != cudaSuccess)
            return nullptr;
        for (int s = 0; s < 2; ++s)
            if (cudaEventCreateWithFlags(&h.in_ready[s], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h.fwd_done[s], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h.out_free[s], cudaEventDisableTiming) != cudaSuccess)
                return nullptr;
        h.ok = true;
    }
    return &h;
}

size_t elem_bytes(mclahe_dtype t) { return t == MCLAHE_U16 ? 2 : t == MCLAHE_U8 ? 1 : 4; }

}  // namespace
}  // namespace mclahe

using namespace mclahe;

extern "C" mclahe_status mclahe_forward_host(mclahe_plan_t p, mclahe_dtype dtype, int n_vol,
                                             const void *const *h_in, float *const *h_out,
                                             void *const *d_in, float *const *d_out,
                                             void *const *d_ws, size_t ws_bytes, const float *d_clip,
                                             mclahe_stream_t stream) {
    if (!p || n_vol < 0 || (dtype != MCLAHE_F32 && dtype != MCLAHE_U16 && dtype != MCLAHE_U8))
        return MCLAHE_ERR_INVALID_ARG;
    if (n_vol == 0) return MCLAHE_OK;
    if (!h_in || !h_out || !d_in || !d_out || !d_ws) return MCLAHE_ERR_INVALID_ARG;
    if (d_clip && (reinterpret_cast<uintptr_t>(d_clip) & 3)) return MCLAHE_ERR_INVALID_ARG;
    for (int s = 0; s < 2; ++s) {
        const mclahe_status st = check_forward_args(p, d_in[s], d_out[s], d_ws[s], ws_bytes);
        if (st != MCLAHE_OK) return st;
    }
    if (d_in[0] == d_in[1] || d_out[0] == d_out[1] || d_ws[0] == d_ws[1] ||
        static_cast<const void *>(d_out[0]) == d_in[1] || static_cast<const void *>(d_out[1]) == d_in[0])
        return MCLAHE_ERR_INVALID_ARG;
    for (int v = 0; v < n_vol; ++v)
        if (!h_in[v] || !h_out[v]) return MCLAHE_ERR_INVALID_ARG;
    const size_t in_bytes = size_t(p->g.N) * elem_bytes(dtype);
    const size_t out_bytes = size_t(p->g.N) * sizeof(float);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    std::lock_guard<std::mutex> lock(g_host_mutex);
    HostStreams *h = host_streams();
    if (!h) return MCLAHE_ERR_CUDA;
    // the slots may still be in use by work enqueued on the caller's stream
    if (cudaEventRecord(h->start, st) != cudaSuccess || cudaStreamWaitEvent(h->in, h->start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(h->out, h->start, 0) != cudaSuccess)
        return MCLAHE_ERR_CUDA;
    for (int v = 0; v < n_vol; ++v) {
        const int s = v & 1;
        if (v >= 2 && cudaStreamWaitEvent(h->in, h->fwd_done[s], 0) != cudaSuccess) return MCLAHE_ERR_CUDA;
        if (cudaMemcpyAsync(d_in[s], h_in[v], in_bytes, cudaMemcpyHostToDevice, h->in) != cudaSuccess ||
            cudaEventRecord(h->in_ready[s], h->in) != cudaSuccess)
            return MCLAHE_ERR_CUDA;
        if (cudaStreamWaitEvent(st, h->in_ready[s], 0) != cudaSuccess) return MCLAHE_ERR_CUDA;
        if (v >= 2 && cudaStreamWaitEvent(st, h->out_free[s], 0) != cudaSuccess) return MCLAHE_ERR_CUDA;
        const mclahe_status fs = mclahe_forward_typed(p, dtype, d_in[s], d_out[s], d_ws[s], ws_bytes,
                                                      d_clip ? d_clip + v : nullptr, stream);
        if (fs != MCLAHE_OK) return fs;
        if (cudaEventRecord(h->fwd_done[s], st) != cudaSuccess ||
            cudaStreamWaitEvent(h->out, h->fwd_done[s], 0) != cudaSuccess ||
            cudaMemcpyAsync(h_out[v], d_out[s], out_bytes, cudaMemcpyDeviceToHost, h->out) != cudaSuccess ||
            cudaEventRecord(h->out_free[s], h->out) != cudaSuccess)
            return MCLAHE_ERR_CUDA;
    }
    // the caller's stream continues after the last copies out
    for (int s = 0; s < 2 && s < n_vol; ++s)
        if (cudaStreamWaitEvent(st, h->out_free[s], 0) != cudaSuccess) return MCLAHE_ERR_CUDA;
    return MCLAHE_OK;
}
