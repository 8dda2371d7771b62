// batch.cu -- many volumes in one pass per phase (no counterpart in the paper).
#include "mclahe_internal.cuh"

extern "C" {

size_t mclahe_batch_workspace_bytes(int n_vol, const mclahe_plan_t *plans) {
    (void)n_vol;
    (void)plans;
    return 0;
}

mclahe_status mclahe_batch(int n_vol, const mclahe_plan_t *plans, const float *const *d_in,
                           float *const *d_out, void *d_ws, size_t ws_bytes, const float *d_clip,
                           mclahe_stream_t stream, int use_graph) {
    (void)n_vol; (void)plans; (void)d_in; (void)d_out; (void)d_ws; (void)ws_bytes;
    (void)d_clip; (void)stream; (void)use_graph;
    return MCLAHE_ERR_UNSUPPORTED;
}

mclahe_status mclahe_autotune(mclahe_plan_t plan, const float *d_in, float *d_out, void *d_ws,
                              size_t ws_bytes, mclahe_stream_t stream) {
    (void)plan; (void)d_in; (void)d_out; (void)d_ws; (void)ws_bytes; (void)stream;
    return MCLAHE_ERR_UNSUPPORTED;
}

}
