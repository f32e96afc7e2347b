// C ABI: nvd_ge_distance_batched (placeholder until the persistent kernel lands).
#include "graph.h"

extern "C" int nvd_ge_distance_batched(const nvd_graph_t *graphs, int32_t G, const int32_t *k_per,
                                       const void *const *x, const void *const *y, int32_t xdtype,
                                       const nvd_solve_opts *opts, double *d2_out, nvd_solve_stats *stats,
                                       nvd_stream_t stream) {
    nvd::clear_error();
    nvd::set_error("nvd_ge_distance_batched: not built yet");
    return NVD_ERR_UNSUPPORTED;
}
