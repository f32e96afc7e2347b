// MIXED-mode (FP32 PCG inside FP64 iterative refinement) tile solver instantiations.
#include "dispatch.h"
#include "solver.cuh"

namespace nvd {

template <class TWN, class TX>
static int mixed_kt(nvd_graph_s *g, const Ctx &c, const Plan *pl64, SolveWs &w, const nvd_solve_opts &o,
                    const TileIO &io, cudaStream_t s, int KT, std::vector<int> &it,
                    std::vector<double> &rr, int *steps, int *conv) {
    switch (KT) {
        case 1: return tile_mixed<TWN, 1, TX>(g, c, pl64, w, o, io, s, it, rr, steps, conv);
        case 4: return tile_mixed<TWN, 4, TX>(g, c, pl64, w, o, io, s, it, rr, steps, conv);
        case 8: return tile_mixed<TWN, 8, TX>(g, c, pl64, w, o, io, s, it, rr, steps, conv);
        case 16: return tile_mixed<TWN, 16, TX>(g, c, pl64, w, o, io, s, it, rr, steps, conv);
        case 32: return tile_mixed<TWN, 32, TX>(g, c, pl64, w, o, io, s, it, rr, steps, conv);
    }
    set_error("unsupported tile width %d", KT);
    return NVD_ERR_INVALID_ARG;
}

int run_tile_mixed(nvd_graph_s *g, const Ctx &c, const Plan *pl64, SolveWs &w, const nvd_solve_opts &o,
                   const TileIO &io, cudaStream_t s, int KT, int xdt, std::vector<int> &iters,
                   std::vector<double> &relres, int *steps, int *conv) {
    if (g->wdtype == NVD_F64)
        return xdt == NVD_F64 ? mixed_kt<double, double>(g, c, pl64, w, o, io, s, KT, iters, relres, steps, conv)
                              : mixed_kt<double, float>(g, c, pl64, w, o, io, s, KT, iters, relres, steps, conv);
    return xdt == NVD_F64 ? mixed_kt<float, double>(g, c, pl64, w, o, io, s, KT, iters, relres, steps, conv)
                          : mixed_kt<float, float>(g, c, pl64, w, o, io, s, KT, iters, relres, steps, conv);
}

}  // namespace nvd
