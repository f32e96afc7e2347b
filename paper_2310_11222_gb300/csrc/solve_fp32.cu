// FP32-mode tile solver instantiations.
#include "dispatch.h"
#include "solver.cuh"

namespace nvd {

template <class TX>
static int fp32_kt(nvd_graph_s *g, const Ctx &c, SolveWs &w, const nvd_solve_opts &o,
                   const TileIO &io, cudaStream_t s, int KT) {
    switch (KT) {
        case 1: return tile_pcg<float, float, float, 1, TX>(g, c, w, o, io, s);
        case 4: return tile_pcg<float, float, float, 4, TX>(g, c, w, o, io, s);
        case 8: return tile_pcg<float, float, float, 8, TX>(g, c, w, o, io, s);
        case 16: return tile_pcg<float, float, float, 16, TX>(g, c, w, o, io, s);
        case 32: return tile_pcg<float, float, float, 32, TX>(g, c, w, o, io, s);
    }
    set_error("unsupported tile width %d", KT);
    return NVD_ERR_INVALID_ARG;
}

int run_tile_fp32(nvd_graph_s *g, const Ctx &c, SolveWs &w, const nvd_solve_opts &o,
                  const TileIO &io, cudaStream_t s, int KT, int xdt) {
    Ctx c32 = c;
    const float *w32 = nullptr;
    NVD_TRY(get_w32(g, &w32, s));
    c32.w = w32;
    return xdt == NVD_F64 ? fp32_kt<double>(g, c32, w, o, io, s, KT) : fp32_kt<float>(g, c32, w, o, io, s, KT);
}

}  // namespace nvd
