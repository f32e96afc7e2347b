// FP64-mode tile solver instantiations (KT in {1,4,8,16,32} x weight type x input type).
#include "dispatch.h"
#include "solver.cuh"

namespace nvd {

template <class TW, class TX>
static int fp64_kt(nvd_graph_s *g, const Ctx &c, SolveWs &w, const nvd_solve_opts &o,
                   const TileIO &io, cudaStream_t s, int KT) {
    switch (KT) {
        case 1: return tile_pcg<double, TW, double, 1, TX>(g, c, w, o, io, s);
        case 4: return tile_pcg<double, TW, double, 4, TX>(g, c, w, o, io, s);
        case 8: return tile_pcg<double, TW, double, 8, TX>(g, c, w, o, io, s);
        case 16: return tile_pcg<double, TW, double, 16, TX>(g, c, w, o, io, s);
        case 32: return tile_pcg<double, TW, double, 32, TX>(g, c, w, o, io, s);
    }
    set_error("unsupported tile width %d", KT);
    return NVD_ERR_INVALID_ARG;
}

int run_tile_fp64(nvd_graph_s *g, const Ctx &c, SolveWs &w, const nvd_solve_opts &o,
                  const TileIO &io, cudaStream_t s, int KT, int xdt) {
    if (g->wdtype == NVD_F64)
        return xdt == NVD_F64 ? fp64_kt<double, double>(g, c, w, o, io, s, KT)
                              : fp64_kt<double, float>(g, c, w, o, io, s, KT);
    return xdt == NVD_F64 ? fp64_kt<float, double>(g, c, w, o, io, s, KT)
                          : fp64_kt<float, float>(g, c, w, o, io, s, KT);
}

int run_collect(const Ctx &c, int KT, ColResult *res, double *d2dev, int64_t d2_stride, int n_owner,
                cudaStream_t s) {
    const int nthr = n_owner * KT;
    const int grid = (nthr + 127) / 128;
    switch (KT) {
        case 1: k_collect<1><<<grid, 128, 0, s>>>(c, res, d2dev, d2_stride); break;
        case 4: k_collect<4><<<grid, 128, 0, s>>>(c, res, d2dev, d2_stride); break;
        case 8: k_collect<8><<<grid, 128, 0, s>>>(c, res, d2dev, d2_stride); break;
        case 16: k_collect<16><<<grid, 128, 0, s>>>(c, res, d2dev, d2_stride); break;
        case 32: k_collect<32><<<grid, 128, 0, s>>>(c, res, d2dev, d2_stride); break;
        default: set_error("unsupported tile width %d", KT); return NVD_ERR_INVALID_ARG;
    }
    note_launch();
    NVD_TRY_CUDA(cudaGetLastError());
    return NVD_OK;
}

int run_apply(nvd_graph_s *g, const Ctx &c, const void *x, void *y, int dtype, cudaStream_t s) {
    dev::EpiApply epi;
    if (dtype == NVD_F64) {
        const double bytes = spmm_bytes(g, 1, 8, g->wdtype == NVD_F64 ? 8 : 4, 8);
        if (g->wdtype == NVD_F64)
            return launch_spmm<double, double, double, 1>(c, epi, (const double *)x, (double *)y, s, bytes);
        return launch_spmm<double, float, double, 1>(c, epi, (const double *)x, (double *)y, s, bytes);
    }
    const double bytes = spmm_bytes(g, 1, 4, 4, 4);
    return launch_spmm<float, float, float, 1>(c, epi, (const float *)x, (float *)y, s, bytes);
}

}  // namespace nvd
