// Runtime-to-template dispatch of the tile solvers (internal).  Each function is
// defined in its own translation unit so the template instantiations compile in
// parallel.
#pragma once

#include <vector>

#include "graph.h"

namespace nvd {

struct SolveWs;
struct TileIO;

// FP64 mode: TV = TA = double, TW = graph weight type.
int run_tile_fp64(nvd_graph_s *g, const Ctx &c, SolveWs &w, const nvd_solve_opts &o,
                  const TileIO &io, cudaStream_t s, int KT, int xdt);
// FP32 mode: TV = TA = TW = float.
int run_tile_fp32(nvd_graph_s *g, const Ctx &c, SolveWs &w, const nvd_solve_opts &o,
                  const TileIO &io, cudaStream_t s, int KT, int xdt);
// MIXED mode: FP32 inner solves, FP64 refinement over the graph's weight type.
int run_tile_mixed(nvd_graph_s *g, const Ctx &c, const Plan *pl64, SolveWs &w, const nvd_solve_opts &o,
                   const TileIO &io, cudaStream_t s, int KT, int xdt, std::vector<int> &iters,
                   std::vector<double> &relres, int *steps, int *conv);
// One persistent cooperative launch solving a whole tile (FP64 or FP32 mode);
// c.owners / c.own0 describe the owners, a the buffers.
int run_persistent(nvd_graph_s *g, const Ctx &c, const PersistArgs &a, int mode, int KT, int xdt,
                   cudaStream_t s);
// k_collect<KT> launch.
int run_collect(const Ctx &c, int KT, ColResult *res, double *d2dev, int64_t d2_stride,
                int n_owner, cudaStream_t s);
// nvd_ge_distance without z_out / stats (used by the tuner to time configurations).
int ge_distance_internal(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdt,
                         const nvd_solve_opts *opts, double *d2_out, cudaStream_t s);
// nvd_ge_distance with NVD_SOLVE_ELIMINATE: degree-1/2 nodes eliminated exactly,
// PCG on the reduced graph (elim.cu).
// idx: x, y are [k] device int32 node ids (indicator pairs), as in the resistance calls.
int elim_distance(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdt,
                  const nvd_solve_opts *opts, double *d2_out, void *z_out, nvd_solve_stats *stats,
                  cudaStream_t s, bool idx = false);
// y = L x for one contiguous column (internal order), dtype = F32 or F64.
int run_apply(nvd_graph_s *g, const Ctx &c, const void *x, void *y, int dtype, cudaStream_t s);

}  // namespace nvd
