// Persistent-solve instantiations and the cooperative launch.
#include <algorithm>

#include "dispatch.h"
#include "persistent.cuh"
#include "solver.cuh"

namespace nvd {

template <class TV, class TW, class TA, int KT, class TX>
static int launch_persistent(nvd_graph_s *g, const Ctx &c, const PersistArgs &a, cudaStream_t s) {
    auto kern = k_persistent<TV, TW, TA, KT, TX>;
    if (c.sl_h != sp_slice_rows(KT, (int)sizeof(TV))) {
        set_error("internal: SpMV plan built for another tile width or precision");
        return NVD_ERR_UNSUPPORTED;
    }
    int per_sm = 0;
    NVD_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, 0));
    if (per_sm < 1) {
        set_error("persistent kernel does not fit on an SM");
        return NVD_ERR_UNSUPPORTED;
    }
    // one co-resident wave (the grid barrier needs every CTA resident); every phase and
    // the per-(owner, column) results loop over the grid, so any number of owners fits
    const int64_t resident = (int64_t)per_sm * g->num_sms;
    const int64_t need_res = ((int64_t)a.n_owner * KT + NT - 1) / NT;
    int64_t grid = std::max<int64_t>({c.n_sblk, c.n_vblk, need_res, 1});
    grid = std::min(grid, resident);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    NVD_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern, c, a));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusNone) note_launch();   // replays of a capture are counted by the caller
    return NVD_OK;
}

template <class TV, class TW, class TA, class TX>
static int persist_kt(nvd_graph_s *g, const Ctx &c, const PersistArgs &a, int KT, cudaStream_t s) {
    switch (KT) {
        case 1: return launch_persistent<TV, TW, TA, 1, TX>(g, c, a, s);
        case 4: return launch_persistent<TV, TW, TA, 4, TX>(g, c, a, s);
        case 8: return launch_persistent<TV, TW, TA, 8, TX>(g, c, a, s);
        case 16: return launch_persistent<TV, TW, TA, 16, TX>(g, c, a, s);
        case 32: return launch_persistent<TV, TW, TA, 32, TX>(g, c, a, s);
    }
    set_error("unsupported tile width %d", KT);
    return NVD_ERR_INVALID_ARG;
}

int run_persistent(nvd_graph_s *g, const Ctx &c, const PersistArgs &a, int mode, int KT, int xdt,
                   cudaStream_t s) {
    if (mode == NVD_MODE_FP64) {
        if (g->wdtype == NVD_F64)
            return xdt == NVD_F64 ? persist_kt<double, double, double, double>(g, c, a, KT, s)
                                  : persist_kt<double, double, double, float>(g, c, a, KT, s);
        return xdt == NVD_F64 ? persist_kt<double, float, double, double>(g, c, a, KT, s)
                              : persist_kt<double, float, double, float>(g, c, a, KT, s);
    }
    if (mode == NVD_MODE_FP32) {
        Ctx c32 = c;
        const float *w32 = nullptr;
        NVD_TRY(get_w32(g, &w32, s));
        c32.w = w32;
        return xdt == NVD_F64 ? persist_kt<float, float, float, double>(g, c32, a, KT, s)
                              : persist_kt<float, float, float, float>(g, c32, a, KT, s);
    }
    set_error("the persistent solve supports the FP64 and FP32 modes");
    return NVD_ERR_UNSUPPORTED;
}

}  // namespace nvd
