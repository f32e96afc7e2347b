// Internal graph handle, device buffers and work plans (host side).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.h"
#include "nvd.h"

namespace nvd {

// NVTX range around a phase of a call (graph creation, plan build, one tile, one
// refinement step, ...), for profilers that attach; without one it costs a call.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Thread-local error detail for nvd_last_error().
void set_error(const char *fmt, ...);
void clear_error();

#define NVD_TRY_CUDA(call)                                                                 \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ::nvd::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                             __FILE__, __LINE__);                                          \
            return e_ == cudaErrorMemoryAllocation ? NVD_ERR_OOM : NVD_ERR_CUDA;           \
        }                                                                                  \
    } while (0)

#define NVD_TRY(call)                       \
    do {                                    \
        int s_ = (call);                    \
        if (s_ != NVD_OK) return s_;        \
    } while (0)

// Owned device allocation.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // (Re)allocate to exactly `b` bytes (contents undefined).
    int alloc(size_t b);
    // Grow to at least `b` bytes (contents undefined after growth).
    int ensure(size_t b) { return b <= bytes && p ? NVD_OK : alloc(b); }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Tunable parameters of the SpMV work decomposition, in percent of the built-in
// defaults: the light-row limit (rows above it are split into heavy sub-items) and
// the number of light CTA blocks per launch.
struct SpParams {
    int32_t row_max_pct = 100;
    int32_t blocks_pct = 100;
    int32_t gather = 0;          // multi-column SpMM: 0 register slices, 1 register stream, 2 TMA stream,
                                 // 3 asynchronous-copy stream
                                 // (2 only where tma_tile holds, else 1); the tuner tries the others
    int32_t l2_hot = 0;          // 1: the multi-column SpMM keeps the gathered vector's hot rows (the
                                 // degree-ordered head of the largest component) persisting in L2
};

// Work decomposition for one (KT, vector size, accumulator size, SpParams).
struct Plan {
    int KT = 0, szv = 0, sza = 0;
    SpParams sp;
    int64_t n_items = 0, n_sblk = 0, n_heavy = 0, n_chunks = 0, n_vblk = 0;
    int64_t n_slices = 0, n_sl_entries = 0;
    DevBuf items, sblk, vblk, seg_sblk_off, seg_heavy_off, seg_vblk_off, hcount;
    DevBuf sl_base, sl_row, sl_col, sl_w;   // sliced light rows (weights in the plan's TW)
    DevBuf sl_wsplit;                       // per light block, the warps' contiguous slice runs
    DevBuf sl_wrun;                         // stream plans: per (block, warp) {first entry, steps}
    bool stream = false;                    // stream layout (stream.cuh)
    bool tma = false;                       // stream plan gathered by TMA
    bool acopy = false;                     // stream plan gathered by per-lane asynchronous copies
    int64_t n_light_slices = 0;             // stream plans: heavy-chunk slices follow the light ones
    int64_t part_slots() const {
        int64_t a = n_sblk + n_heavy;
        return a > n_vblk ? a : n_vblk;
    }
};

}  // namespace nvd

namespace nvd {
struct ElimState;   // exact low-degree elimination (elim.cu)
void elim_state_delete(ElimState *e);
}  // namespace nvd

struct nvd_graph_s {
    uint64_t id = 0;             // unique per handle (cache keys)
    int device = 0;
    int num_sms = 0;
    int64_t n = 0, nnz = 0;      // after cleaning (self-loops dropped, repeats merged)
    int64_t nnz_user = 0;        // entries given to nvd_graph_create
    int32_t wdtype = NVD_F64;
    // internal CSR (component-contiguous node order), arrays padded to 4 entries
    nvd::DevBuf rowptr, colidx, w, w32;   // w in wdtype; w32 = FP32 copy when wdtype is F64 (lazy)
    nvd::DevBuf deg64, dinv64, deg32, dinv32;
    nvd::DevBuf perm;            // int32 internal -> user node; empty when identity
    nvd::DevBuf uent;            // int64 user entry -> internal entry (-1 dropped); empty when identity
    // inverse of uent for nvd_graph_set_weights (built on first use): the user entries
    // of internal entry e are ient_src[ient_ptr[e] .. ient_ptr[e+1]), increasing
    nvd::DevBuf ient_ptr, ient_src;
    int32_t ncomp = 0, nseg = 0;
    bool reordered = false;      // NVD_GRAPH_REORDER_DEGREE: nodes by degree inside each component
    int64_t hot_begin = 0, hot_rows = 0;   // reordered: the largest segment's rows (highest degree first)
    int64_t n_singleton = 0;
    std::vector<int64_t> h_rowptr, h_seg_begin, h_seg_end;
    std::vector<int32_t> h_seg_of;  // user node -> its segment (-1: isolated node)
    nvd::DevBuf seg_begin, seg_end, seg_owner;
    nvd::SpParams sp;            // parameters of plans built from now on (nvd_graph_tune)
    int32_t tuned_kt[3] = {0, 0, 0};          // per solve mode: tile width chosen by the tuner (0 = none)
    int32_t tuned_persistent[3] = {0, 0, 0};  // per solve mode: 1 = persistent launch was faster
    int32_t tuned_fold[3] = {0, 0, 0};        // per solve mode: 1 = two kernels per iteration were faster
    std::map<int64_t, std::unique_ptr<nvd::Plan>> plans;
    std::map<std::string, std::unique_ptr<nvd::DevBuf>> ws;  // named lazily-grown workspace
    // host-input staging: a copy stream and per-slot events (two slots), created on
    // first use, so the next tile's host-to-device copy overlaps the current solve
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
    // degree-1/2 nodes eliminated exactly and the reduced graph (nvd_graph_eliminate)
    std::unique_ptr<nvd::ElimState, void (*)(nvd::ElimState *)> elim{nullptr, nvd::elim_state_delete};
    ~nvd_graph_s();

    void *wsp(const std::string &name, size_t bytes, int *st);
    int64_t device_bytes() const;
};

namespace nvd {

// Work plan for (KT, szv, sza), built on first use and cached in the handle.  A stream
// plan (SpParams::gather >= 1, KT > 1) is laid out for the stream SpMM only
// (k_spmm_stream, k_spmm_tma); launches that run the register-slice path (the
// persistent kernel) ask for allow_stream = false.
int get_plan(nvd_graph_s *g, int KT, int szv, int sza, Plan **out, bool allow_stream = true);
// FP32 weights for the FP32 paths (the FP64 weights rounded once, cached).
int get_w32(nvd_graph_s *g, const float **out, cudaStream_t s);
// Ctx fields that depend only on the graph and a plan.
void fill_graph_ctx(const nvd_graph_s *g, const Plan *pl, Ctx *c);
// Only the SpMV/SpMM work-decomposition fields of a Ctx.
void set_sp_plan(Ctx *c, const Plan *pl);

// Tensor map of a [rows][kt] array of szv-byte values (row-major, 16-byte aligned
// base) for TMA row gathers: one box = one whole row.  Encoded once per
// (address, shape) and cached.
int tma_map(const void *base, int64_t rows, int kt, int szv, CUtensorMap *out);

// Bytes of L2 this process may keep persisting for one access-policy window on the
// current device (the set-aside is requested once per device, on first use); 0 if
// the device has none.
size_t l2_persist_bytes();

// Blocks per kernel launch the planner aims for (about two waves of 8 CTAs per SM).
int target_blocks(const nvd_graph_s *g);
// Fresh handle id.
uint64_t next_graph_id();

}  // namespace nvd
