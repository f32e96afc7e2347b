// Device code of the GE-distance solver, part 4: the multi-column SpMM of the PCG
// iteration (Section 3.2) over a "stream" plan (internal; sm_103a).
//
// A stream plan stores every step a warp takes in one contiguous run of the sliced
// arrays, so a warp needs no per-slice bookkeeping loads and can fetch ahead across
// slice boundaries.  A step is H entries side by side (one per lane group, H = 32 /
// lanes per row).
//   Light slice (H rows of a block, sorted by length): its first step gathers the
//   rows' own vector rows, with the rows' degrees as weights (sign bit set: empty lane
//   group) and the rows' ids as columns; the following steps hold the rows' entries
//   (rows shorter than the slice padded with zero weights on their own column); the
//   weights of the slice's last step carry the sign bit.  The row epilogue
//   q_i = d_i p_i - sum_j w_ij p_j then runs from registers.
//   Heavy-row chunk (a row above the light-row limit, cut into chunks of 64 steps):
//   entries j*H + g of the chunk at step j, lane group g; the lane groups' sums are
//   added by a fixed butterfly and the chunks of a row combined in chunk order by the
//   warp that finishes the row's last chunk (counter hcount).
// Each warp of a light block takes the run of its block's slices that the planner
// cut for it (the running entry count closest to an equal share); each warp of a
// heavy block one chunk.  Every thread therefore adds the same rows in the same order
// on every run, and the row sums are those of the register path (kernels.cuh): each
// row's products in entry order.
//
// Two engines fetch the gathered rows: registers (reg_stream: a batch of STREAM_U
// steps in flight per lane, their columns and weights loaded a batch ahead with one
// coalesced load per lane) and TMA (tma.cuh, tiles whose rows are 64 or 128 bytes:
// tile::gather4 into shared-memory rings).
#pragma once

#include "tma.cuh"

namespace nvd {

// Steps a lane keeps in flight in the register engine.
#ifndef NVD_STREAM_U
#define NVD_STREAM_U 8
#endif
constexpr int STREAM_U = NVD_STREAM_U;

namespace dev {

// The row-side work of a stream: light slices (own row, entries, epilogue) and heavy
// chunks (partial row sum, split-row combination).  One object per lane.
template <class TV, class TA, int KT, class Epi>
struct StreamRows {
    typedef SpCfg<TV, TA, KT> C;
    static constexpr int VEC = C::VEC, LPR = C::LPR, ND = Epi::ND;
    typedef typename Epi::template D<TV> DT;
    const Ctx &c;
    Epi e;
    TV *dst;
    int col0;
    DT (&dot)[ND > 0 ? ND : 1][VEC];
    TA acc[VEC];
    TV own[VEC];
    TA dg = 0;
    int32_t row = 0;
    bool first = true, valid = false;

    __device__ __forceinline__ StreamRows(const Ctx &c_, const Epi &epi, int seg, int col0_, TV *dst_,
                                          DT (&dot_)[ND > 0 ? ND : 1][VEC])
        : c(c_), e(epi), dst(dst_), col0(col0_), dot(dot_) {
        e.prep(c, seg, col0);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0;
    }
    // One step of a light slice: pv = this lane's 16 bytes of the gathered row, w its
    // row's weight (degree on a slice's first step), col its row's column (the row id
    // on a slice's first step).  `first` and the last-step sign are the same for every
    // lane of the warp.
    __device__ __forceinline__ void light(const TV (&pv)[VEC], TA w, int32_t col) {
        const bool neg = signbit(w) != 0;
        const TA mag = fabs(w);
        if (first) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) own[v] = pv[v];
            dg = mag;
            valid = !neg;
            row = col;
            first = false;
            return;
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] += mag * (TA)pv[v];
        if (neg) {
            if (valid) e.template elem<TV, TA, VEC>(c, row, col0, KT, own, acc, dg, dst, dot);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] = 0;
            first = true;
        }
    }
    __device__ __forceinline__ void heavy(const TV (&pv)[VEC], TA w) {
        const TA mag = fabs(w);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] += mag * (TA)pv[v];
    }
    // End of a heavy chunk (whole warp): its partial row sum into hsum; the warp that
    // completes the row adds the chunks in chunk order and writes the row and its
    // partial-slot inner products.
    __device__ __forceinline__ void heavy_finish(const SpItem &it, const TV *__restrict__ src) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] += __shfl_xor_sync(NVD_FULLMASK, acc[v], off);
        if (lane < LPR) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) c.hsum[(int64_t)(it.hbase + it.hchunk) * KT + col0 + v] = (double)acc[v];
        }
        __threadfence();
        __syncwarp();
        int fin = 0;
        if (lane == 0) fin = atomicAdd(c.hcount + it.hrow, 1) == it.nchunk - 1;
        fin = __shfl_sync(NVD_FULLMASK, fin, 0);
        if (fin) {
            __threadfence();
            if (lane < LPR) {
                TA rs[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    double sum = 0.0;
                    for (int q = 0; q < it.nchunk; ++q) sum += __ldcg(c.hsum + (int64_t)(it.hbase + q) * KT + col0 + v);
                    rs[v] = (TA)sum;
                }
                TV ow[VEC];
                ldv<LdRO, TV, VEC>(src + (int64_t)it.r0 * KT + col0, ow);
                DT hdot[ND > 0 ? ND : 1][VEC];
#pragma unroll
                for (int d = 0; d < (ND > 0 ? ND : 1); ++d)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) dot_zero(hdot[d][v]);
                e.template elem<TV, TA, VEC>(c, it.r0, col0, KT, ow, rs, __ldg(deg_of<TA>(c) + it.r0), dst, hdot);
                if constexpr (ND > 0) {
                    const int64_t hs = c.n_sblk + it.hrow;
#pragma unroll
                    for (int d = 0; d < ND; ++d)
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            c.part[((int64_t)d * c.part_stride + hs) * KT + col0 + v] = dot_get(hdot[d][v]);
                }
            }
            if (lane == 0) atomicExch(c.hcount + it.hrow, 0);
        }
        __syncwarp();
    }
};

// Register engine: steps [0, T) of the run starting at entry E0.  Per batch of
// STREAM_U steps each lane gathers its 16 bytes of every step's row (all in flight
// together), while the columns and weights of the batch after next are loaded: lane
// l holds entries k*32 + l of a batch (k < NL), and the lane of group g at step s
// takes entry s*H + g by a shuffle.  f(pv, w, col) is called for every step in order.
template <class TV, class TA, int KT, class F>
__device__ __forceinline__ void reg_stream(const Ctx &c, int64_t E0, int64_t T, const TV *__restrict__ src,
                                           F &&f) {
    typedef SpCfg<TV, TA, KT> C;
    constexpr int VEC = C::VEC, LPR = C::LPR, H = C::G, U = STREAM_U;
    constexpr int NL = (U * H + 31) / 32;
    static_assert(32 % H == 0, "a lane group's step entry sits in one 32-entry part of a batch");
    const int lane = threadIdx.x & 31, gid = lane / LPR, col0 = (lane % LPR) * VEC;
    const int32_t *__restrict__ cols = c.sl_col + E0;
    const TA *__restrict__ ws = reinterpret_cast<const TA *>(c.sl_w) + E0;
    const int64_t NE = T * H;
    int mc[NL], nc[NL];
    TA mw[NL], nw[NL];
    auto load_meta = [&](int64_t t0, int (&oc)[NL], TA (&ow)[NL]) {
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int64_t e = t0 * H + k * 32 + lane;
            if (k * 32 + lane < U * H && e < NE) {
                oc[k] = __ldcs(cols + e);
                ow[k] = __ldcs(ws + e);
            }
        }
    };
    load_meta(0, mc, mw);
    load_meta(U, nc, nw);
    for (int64_t t0 = 0; t0 < T; t0 += U) {
        TV pv[U][VEC];
        int cc[U];
#pragma unroll
        for (int s = 0; s < U; ++s) {
            cc[s] = __shfl_sync(NVD_FULLMASK, mc[(s * H) / 32], (s * H + gid) % 32);
            if (t0 + s < T) ldv<LdRO, TV, VEC>(src + (int64_t)cc[s] * KT + col0, pv[s]);
        }
        TA cw[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            cw[k] = mw[k];
            mc[k] = nc[k];
            mw[k] = nw[k];
        }
        load_meta(t0 + 2 * U, nc, nw);
#pragma unroll
        for (int s = 0; s < U; ++s) {
            if (t0 + s < T) {
                const TA w = __shfl_sync(NVD_FULLMASK, cw[(s * H) / 32], (s * H + gid) % 32);
                f(pv[s], w, cc[s]);
            }
        }
    }
}

// One CTA block b of a stream plan (see the top of this file); ENGINE 0 registers,
// 1 TMA (`ring`: this CTA's 128-byte aligned ring area, `tm`: the tensor map of src),
// 2 per-lane asynchronous copies into the same ring.  Then the block's inner-product
// partials and the segment arrival, as in the register path.  `smem` is the register
// path's layout (reduction scratch and totals).
template <int ENGINE, class TV, class TW, class TA, int KT, class Epi>
__device__ void spmm_block_stream(const Ctx &c, const Epi &epi, const TV *__restrict__ src, TV *__restrict__ dst,
                                  int64_t b, char *ring, char *smem, const CUtensorMap *tm) {
    typedef SpCfg<TV, TA, KT> C;
    constexpr int VEC = C::VEC, LPR = C::LPR, H = C::G, ND = Epi::ND;
    constexpr int RB = KT * (int)sizeof(TV);       // bytes of one gathered row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane / LPR, col0 = (lane % LPR) * VEC;
    const Block blk = c.sblk[b];
    const int seg = blk.seg;
    double *red = reinterpret_cast<double *>(smem + C::ACC);
    double *tot = red + C::RED;
    typename Epi::template D<TV> dot[ND > 0 ? ND : 1][VEC];
#pragma unroll
    for (int d = 0; d < (ND > 0 ? ND : 1); ++d)
#pragma unroll
        for (int v = 0; v < VEC; ++v) dot_zero(dot[d][v]);
    const bool live = !Epi::NEEDS_LIVE || seg_live<KT>(c, seg);
    const longlong2 run = live ? c.sl_wrun[b * NWARP + warp] : make_longlong2(0, 0);
    const int64_t E0 = run.x, T = run.y;
    if (T > 0) {
        StreamRows<TV, TA, KT, Epi> rows(c, epi, seg, col0, dst, dot);
        bool ok = true;
        if constexpr (ENGINE == 2) {
            static_assert(H * RB == TMA_STEP_BYTES && (H == 4 || H == 8), "one step is 512 bytes of 4 or 8 rows");
            static_assert(TMA_STEP_BYTES + H * (int)sizeof(TA) <= TMA_IDS_OFFSET, "weights fit the slot");
            static_assert(VEC * (int)sizeof(TV) == 16, "16-byte lane vectors");
            char *wring = ring + warp * TMA_SLOTS * TMA_SLOT_BYTES;
            auto slot_values = [&](const char *slot, TV (&pv)[VEC], TA &w, int32_t &col) {
                SmemVec<TV, VEC>::ld(slot + lane * 16, pv);
                w = *reinterpret_cast<const TA *>(slot + TMA_STEP_BYTES + gid * (int)sizeof(TA));
                col = reinterpret_cast<const int32_t *>(slot + TMA_IDS_OFFSET)[gid];
            };
            if (blk.pad == 0) {
                acopy_stream<H, RB, TV, TA, KT>(c, E0, T, src, wring, [&](int64_t, const char *slot) {
                    TV pv[VEC];
                    TA w;
                    int32_t col;
                    slot_values(slot, pv, w, col);
                    rows.light(pv, w, col);
                    return true;
                });
            } else {
                acopy_stream<H, RB, TV, TA, KT>(c, E0, T, src, wring, [&](int64_t, const char *slot) {
                    TV pv[VEC];
                    TA w;
                    int32_t col;
                    slot_values(slot, pv, w, col);
                    rows.heavy(pv, w);
                    return true;
                });
            }
        } else if constexpr (ENGINE == 1) {
            static_assert(H * RB == TMA_STEP_BYTES && (H == 4 || H == 8), "one step is 512 bytes of 4 or 8 rows");
            static_assert(TMA_STEP_BYTES + H * (int)sizeof(TA) <= TMA_IDS_OFFSET, "weights fit the slot");
            static_assert(VEC * (int)sizeof(TV) == 16, "16-byte lane vectors");
            char *wring = ring + warp * TMA_SLOTS * TMA_SLOT_BYTES;
            uint64_t *bars =
                reinterpret_cast<uint64_t *>(ring + NWARP * TMA_SLOTS * TMA_SLOT_BYTES) + warp * TMA_SLOTS;
            if (lane == 0)
                for (int q = 0; q < TMA_SLOTS; ++q) mbar_init(bars + q, 1);
            fence_mbar_init();
            fence_proxy_async_smem();
            __syncwarp();
            auto slot_values = [&](const char *slot, TV (&pv)[VEC], TA &w, int32_t &col) {
                SmemVec<TV, VEC>::ld(slot + lane * 16, pv);
                w = *reinterpret_cast<const TA *>(slot + TMA_STEP_BYTES + gid * (int)sizeof(TA));
                col = reinterpret_cast<const int32_t *>(slot + TMA_IDS_OFFSET)[gid];
            };
            if (blk.pad == 0) {
                ok = tma_stream<H, RB, TA>(c, E0, T, wring, bars, tm, [&](int64_t, const char *slot) {
                    TV pv[VEC];
                    TA w;
                    int32_t col;
                    slot_values(slot, pv, w, col);
                    rows.light(pv, w, col);
                    return true;
                });
            } else {
                ok = tma_stream<H, RB, TA>(c, E0, T, wring, bars, tm, [&](int64_t, const char *slot) {
                    TV pv[VEC];
                    TA w;
                    int32_t col;
                    slot_values(slot, pv, w, col);
                    rows.heavy(pv, w);
                    return true;
                });
            }
        } else {
            if (blk.pad == 0)
                reg_stream<TV, TA, KT>(c, E0, T, src,
                                       [&](const TV (&pv)[VEC], TA w, int32_t col) { rows.light(pv, w, col); });
            else
                reg_stream<TV, TA, KT>(c, E0, T, src,
                                       [&](const TV (&pv)[VEC], TA w, int32_t) { rows.heavy(pv, w); });
        }
        if (ok && blk.pad != 0) rows.heavy_finish(c.items[blk.i0 + warp], src);
        if (!ok && lane == 0) atomicCAS(c.err, 0, NVD_ERR_TIMEOUT);
    }
    if constexpr (ND > 0) {
        double dd[ND][VEC];
        dot_to_double(dot, dd);
        block_reduce_cols<ND, KT, VEC>(dd, red, tot);
        const int64_t s0 = c.seg_sblk_off[seg];
        const int32_t cnt = c.seg_sblk_off[seg + 1] - (int32_t)s0;
        const int64_t h0 = c.n_sblk + c.seg_heavy_off[seg];
        const int32_t hcnt = c.seg_heavy_off[seg + 1] - c.seg_heavy_off[seg];
        seg_arrive<ND, KT>(c, epi.fin, seg, b, tot, s0, cnt, h0, hcnt, red);
    }
}

}  // namespace dev
}  // namespace nvd
