// Device code of the GE-distance solver, part 3: the TMA engine of the stream SpMM
// (stream.cuh) for tiles whose rows are 64 or 128 bytes (internal; sm_103a).
//
// One stream step gathers H neighbour rows of KT values, 512 bytes in all (H * KT *
// sizeof(TV) = 32 lanes * 16 bytes), and a TMA tile::gather4 instruction fetches 4
// such rows by their indices into shared memory.  Each warp has a ring of TMA_SLOTS
// step slots; lanes issue the gathers (and a bulk copy of the step's H weights) for
// TMA_ROUND steps at once, one step per lane, so up to 2 * TMA_ROUND * 512 bytes per
// warp are in flight without holding registers.  Every step completes an mbarrier
// (arrival plus transaction bytes); the warp waits on it and each lane reads its 16
// bytes of the step (lane group = row), its row's weight and column.
//
// Every wait is bounded: a step that has not arrived after about one second sets
// NVD_ERR_TIMEOUT in c.err, the warp waits (again bounded) for the copies it
// issued, and stops.
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace nvd {

// Ring of one warp: TMA_SLOTS step slots of 512 bytes of gathered rows (128-byte
// aligned) followed by the step's weights (at most 8 of 8 bytes).
constexpr int TMA_SLOTS = 16;
constexpr int TMA_ROUND = TMA_SLOTS / 2;
constexpr int TMA_STEP_BYTES = 512;
constexpr int TMA_IDS_OFFSET = 576;   // the step's column indices (row ids of a slice's first step)
constexpr int TMA_SLOT_BYTES = 640;
// Dynamic shared memory of the TMA SpMM kernel: 128 bytes of alignment slack, the
// rings and mbarriers of the NWARP warps, then the register path's layout (split
// rows, reduction scratch, totals).
constexpr int tma_ring_bytes() { return 128 + NWARP * TMA_SLOTS * (TMA_SLOT_BYTES + 8); }

namespace dev {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Make mbarrier initialisation and earlier shared-memory accesses of the generic
// proxy visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of `parity` to complete, at most about `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer_ns();
    for (uint32_t spin = 1;; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 63u) == 0 && gtimer_ns() - t0 > limit_ns) return false;
    }
}
// Four rows (y0..y3) of a 2-D tensor, columns [x, x + box width), into dst.
__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *tm, int32_t x, int32_t y0, int32_t y1,
                                            int32_t y2, int32_t y3, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(smem_addr(bar))
        : "memory");
}
// Contiguous global -> shared copy (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

template <class T, int V> struct SmemVec;
template <> struct SmemVec<float, 4> {
    static __device__ __forceinline__ void ld(const char *p, float (&o)[4]) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    }
};
template <> struct SmemVec<double, 2> {
    static __device__ __forceinline__ void ld(const char *p, double (&o)[2]) {
        const double2 a = *reinterpret_cast<const double2 *>(p);
        o[0] = a.x; o[1] = a.y;
    }
};

// The step stream of one warp: steps [E0 / H, E0 / H + T) of the plan's sliced
// arrays (light slices, or one heavy-row chunk), TMA_SLOTS slots in flight.  Lane l
// < TMA_ROUND issues step (round * TMA_ROUND + l): the 4 or 8 gathered rows, a bulk
// copy of the step's H weights and an ordinary shared store of its H column indices
// (the rows of a light slice's first step); its columns are loaded two rounds ahead.
// At the start of round k (k >= 1) round k - 1 has been read by every lane, so its
// slots take round k + 1.  consume(t, slot) is called for every step in order, by
// all lanes; it returns false to stop early.  Returns false if a wait gave up (then
// NVD_ERR_TIMEOUT is in c.err and the copies in flight have been waited for).
template <int H, int RB, class TA, class Consume>
__device__ __forceinline__ bool tma_stream(const Ctx &c, int64_t E0, int64_t T, char *wring, uint64_t *bars,
                                           const CUtensorMap *tm, Consume &&consume) {
    constexpr int Q = H / 4;
    constexpr uint32_t WB = H * (uint32_t)sizeof(TA);
    const int lane = threadIdx.x & 31;
    const TA *__restrict__ slw = reinterpret_cast<const TA *>(c.sl_w);
    int4 cq1[Q], cq2[Q];
    auto load_cols = [&](int64_t t, int4 (&o)[Q]) {
        if (lane < TMA_ROUND && t < T) {
#pragma unroll
            for (int q = 0; q < Q; ++q) o[q] = __ldcs(reinterpret_cast<const int4 *>(c.sl_col + E0 + t * H) + q);
        }
    };
    auto issue = [&](int64_t t, const int4 (&o)[Q]) {
        if (lane < TMA_ROUND && t < T) {
            const int sl = (int)(t % TMA_SLOTS);
            char *slot = wring + sl * TMA_SLOT_BYTES;
            int4 *ids = reinterpret_cast<int4 *>(slot + TMA_IDS_OFFSET);
#pragma unroll
            for (int q = 0; q < Q; ++q) ids[q] = o[q];
            mbar_arrive_expect_tx(bars + sl, TMA_STEP_BYTES + WB);
#pragma unroll
            for (int q = 0; q < Q; ++q) tma_gather4(slot + q * 4 * RB, tm, 0, o[q].x, o[q].y, o[q].z, o[q].w, bars + sl);
            tma_bulk_g2s(slot + TMA_STEP_BYTES, slw + E0 + t * H, WB, bars + sl);
        }
    };
    {
        int4 c0[Q];
        load_cols(lane, c0);
        load_cols(TMA_ROUND + lane, cq1);
        load_cols(2 * TMA_ROUND + lane, cq2);
        issue(lane, c0);
        issue(TMA_ROUND + lane, cq1);
#pragma unroll
        for (int q = 0; q < Q; ++q) cq1[q] = cq2[q];
        load_cols(3 * TMA_ROUND + lane, cq2);
    }
    __syncwarp();
    int64_t t = 0;
    for (; t < T; ++t) {
        if (t >= TMA_ROUND && t % TMA_ROUND == 0) {
            __syncwarp();
            fence_proxy_async_smem();
            issue(t + TMA_ROUND + lane, cq1);
#pragma unroll
            for (int q = 0; q < Q; ++q) cq1[q] = cq2[q];
            load_cols(t + 3 * TMA_ROUND + lane, cq2);
            __syncwarp();
        }
        const int sl = (int)(t % TMA_SLOTS);
        const bool ok = mbar_wait_bounded(bars + sl, (uint32_t)((t / TMA_SLOTS) & 1), 1000000000ull);
        if (!__all_sync(NVD_FULLMASK, ok)) break;   // the warp leaves together
        if (!consume(t, (const char *)(wring + sl * TMA_SLOT_BYTES))) {
            ++t;
            break;
        }
    }
    if (t < T) {
        // stopped early: wait (bounded) for the copies still in flight
        const int64_t issued = ((t / TMA_ROUND) + 2) * TMA_ROUND;
        bool timed_out = false;
        for (int64_t u = t; u < issued && u < T; ++u)
            timed_out |= !mbar_wait_bounded(bars + (int)(u % TMA_SLOTS), (uint32_t)((u / TMA_SLOTS) & 1),
                                            100000000ull);
        __syncwarp();
        (void)timed_out;
        return false;
    }
    __syncwarp();
    return true;
}

// ------------------------------------------------------------------ per-lane asynchronous copies

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Steps per round and rounds in flight of the asynchronous-copy engine (the ring is
// the TMA engine's: TMA_SLOTS slots of TMA_SLOT_BYTES per warp).
constexpr int ACOPY_ROUND = 4;
constexpr int ACOPY_DEPTH = TMA_SLOTS / ACOPY_ROUND;

// The step stream of one warp as in tma_stream, with the rows fetched by ordinary
// per-lane asynchronous copies (cp.async) instead of the TMA unit: lane (g, sub)
// copies its own 16 bytes of row g of every step -- the bytes it reads back when the
// step is consumed -- so a lane only waits for its own copies (cp.async.wait_group),
// and the copies go through the load path like register gathers, without holding
// registers while in flight.  Rounds of ACOPY_ROUND steps, ACOPY_DEPTH rounds in
// flight; at the start of round k (its copies waited for), round k + DEPTH - 1 is
// issued into the slots of round k - 1, which every lane has read.  The lanes that
// loaded a round's columns and weights (entry s*H + g of the round in lane s*H + g)
// store them into the step's slot; the copy of step s row g takes its column by a
// shuffle.  consume(t, slot) as for tma_stream.  No wait can hang: wait_group waits
// for this lane's own copies, which always complete.
template <int H, int RB, class TV, class TA, int KT, class Consume>
__device__ __forceinline__ void acopy_stream(const Ctx &c, int64_t E0, int64_t T, const TV *__restrict__ src,
                                             char *wring, Consume &&consume) {
    constexpr int R = ACOPY_ROUND, DEPTH = ACOPY_DEPTH, LPR = RB / 16, VEC = 16 / (int)sizeof(TV);
    static_assert(R * H <= 32 && DEPTH >= 2 && LPR * H == 32, "one round's entries fit the warp's lanes");
    const int lane = threadIdx.x & 31, gid = lane / LPR, sub = lane % LPR;
    const int32_t *__restrict__ cols = c.sl_col + E0;
    const TA *__restrict__ ws = reinterpret_cast<const TA *>(c.sl_w) + E0;
    const int64_t NE = T * H;
    const int64_t NR = (T + R - 1) / R;   // rounds
    // meta of a round: lane l < R*H holds entry l (step l / H, row l % H)
    auto load_meta = [&](int64_t k, int &oc, TA &ow) {
        const int64_t e = k * (R * H) + lane;
        oc = 0;
        ow = 0;
        if (lane < R * H && e < NE) {
            oc = __ldcs(cols + e);
            ow = __ldcs(ws + e);
        }
    };
    auto issue = [&](int64_t k, int mc, TA mw) {
        if (k < NR) {
            if (lane < R * H) {
                const int64_t t = k * R + lane / H;
                if (t < T) {
                    char *slot = wring + (int)(t % TMA_SLOTS) * TMA_SLOT_BYTES;
                    reinterpret_cast<TA *>(slot + TMA_STEP_BYTES)[lane % H] = mw;
                    reinterpret_cast<int32_t *>(slot + TMA_IDS_OFFSET)[lane % H] = mc;
                }
            }
#pragma unroll
            for (int s = 0; s < R; ++s) {
                const int col = __shfl_sync(NVD_FULLMASK, mc, s * H + gid);
                const int64_t t = k * R + s;
                if (t < T)
                    cp_async16(wring + (int)(t % TMA_SLOTS) * TMA_SLOT_BYTES + gid * RB + sub * 16,
                               src + (int64_t)col * KT + sub * VEC);
            }
        }
        cp_async_commit();   // an empty group past the end keeps the group count
    };
    // meta two rounds ahead of its issue
    int c0, c1;
    TA w0, w1;
    {
        int mc;
        TA mw;
#pragma unroll
        for (int k = 0; k < DEPTH - 1; ++k) {
            load_meta(k, mc, mw);
            issue(k, mc, mw);
        }
        load_meta(DEPTH - 1, c0, w0);
        load_meta(DEPTH, c1, w1);
    }
    int64_t t = 0;
    for (int64_t k = 0; k < NR; ++k) {
        __syncwarp();                       // round k - 1 has been read by every lane
        issue(k + DEPTH - 1, c0, w0);
        c0 = c1;
        w0 = w1;
        load_meta(k + DEPTH + 1, c1, w1);
        cp_async_wait<DEPTH - 1>();         // this lane's copies of round k have landed
        __syncwarp();                       // and every lane's slot stores of round k are visible
        bool go = true;
        for (int s = 0; s < R && t < T; ++s, ++t) {
            go = consume(t, (const char *)(wring + (int)(t % TMA_SLOTS) * TMA_SLOT_BYTES));
            if (!go) break;
        }
        if (!go) break;
    }
    cp_async_wait_all();
    __syncwarp();
}

}  // namespace dev
}  // namespace nvd
