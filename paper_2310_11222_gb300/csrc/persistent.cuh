// Persistent PCG: the whole solve of one tile in one cooperative kernel (internal).
//
// The same block routines as the host-driven path (kernels.cuh) run phase after
// phase; a grid-wide barrier separates the phases instead of kernel boundaries,
// and the loop ends on the device when every (segment, column) has left the
// active set (convergence, breakdown or max_iter), so no host round trip is
// needed.  Loads of data written earlier in the same launch use the coherent
// (L2) path.  With many owners this is the batched solve: the block-diagonal
// Laplacian of G graphs, each (graph, pair) with its own CG scalars.
#pragma once

#include "vecops.cuh"

namespace nvd {
namespace dev {

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (all CTAs co-resident).  Sense by
// generation counter; the wait is bounded (2 s): on timeout the CTA records
// NVD_ERR_TIMEOUT in c.err and every CTA leaves at its next barrier.
__device__ __forceinline__ bool grid_sync(const Ctx &c) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = atomicAdd(c.bar_gen, 0u);
        __threadfence();
        const unsigned arrived = atomicAdd(c.bar_count, 1u);
        if (arrived == gridDim.x - 1 + (unsigned)c.bar_extra) {
            atomicExch(c.bar_count, 0u);
            __threadfence();
            atomicAdd(c.bar_gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (atomicAdd(c.bar_gen, 0u) == gen) {
                if (__ldcg(c.err) != 0) break;
                if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > 2000000000ull) {
                    atomicCAS(c.err, 0, NVD_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return __ldcg(c.err) == 0;
}

// Lane vectors per trip of the vector phases: the whole solve is one kernel, so its
// register budget is the largest phase's; 16-byte lane vectors take 2 per trip.
template <class TV, int KT>
constexpr int persist_unroll() { return VecCfg<TV, KT>::VEC * (int)sizeof(TV) >= 16 ? 2 : 4; }

// One phase over all blocks of the grid-stride loop.  (Out-of-line phases spilled
// less but ran slower: call overhead and saved registers on every block.)
template <class TV, int KT, class Op, int U>
__device__ __forceinline__ void vec_phase(const Ctx &c, const Op op, char *smem) {
    for (int64_t b = blockIdx.x; b < c.n_vblk; b += gridDim.x) vec_block<TV, KT, Op, U>(c, op, b, smem);
}
template <class TV, class TW, class TA, int KT, class Epi>
__device__ __forceinline__ void spmm_phase(const Ctx &c, const Epi epi, const TV *src, TV *dst, char *smem) {
    for (int64_t b = blockIdx.x; b < c.n_sblk; b += gridDim.x)
        spmm_block<LdCoh, TV, TW, TA, KT>(c, epi, src, dst, b, smem);
}

// One tile: form delta, PCG to convergence, d^2, optional z_out, per-owner results.
template <class TV, class TW, class TA, int KT, class TX>
__device__ void persistent_solve(const Ctx &c, const PersistArgs &a, char *smem) {
    constexpr int PU = persist_unroll<TV, KT>();
    TV *x = (TV *)a.x, *r = (TV *)a.r, *p = (TV *)a.p, *q = (TV *)a.q, *u = (TV *)a.u;
    // delta = x - y, segment sums
    {
        OpFormDelta<TX, KT> fd;
        fd.delta = a.delta;
        fd.fin.KT = KT;
        vec_phase<double, KT, decltype(fd), PU>(c, fd, smem);
    }
    if (!grid_sync(c)) return;
    {
        OpInit<TV, KT, LdCoh> oi;
        oi.src = a.delta;
        oi.writeback = a.delta;
        oi.x = x;
        oi.r = r;
        oi.p = a.fold ? u : p;
        oi.fin.KT = KT;
        vec_phase<TV, KT, decltype(oi), PU>(c, oi, smem);
    }
    if (!grid_sync(c)) return;
    EpiLap epi;
    epi.fin.KT = KT;
    EpiLapDir<TV, KT> epd;
    epd.p = p;
    epd.q = q;
    epd.fin.KT = KT;
    OpUpdate<TV, KT, LdCoh> ou;
    ou.x = x;
    ou.r = r;
    ou.p = p;
    ou.q = q;
    ou.u = u;
    ou.fin.KT = KT;
    OpResid<TV, KT, LdCoh> orr;
    orr.r = r;
    orr.q = q;
    orr.fin.KT = KT;
    OpStepDir<TV, KT, LdCoh> od;
    od.x = x;
    od.r = r;
    od.p = p;
    // the device deactivates every column by max_iter, so this loop is bounded;
    // a.fold: two phases per iteration (SpMV on u with the direction update folded
    // in, then the x/r/u update), else three (SpMV on p, residual, direction with
    // the x step -- always run, it takes the last step of a converged column)
    for (int it = 0; it <= c.max_iter; ++it) {
        if (__ldcg(c.n_active) == 0) break;
        if (a.fold) {
            spmm_phase<TV, TW, TA, KT>(c, epd, u, q, smem);
            if (!grid_sync(c)) return;
            vec_phase<TV, KT, decltype(ou), PU>(c, ou, smem);
            if (!grid_sync(c)) return;
            continue;
        }
        spmm_phase<TV, TW, TA, KT>(c, epi, p, q, smem);
        if (!grid_sync(c)) return;
        vec_phase<TV, KT, decltype(orr), PU>(c, orr, smem);
        if (!grid_sync(c)) return;
        vec_phase<TV, KT, decltype(od), PU>(c, od, smem);
        if (!grid_sync(c)) return;
    }
    {
        OpFinal<TV, KT, LdCoh> of;
        of.x = x;
        of.delta = a.delta;
        of.fin.KT = KT;
        of.fin.set_d2 = true;
        vec_phase<TV, KT, decltype(of), PU>(c, of, smem);
    }
    if (!grid_sync(c)) return;
    if (a.write_z) {
        OpZout<TV, TX, KT, LdCoh> oz;
        oz.src = x;
        oz.meanv = c.meanx;
        vec_phase<TV, KT, decltype(oz), PU>(c, oz, smem);
    }
    // per (owner, column) results (grid-stride: any number of owners)
    for (int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; tid < (int64_t)a.n_owner * KT;
         tid += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(tid / KT), j = (int)(tid % KT);
        const Owner &ow = c.owners ? c.owners[o] : c.own0;
        ColResult rs{0.0, 0.0, 0.0, 0, NVD_OK};
        for (int sg = ow.seg0; sg < ow.seg1; ++sg) {
            const int64_t i = (int64_t)sg * KT + j;
            rs.d2 += __ldcg(c.d2 + i);
            rs.rr += __ldcg(c.rr + i);
            rs.rr0 += __ldcg(c.rr0 + i);
            rs.iters = max(rs.iters, __ldcg(c.iters + i));
            const int st = __ldcg(c.status + i);
            if (st == NVD_ERR_NUMERIC || (st == NVD_ERR_NOT_CONVERGED && rs.status == NVD_OK)) rs.status = st;
        }
        a.res[tid] = rs;
    }
}

// Shared memory of the persistent kernel: the larger of the SpMM and vector needs.
template <class TV, class TA, int KT>
struct PersistSmem {
    static constexpr int A = SpCfg<TV, TA, KT>::SMEM, B = vec_smem_bytes(KT);
    static constexpr int BYTES = A > B ? A : B;
};

}  // namespace dev

template <class TV, class TW, class TA, int KT, class TX>
__global__ void __launch_bounds__(NT, 2) k_persistent(Ctx c, PersistArgs a) {
    __shared__ __align__(16) char smem[dev::PersistSmem<TV, TA, KT>::BYTES];
    dev::persistent_solve<TV, TW, TA, KT, TX>(c, a, smem);
}

}  // namespace nvd
