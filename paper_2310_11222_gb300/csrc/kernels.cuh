// Device code of the GE-distance solver (internal; sm_103a).
//
// The method (Section 3.1, GE equation; Section 3.2 Laplacian solvers): solve
// L z = P(x - y) by Jacobi-preconditioned conjugate gradient and take
// (x - y)^T z.  Every pass over the data is one of the "block" routines below;
// the host-driven solver launches them as separate kernels, the persistent
// solver calls them inside one cooperative kernel separated by grid barriers.
//
// Work layout: block vectors are [n][KT] row-major (KT right-hand sides side by
// side, one 16-byte-aligned row per node), the graph is CSR in internal node
// order where every connected component ("segment") is a contiguous node range,
// plus a sliced copy of its light rows (see Ctx::sl_*).  Each CTA block covers
// work of one segment (slices, heavy sub-items or a row range) and owns one
// partial-sum slot per inner product; the last block of a segment to finish
// (atomic arrival counters) adds the segment's slots -- directly in slot order,
// or, for many slots, the sums of groups of consecutive slots that each group's
// last writer formed -- and updates the per-(segment, column) CG scalars, so
// every reduction is deterministic and needs no extra launch.
#pragma once

#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "common.h"

namespace nvd {
namespace dev {

#define NVD_FULLMASK 0xffffffffu

// Entries each lane keeps in flight per pass of the single-RHS SpMV row loop.
#ifndef SPMV1_UNROLL
#define SPMV1_UNROLL 4
#endif
// Gathered neighbour rows each lane group keeps in flight in the multi-RHS SpMM
// (FP64 rows: 2, their products already keep the FP64 pipe busy; FP32 rows: 4).
#ifndef SPMM_UNROLL_F64
#define SPMM_UNROLL_F64 2
#endif
#ifndef SPMM_UNROLL_F32
#define SPMM_UNROLL_F32 4
#endif

// ------------------------------------------------------------------ loads/stores

// Read-only data path: data not written by any CTA during the kernel.
struct LdRO {
    template <class T>
    static __device__ __forceinline__ T ld(const T *p) { return __ldg(p); }
};
// Coherent path (L2): data written by other CTAs earlier in the same kernel
// (persistent kernel; L1 is not coherent across SMs).
struct LdCoh {
    template <class T>
    static __device__ __forceinline__ T ld(const T *p) { return __ldcg(p); }
};

template <class T, int V> struct VecOf;
template <> struct VecOf<float, 1> { typedef float t; };
template <> struct VecOf<float, 2> { typedef float2 t; };
template <> struct VecOf<float, 4> { typedef float4 t; };
template <> struct VecOf<double, 1> { typedef double t; };
template <> struct VecOf<double, 2> { typedef double2 t; };

__device__ __forceinline__ void unpack(float a, float (&o)[1]) { o[0] = a; }
__device__ __forceinline__ void unpack(float2 a, float (&o)[2]) { o[0] = a.x; o[1] = a.y; }
__device__ __forceinline__ void unpack(float4 a, float (&o)[4]) {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void unpack(double a, double (&o)[1]) { o[0] = a; }
__device__ __forceinline__ void unpack(double2 a, double (&o)[2]) { o[0] = a.x; o[1] = a.y; }
__device__ __forceinline__ float pack(const float (&o)[1]) { return o[0]; }
__device__ __forceinline__ float2 pack(const float (&o)[2]) { return make_float2(o[0], o[1]); }
__device__ __forceinline__ float4 pack(const float (&o)[4]) {
    return make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ double pack(const double (&o)[1]) { return o[0]; }
__device__ __forceinline__ double2 pack(const double (&o)[2]) { return make_double2(o[0], o[1]); }

// Plain (default-cached) loads for data this kernel may also write.
struct LdPlain {
    template <class T>
    static __device__ __forceinline__ T ld(const T *p) { return *p; }
};

// V consecutive elements, naturally aligned; wider than 16 bytes = several 16-byte loads.
template <class LD, class T, int V>
__device__ __forceinline__ void ldv(const T *p, T (&o)[V]) {
    if constexpr (V * sizeof(T) <= 16) {
        unpack(LD::ld(reinterpret_cast<const typename VecOf<T, V>::t *>(p)), o);
    } else {
        constexpr int H = V / 2;
        T a[H], b[H];
        ldv<LD, T, H>(p, a);
        ldv<LD, T, H>(p + H, b);
#pragma unroll
        for (int i = 0; i < H; ++i) {
            o[i] = a[i];
            o[H + i] = b[i];
        }
    }
}
template <class T, int V>
__device__ __forceinline__ void stv(T *p, const T (&o)[V]) {
    if constexpr (V * sizeof(T) <= 16) {
        *reinterpret_cast<typename VecOf<T, V>::t *>(p) = pack(o);
    } else {
        constexpr int H = V / 2;
        T a[H], b[H];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            a[i] = o[i];
            b[i] = o[H + i];
        }
        stv<T, H>(p, a);
        stv<T, H>(p + H, b);
    }
}

// Four consecutive CSR weights starting at a multiple of 4 (streaming, evict-first).
__device__ __forceinline__ void ld4_stream(const float *p, float (&o)[4]) {
    float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void ld4_stream(const double *p, double (&o)[4]) {
    double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// Elements per lane-vector for a [n][KT] array of T (16-byte loads when possible).
template <class T, int KT>
struct VecCfg {
    static constexpr int VEC = (KT * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : KT;
    static constexpr int CG = KT / VEC;  // lane-vectors per row
};

__device__ __forceinline__ const Owner &owner_of(const Ctx &c, int seg) {
    return c.owners ? c.owners[c.seg_owner[seg]] : c.own0;
}

template <class T> __device__ __forceinline__ const T *dinv_of(const Ctx &c);
template <> __device__ __forceinline__ const float *dinv_of<float>(const Ctx &c) { return c.dinv32; }
template <> __device__ __forceinline__ const double *dinv_of<double>(const Ctx &c) { return c.dinv64; }
template <class T> __device__ __forceinline__ const T *deg_of(const Ctx &c);
template <> __device__ __forceinline__ const float *deg_of<float>(const Ctx &c) { return c.deg32; }
template <> __device__ __forceinline__ const double *deg_of<double>(const Ctx &c) { return c.deg64; }

// ------------------------------------------------------------------ reductions

// Per-thread partial sums of inner products.  FP64 vectors: an FP64 accumulator.
// FP32 vectors: a double-float accumulator (hi + lo, about 48 significant bits)
// fed with the exact product of two floats (p = a*b and e = fma(a, b, -p) give
// a*b = p + e) and Knuth's two-sum, all on the FP32 pipe -- on this part FP64
// runs at 1/64 of the FP32 rate, and one FP64 multiply-add plus two conversions
// per element made the FP64 unit the limit of every FP32 pass.  The thread's
// partial is converted to FP64 (hi + lo) before the block and grid reductions,
// which run in FP64.  The _rn intrinsics keep the compiler from fusing the
// error-free steps.
struct DFloat {
    float hi, lo;
};
template <class TV> struct DotOf { typedef double type; };
template <> struct DotOf<float> { typedef DFloat type; };

__device__ __forceinline__ void dot_zero(double &d) { d = 0.0; }
__device__ __forceinline__ void dot_zero(DFloat &d) { d.hi = 0.f; d.lo = 0.f; }
__device__ __forceinline__ double dot_get(double d) { return d; }
__device__ __forceinline__ double dot_get(const DFloat &d) { return (double)d.hi + (double)d.lo; }
__device__ __forceinline__ void dot_add(double &d, double a) { d += a; }
__device__ __forceinline__ void dot_fma(double &d, double a, double b) { d = fma(a, b, d); }
__device__ __forceinline__ void dot_add(DFloat &d, float a) {
    const float s = __fadd_rn(d.hi, a);          // two-sum: s + t = d.hi + a exactly
    const float bb = __fsub_rn(s, d.hi);
    const float t = __fadd_rn(__fsub_rn(d.hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
    d.hi = s;
    d.lo = __fadd_rn(d.lo, t);
}
__device__ __forceinline__ void dot_fma(DFloat &d, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);         // a*b - p, exact
    const float s = __fadd_rn(d.hi, p);
    const float bb = __fsub_rn(s, d.hi);
    const float t = __fadd_rn(__fsub_rn(d.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    d.hi = s;
    d.lo = __fadd_rn(d.lo, __fadd_rn(t, e));
}

// FP64 copy of a thread's partial sums.
template <int ND, int VEC, class D>
__device__ __forceinline__ void dot_to_double(const D (&a)[ND][VEC], double (&o)[ND][VEC]) {
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[d][v] = dot_get(a[d][v]);
}

// Block-wide per-column sums.  Thread t holds acc[d][v] for column
// (t % CG) * VEC + v.  On return tot[d * KT + j] (shared) holds the block total,
// summed in a fixed order (KT = 1: per lane over the warps, then a butterfly;
// KT > 1: warp butterfly, then warps 0..7).
template <int ND, int KT, int VEC>
__device__ __forceinline__ void block_reduce_cols(double (&acc)[ND > 0 ? ND : 1][VEC], double *red,
                                                  double *tot) {
    if constexpr (ND > 0 && KT == 1) {
        // one column: each sum's NT partials go to shared memory and warp d adds
        // sum d (lane l: partials l, l+32, ... in order, then a butterfly), which
        // takes far fewer FP64 instructions than a butterfly in every warp
        static_assert(ND <= 4, "reduction scratch holds 4 sums");
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int d = 0; d < ND; ++d) red[d * NT + threadIdx.x] = acc[d][0];
        __syncthreads();
        if (warp < ND) {
            double s = red[warp * NT + lane];
#pragma unroll
            for (int k = 1; k < NWARP; ++k) s += red[warp * NT + k * 32 + lane];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(NVD_FULLMASK, s, off);
            if (lane == 0) tot[warp] = s;
        }
        __syncthreads();
    } else if constexpr (ND > 0) {
        constexpr int CG = KT / VEC;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int off = CG; off < 32; off <<= 1)
#pragma unroll
            for (int d = 0; d < ND; ++d)
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                    acc[d][v] += __shfl_xor_sync(NVD_FULLMASK, acc[d][v], off);
        if (lane < CG) {
#pragma unroll
            for (int d = 0; d < ND; ++d)
#pragma unroll
                for (int v = 0; v < VEC; ++v) red[(warp * ND + d) * KT + lane * VEC + v] = acc[d][v];
        }
        __syncthreads();
        if (threadIdx.x < ND * KT) {
            const int d = threadIdx.x / KT, j = threadIdx.x % KT;
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NWARP; ++w) s += red[(w * ND + d) * KT + j];
            tot[threadIdx.x] = s;
        }
        __syncthreads();
    }
}

constexpr int pow2floor(int x) { return x >= 256 ? 256 : x >= 128 ? 128 : x >= 64 ? 64 : x >= 32 ? 32
                                       : x >= 16 ? 16 : x >= 8 ? 8 : x >= 4 ? 4 : x >= 2 ? 2 : 1; }

// Cross-block sums.  Every block of a pass owns one partial-sum slot per inner
// product; a split row's finishing chunk owns one more ("heavy" slot).  The sum
// over a segment's slots is taken in a fixed order, so it does not depend on
// which block finishes last:
//   few slots: the segment's last block to arrive adds all slots in slot order;
//   many slots: the slots form arrival groups of SLOT_GROUP consecutive slots; the
//     last writer of a group adds that group in slot order into the group's sum
//     (gpart, at the group's first slot) and arrives on the segment; the last
//     group to arrive adds the group sums in group order.  The tail of a pass (the
//     work left once every other block is done) then reads a few hundred group
//     sums instead of every slot -- one SM reading tens of thousands of slots took
//     a large part of a multi-column SpMM.
constexpr int SLOT_GROUP = 32;
// Slots x sums up to which one block adds the segment's slots itself.
constexpr int FLAT_SUMS_MAX = 16384;

// Block-wide, fixed order: for each sum p = d * KT + j (P = ND * KT of them),
//   sums[p] = sum_k a[(d * stride + a0 + k * as) * KT + j], k < an
//           + sum_k b[(d * stride + b0 + k * bs) * KT + j], k < bn
// (thread `sub` of the TPP threads of sum p takes k = sub, sub + TPP, ... of each
// range in order; the TPP partials are then added by a fixed butterfly).
// `sums` holds P doubles and `red` at least 128 + NWARP doubles of shared scratch
// (sums may alias red).
template <int ND, int KT>
__device__ __forceinline__ void block_sum_slots(const double *a, int64_t a0, int32_t an, int32_t as,
                                                const double *b, int64_t b0, int32_t bn, int32_t bs,
                                                int64_t stride, double *red) {
    constexpr int P = ND * KT;
    constexpr int TPP = pow2floor(NT / P);
    const int pair = threadIdx.x / TPP, sub = threadIdx.x % TPP;
    double s = 0.0;
    if (pair < P) {
        const int d = pair / KT, j = pair % KT;
        const double *pa = a + (d * stride + a0) * KT + j;
        const int64_t sa = (int64_t)as * KT;
        // eight independent loads in flight, added in slot order
        int i = sub;
        for (; i + 7 * TPP < an; i += 8 * TPP) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(pa + (int64_t)(i + u * TPP) * sa);
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; i < an; i += TPP) s += __ldcg(pa + (int64_t)i * sa);
        if (bn > 0) {
            const double *pb = b + (d * stride + b0) * KT + j;
            const int64_t sb = (int64_t)bs * KT;
            i = sub;
            for (; i + 7 * TPP < bn; i += 8 * TPP) {
                double v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcg(pb + (int64_t)(i + u * TPP) * sb);
#pragma unroll
                for (int u = 0; u < 8; ++u) s += v[u];
            }
            for (; i < bn; i += TPP) s += __ldcg(pb + (int64_t)i * sb);
        }
    }
    constexpr int WOFF = TPP < 32 ? TPP : 32;
#pragma unroll
    for (int off = WOFF / 2; off > 0; off >>= 1) s += __shfl_xor_sync(NVD_FULLMASK, s, off);
    double *sums = red;          // [P]
    double *wsum = red + 128;    // [NWARP] (only when TPP > 32)
    if constexpr (TPP > 32) {
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
        __syncthreads();
        if (sub == 0 && pair < P) {
            double t = 0.0;
            for (int w = 0; w < TPP / 32; ++w) t += wsum[pair * (TPP / 32) + w];
            sums[pair] = t;
        }
    } else {
        __syncthreads();         // the caller may have read red just before
        if (sub == 0 && pair < P) sums[pair] = s;
    }
    __syncthreads();
}

// After this block's writes to a slot of group [f, f + m): count the arrival; the
// group's last writer adds the group into gpart at f.  Returns (block-uniformly)
// whether this block did.
template <int ND, int KT>
__device__ __forceinline__ bool group_arrive(const Ctx &c, int64_t f, int32_t m, double *red) {
    __shared__ int s_glast;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_glast = (atomicAdd(&c.gcount[f], 1u) == (unsigned)(m - 1));
    __syncthreads();
    if (!s_glast) return false;
    __threadfence();
    block_sum_slots<ND, KT>(c.part, f, m, 1, nullptr, 0, 0, 0, c.part_stride, red);
    if (threadIdx.x < ND * KT) {
        const int d = threadIdx.x / KT, j = threadIdx.x % KT;
        c.gpart[((int64_t)d * c.part_stride + f) * KT + j] = red[threadIdx.x];
    }
    if (threadIdx.x == 0) atomicExch(&c.gcount[f], 0u);
    return true;
}

__device__ __forceinline__ int32_t n_groups(int32_t cnt) { return (cnt + SLOT_GROUP - 1) / SLOT_GROUP; }

// The segment adds its slots itself (one level) when they are few, unless split
// rows arrive in groups of their own (hgroup) and the segment has some.
template <int ND, int KT>
__device__ __forceinline__ bool seg_flat(int32_t cnt, int32_t hcnt, bool hgroup) {
    return (int64_t)(cnt + hcnt) * ND * KT <= FLAT_SUMS_MAX && (!hgroup || hcnt == 0);
}

// Arrival of a group sum on its segment; the last group adds the block groups then
// the heavy groups (hgroup; else the heavy slots themselves) and calls
// fin(c, seg, j, sums) for each column j.
template <int ND, int KT, class Fin>
__device__ void seg_group_arrive(const Ctx &c, const Fin &fin, int seg, int64_t s0, int32_t cnt, int64_t h0,
                                 int32_t hcnt, bool hgroup, double *red) {
    __shared__ int s_last;
    const int32_t ng = n_groups(cnt) + (hgroup ? n_groups(hcnt) : 0);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&c.counter[seg], 1u) == (unsigned)(ng - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (hgroup)
        block_sum_slots<ND, KT>(c.gpart, s0, n_groups(cnt), SLOT_GROUP, c.gpart, h0, n_groups(hcnt), SLOT_GROUP,
                                c.part_stride, red);
    else
        block_sum_slots<ND, KT>(c.gpart, s0, n_groups(cnt), SLOT_GROUP, c.part, h0, hcnt, 1, c.part_stride, red);
    if (threadIdx.x < KT) {
        double v[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) v[d] = red[d * KT + threadIdx.x];
        fin(c, seg, threadIdx.x, v);
    }
    if (threadIdx.x == 0) atomicExch(&c.counter[seg], 0u);
    __syncthreads();
}

// Publish this block's partials (tot, shared) into `slot` and arrive: the segment's
// blocks are slots [s0, s0 + cnt), its split-row slots [h0, h0 + hcnt).  The block
// that completes the segment calls fin(c, seg, j, sums) for each column j (one
// thread per column).  `red` needs NT doubles of shared scratch.  hgroup: the
// split rows' slots arrive themselves (heavy_arrive), in groups; every block of the
// pass must pass the same value, and it may be true only if every split row of the
// segment is finished in this pass.
template <int ND, int KT, class Fin>
__device__ void seg_arrive(const Ctx &c, const Fin &fin, int seg, int64_t slot, const double *tot,
                           int64_t s0, int32_t cnt, int64_t h0, int32_t hcnt, double *red, bool hgroup = false) {
    static_assert(ND > 0, "arrival needs a reduction");
    __shared__ int s_last;
    if (threadIdx.x < ND * KT) {
        const int d = threadIdx.x / KT, j = threadIdx.x % KT;
        c.part[((int64_t)d * c.part_stride + slot) * KT + j] = tot[threadIdx.x];
    }
    if (!seg_flat<ND, KT>(cnt, hcnt, hgroup)) {
        const int64_t f = s0 + (slot - s0) / SLOT_GROUP * SLOT_GROUP;
        const int32_t m = (int32_t)(s0 + cnt - f < SLOT_GROUP ? s0 + cnt - f : SLOT_GROUP);
        if (group_arrive<ND, KT>(c, f, m, red)) seg_group_arrive<ND, KT>(c, fin, seg, s0, cnt, h0, hcnt, hgroup, red);
        return;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&c.counter[seg], 1u) == (unsigned)(cnt - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    block_sum_slots<ND, KT>(c.part, s0, cnt, 1, c.part, h0, hcnt, 1, c.part_stride, red);
    if (threadIdx.x < KT) {
        double v[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) v[d] = red[d * KT + threadIdx.x];
        fin(c, seg, threadIdx.x, v);
    }
    if (threadIdx.x == 0) atomicExch(&c.counter[seg], 0u);
    __syncthreads();
}

// A split row's finishing chunk (a whole block) has written the row's slot hs:
// arrive on the row's heavy group and, if that completes it, on the segment.
template <int ND, int KT, class Fin>
__device__ void heavy_arrive(const Ctx &c, const Fin &fin, int seg, int64_t hs, double *red) {
    const int64_t s0 = c.seg_sblk_off[seg];
    const int32_t cnt = c.seg_sblk_off[seg + 1] - (int32_t)s0;
    const int64_t h0 = c.n_sblk + c.seg_heavy_off[seg];
    const int32_t hcnt = c.seg_heavy_off[seg + 1] - c.seg_heavy_off[seg];
    const int64_t f = h0 + (hs - h0) / SLOT_GROUP * SLOT_GROUP;
    const int32_t m = (int32_t)(h0 + hcnt - f < SLOT_GROUP ? h0 + hcnt - f : SLOT_GROUP);
    if (group_arrive<ND, KT>(c, f, m, red)) seg_group_arrive<ND, KT>(c, fin, seg, s0, cnt, h0, hcnt, true, red);
}

// Is any column of the segment still iterating?  (Constant during one phase:
// only the segment's own finalizer changes it, after all its blocks arrived.)
template <int KT>
__device__ __forceinline__ bool seg_live(const Ctx &c, int seg) {
    int a = 0;
#pragma unroll
    for (int j = 0; j < KT; ++j) a |= __ldcg(c.active + (int64_t)seg * KT + j);
    return a != 0;
}

// ------------------------------------------------------------------ finalizers
// Run by one thread per column in the last block of a segment.

struct FinNone {
    __device__ void operator()(const Ctx &, int, int, const double *) const {}
};

// Per-segment mean of the right-hand side (projection P, Section 3.1: L^+
// annihilates constants on every component).
struct FinMean {
    __device__ void operator()(const Ctx &c, int seg, int j, const double *s) const {
        const double sz = (double)(c.seg_end[seg] - c.seg_begin[seg]);
        c.mean[(int64_t)seg * KT + j] = s[0] / sz;
    }
    int KT;
};

// PCG start: rho = r^T D^-1 r, rr0 = |r|^2; a column iterates if it is a real
// pair of this owner and its right-hand side is non-zero.  keep_rr0 (warm start,
// r = P(delta - L z0)): rr0 stays |P delta|^2 from the first start, and a column
// whose start already meets the residual test does not iterate.
struct FinInit {
    int KT;
    bool keep_rr0 = false;
    __device__ void operator()(const Ctx &c, int seg, int j, const double *s) const {
        const int64_t i = (int64_t)seg * KT + j;
        const bool valid = j < owner_of(c, seg).kc;
        const double rho = s[0], rr = s[1];
        c.rho[i] = rho;
        c.rr[i] = rr;
        if (!keep_rr0) c.rr0[i] = rr;
        c.alpha[i] = 0.0;
        c.beta[i] = 0.0;
        c.iters[i] = 0;
        if (c.d2stop > 0.0) {
            c.hs_sum[i] = 0.0;
            for (int w = 0; w < d2_window(); ++w) c.hs_hist[i * d2_window() + w] = 0.0;
        }
        const bool finite = isfinite(rr) && isfinite(rho);
        c.status[i] = (valid && !finite) ? NVD_ERR_NUMERIC : NVD_OK;
        const bool act = valid && finite && rr > 0.0 && rho > 0.0 && !(keep_rr0 && rr <= c.rtol2 * c.rr0[i]);
        c.active[i] = act ? 1 : 0;
        if (act) atomicAdd(c.n_active, 1);
    }
};

// After q = L p: alpha = rho / p^T q.  Loss of positivity is recorded in status
// and acted on by FinUpdate (so n_active only changes in FinInit/FinUpdate).
struct FinAlpha {
    int KT;
    __device__ void operator()(const Ctx &c, int seg, int j, const double *s) const {
        const int64_t i = (int64_t)seg * KT + j;
        if (!c.active[i]) {
            c.alpha[i] = 0.0;
            return;
        }
        const double pq = s[0];
        if (pq > 0.0 && isfinite(pq)) {
            c.alpha[i] = c.rho[i] / pq;
        } else {
            c.alpha[i] = 0.0;
            c.status[i] = NVD_ERR_NUMERIC;
        }
    }
};

// After x += alpha p, r -= alpha q: convergence test on |r|^2 <= rtol^2 |r0|^2,
// beta = rho_new / rho.
//
// With c.d2stop > 0 a column also stops when its d^2 is accurate enough.  From
// x_0 = 0, step k raises delta^T x by exactly t_k = alpha_k rho_k (rho_k =
// r_k^T D^-1 r_k), and the remaining gap d^2 - delta^T x_k = |x* - x_k|_L^2 is the
// sum of the terms still to come (the Hestenes-Stiefel identity behind the CG
// error estimates of Strakos and Tichy).  The terms shrink about geometrically
// once CG settles, so the gap is extrapolated as t_k q / (1 - q) with q the largest
// ratio of consecutive terms over the last d2_window() steps; the column stops when
// that is at most d2_safety() * d2stop of the sum so far and q < 0.95 (no stop
// while the terms are not clearly shrinking).  This is an estimate, not a bound.
struct FinBeta {
    int KT;
    __device__ void operator()(const Ctx &c, int seg, int j, const double *s) const {
        const int64_t i = (int64_t)seg * KT + j;
        if (!c.active[i]) return;
        const int it = c.iters[i] + 1;
        c.iters[i] = it;
        const double rho_new = s[0], rr = s[1];
        c.rr[i] = rr;
        bool d2_done = false;
        if (c.d2stop > 0.0) {
            double *h = c.hs_hist + i * d2_window();   // t_{k-1}, t_{k-2}, ...
            const double t = c.alpha[i] * c.rho[i];
            const double sum = c.hs_sum[i] + t;
            c.hs_sum[i] = sum;
            bool ok = it > d2_window() && t > 0.0;
            double q = 0.0, nxt = t;
            for (int w = 0; w < d2_window(); ++w) {
                const double prev = h[w];
                ok = ok && prev > 0.0;
                if (prev > 0.0) q = fmax(q, nxt / prev);
                h[w] = nxt;
                nxt = prev;
            }
            d2_done = ok && q < 0.95 && t * q <= d2_safety() * c.d2stop * sum * (1.0 - q);
        }
        int st = -1;
        if (c.status[i] == NVD_ERR_NUMERIC || !isfinite(rr) || !isfinite(rho_new))
            st = NVD_ERR_NUMERIC;
        else if (rr <= c.rtol2 * c.rr0[i] || d2_done)
            st = NVD_OK;
        else if (it >= c.max_iter)
            st = NVD_ERR_NOT_CONVERGED;
        if (st >= 0) {
            c.status[i] = st;
            c.active[i] = 0;
            c.beta[i] = 0.0;
            atomicSub(c.n_active, 1);
        } else {
            c.beta[i] = rho_new / c.rho[i];
            c.rho[i] = rho_new;
        }
    }
};

// End of a solve: mean of x per segment, d^2 = delta^T x (Section 3.1; with x
// projected afterwards, delta^T P x = delta^T x because P delta = delta).
struct FinFinal {
    int KT;
    bool set_d2;  // false after refinement: d^2 is the variational value of FinResid
    __device__ void operator()(const Ctx &c, int seg, int j, const double *s) const {
        const int64_t i = (int64_t)seg * KT + j;
        const double sz = (double)(c.seg_end[seg] - c.seg_begin[seg]);
        c.meanx[i] = s[0] / sz;
        if (set_d2) c.d2[i] = s[1];
    }
};

// FP64 residual of iterative refinement, r = delta - L z:
//   d^2 (variational) = 2 delta^T z - z^T L z = delta^T z + z^T r,
// error -|z* - z|_L^2 (quadratic in the error of z); mean(r) for the next projection.
struct FinResid {
    int KT;
    __device__ void operator()(const Ctx &c, int seg, int j, const double *s) const {
        const int64_t i = (int64_t)seg * KT + j;
        const double sz = (double)(c.seg_end[seg] - c.seg_begin[seg]);
        c.dz[i] = s[0];
        c.zr[i] = s[1];
        c.rr[i] = s[2];
        c.d2[i] = s[0] + s[1];
        c.mean[i] = s[3] / sz;
    }
};

// ------------------------------------------------------------------ SpMV / SpMM epilogues
// elem(): row i, columns col0..col0+VEC-1; own = src[i][cols], acc = sum_j w_ij src[j][cols].

// q = L p = D p - W p, and p^T q for alpha.
struct EpiLap {
    static constexpr int ND = 1;
    static constexpr bool NEEDS_LIVE = true;   // CG step: converged segments skip the work
    template <class TV> using D = typename DotOf<TV>::type;
    __device__ __forceinline__ void prep(const Ctx &, int, int) {}
    template <class TV, class TA, int VEC, class DT>
    __device__ __forceinline__ void elem(const Ctx &, int64_t i, int col0, int KT, const TV (&own)[VEC],
                                         const TA (&acc)[VEC], TA degi, TV *dst, DT (&dot)[1][VEC]) const {
        TV y[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            y[v] = (TV)(degi * (TA)own[v] - acc[v]);
            dot_fma(dot[0][v], own[v], y[v]);
        }
        stv(dst + i * KT + col0, y);
    }
    FinAlpha fin;
};

// The CG step with the direction update folded in.  The SpMV runs on the
// preconditioned residual u = D^-1 r instead of the direction p; with
// w = L u the new direction and its image follow row by row,
//     p = u + beta p_old,   q = L p = w + beta q_old,
// (q by the recurrence instead of a second product), and p^T q gives alpha.  This
// is the same CG (same alpha, beta, x, r in exact arithmetic) with one pass over
// the vectors fewer per iteration.  beta = 0 on the first iteration selects
// p = u, q = w (p_old, q_old are not read then); columns that stopped keep p, q.
template <class TVD, int KT>
struct EpiLapDir {
    static constexpr int ND = 1;
    static constexpr bool NEEDS_LIVE = true;
    static constexpr int VM = VecCfg<TVD, KT>::VEC;
    template <class TV> using D = typename DotOf<TV>::type;
    TVD *p, *q;
    TVD be[VM];
    unsigned act;   // bit v: column col0 + v still iterating
    __device__ __forceinline__ void prep(const Ctx &c, int seg, int col0) {
        act = 0;
#pragma unroll
        for (int v = 0; v < VM; ++v) {
            be[v] = (TVD)__ldcg(c.beta + (int64_t)seg * KT + col0 + v);
            if (__ldcg(c.active + (int64_t)seg * KT + col0 + v)) act |= 1u << v;
        }
    }
    template <class TV, class TA, int VEC, class DT>
    __device__ __forceinline__ void elem(const Ctx &, int64_t i, int col0, int, const TV (&own)[VEC],
                                         const TA (&acc)[VEC], TA degi, TV *, DT (&dot)[1][VEC]) const {
        static_assert(VEC == VM, "tile layout");
        const int64_t o = i * KT + col0;
        if (!act) return;
        bool first = true;
#pragma unroll
        for (int v = 0; v < VEC; ++v) first = first && !(be[v] != (TVD)0);
        TV pv[VEC], qv[VEC];
        if (!first) {
            ldv<LdPlain, TV, VEC>(p + o, pv);
            ldv<LdPlain, TV, VEC>(q + o, qv);
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const TV w = (TV)(degi * (TA)own[v] - acc[v]);
            const TV b = be[v];
            const TV pn = first ? own[v] : own[v] + b * pv[v];
            const TV qn = first ? w : w + b * qv[v];
            if (act & (1u << v)) {
                pv[v] = pn;
                qv[v] = qn;
                dot_fma(dot[0][v], pn, qn);
            }
        }
        stv(p + o, pv);
        stv(q + o, qv);
    }
    FinAlpha fin;
};

// y = L x only (operator application, no reduction).
struct EpiApply {
    static constexpr int ND = 0;
    static constexpr bool NEEDS_LIVE = false;
    template <class TV> using D = double;
    __device__ __forceinline__ void prep(const Ctx &, int, int) {}
    template <class TV, class TA, int VEC, class DT>
    __device__ __forceinline__ void elem(const Ctx &, int64_t i, int col0, int KT, const TV (&own)[VEC],
                                         const TA (&acc)[VEC], TA degi, TV *dst, DT (&)[1][VEC]) const {
        TV y[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) y[v] = (TV)(degi * (TA)own[v] - acc[v]);
        stv(dst + i * KT + col0, y);
    }
    FinNone fin;
};

// FP64 refinement residual r = delta - L z with delta^T z, z^T r, r^T r, sum r.
struct EpiResid {
    static constexpr int ND = 4;
    static constexpr bool NEEDS_LIVE = false;  // runs after the inner solve, always on every segment
    const double *delta;
    template <class TV> using D = double;
    __device__ __forceinline__ void prep(const Ctx &, int, int) {}
    template <class TV, class TA, int VEC>
    __device__ __forceinline__ void elem(const Ctx &, int64_t i, int col0, int KT, const TV (&own)[VEC],
                                         const TA (&acc)[VEC], TA degi, TV *dst,
                                         double (&dot)[4][VEC]) const {
        double dl[VEC];
        ldv<LdRO, double, VEC>(delta + i * KT + col0, dl);
        TV y[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const double lz = (double)degi * (double)own[v] - (double)acc[v];
            const double rv = dl[v] - lz;
            y[v] = (TV)rv;
            dot[0][v] += dl[v] * (double)own[v];
            dot[1][v] += (double)own[v] * rv;
            dot[2][v] += rv * rv;
            dot[3][v] += rv;
        }
        stv(dst + i * KT + col0, y);
    }
    FinResid fin;
};

// ------------------------------------------------------------------ SpMV / SpMM block

// Lane layout of the multi-column SpMM and the shared memory of a CTA: the row
// accumulators of one split row (KT x sza), the reduction scratch and the totals.
template <class TV, class TA, int KT>
struct SpCfg {
    static constexpr int VEC = VecCfg<TV, KT>::VEC;
    static constexpr int LPR = KT / VEC;          // lanes per gathered row vector
    static constexpr int G = 32 / LPR;            // rows per warp (rows per slice)
    static constexpr int ND_MAX = 4;
    static constexpr int RED = red_doubles(KT);
    static constexpr int ACC = KT == 1 ? 0 : ((KT * (int)sizeof(TA) + 15) / 16) * 16;
    // one column: the light rows' row sums (sp_span_max of them) live in the
    // reduction scratch; their presence bits and the slice counter follow the
    // totals (several columns: the slice counter)
    static constexpr int HAS = KT == 1 ? sp_span_max() / 32 * 4 + 16 : 16;
    static_assert(KT != 1 || RED * 8 >= sp_span_max() * (int)sizeof(TA), "row sums fit the scratch");
    static constexpr int SMEM = ACC + RED * 8 + ND_MAX * KT * 8 + HAS;
};

// Row epilogue of a split row: rows [r0, r1) with their neighbour sums in s_acc.
template <class LD, class TV, class TA, int KT, class Epi, class DT>
__device__ __forceinline__ void spmm_epilogue(const Ctx &c, const Epi &epi, int seg, const TV *src, TV *dst,
                                              int64_t r0, int64_t r1, const TA *s_acc,
                                              DT (&dot)[Epi::ND > 0 ? Epi::ND : 1][SpCfg<TV, TA, KT>::VEC]) {
    constexpr int VEC = SpCfg<TV, TA, KT>::VEC, CG = KT / VEC;
    const TA *deg = deg_of<TA>(c);
    const int64_t ne = (r1 - r0) * CG;
    for (int64_t t = threadIdx.x; t < ne; t += NT) {
        const int64_t li = t / CG;
        const int col0 = (int)(t % CG) * VEC;
        const int64_t i = r0 + li;
        TV own[VEC];
        ldv<LD, TV, VEC>(src + i * KT + col0, own);
        TA acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = s_acc[li * KT + col0 + v];
        Epi e = epi;
        e.prep(c, seg, col0);
        e.template elem<TV, TA, VEC>(c, i, col0, KT, own, acc, __ldg(deg + i), dst, dot);
    }
}

// One chunk [e0, e1) of a split row r0 (merge-path style row splitting): block-wide
// partial row sum into hsum; the chunk that arrives last adds the chunks in chunk
// order, applies the row epilogue and writes the row's partial slot.
template <class LD, class TV, class TW, class TA, int KT, class Epi>
__device__ __forceinline__ void spmm_chunk(const Ctx &c, const Epi &epi, int seg, const TV *__restrict__ src,
                                           TV *__restrict__ dst, const SpItem &it, TA *s_acc, double *red) {
    typedef SpCfg<TV, TA, KT> C;
    constexpr int VEC = C::VEC, LPR = C::LPR, G = C::G, ND = Epi::ND;
    const TW *__restrict__ w = reinterpret_cast<const TW *>(c.w);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // ---------------- chunk [e0, e1) of split row r0
    const int64_t i = it.r0;
    double *chunk = red;  // [KT] block total of this chunk
    if constexpr (KT == 1) {
        TA s = 0;
        for (int64_t eb = (it.e0 & ~(int64_t)3) + 4 * threadIdx.x; eb < it.e1; eb += 4 * NT) {
            const int4 c4 = __ldcs(reinterpret_cast<const int4 *>(c.colidx + eb));
            TW w4[4];
            ld4_stream(w + eb, w4);
            const int cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (eb + q >= it.e0 && eb + q < it.e1) s += (TA)w4[q] * (TA)LD::ld(src + cc[q]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(NVD_FULLMASK, s, off);
        if (lane == 0) red[NT / 2 + warp] = (double)s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < NWARP; ++q) t += red[NT / 2 + q];
            chunk[0] = t;
        }
    } else {
        const int gi = lane / LPR, col0 = (lane % LPR) * VEC;
        TA acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0;
        // entries e, e + S, e + 2S, ... of this lane group (S = NWARP * G), U of them
        // gathered together before their products are added in entry order (one in the
        // persistent kernel, LdCoh, whose registers are already at its cap: the unrolled
        // form made its batched solve 43% slower; the sums are the same either way)
        constexpr int U = std::is_same<LD, LdCoh>::value ? 1 : sizeof(TV) == 8 ? SPMM_UNROLL_F64 : SPMM_UNROLL_F32;
        constexpr int64_t S = (int64_t)NWARP * G;
        for (int64_t e = it.e0 + warp * G + gi; e < it.e1; e += U * S) {
            int ca[U];
            TA wa[U];
            TV pa[U][VEC];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (e + u * S < it.e1) {
                    ca[u] = __ldcs(c.colidx + e + u * S);
                    wa[u] = (TA)__ldcs(w + e + u * S);
                }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (e + u * S < it.e1) ldv<LD, TV, VEC>(src + (int64_t)ca[u] * KT + col0, pa[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (e + u * S < it.e1)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] += wa[u] * (TA)pa[u][v];
        }
#pragma unroll
        for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] += __shfl_xor_sync(NVD_FULLMASK, acc[v], off);
        if (gi == 0) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) red[KT + warp * KT + col0 + v] = (double)acc[v];
        }
        __syncthreads();
        if (threadIdx.x < KT) {
            double t = 0.0;
            for (int q = 0; q < NWARP; ++q) t += red[KT + q * KT + threadIdx.x];
            chunk[threadIdx.x] = t;
        }
    }
    __syncthreads();
    __shared__ int s_fin;
    if (threadIdx.x < KT) c.hsum[(int64_t)(it.hbase + it.hchunk) * KT + threadIdx.x] = chunk[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        s_fin = (atomicAdd(c.hcount + it.hrow, 1) == it.nchunk - 1);
    __syncthreads();
    if (s_fin) {
        __threadfence();
        if (threadIdx.x < KT) {
            double t = 0.0;
            for (int q = 0; q < it.nchunk; ++q)
                t += __ldcg(c.hsum + (int64_t)(it.hbase + q) * KT + threadIdx.x);
            s_acc[threadIdx.x] = (TA)t;
        }
        if (threadIdx.x == 0) atomicExch(c.hcount + it.hrow, 0);
        __syncthreads();
        typename Epi::template D<TV> hdot[ND > 0 ? ND : 1][VEC];
#pragma unroll
        for (int d = 0; d < (ND > 0 ? ND : 1); ++d)
#pragma unroll
            for (int v = 0; v < VEC; ++v) dot_zero(hdot[d][v]);
        spmm_epilogue<LD, TV, TA, KT, Epi>(c, epi, seg, src, dst, i, i + 1, s_acc, hdot);
        if constexpr (ND > 0) {
            constexpr int CG = KT / VEC;
            if (threadIdx.x < CG) {
                const int64_t hs = c.n_sblk + it.hrow;
#pragma unroll
                for (int d = 0; d < ND; ++d)
#pragma unroll
                    for (int v = 0; v < VEC; ++v)
                        c.part[((int64_t)d * c.part_stride + hs) * KT + threadIdx.x * VEC + v] = dot_get(hdot[d][v]);
            }
            heavy_arrive<ND, KT>(c, epi.fin, seg, c.n_sblk + it.hrow, red);
        }
    }
    __syncthreads();

}

// Whole-warp part of the single-RHS SpMV: one long row (kind 2) or one chunk of a
// split row (kind 1).  Kept out of line so the short-row loop keeps few registers.
template <class LD, class TV, class TW, class TA, class Epi>
__device__ __noinline__ void spmv1_long(const Ctx &c, const Epi &epi_in, int seg, const TV *__restrict__ src,
                                        TV *__restrict__ dst, const SpItem &it,
                                        typename Epi::template D<TV> (&dot)[Epi::ND > 0 ? Epi::ND : 1][1]) {
    constexpr int ND = Epi::ND;
    Epi epi = epi_in;
    epi.prep(c, seg, 0);
    const int lane = threadIdx.x & 31;
    const TW *__restrict__ w = reinterpret_cast<const TW *>(c.w);
    const TA *__restrict__ deg = deg_of<TA>(c);
        const int64_t i = it.r0;
        TA s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        for (int64_t qb = (it.e0 & ~(int64_t)3) + 4 * lane; qb < it.e1; qb += 128) {
            const int4 cq = __ldcs(reinterpret_cast<const int4 *>(c.colidx + qb));
            TW wq[4];
            ld4_stream(w + qb, wq);
            const bool in0 = qb >= it.e0 && qb < it.e1, in1 = qb + 1 >= it.e0 && qb + 1 < it.e1;
            const bool in2 = qb + 2 >= it.e0 && qb + 2 < it.e1, in3 = qb + 3 >= it.e0 && qb + 3 < it.e1;
            if (in0) s0 += (TA)wq[0] * (TA)LD::ld(src + cq.x);
            if (in1) s1 += (TA)wq[1] * (TA)LD::ld(src + cq.y);
            if (in2) s2 += (TA)wq[2] * (TA)LD::ld(src + cq.z);
            if (in3) s3 += (TA)wq[3] * (TA)LD::ld(src + cq.w);
        }
        TA sum = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(NVD_FULLMASK, sum, off);
        if (it.kind == 2) {
            if (lane == 0) {
                TV own[1] = {LD::ld(src + i)};
                const TA acc[1] = {sum};
                epi.template elem<TV, TA, 1>(c, i, 0, 1, own, acc, __ldg(deg + i), dst, dot);
            }
        } else {
            int fin = 0;
            if (lane == 0) {
                c.hsum[it.hbase + it.hchunk] = (double)sum;
                __threadfence();
                fin = (atomicAdd(c.hcount + it.hrow, 1) == it.nchunk - 1);
            }
            fin = __shfl_sync(NVD_FULLMASK, fin, 0);
            if (fin && lane == 0) {
                __threadfence();
                double t = 0.0;
                for (int q = 0; q < it.nchunk; ++q) t += __ldcg(c.hsum + it.hbase + q);
                atomicExch(c.hcount + it.hrow, 0);
                TV own[1] = {LD::ld(src + i)};
                const TA acc[1] = {(TA)t};
                typename Epi::template D<TV> hdot[ND > 0 ? ND : 1][1];
#pragma unroll
                for (int d = 0; d < (ND > 0 ? ND : 1); ++d) dot_zero(hdot[d][0]);
                epi.template elem<TV, TA, 1>(c, i, 0, 1, own, acc, __ldg(deg + i), dst, hdot);
                if constexpr (ND > 0) {
#pragma unroll
                    for (int d = 0; d < ND; ++d)
                        c.part[(int64_t)d * c.part_stride + c.n_sblk + it.hrow] = dot_get(hdot[d][0]);
                }
            }
        }

}

// Single right-hand side (KT = 1) SpMV block.  Warps never wait for each other
// until the block's final reduction, so many independent load chains are in
// flight per SM.
//   light block (pad 0): slices of the sliced light-row layout, one row per lane;
//   heavy block (pad 1): up to 8 sub-items, one per warp: a long row (kind 2) or a
//           chunk of a split row (kind 1, see spmv1_long).
template <class LD, class TV, class TW, class TA, class Epi>
__device__ void spmv1_block(const Ctx &c, const Epi &epi, const TV *__restrict__ src, TV *__restrict__ dst,
                            int64_t b, char *smem) {
    constexpr int ND = Epi::ND;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *red = reinterpret_cast<double *>(smem);
    double *tot = red + red_doubles(1);
    const TA *__restrict__ deg = deg_of<TA>(c);
    const Block blk = c.sblk[b];
    const int seg = blk.seg;
    typename Epi::template D<TV> dot[ND > 0 ? ND : 1][1];
#pragma unroll
    for (int d = 0; d < (ND > 0 ? ND : 1); ++d) dot_zero(dot[d][0]);
    const bool live = !Epi::NEEDS_LIVE || seg_live<1>(c, seg);
    if (live) {
        if (blk.pad == 0) {
            // light slices [i0, i1): a warp takes the next slice of 32 rows, one
            // row per lane; entry j of the 32 rows is one coalesced load of columns
            // and of weights, the gathers of SPMV1_UNROLL entries are in flight
            // before their products, and each lane adds its row's products in entry
            // order into one accumulator (no cross-lane sum).  The row sums go to
            // shared memory by row (rows r0 .. r0 + nr - 1; a bit marks each light
            // row of the span) and the row epilogue then runs in row order, so its
            // loads and stores of the own row are coalesced.
            TA *s_acc = reinterpret_cast<TA *>(red);   // [nr]; the reduction scratch is free until the end
            unsigned *s_has = reinterpret_cast<unsigned *>(tot + SpCfg<TV, TA, 1>::ND_MAX);
            int *s_next = reinterpret_cast<int *>(s_has + sp_span_max() / 32);
            const int32_t r0 = blk.r0, nr = blk.nr;
            for (int t = threadIdx.x; t < (nr + 31) / 32; t += NT) s_has[t] = 0u;
            if (threadIdx.x == 0) *s_next = 0;
            __syncthreads();
            const TW *__restrict__ slw = reinterpret_cast<const TW *>(c.sl_w);
            const int64_t ns = blk.i1 - blk.i0;
            for (;;) {
                // the next slice of the block, longest first, to whichever warp is
                // free (the warps finish together however the lengths fall)
                int q = 0;
                if (lane == 0) q = atomicAdd(s_next, 1);
                q = __shfl_sync(NVD_FULLMASK, q, 0);
                if (q >= ns) break;
                const int64_t sl = blk.i0 + q;
                const int64_t base = __ldg(c.sl_base + sl);
                const int L = (int)((__ldg(c.sl_base + sl + 1) - base) >> 5);
                const int32_t i = __ldg(c.sl_row + sl * 32 + lane);
                const int32_t *__restrict__ cp = c.sl_col + base + lane;
                const TW *__restrict__ wp = slw + base + lane;
                // L is the same for the whole warp, so the bounds tests below are
                // uniform branches (the last step issues only its valid entries,
                // all of them in flight together)
                constexpr int U = SPMV1_UNROLL;
                TA acc = 0;
                int cu[U] = {};
                TW wu[U] = {};
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (u < L) {
                        cu[u] = __ldcs(cp + u * 32);
                        wu[u] = __ldcs(wp + u * 32);
                    }
                for (int j = 0; j < L; j += U) {
                    // the next step's columns and weights are loaded while this
                    // step's gathers are in flight
                    int cn[U] = {};
                    TW wn[U] = {};
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (j + U + u < L) {
                            cn[u] = __ldcs(cp + (j + U + u) * 32);
                            wn[u] = __ldcs(wp + (j + U + u) * 32);
                        }
                    TV pv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (j + u < L) pv[u] = LD::ld(src + cu[u]);
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (j + u < L) acc += (TA)wu[u] * (TA)pv[u];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        cu[u] = cn[u];
                        wu[u] = wn[u];
                    }
                }
                if (i >= 0) {
                    const int t = i - r0;
                    s_acc[t] = acc;
                    atomicOr(s_has + (t >> 5), 1u << (t & 31));
                }
            }
            __syncthreads();
            Epi e = epi;
            e.prep(c, seg, 0);
            for (int t = threadIdx.x; t < nr; t += NT) {
                if (!((s_has[t >> 5] >> (t & 31)) & 1u)) continue;   // a heavy row inside the span
                const int64_t i = (int64_t)r0 + t;
                const TV own[1] = {LD::ld(src + i)};
                const TA av[1] = {s_acc[t]};
                e.template elem<TV, TA, 1>(c, i, 0, 1, own, av, __ldg(deg + i), dst, dot);
            }
            __syncthreads();   // s_acc aliases the reduction scratch
        } else {
            // heavy sub-items (long rows, chunks of split rows), one warp each
            for (int64_t si = blk.i0 + warp; si < blk.i1; si += NWARP) {
                const SpItem it = c.items[si];
                spmv1_long<LD, TV, TW, TA, Epi>(c, epi, seg, src, dst, it, dot);
            }
        }
    }
    if constexpr (ND > 0) {
        double dd[ND][1];
        dot_to_double(dot, dd);
        block_reduce_cols<ND, 1, 1>(dd, red, tot);
        const int64_t s0 = c.seg_sblk_off[seg];
        const int32_t cnt = c.seg_sblk_off[seg + 1] - (int32_t)s0;
        const int64_t h0 = c.n_sblk + c.seg_heavy_off[seg];
        const int32_t hcnt = c.seg_heavy_off[seg + 1] - c.seg_heavy_off[seg];
        seg_arrive<ND, 1>(c, epi.fin, seg, b, tot, s0, cnt, h0, hcnt, red);
    }
}

// A warp's fixed run of light slices [s_lo, s_hi) of a multi-column SpMM (tiles
// where U steps of G rows span at most 16 entries: 128-byte FP32 rows and the FP64
// tiles; with 8 rows per slice the per-step loop of spmm_block measured 1.6% faster,
// with 4 this form 2% faster).  Products are added in entry
// order exactly as in the per-step loop; what changes is how the slices' columns
// and weights reach the lanes: the run's entries are one contiguous stream, read
// 32 at a time by the whole warp (one coalesced load each of columns and weights)
// into a window of two such chunks, and handed to the lanes by shuffles; the
// chunk after the window and the next slice's bounds and row id are loaded while
// the current gathers are in flight.  The chain per U steps is then one gather
// latency instead of a column load followed by a gather.
template <class LD, class TV, class TW, class TA, int KT, class Epi>
__device__ __forceinline__ void spmm_light_run(const Ctx &c, Epi &e, const TV *__restrict__ src,
                                               TV *__restrict__ dst, int64_t s_lo, int64_t s_hi,
                                               typename Epi::template D<TV> (&dot)[Epi::ND > 0 ? Epi::ND : 1]
                                                                                  [SpCfg<TV, TA, KT>::VEC]) {
    typedef SpCfg<TV, TA, KT> C;
    constexpr int VEC = C::VEC, LPR = C::LPR, G = C::G;
    constexpr int U = sizeof(TV) == 8 ? SPMM_UNROLL_F64 : SPMM_UNROLL_F32;
    static_assert(U * G <= 32 && 32 % G == 0, "U steps of a slice fit one 32-entry chunk");
    if (s_lo >= s_hi) return;
    const int lane = threadIdx.x & 31;
    const int gid = lane / LPR, col0 = (lane % LPR) * VEC;
    const TA *__restrict__ deg = deg_of<TA>(c);
    // entries of the run relative to its first (a run holds far fewer than 2^31)
    const int64_t e_lo = __ldg(c.sl_base + s_lo);
    const int32_t *__restrict__ slc = c.sl_col + e_lo;
    const TW *__restrict__ slw = reinterpret_cast<const TW *>(c.sl_w) + e_lo;
    const int n_e = (int)(__ldg(c.sl_base + s_hi) - e_lo);
    int base = 0;
    int nb = (int)(__ldg(c.sl_base + s_lo + 1) - e_lo);
    int32_t i = __ldg(c.sl_row + s_lo * G + gid);
    // window [wb, wb + 64): chunk (mc, mw) then chunk (nc, nw)
    int wb = 0;
    int mc = 0, nc = 0;
    TW mw = 0, nw = 0;
    if (lane < n_e) {
        mc = __ldcs(slc + lane);
        mw = __ldcs(slw + lane);
    }
    if (32 + lane < n_e) {
        nc = __ldcs(slc + 32 + lane);
        nw = __ldcs(slw + 32 + lane);
    }
    for (int64_t sl = s_lo; sl < s_hi; ++sl) {
        const int L = (nb - base) / G;
        // the next slice's end and row id, in flight during this slice
        int nb2 = nb;
        int32_t i2 = -1;
        if (sl + 1 < s_hi) {
            nb2 = (int)(__ldg(c.sl_base + sl + 2) - e_lo);
            i2 = __ldg(c.sl_row + (sl + 1) * G + gid);
        }
        TV own[VEC];
        TA dg = 0;
        if (i >= 0) {
            ldv<LD, TV, VEC>(src + (int64_t)i * KT + col0, own);
            dg = __ldg(deg + i);
        }
        TA acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0;
        for (int j = 0; j < L; j += U) {
            const int pos = base + j * G;
            if (pos >= wb + 32) {   // slide the window by one chunk
                mc = nc;
                mw = nw;
                wb += 32;
                nc = 0;
                nw = 0;
                if (wb + 32 + lane < n_e) {
                    nc = __ldcs(slc + wb + 32 + lane);
                    nw = __ldcs(slw + wb + 32 + lane);
                }
            }
            const int ob = pos - wb;   // < 32, a multiple of G
            int cu[U];
            TA wu[U];
            TV pv[U][VEC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                // step j + u is entries ob + u*G .. + G - 1 of the window: all in the
                // first chunk or all in the second (G divides 32), the same for every lane
                const bool lo = ob + u * G < 32;
                const int sl_lane = (ob + u * G + gid) & 31;
                cu[u] = __shfl_sync(NVD_FULLMASK, lo ? mc : nc, sl_lane);
                wu[u] = (TA)__shfl_sync(NVD_FULLMASK, lo ? mw : nw, sl_lane);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j + u < L) ldv<LD, TV, VEC>(src + (int64_t)cu[u] * KT + col0, pv[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j + u < L)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] += wu[u] * (TA)pv[u][v];
        }
        if (i >= 0) e.template elem<TV, TA, VEC>(c, i, col0, KT, own, acc, dg, dst, dot);
        base = nb;
        nb = nb2;
        i = i2;
    }
}

// One SpMV/SpMM block b: its slices or heavy sub-items, then the segment arrival.
template <class LD, class TV, class TW, class TA, int KT, class Epi>
__device__ void spmm_block(const Ctx &c, const Epi &epi, const TV *__restrict__ src, TV *__restrict__ dst,
                           int64_t b, char *smem) {
    if constexpr (KT == 1) {
        spmv1_block<LD, TV, TW, TA, Epi>(c, epi, src, dst, b, smem);
        return;
    }
    typedef SpCfg<TV, TA, KT> C;
    constexpr int VEC = C::VEC, LPR = C::LPR, G = C::G, ND = Epi::ND;
    TA *s_acc = reinterpret_cast<TA *>(smem);
    double *red = reinterpret_cast<double *>(smem + C::ACC);
    double *tot = red + C::RED;
    const int lane = threadIdx.x & 31;
    const Block blk = c.sblk[b];
    const int seg = blk.seg;

    typename Epi::template D<TV> dot[ND > 0 ? ND : 1][VEC];
#pragma unroll
    for (int d = 0; d < (ND > 0 ? ND : 1); ++d)
#pragma unroll
        for (int v = 0; v < VEC; ++v) dot_zero(dot[d][v]);

    const bool live = !Epi::NEEDS_LIVE || seg_live<KT>(c, seg);
    if (live) {
        if (blk.pad == 0) {
            // light slices: warp w takes its fixed run of the block's slices (cut
            // where the running entry count is closest to an equal share, as the TMA
            // path does), so every thread adds the same rows in the same order on
            // every run; a slice has G rows, the LPR lanes of group `gid` own its row
            // gid, lane `sub` of the group columns col0..col0+VEC-1, so a row needs
            // no cross-lane sum; entry j of the G rows is one load of columns and of
            // weights, SPMM_UNROLL_* gathered neighbour rows are in flight, products
            // are added in entry order
            const int gid = lane / LPR, col0 = (lane % LPR) * VEC;
            const TA *__restrict__ deg = deg_of<TA>(c);
            const TW *__restrict__ slw = reinterpret_cast<const TW *>(c.sl_w);
            Epi e = epi;
            e.prep(c, seg, col0);
            const int32_t *split = c.sl_wsplit + b * (NWARP + 1);
            const int warp = threadIdx.x >> 5;
            const int64_t s_hi = blk.i0 + __ldg(split + warp + 1);
            constexpr int U = sizeof(TV) == 8 ? SPMM_UNROLL_F64 : SPMM_UNROLL_F32;
            if constexpr (U * G <= 16) {
                spmm_light_run<LD, TV, TW, TA, KT, Epi>(c, e, src, dst, blk.i0 + __ldg(split + warp), s_hi, dot);
            } else
            for (int64_t sl = blk.i0 + __ldg(split + warp); sl < s_hi; ++sl) {
                const int64_t base = __ldg(c.sl_base + sl);
                const int L = (int)((__ldg(c.sl_base + sl + 1) - base) / G);
                const int32_t i = __ldg(c.sl_row + sl * G + gid);
                TV own[VEC];
                TA dg = 0;
                if (i >= 0) {
                    ldv<LD, TV, VEC>(src + (int64_t)i * KT + col0, own);
                    dg = __ldg(deg + i);
                }
                const int32_t *__restrict__ cp = c.sl_col + base + gid;
                const TW *__restrict__ wp = slw + base + gid;
                TA acc[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[v] = 0;
                for (int j = 0; j < L; j += U) {   // uniform bounds tests, as for KT = 1
                    int cu[U];
                    TA wu[U];
                    TV pv[U][VEC];
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (j + u < L) {
                            cu[u] = __ldcs(cp + (j + u) * G);
                            wu[u] = (TA)__ldcs(wp + (j + u) * G);
                        }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (j + u < L) ldv<LD, TV, VEC>(src + (int64_t)cu[u] * KT + col0, pv[u]);
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (j + u < L)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[v] += wu[u] * (TA)pv[u][v];
                }
                if (i >= 0) e.template elem<TV, TA, VEC>(c, i, col0, KT, own, acc, dg, dst, dot);
            }
        } else {
            // heavy block: chunks of split rows, each taken by the whole CTA
            for (int64_t si = blk.i0; si < blk.i1; ++si) {
                const SpItem it = c.items[si];
                spmm_chunk<LD, TV, TW, TA, KT, Epi>(c, epi, seg, src, dst, it, s_acc, red);
            }
        }
    }
    if constexpr (ND > 0) {
        double dd[ND][VEC];
        dot_to_double(dot, dd);
        block_reduce_cols<ND, KT, VEC>(dd, red, tot);
        const int64_t s0 = c.seg_sblk_off[seg];
        const int32_t cnt = c.seg_sblk_off[seg + 1] - (int32_t)s0;
        const int64_t h0 = c.n_sblk + c.seg_heavy_off[seg];
        const int32_t hcnt = c.seg_heavy_off[seg + 1] - c.seg_heavy_off[seg];
        // split rows arrive by themselves only in a pass that runs them (a segment
        // whose columns have all stopped skips its rows; `live` is the same in
        // every block of the pass)
        seg_arrive<ND, KT>(c, epi.fin, seg, b, tot, s0, cnt, h0, hcnt, red, live);
    }
}

}  // namespace dev
}  // namespace nvd
