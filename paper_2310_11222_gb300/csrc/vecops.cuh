// Device code of the GE-distance solver, part 2: the streaming vector passes of
// the PCG iteration (Section 3.2): forming the projected right-hand side, the
// x/r update with the preconditioned inner products, the direction update and
// the final d^2 sums.  Each pass reads and writes [n][KT] block vectors of one
// CTA block of rows and reduces its inner products like the SpMV (block slot,
// last-arriving block of the segment finalizes).
#pragma once

#include "kernels.cuh"

namespace nvd {
namespace dev {

// ------------------------------------------------------------------ vector passes

// Does a segment need this pass?  NEEDS_LIVE: while a column iterates;
// LIVE_ON_STEP (optional member): while a column has a step to take (alpha != 0);
// otherwise always.
template <class Op, class = void> struct LiveOnStep { static constexpr bool value = false; };
template <class Op> struct LiveOnStep<Op, decltype((void)Op::LIVE_ON_STEP)> {
    static constexpr bool value = Op::LIVE_ON_STEP;
};
template <int KT>
__device__ __forceinline__ bool seg_stepped(const Ctx &c, int seg) {
    bool a = false;
#pragma unroll
    for (int j = 0; j < KT; ++j) a = a || __ldcg(c.alpha + (int64_t)seg * KT + j) != 0.0;
    return a;
}
template <int KT, class Op>
__device__ __forceinline__ bool op_live(const Ctx &c, int seg) {
    if constexpr (LiveOnStep<Op>::value) return seg_stepped<KT>(c, seg);
    else if constexpr (Op::NEEDS_LIVE) return seg_live<KT>(c, seg);
    else return true;
}

// Generic streaming pass over rows [i0, i1) of one segment.  Op provides ND,
// NEEDS_LIVE (see op_live), a register type R, setup(c, seg, col0), load(c, i,
// col0, R&) and apply(c, i, col0, R&, dot) with per-thread partial sums of type
// Op::D (see DotOf).  Each thread handles U lane-vectors per trip with all U loads
// issued before the first use.
template <class TV, int KT, class Op, int U = 4>
__device__ void vec_block(const Ctx &c, Op op, int64_t b, char *smem) {
    constexpr int VEC = VecCfg<TV, KT>::VEC, CG = KT / VEC, ND = Op::ND;
    double *red = reinterpret_cast<double *>(smem);
    double *tot = red + red_doubles(KT);
    const Block blk = c.vblk[b];
    const int seg = blk.seg;
    const int col0 = (int)(threadIdx.x % CG) * VEC;
    typename Op::D dot[ND > 0 ? ND : 1][VEC];
#pragma unroll
    for (int d = 0; d < (ND > 0 ? ND : 1); ++d)
#pragma unroll
        for (int v = 0; v < VEC; ++v) dot_zero(dot[d][v]);
    if (op_live<KT, Op>(c, seg)) {
        op.setup(c, seg, col0);
        const int64_t t1 = blk.i1 * CG;
        for (int64_t t = blk.i0 * CG + threadIdx.x; t < t1; t += (int64_t)NT * U) {
            typename Op::R regs[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t tu = t + (int64_t)u * NT;
                if (tu < t1) op.load(c, tu / CG, col0, regs[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t tu = t + (int64_t)u * NT;
                if (tu < t1) op.apply(c, tu / CG, col0, regs[u], dot);
            }
        }
    }
    if constexpr (ND > 0) {
        double dd[ND][VEC];
        dot_to_double(dot, dd);
        block_reduce_cols<ND, KT, VEC>(dd, red, tot);
        const int64_t s0 = c.seg_vblk_off[seg];
        const int32_t cnt = c.seg_vblk_off[seg + 1] - (int32_t)s0;
        seg_arrive<ND, KT>(c, op.fin, seg, b, tot, s0, cnt, 0, 0, red);
    }
}

// delta = x - y for this tile (user layout [k][n], optional node permutation) into
// [n][KT] FP64; per-segment sums for the projection.
template <class TX, int KT>
struct OpFormDelta {
    static constexpr int ND = 1, VEC = VecCfg<double, KT>::VEC;
    static constexpr bool NEEDS_LIVE = false;
    struct R { double d[VEC]; };
    typedef double D;
    double *delta;
    FinMean fin;
    const TX *X, *Y;
    int64_t base, ld;
    int kc, idx;
    __device__ void setup(const Ctx &c, int seg, int) {
        const Owner &o = owner_of(c, seg);
        X = reinterpret_cast<const TX *>(o.x);
        Y = reinterpret_cast<const TX *>(o.y);
        base = o.base;
        ld = o.ld;
        kc = o.kc;
        idx = o.idx & 1;
    }
    __device__ __forceinline__ void load(const Ctx &c, int64_t i, int col0, R &r) const {
        const int64_t u = (c.perm ? (int64_t)__ldg(c.perm + i) : i) - base;
        if (idx) {
            // node-id pairs: column j is the indicator difference e_x[j] - e_y[j]
            const int32_t *Xi = reinterpret_cast<const int32_t *>(X), *Yi = reinterpret_cast<const int32_t *>(Y);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int j = col0 + v;
                r.d[v] = j < kc ? (double)(u == (int64_t)__ldg(Xi + j)) - (double)(u == (int64_t)__ldg(Yi + j)) : 0.0;
            }
            return;
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int j = col0 + v;
            r.d[v] = j < kc ? (double)__ldg(X + (int64_t)j * ld + u) - (double)__ldg(Y + (int64_t)j * ld + u) : 0.0;
        }
    }
    __device__ __forceinline__ void apply(const Ctx &, int64_t i, int col0, R &r, double (&dot)[1][VEC]) const {
#pragma unroll
        for (int v = 0; v < VEC; ++v) dot[0][v] += r.d[v];
        stv(delta + i * KT + col0, r.d);
    }
};

// PCG start from x = 0: r = P src (src minus its segment mean, optionally written
// back), u = D^-1 r, p = u; r^T u and |r|^2.
template <class TV, int KT, class LD = LdPlain>
struct OpInit {
    static constexpr int ND = 2, VEC = VecCfg<TV, KT>::VEC;
    static constexpr bool NEEDS_LIVE = false;
    struct R { double s[VEC]; TV di; };
    typedef typename DotOf<TV>::type D;
    const double *src;
    double *writeback;
    TV *x, *r, *p;
    bool zero_x = true;   // false: keep x (warm start)
    FinInit fin;
    double mu[VEC];
    __device__ void setup(const Ctx &c, int seg, int col0) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) mu[v] = __ldcg(c.mean + (int64_t)seg * KT + col0 + v);
    }
    __device__ __forceinline__ void load(const Ctx &c, int64_t i, int col0, R &q) const {
        ldv<LD, double, VEC>(src + i * KT + col0, q.s);
        q.di = __ldg(dinv_of<TV>(c) + i);
    }
    __device__ __forceinline__ void apply(const Ctx &, int64_t i, int col0, R &q, D (&dot)[2][VEC]) const {
        const int64_t o = i * KT + col0;
        TV rv[VEC], uv[VEC], zv[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            q.s[v] -= mu[v];
            rv[v] = (TV)q.s[v];
            uv[v] = q.di * rv[v];
            zv[v] = (TV)0;
            dot_fma(dot[0][v], rv[v], uv[v]);
            dot_fma(dot[1][v], rv[v], rv[v]);
        }
        if (writeback) stv(writeback + o, q.s);
        stv(r + o, rv);
        stv(p + o, uv);
        if (zero_x) stv(x + o, zv);
    }
};

// x = z0, a saved solution in the user's layout ([kc][ld], e.g. z_out of an
// earlier call) cast to TV, for a warm start; padding columns (j >= kc) get 0.
template <class TV, class TX, int KT, class LD = LdPlain>
struct OpLoadX {
    static constexpr int ND = 0, VEC = VecCfg<TV, KT>::VEC;
    static constexpr bool NEEDS_LIVE = false;
    struct R { double s[VEC]; };
    typedef double D;
    const TX *Z0;
    TV *x;
    FinNone fin;
    int64_t base, ld;
    int kc;
    __device__ void setup(const Ctx &c, int seg, int) {
        const Owner &o = owner_of(c, seg);
        base = o.base;
        ld = o.ld;
        kc = o.kc;
    }
    __device__ __forceinline__ void load(const Ctx &c, int64_t i, int col0, R &g) const {
        const int64_t u = (c.perm ? (int64_t)__ldg(c.perm + i) : i) - base;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int j = col0 + v;
            g.s[v] = j < kc ? (double)__ldg(Z0 + (int64_t)j * ld + u) : 0.0;
        }
    }
    __device__ __forceinline__ void apply(const Ctx &, int64_t i, int col0, R &g, double (&)[1][VEC]) const {
        TV xv[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) xv[v] = (TV)g.s[v];
        stv(x + i * KT + col0, xv);
    }
};

// x += alpha p, r -= alpha q, u = D^-1 r (stored when u is set: the next SpMV
// runs on it); r^T u and |r|^2.
template <class TV, int KT, class LD = LdPlain>
struct OpUpdate {
    static constexpr int ND = 2, VEC = VecCfg<TV, KT>::VEC;
    static constexpr bool NEEDS_LIVE = true;
    struct R { TV x[VEC], r[VEC], p[VEC], q[VEC]; TV di; };
    typedef typename DotOf<TV>::type D;
    TV *x, *r;
    const TV *p, *q;
    TV *u = nullptr;
    FinBeta fin;
    TV al[VEC];
    __device__ void setup(const Ctx &c, int seg, int col0) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) al[v] = (TV)__ldcg(c.alpha + (int64_t)seg * KT + col0 + v);
    }
    __device__ __forceinline__ void load(const Ctx &c, int64_t i, int col0, R &g) const {
        const int64_t o = i * KT + col0;
        ldv<LD, TV, VEC>(x + o, g.x);
        ldv<LD, TV, VEC>(r + o, g.r);
        ldv<LD, TV, VEC>(p + o, g.p);
        ldv<LD, TV, VEC>(q + o, g.q);
        g.di = __ldg(dinv_of<TV>(c) + i);
    }
    __device__ __forceinline__ void apply(const Ctx &, int64_t i, int col0, R &g, D (&dot)[2][VEC]) const {
        const int64_t o = i * KT + col0;
        TV uv[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            g.x[v] += al[v] * g.p[v];
            g.r[v] -= al[v] * g.q[v];
            uv[v] = g.di * g.r[v];
            dot_fma(dot[0][v], g.r[v], uv[v]);
            dot_fma(dot[1][v], g.r[v], g.r[v]);
        }
        stv(x + o, g.x);
        stv(r + o, g.r);
        if (u) stv(u + o, uv);
    }
};

// The three-kernel iteration moves as few [n][KT] vectors as it can: after the
// SpMV (q = L p, p^T q) the residual pass only reads r, q and D^-1 and writes r;
// the direction pass then takes the x step with the p it reads anyway and forms
// the next direction from r and D^-1 (no stored D^-1 r):
//     residual pass   r -= alpha q;  r^T D^-1 r, |r|^2          (3 vectors)
//     direction pass  x += alpha p;  p = D^-1 r + beta p        (5 vectors)
// against 7 + 3 when the update pass also moves x and stores u = D^-1 r.

// r -= alpha q; r^T D^-1 r and |r|^2 for beta and the convergence test.
template <class TV, int KT, class LD = LdPlain>
struct OpResid {
    static constexpr int ND = 2, VEC = VecCfg<TV, KT>::VEC;
    static constexpr bool NEEDS_LIVE = true;
    struct R { TV r[VEC], q[VEC]; TV di; };
    typedef typename DotOf<TV>::type D;
    TV *r;
    const TV *q;
    FinBeta fin;
    TV al[VEC];
    __device__ void setup(const Ctx &c, int seg, int col0) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) al[v] = (TV)__ldcg(c.alpha + (int64_t)seg * KT + col0 + v);
    }
    __device__ __forceinline__ void load(const Ctx &c, int64_t i, int col0, R &g) const {
        const int64_t o = i * KT + col0;
        ldv<LD, TV, VEC>(r + o, g.r);
        ldv<LD, TV, VEC>(q + o, g.q);
        g.di = __ldg(dinv_of<TV>(c) + i);
    }
    __device__ __forceinline__ void apply(const Ctx &, int64_t i, int col0, R &g, D (&dot)[2][VEC]) const {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            g.r[v] -= al[v] * g.q[v];
            const TV uv = g.di * g.r[v];
            dot_fma(dot[0][v], g.r[v], uv);
            dot_fma(dot[1][v], g.r[v], g.r[v]);
        }
        stv(r + i * KT + col0, g.r);
    }
};

// x += alpha p (the step whose alpha the last SpMV set), then p = D^-1 r + beta p
// on the columns still iterating.  A segment runs this pass while any of its
// columns has a non-zero alpha -- also when its last column converged in the
// residual pass just before, whose x step is still due; alpha is 0 for columns
// that had stopped before the SpMV, so their x and p stay as they are.
template <class TV, int KT, class LD = LdPlain>
struct OpStepDir {
    static constexpr int ND = 0, VEC = VecCfg<TV, KT>::VEC;
    static constexpr bool NEEDS_LIVE = false;
    static constexpr bool LIVE_ON_STEP = true;
    struct R { TV x[VEC], r[VEC], p[VEC]; TV di; };
    typedef double D;
    TV *x;
    const TV *r;
    TV *p;
    FinNone fin;
    TV al[VEC], be[VEC];
    bool act[VEC];
    __device__ void setup(const Ctx &c, int seg, int col0) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int64_t i = (int64_t)seg * KT + col0 + v;
            al[v] = (TV)__ldcg(c.alpha + i);
            be[v] = (TV)__ldcg(c.beta + i);
            act[v] = __ldcg(c.active + i) != 0;
        }
    }
    __device__ __forceinline__ void load(const Ctx &c, int64_t i, int col0, R &g) const {
        const int64_t o = i * KT + col0;
        ldv<LD, TV, VEC>(x + o, g.x);
        ldv<LD, TV, VEC>(r + o, g.r);
        ldv<LD, TV, VEC>(p + o, g.p);
        g.di = __ldg(dinv_of<TV>(c) + i);
    }
    __device__ __forceinline__ void apply(const Ctx &, int64_t i, int col0, R &g, double (&)[1][VEC]) const {
        const int64_t o = i * KT + col0;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            g.x[v] += al[v] * g.p[v];
            g.p[v] = act[v] ? g.di * g.r[v] + be[v] * g.p[v] : g.p[v];
        }
        stv(x + o, g.x);
        stv(p + o, g.p);
    }
};

// sum of x and delta^T x per segment (end of solve).
template <class TV, int KT, class LD = LdPlain>
struct OpFinal {
    static constexpr int ND = 2, VEC = VecCfg<TV, KT>::VEC;
    static constexpr bool NEEDS_LIVE = false;
    struct R { TV x[VEC]; double d[VEC]; };
    typedef double D;
    const TV *x;
    const double *delta;
    FinFinal fin;
    __device__ void setup(const Ctx &, int, int) {}
    __device__ __forceinline__ void load(const Ctx &, int64_t i, int col0, R &g) const {
        const int64_t o = i * KT + col0;
        ldv<LD, TV, VEC>(x + o, g.x);
        ldv<LD, double, VEC>(delta + o, g.d);
    }
    __device__ __forceinline__ void apply(const Ctx &, int64_t, int, R &g, double (&dot)[2][VEC]) const {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            dot[0][v] += (double)g.x[v];
            dot[1][v] += g.d[v] * (double)g.x[v];
        }
    }
};

// z_out = src - mean_seg(src) in the user layout [k][n] (optionally permuted).
template <class TS, class TZ, int KT, class LD = LdPlain>
struct OpZout {
    static constexpr int ND = 0, VEC = VecCfg<TS, KT>::VEC;
    static constexpr bool NEEDS_LIVE = false;
    struct R { TS s[VEC]; };
    typedef double D;
    const TS *src;
    const double *meanv;
    FinNone fin;
    TZ *Z;
    int64_t base, ld;
    int kc;
    double mu[VEC];
    __device__ void setup(const Ctx &c, int seg, int col0) {
        const Owner &o = owner_of(c, seg);
        Z = reinterpret_cast<TZ *>(o.z);
        base = o.base;
        ld = o.ld;
        kc = o.kc;
#pragma unroll
        for (int v = 0; v < VEC; ++v) mu[v] = __ldcg(meanv + (int64_t)seg * KT + col0 + v);
    }
    __device__ __forceinline__ void load(const Ctx &, int64_t i, int col0, R &g) const {
        ldv<LD, TS, VEC>(src + i * KT + col0, g.s);
    }
    __device__ __forceinline__ void apply(const Ctx &c, int64_t i, int col0, R &g, double (&)[1][VEC]) const {
        if (!Z) return;
        const int64_t u = (c.perm ? (int64_t)__ldg(c.perm + i) : i) - base;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int j = col0 + v;
            if (j < kc) Z[(int64_t)j * ld + u] = (TZ)((double)g.s[v] - mu[v]);
        }
    }
};

// z64 += x (FP32 correction of one refinement step, accumulated in FP64).
template <class TV, int KT, class LD = LdPlain>
struct OpAccum {
    static constexpr int ND = 0, VEC = VecCfg<TV, KT>::VEC;
    static constexpr bool NEEDS_LIVE = false;
    struct R { TV x[VEC]; double z[VEC]; };
    typedef double D;
    const TV *x;
    double *z;
    FinNone fin;
    __device__ void setup(const Ctx &, int, int) {}
    __device__ __forceinline__ void load(const Ctx &, int64_t i, int col0, R &g) const {
        const int64_t o = i * KT + col0;
        ldv<LD, TV, VEC>(x + o, g.x);
        ldv<LD, double, VEC>(z + o, g.z);
    }
    __device__ __forceinline__ void apply(const Ctx &, int64_t i, int col0, R &g, double (&)[1][VEC]) const {
#pragma unroll
        for (int v = 0; v < VEC; ++v) g.z[v] += (double)g.x[v];
        stv(z + i * KT + col0, g.z);
    }
};

}  // namespace dev
}  // namespace nvd
