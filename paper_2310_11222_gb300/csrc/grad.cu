// C ABI: nvd_ge_grad -- adjoint of d^2 = delta^T L^+ delta (no new solve).
//
// With z = L^+ delta (mean-zero per component) and upstream weights gbar_j:
//   d(d^2)/dx = 2 z,  d(d^2)/dy = -2 z                       (L^+ symmetric)
//   d(d^2)/dW_uv = -z^T (dL/dW_uv) z = -1/2 (z_u - z_v)^2    per stored entry,
// from dL^+ = -L^+ dL L^+ (the null space is fixed while weights stay positive)
// and dL/dW_uv = 1/2 (e_u - e_v)(e_u - e_v)^T for the operator built from
// W_sym = (W + W^T)/2.  The two stored entries of an undirected edge thus sum to
// -(z_u - z_v)^2, the derivative with respect to the edge weight.
//
// The weight gradient is an edge gather over the CSR: z is first laid out as
// [n][KT] tiles (one 16-byte aligned row per node) so each stored entry reads one
// contiguous row of its neighbour, like the SpMM.
#include <algorithm>
#include <cstring>

#include "graph.h"
#include "kernels.cuh"

using namespace nvd;

namespace {

// zt[i][j] = z[c0 + j][user(i)] (0 beyond k), 32 rows per CTA through shared memory.
template <class TZ, int KT>
__global__ void k_z_tile(const TZ *__restrict__ z, int64_t n, int k, int c0, const int32_t *__restrict__ perm,
                         TZ *__restrict__ zt) {
    __shared__ TZ tile[32][KT + 1];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    for (int t = threadIdx.x; t < 32 * KT; t += blockDim.x) {
        const int li = t % 32, j = t / 32;
        const int64_t i = i0 + li;
        TZ v = 0;
        if (i < n && c0 + j < k) {
            const int64_t u = perm ? (int64_t)perm[i] : i;
            v = z[(int64_t)(c0 + j) * n + u];
        }
        tile[li][j] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * KT; t += blockDim.x) {
        const int j = t % KT, li = t / KT;
        const int64_t i = i0 + li;
        if (i < n) zt[i * KT + j] = tile[li][j];
    }
}

// One warp per row u: for every stored entry e = (u, v),
//   g[e] (+)= -1/2 sum_j gbar_j (zt[u][j] - zt[v][j])^2.
template <class TZ, class TG, int KT, bool ACC>
__global__ void __launch_bounds__(256) k_grad_edges(int64_t n, const int64_t *__restrict__ rowptr,
                                                    const int32_t *__restrict__ colidx,
                                                    const TZ *__restrict__ zt, const double *__restrict__ gb,
                                                    TG *__restrict__ g) {
    constexpr int VEC = dev::VecCfg<TZ, KT>::VEC, LPR = KT / VEC, G = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int gi = lane / LPR, sub = lane % LPR, col0 = sub * VEC;
    double gbl[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) gbl[v] = gb[col0 + v];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nw) {
        const int64_t e0 = __ldg(rowptr + u), e1 = __ldg(rowptr + u + 1);
        if (e0 == e1) continue;
        TZ own[VEC];
        dev::ldv<dev::LdRO, TZ, VEC>(zt + u * KT + col0, own);
        for (int64_t eb = e0; eb < e1; eb += G) {
            const int64_t e = eb + gi;
            const bool ok = e < e1;
            double s = 0.0;
            if (ok) {
                const int32_t v = __ldcs(colidx + e);
                TZ zv[VEC];
                dev::ldv<dev::LdRO, TZ, VEC>(zt + (int64_t)v * KT + col0, zv);
#pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    const double d = (double)own[q] - (double)zv[q];
                    s += gbl[q] * d * d;
                }
            }
#pragma unroll
            for (int off = 1; off < LPR; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (ok && sub == 0) {
                const double val = -0.5 * s;
                if (ACC) g[e] = (TG)((double)g[e] + val);
                else g[e] = (TG)val;
            }
        }
    }
}

// grad_w[e] = g_int[uent[e]] (0 for dropped self-loops), converted to TW.
template <class TW>
__global__ void k_grad_scatter(const double *__restrict__ gint, const int64_t *__restrict__ uent,
                               int64_t nnz_user, TW *__restrict__ gw) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_user;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = uent ? uent[e] : e;
        gw[e] = m >= 0 ? (TW)gint[m] : (TW)0;
    }
}

// grad_x = 2 gbar_j z, grad_y = -grad_x.  Column j of [k][n] on blockIdx.y (and its
// grid stride): the factor 2 gbar_j is one value per column, so an element costs one
// multiply and no index division (the FP64 unit, 1/64 of the FP32 rate, had bounded
// the per-element form).
template <class TZ>
__global__ void k_grad_xy(const TZ *__restrict__ z, int64_t n, int k, const double *__restrict__ gbar,
                          TZ *gx, TZ *gy) {
    for (int j = blockIdx.y; j < k; j += gridDim.y) {
        const double cj = 2.0 * gbar[j];
        const TZ *zj = z + (int64_t)j * n;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const double v = cj * (double)zj[i];
            if (gx) gx[(int64_t)j * n + i] = (TZ)v;
            if (gy) gy[(int64_t)j * n + i] = (TZ)(-v);
        }
    }
}

int grid_cap(int64_t work, int num_sms) {
    int64_t b = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms * 32));
}

template <class TZ, class TW, int KT>
int grad_w_impl(nvd_graph_s *g, int k, const TZ *z, const double *gbar, TW *grad_w, cudaStream_t s) {
    int st = NVD_OK;
    const int ntile = (k + KT - 1) / KT;
    double *gbp = (double *)g->wsp("grad_gbar", (size_t)ntile * KT * 8, &st);
    TZ *zt = (TZ *)g->wsp("grad_zt", (size_t)g->n * KT * sizeof(TZ), &st);
    if (st) return st;
    NVD_TRY_CUDA(cudaMemsetAsync(gbp, 0, (size_t)ntile * KT * 8, s));
    NVD_TRY_CUDA(cudaMemcpyAsync(gbp, gbar, (size_t)k * 8, cudaMemcpyDeviceToDevice, s));
    const bool direct = (ntile == 1) && !g->uent.p;
    double *gint = nullptr;
    if (!direct) {
        gint = (double *)g->wsp("grad_gint", (size_t)std::max<int64_t>(g->nnz, 1) * 8, &st);
        if (st) return st;
    }
    const int zgrid = (int)((g->n + 31) / 32);
    const int egrid = grid_cap(g->n * 32, g->num_sms);
    for (int t = 0; t < ntile; ++t) {
        k_z_tile<TZ, KT><<<zgrid, 256, 0, s>>>(z, g->n, k, t * KT, g->perm.as<int32_t>(), zt);
        if (direct) {
            k_grad_edges<TZ, TW, KT, false><<<egrid, 256, 0, s>>>(g->n, g->rowptr.as<int64_t>(),
                                                                   g->colidx.as<int32_t>(), zt, gbp, grad_w);
        } else if (t == 0) {
            k_grad_edges<TZ, double, KT, false><<<egrid, 256, 0, s>>>(
                g->n, g->rowptr.as<int64_t>(), g->colidx.as<int32_t>(), zt, gbp + t * KT, gint);
        } else {
            k_grad_edges<TZ, double, KT, true><<<egrid, 256, 0, s>>>(
                g->n, g->rowptr.as<int64_t>(), g->colidx.as<int32_t>(), zt, gbp + t * KT, gint);
        }
        NVD_TRY_CUDA(cudaGetLastError());
    }
    if (!direct) {
        k_grad_scatter<TW><<<grid_cap(g->nnz_user, g->num_sms), 256, 0, s>>>(gint, g->uent.as<int64_t>(),
                                                                             g->nnz_user, grad_w);
        NVD_TRY_CUDA(cudaGetLastError());
    }
    return NVD_OK;
}

template <class TZ, class TW>
int grad_w_kt(nvd_graph_s *g, int k, const TZ *z, const double *gbar, TW *grad_w, cudaStream_t s) {
    if (k <= 1) return grad_w_impl<TZ, TW, 1>(g, k, z, gbar, grad_w, s);
    if (k <= 4) return grad_w_impl<TZ, TW, 4>(g, k, z, gbar, grad_w, s);
    if (k <= 8) return grad_w_impl<TZ, TW, 8>(g, k, z, gbar, grad_w, s);
    if (k <= 16) return grad_w_impl<TZ, TW, 16>(g, k, z, gbar, grad_w, s);
    return grad_w_impl<TZ, TW, 32>(g, k, z, gbar, grad_w, s);
}

int grad_impl(nvd_graph_t g, int32_t k, const void *z, int32_t zdt, const double *gbar, void *grad_w,
              void *grad_x, void *grad_y, cudaStream_t s) {
    if (!g || k < 0 || (zdt != NVD_F32 && zdt != NVD_F64) || (k > 0 && (!z || !gbar))) {
        set_error("nvd_ge_grad: invalid argument");
        return NVD_ERR_INVALID_ARG;
    }
    if (k == 0) return NVD_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) cudaSetDevice(g->device);
    int rc = NVD_OK;
    if (grad_x || grad_y) {
        // about 32 CTAs per SM in all, spread over the columns
        const int gy = std::min(k, 65535);
        const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((g->n + 255) / 256,
                                                                   ((int64_t)g->num_sms * 32 + gy - 1) / gy));
        const dim3 grid((unsigned)gx, (unsigned)gy);
        if (zdt == NVD_F64)
            k_grad_xy<double><<<grid, 256, 0, s>>>((const double *)z, g->n, k, gbar, (double *)grad_x,
                                                   (double *)grad_y);
        else
            k_grad_xy<float><<<grid, 256, 0, s>>>((const float *)z, g->n, k, gbar, (float *)grad_x,
                                                  (float *)grad_y);
        if (cudaGetLastError() != cudaSuccess) rc = NVD_ERR_CUDA;
    }
    if (rc == NVD_OK && grad_w && g->nnz_user > 0) {
        if (g->nnz == 0) {
            rc = cudaMemsetAsync(grad_w, 0, (size_t)g->nnz_user * (g->wdtype == NVD_F64 ? 8 : 4), s) == cudaSuccess
                     ? NVD_OK : NVD_ERR_CUDA;
        } else if (zdt == NVD_F64) {
            rc = g->wdtype == NVD_F64 ? grad_w_kt<double, double>(g, k, (const double *)z, gbar, (double *)grad_w, s)
                                      : grad_w_kt<double, float>(g, k, (const double *)z, gbar, (float *)grad_w, s);
        } else {
            rc = g->wdtype == NVD_F64 ? grad_w_kt<float, double>(g, k, (const float *)z, gbar, (double *)grad_w, s)
                                      : grad_w_kt<float, float>(g, k, (const float *)z, gbar, (float *)grad_w, s);
        }
    }
    if (rc == NVD_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("nvd_ge_grad: %s", cudaGetErrorString(e));
            rc = NVD_ERR_CUDA;
        }
    }
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    return rc;
}

}  // namespace

extern "C" int nvd_ge_grad(nvd_graph_t g, int32_t k, const void *z, int32_t zdtype, const double *gbar,
                           void *grad_w, void *grad_x, void *grad_y, nvd_stream_t stream) {
    clear_error();
    TraceRange trace("nvd_ge_grad");
    try {
        return grad_impl(g, k, z, zdtype, gbar, grad_w, grad_x, grad_y, (cudaStream_t)stream);
    } catch (...) {
        set_error("nvd_ge_grad: unexpected host exception");
        return NVD_ERR_CUDA;
    }
}
