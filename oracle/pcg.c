/*
 * Oracle: plain FP64 Jacobi-preconditioned conjugate gradient for the GE distance.
 *
 * TEST INFRASTRUCTURE ONLY.  Used by tests/, the smoke check and the CPU-baseline
 * leg of the bench; the library never links or calls it.  Shares no code with
 * the CUDA path.
 *
 * What it computes (Section 3.1, GE equation; Section 3.2 Laplacian solvers;
 * the "CG" solver of Table 1):
 *     d^2 = (x - y)^T L^+ (x - y)
 * without forming L^+: with delta projected mean-zero on every connected
 * component (L^+ annihilates per-component constants), solve L z = delta by the
 * textbook preconditioned conjugate gradient with the Jacobi preconditioner
 * M = D (the weighted degrees), from z = 0, then d^2 = delta^T z with z projected
 * mean-zero per component.
 *
 * Stopping rule: the recursively updated residual is checked every iteration;
 * when ||r|| <= rtol ||delta|| the true residual delta - L z is formed and, if it
 * also meets the target, the solve ends; otherwise CG restarts from the current
 * z with the true residual.
 *
 * Input: a symmetric CSR adjacency (both directions stored), weights > 0,
 * self-loops ignored.  L_uv = -w_uv, L_uu = sum_v w_uv.
 *
 * Threads: loops over nodes are split statically over `nthreads` OpenMP threads;
 * every inner product sums per-thread partials in thread order, so results are
 * repeatable for a fixed thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

typedef struct {
    int64_t n;
    const int64_t *rowptr;
    const int32_t *colidx;
    const double *w;
    double *deg;
    int32_t *comp;
    int64_t ncomp;
    int64_t *comp_size;
    int nthreads;
    double *part;      /* [nthreads] partial sums */
    double *csum;      /* [nthreads * ncomp] per-thread per-component sums */
} graph_t;

/* Connected components by breadth-first search, numbered by smallest node. */
static int64_t bfs_components(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                              int32_t *comp) {
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) comp[i] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (comp[s] >= 0) continue;
        int64_t head = 0, tail = 0;
        comp[s] = (int32_t)c;
        queue[tail++] = s;
        while (head < tail) {
            int64_t u = queue[head++];
            for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                int64_t v = colidx[e];
                if (comp[v] < 0) {
                    comp[v] = (int32_t)c;
                    queue[tail++] = v;
                }
            }
        }
        ++c;
    }
    free(queue);
    return c;
}

/* sum_i a_i b_i with per-thread partials summed in thread order. */
static double dot(const graph_t *g, const double *a, const double *b) {
    const int64_t n = g->n;
#pragma omp parallel num_threads(g->nthreads)
    {
        int t = omp_get_thread_num(), nt = omp_get_num_threads();
        int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
        double s = 0.0;
        for (int64_t i = lo; i < hi; ++i) s += a[i] * b[i];
        g->part[t] = s;
        if (t == 0)
            for (int u = nt; u < g->nthreads; ++u) g->part[u] = 0.0;
    }
    double s = 0.0;
    for (int t = 0; t < g->nthreads; ++t) s += g->part[t];
    return s;
}

/* y = L x = D x - W x. */
static void lap_apply(const graph_t *g, const double *x, double *y) {
    const int64_t n = g->n;
#pragma omp parallel for schedule(static) num_threads(g->nthreads)
    for (int64_t u = 0; u < n; ++u) {
        double s = 0.0;
        for (int64_t e = g->rowptr[u]; e < g->rowptr[u + 1]; ++e) {
            int64_t v = g->colidx[e];
            if (v != u) s += g->w[e] * x[v];
        }
        y[u] = g->deg[u] * x[u] - s;
    }
}

/* v <- v - mean_c(v) on every connected component c. */
static void project(const graph_t *g, double *v) {
    const int64_t n = g->n, nc = g->ncomp;
#pragma omp parallel num_threads(g->nthreads)
    {
        int t = omp_get_thread_num(), nt = omp_get_num_threads();
        double *cs = g->csum + (size_t)t * (size_t)nc;
        for (int64_t c = 0; c < nc; ++c) cs[c] = 0.0;
        int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
        for (int64_t i = lo; i < hi; ++i) cs[g->comp[i]] += v[i];
        if (t == 0)
            for (int u = nt; u < g->nthreads; ++u)
                memset(g->csum + (size_t)u * (size_t)nc, 0, sizeof(double) * (size_t)nc);
    }
    double *mean = (double *)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    for (int64_t c = 0; c < nc; ++c) {
        double s = 0.0;
        for (int t = 0; t < g->nthreads; ++t) s += g->csum[(size_t)t * (size_t)nc + c];
        mean[c] = s / (double)g->comp_size[c];
    }
#pragma omp parallel for schedule(static) num_threads(g->nthreads)
    for (int64_t i = 0; i < n; ++i) v[i] -= mean[g->comp[i]];
    free(mean);
}

/* Solve L z = delta (delta already projected) by Jacobi PCG.  Returns the number of
 * iterations, or -1 if max_iter was reached first.  *relres gets the final true
 * relative residual. */
static int64_t pcg_solve(const graph_t *g, const double *delta, double rtol, int64_t max_iter,
                         double *z, double *relres, double *r, double *u, double *p,
                         double *q) {
    const int64_t n = g->n;
    double dnorm = sqrt(dot(g, delta, delta));
    memset(z, 0, sizeof(double) * (size_t)n);
    if (dnorm == 0.0) {
        *relres = 0.0;
        return 0;
    }
    memcpy(r, delta, sizeof(double) * (size_t)n);
    int64_t it = 0;
    for (int restarts = 0;; ++restarts) {
        /* (re)start: u = D^{-1} r, p = u, rho = r.u */
#pragma omp parallel for schedule(static) num_threads(g->nthreads)
        for (int64_t i = 0; i < n; ++i) {
            u[i] = g->deg[i] > 0.0 ? r[i] / g->deg[i] : 0.0;
            p[i] = u[i];
        }
        double rho = dot(g, r, u);
        double rnorm = sqrt(dot(g, r, r));
        while (rnorm > rtol * dnorm && it < max_iter) {
            lap_apply(g, p, q);
            double pq = dot(g, p, q);
            if (!(pq > 0.0)) break;
            double alpha = rho / pq;
#pragma omp parallel for schedule(static) num_threads(g->nthreads)
            for (int64_t i = 0; i < n; ++i) {
                z[i] += alpha * p[i];
                r[i] -= alpha * q[i];
                u[i] = g->deg[i] > 0.0 ? r[i] / g->deg[i] : 0.0;
            }
            double rho_new = dot(g, r, u);
            rnorm = sqrt(dot(g, r, r));
            double beta = rho_new / rho;
            rho = rho_new;
#pragma omp parallel for schedule(static) num_threads(g->nthreads)
            for (int64_t i = 0; i < n; ++i) p[i] = u[i] + beta * p[i];
            ++it;
        }
        /* true residual */
        lap_apply(g, z, q);
#pragma omp parallel for schedule(static) num_threads(g->nthreads)
        for (int64_t i = 0; i < n; ++i) r[i] = delta[i] - q[i];
        project(g, r);
        double tnorm = sqrt(dot(g, r, r));
        *relres = tnorm / dnorm;
        if (tnorm <= rtol * dnorm) return it;
        if (it >= max_iter || restarts >= 50) return -1;
    }
}

/*
 * For every pair j (rows of X and Y, [k][n] row-major):
 *   d2[j] = (P delta_j)^T z_j,  z_j = L^+ delta_j (projected), delta_j = X_j - Y_j.
 * Z (optional, [k][n]) receives z_j.  iters[j] / relres[j] receive the iteration
 * count (-1 = not converged) and the final true relative residual.
 * Returns 0 when every pair converged, 1 otherwise, -1 on bad arguments.
 */
int oracle_ge_pcg(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *w,
                  int64_t k, const double *X, const double *Y, double rtol, int64_t max_iter,
                  int nthreads, double *d2, double *Z, int64_t *iters, double *relres) {
    if (n <= 0 || k < 0 || nthreads <= 0) return -1;
    graph_t g;
    g.n = n;
    g.rowptr = rowptr;
    g.colidx = colidx;
    g.w = w;
    g.nthreads = nthreads;
    g.deg = (double *)malloc(sizeof(double) * (size_t)n);
    g.comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    g.part = (double *)calloc((size_t)nthreads, sizeof(double));
    g.ncomp = bfs_components(n, rowptr, colidx, g.comp);
    g.comp_size = (int64_t *)calloc((size_t)g.ncomp, sizeof(int64_t));
    g.csum = (double *)calloc((size_t)nthreads * (size_t)g.ncomp, sizeof(double));
    for (int64_t i = 0; i < n; ++i) g.comp_size[g.comp[i]]++;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t u = 0; u < n; ++u) {
        double s = 0.0;
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e)
            if (colidx[e] != u) s += w[e];
        g.deg[u] = s;
    }
    size_t nb = sizeof(double) * (size_t)n;
    double *delta = (double *)malloc(nb), *z = (double *)malloc(nb), *r = (double *)malloc(nb);
    double *u = (double *)malloc(nb), *p = (double *)malloc(nb), *q = (double *)malloc(nb);
    int status = 0;
    for (int64_t j = 0; j < k; ++j) {
        const double *x = X + (size_t)j * (size_t)n, *y = Y + (size_t)j * (size_t)n;
#pragma omp parallel for schedule(static) num_threads(nthreads)
        for (int64_t i = 0; i < n; ++i) delta[i] = x[i] - y[i];
        project(&g, delta);
        double rr;
        int64_t it = pcg_solve(&g, delta, rtol, max_iter, z, &rr, r, u, p, q);
        project(&g, z);
        d2[j] = dot(&g, delta, z);
        if (Z) memcpy(Z + (size_t)j * (size_t)n, z, nb);
        if (iters) iters[j] = it;
        if (relres) relres[j] = rr;
        if (it < 0) status = 1;
    }
    free(delta); free(z); free(r); free(u); free(p); free(q);
    free(g.deg); free(g.comp); free(g.part); free(g.comp_size); free(g.csum);
    return status;
}

/* Number of connected components (exposed for the host-side tests). */
int64_t oracle_components(int64_t n, const int64_t *rowptr, const int32_t *colidx,
                          int32_t *comp) {
    return bfs_components(n, rowptr, colidx, comp);
}
