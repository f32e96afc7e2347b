/*
 * nvd.h -- C ABI of the GB300 Generalized-Euclidean node-vector distance library.
 *
 * The library computes, for node vectors x and y on a weighted undirected graph,
 *
 *     d(x, y)^2 = (x - y)^T L^+ (x - y)                 (Section 3.1, GE equation)
 *
 * where L = D - W is the graph Laplacian and L^+ its Moore-Penrose pseudoinverse,
 * without ever forming L^+: it solves L z = x - y with a Laplacian solver
 * (Section 3.2) -- here a Jacobi-preconditioned conjugate gradient (the "CG"
 * solver of Table 1) built from hand-written sm_103a kernels -- and returns
 * (x - y)^T z.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an nvd_status (0 = NVD_OK) and never throws or aborts.
 *    nvd_last_error() gives a one-line description of the most recent failure on
 *    the calling thread.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All device work is ordered on that stream.  Unless a flag below
 *    says otherwise, a call returns after its results are available to the
 *    caller (it synchronises the stream once at the end).
 *  - Node vectors use the layout [k][n]: k pairs, one contiguous row of n values
 *    per pair, node order of the CSR given to nvd_graph_create.
 *  - One handle may be used by one thread at a time; distinct handles are
 *    independent.  A handle lives on the CUDA device that was current when it
 *    was created; calls on it make that device current for their duration.
 *  - Sizes: n < 2^31 nodes, nnz < 2^62 stored entries, k < 2^31 pairs.
 */
#ifndef NVD_H_
#define NVD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nvd_graph_s *nvd_graph_t; /* opaque graph handle */
typedef void *nvd_stream_t;              /* cudaStream_t */

typedef enum { NVD_F32 = 0, NVD_F64 = 1 } nvd_dtype;

typedef enum {
    NVD_OK = 0,
    NVD_ERR_INVALID_ARG = 1,   /* bad pointer, size, dtype, flag or CSR layout */
    NVD_ERR_NOT_SYMMETRIC = 2, /* CSR is not a symmetric matrix (structure or values) */
    NVD_ERR_BAD_WEIGHT = 3,    /* a weight is <= 0, NaN or infinite (Section 3.1 needs w > 0) */
    NVD_ERR_OOM = 4,           /* device or host allocation failed */
    NVD_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    NVD_ERR_NOT_CONVERGED = 6, /* some pair did not reach the tolerance (results still written) */
    NVD_ERR_NUMERIC = 7,       /* NaN/Inf or loss of positivity inside the solver */
    NVD_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up (grid barrier) */
    NVD_ERR_UNSUPPORTED = 9    /* valid request the build does not handle */
} nvd_status;

/* ------------------------------------------------------------------ graphs */

#define NVD_GRAPH_DEVICE_PTRS 1u    /* rowptr/colidx/w are device pointers (else host) */
#define NVD_GRAPH_SKIP_SYM_CHECK 2u /* trust the caller: skip the symmetry check */
#define NVD_GRAPH_REORDER_DEGREE 4u /* store each component's nodes by degree, highest first (the rows the
                                       SpMM gathers most form one contiguous run; results in the caller's
                                       node order as always) */

/*
 * nvd_graph_create -- build a graph handle from a CSR adjacency (Section 3.1:
 * undirected graph, positive weights; L = D - W).
 *
 *   n        number of nodes (>= 1).
 *   nnz      number of stored entries (>= 0); rowptr[n] must equal nnz.
 *   rowptr   int64 [n+1], non-decreasing, rowptr[0] = 0.
 *   colidx   int32 [nnz], column of each entry, 0 <= colidx < n.
 *   w        [nnz] weights, float (NVD_F32) or double (NVD_F64) per wdtype;
 *            NULL means every weight is 1.
 *   flags    NVD_GRAPH_* bits.  Without NVD_GRAPH_DEVICE_PTRS the three arrays
 *            are host memory.
 *
 * The matrix must be symmetric (entry (u,v,w) present iff (v,u,w) is); both
 * directions of every edge are stored.  Self-loops are dropped (they do not
 * change L); repeated (u,v) entries are summed (parallel conductances); columns
 * need not be sorted.  The library copies everything it needs: the caller may
 * free its arrays when the call returns.  Connected components are found here;
 * the solver works on each component separately (L^+ annihilates constants on
 * every component, so delta is projected mean-zero per component).
 *
 * Errors: NVD_ERR_INVALID_ARG (n < 1, nnz < 0, NULL pointers, rowptr not
 * monotone or not ending at nnz, column out of range), NVD_ERR_NOT_SYMMETRIC,
 * NVD_ERR_BAD_WEIGHT, NVD_ERR_OOM, NVD_ERR_CUDA.  On failure *out is NULL.
 */
int nvd_graph_create(nvd_graph_t *out, int64_t n, int64_t nnz, const int64_t *rowptr,
                     const int32_t *colidx, const void *w, int32_t wdtype, uint32_t flags,
                     nvd_stream_t stream);

/* nvd_graph_destroy -- release a handle and all its device memory.  NULL is a no-op. */
int nvd_graph_destroy(nvd_graph_t g);

/*
 * nvd_graph_info -- sizes of a handle.  Any output pointer may be NULL.
 *   n, nnz        nodes and stored entries after cleaning (self-loops dropped,
 *                 repeated entries merged);
 *   ncomp         connected components (isolated nodes count as components);
 *   device_bytes  device memory currently held by the handle (graph + workspace).
 */
int nvd_graph_info(nvd_graph_t g, int64_t *n, int64_t *nnz, int32_t *ncomp,
                   int64_t *device_bytes);

/*
 * nvd_graph_set_weights -- new edge weights for the same sparsity pattern (the
 * weighted graphs of Section 3.1; a training loop that updates w between
 * distance evaluations), without rebuilding the handle: no new components,
 * relabelling, plans or tuning.
 *
 *   w       [nnz] weights in the entry order of the CSR given to nvd_graph_create
 *           (the caller's nnz, before cleaning), host memory, or device memory with
 *           NVD_GRAPH_DEVICE_PTRS in flags.
 *   wdtype  must be the handle's weight type (the wdtype of nvd_graph_create).
 *   flags   NVD_GRAPH_DEVICE_PTRS, NVD_GRAPH_SKIP_SYM_CHECK.
 *
 * Entries are mapped as at creation: self-loop entries are dropped (their weight
 * must still be finite and > 0) and repeated (u, v) entries are summed in entry
 * order.  The degrees, D^-1, the FP32 copy of FP64 weights and the sliced copies of
 * every cached work plan are recomputed.  An elimination made by
 * nvd_graph_eliminate is dropped (it depends on the weights): call it again before
 * solving with NVD_SOLVE_ELIMINATE.  Synchronous: returns once the handle holds the
 * new weights.
 *
 * Errors: NVD_ERR_INVALID_ARG (NULL pointer, other dtype, unknown flag),
 * NVD_ERR_BAD_WEIGHT (a weight <= 0, NaN or infinite), NVD_ERR_NOT_SYMMETRIC
 * (w_uv != w_vu after merging), NVD_ERR_OOM, NVD_ERR_CUDA.  On an error the
 * handle keeps its old weights.
 */
int nvd_graph_set_weights(nvd_graph_t g, const void *w, int32_t wdtype, uint32_t flags,
                          nvd_stream_t stream);

/* ------------------------------------------------------------------ solving */

typedef enum {
    NVD_MODE_FP64 = 0,  /* FP64 vectors, FP64 arithmetic throughout */
    NVD_MODE_FP32 = 1,  /* FP32 vectors and SpMV/SpMM, FP64 inner products and scalars */
    NVD_MODE_MIXED = 2  /* FP32 block-PCG inside an FP64 iterative-refinement loop */
} nvd_mode;

#define NVD_SOLVE_SINGLE_RHS 1u   /* solve the k pairs one right-hand side at a time */
#define NVD_SOLVE_D2_DEVICE 2u    /* d2_out is a device pointer (default: host) */
#define NVD_SOLVE_HOST_INPUTS 4u  /* x, y (and z_out) are host pointers; copies are done here */
#define NVD_SOLVE_PERSISTENT 8u   /* run each PCG solve inside one persistent cooperative kernel */
#define NVD_SOLVE_NO_SYNC 16u     /* with NVD_SOLVE_D2_DEVICE and no stats: return without a final sync */
#define NVD_SOLVE_TEST_TIMEOUT 64u /* diagnostic, with NVD_SOLVE_PERSISTENT: the grid barrier waits for
                                     one arrival more than the grid has, so its bounded wait runs out;
                                     the call returns NVD_ERR_TIMEOUT (exercises the timeout path) */
#define NVD_SOLVE_FOLD_DIRECTION 32u /* two kernels per CG iteration: the direction update folded into
                                        an SpMV on D^-1 r (default: three, SpMV on p, x/r update,
                                        direction pass) */
#define NVD_SOLVE_ELIMINATE 256u  /* solve on the handle's reduced graph (nvd_graph_eliminate): degree-1/2
                                     nodes eliminated exactly; device x, y; z_out by back-substitution */
#define NVD_SOLVE_D2_STOP 128u    /* FP64/FP32: a pair also stops once its d^2 is estimated to be
                                     within d2_rtol: step k of CG from z = 0 adds exactly
                                     alpha_k r_k^T D^-1 r_k to delta^T z and the remaining gap is
                                     |z* - z_k|_L^2; the gap is extrapolated from the last terms'
                                     geometric decay (an estimate, not a bound; see the finalizer).
                                     Not with MIXED, nvd_resistance_matrix or nvd_network_variance */

typedef struct {
    int32_t mode;        /* nvd_mode */
    int32_t max_iter;    /* CG iteration limit per solve (MIXED: per inner solve) */
    double rtol;         /* FP64/FP32: stop when ||delta - L z||_2 <= rtol ||delta||_2 per pair
                            (recursive residual); MIXED: tolerance of each inner FP32 solve */
    double d2_rtol;      /* MIXED: stop refining when the relative change of d^2 <= d2_rtol;
                            with NVD_SOLVE_D2_STOP: the d^2 accuracy asked of each pair (< 1) */
    int32_t max_refine;  /* MIXED: limit on outer refinement steps */
    int32_t check_every; /* iterations between host convergence polls (host-driven loop) */
    int32_t kt;          /* right-hand sides per tile: 0 = automatic, else 1, 4, 8, 16 or 32 */
    uint32_t flags;      /* NVD_SOLVE_* bits */
} nvd_solve_opts;

typedef struct {
    int32_t iters;        /* CG iterations used (MIXED: summed over inner solves) */
    int32_t refine_steps; /* MIXED: outer steps; 0 otherwise */
    double rel_resid;     /* final relative residual ||delta - L z|| / ||delta|| (recursive;
                             MIXED: the true FP64 residual of the last refinement step) */
    int32_t status;       /* nvd_status of this pair */
    int32_t reserved;
} nvd_solve_stats;

/* nvd_solve_opts_default -- FP64 mode, rtol 1e-10, max_iter 10000, d2_rtol 1e-8,
 * max_refine 8, check_every 4, kt automatic, no flags. */
void nvd_solve_opts_default(nvd_solve_opts *o);

/* ------------------------------------------------------------------ tuning */

#define NVD_TUNE_SINGLE_RHS 1u   /* tune for one right-hand side at a time (tile width 1) */

typedef struct {
    int32_t kt;            /* chosen right-hand sides per tile */
    int32_t row_max_pct;   /* light-row limit in percent of the default (50, 100 or 200) */
    int32_t blocks_pct;    /* light CTA blocks per SpMV in percent of the default */
    int32_t persistent;    /* 1: one persistent launch per tile was faster */
    int32_t candidates;    /* configurations timed */
    int32_t fold_direction; /* 1: two kernels per iteration (NVD_SOLVE_FOLD_DIRECTION) were faster */
    int32_t gather;        /* multi-column SpMM: 0 register loads per slice (default), 1 register loads
                              over each warp's step stream, 2 TMA gathers over the stream, 3 per-lane
                              asynchronous copies (cp.async) over the stream (2 and 3: tiles whose
                              rows are 64 or 128 bytes; others use 1) */
    int32_t l2_hot;        /* 1: graphs made with NVD_GRAPH_REORDER_DEGREE keep the gathered vector's
                              highest-degree rows persisting in L2 during multi-column SpMMs (this
                              process's L2 set-aside is requested on first use) */
    double ms_per_iter;    /* device time of one PCG iteration of one tile, chosen setting */
    double ms_per_pair_iter; /* ms_per_iter / kt */
} nvd_tune_result;

/*
 * nvd_graph_tune -- choose the work decomposition of the solve (Section 3.2) for
 * this graph by timing it: tile width (k-blocking) for k pairs, the row-split
 * limit (longer rows become split sub-items), the number of SpMV blocks, the
 * gather engine of multi-column SpMMs (register loads per slice, register loads
 * over a warp's step stream, TMA row gathers or per-lane asynchronous copies
 * into shared memory), host-driven
 * versus persistent iterations, and two versus three kernels per iteration
 * (NVD_SOLVE_FOLD_DIRECTION).  Candidates run real solves with
 * seeded synthetic right-hand sides for a fixed number of iterations on
 * `stream`; the winner is stored in the handle and used by later calls of
 * mode `mode` (MIXED is timed as its FP32 inner solve): plans built afterwards
 * use the row split and block count, and nvd_ge_distance uses the tile width
 * when opts.kt = 0 and the launch mode and iteration form when the flags leave
 * them at their defaults.
 * Results do not depend on the choice beyond rounding (each choice is a valid
 * order of the same sums).  Synchronous.
 *   k      number of pairs the later calls will solve (sets the tile-width cost
 *          ceil(k / kt) * per-tile time); flags: NVD_TUNE_* bits.
 *   out    optional; the chosen setting.
 * Memory: 32 n doubles of synthetic input plus the plans of the timed
 * candidates (plans of losing candidates are freed on return).
 * Errors: NVD_ERR_INVALID_ARG (NULL handle, bad mode, k < 1, unknown flag),
 * NVD_ERR_OOM, NVD_ERR_CUDA; on error the handle's previous setting is kept.
 */
int nvd_graph_tune(nvd_graph_t g, int32_t mode, int32_t k, uint32_t flags, nvd_tune_result *out,
                   nvd_stream_t stream);

/*
 * nvd_graph_set_tuning -- apply a setting (for example one nvd_graph_tune chose
 * earlier for the same graph) without timing anything.  Reads kt (0 = no
 * preference), row_max_pct and blocks_pct (10..1000), persistent,
 * fold_direction and l2_hot (0/1), gather (0..3); the other fields are ignored.  Host only; plans built
 * afterwards use it.
 * Errors: NVD_ERR_INVALID_ARG (NULL pointer, bad mode or field).
 */
int nvd_graph_set_tuning(nvd_graph_t g, int32_t mode, const nvd_tune_result *t);

/*
 * nvd_ge_distance -- d^2 = (x_j - y_j)^T L^+ (x_j - y_j) for j < k (Section 3.1,
 * GE equation), by PCG on L z = P(x_j - y_j) (Section 3.2), P the per-component
 * mean-zero projector.  d = sqrt(max(d^2, 0)) is left to the caller.
 *
 *   x, y    [k][n] device arrays (host with NVD_SOLVE_HOST_INPUTS) of xdtype.
 *   d2_out  [k] double, host unless NVD_SOLVE_D2_DEVICE.
 *   z_out   optional [k][n] of xdtype: z_j = L^+ (x_j - y_j), mean-zero on every
 *           component (what nvd_ge_grad consumes).  NULL to skip.
 *   stats   optional [k] host array.
 *
 * FP64 mode returns d^2 = delta^T z at the converged z; MIXED mode returns the
 * variational estimate 2 delta^T z - z^T L z from the FP64 residual (error
 * quadratic in the error of z).  Non-convergence still writes every output and
 * returns NVD_ERR_NOT_CONVERGED; per-pair status is in stats.
 */
int nvd_ge_distance(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdtype,
                    const nvd_solve_opts *opts, double *d2_out, void *z_out,
                    nvd_solve_stats *stats, nvd_stream_t stream);

/*
 * nvd_graph_eliminate -- exact elimination of degree-1 and degree-2 nodes for
 * later solves with NVD_SOLVE_ELIMINATE.  Eliminating a node of the Laplacian
 * leaves the Schur complement, again a graph Laplacian with no fill for such a
 * node: a leaf goes with its edge, a node with neighbours a, c becomes the edge
 * a-c of conductance w_a w_c / d_v (series rule), and for b mean-zero per
 * component b^T L^+ b = b'^T L'^+ b' + b_v^2 / d_v with b'_u = b_u + b_v w_vu / d_v,
 * so d^2 (GE equation, Section 3.1) is the reduced graph's d^2 plus one term per
 * eliminated node, and PCG (Section 3.2) runs on the reduced graph.  Nodes go in
 * rounds of independent sets, so the per-solve forward pass is one parallel step
 * per round.  Builds on the host from the handle's CSR (O(nnz) memory) and keeps
 * the reduced graph in the handle; calling it again rebuilds.  Synchronous.
 *   info    optional: kept nodes, their stored entries, eliminated nodes, rounds.
 * Errors: NVD_ERR_INVALID_ARG (NULL handle), NVD_ERR_OOM, NVD_ERR_CUDA.
 */
typedef struct {
    int64_t n_kept;
    int64_t nnz_kept;
    int64_t n_eliminated;
    int32_t rounds;
    int32_t reserved;
} nvd_elim_info;
int nvd_graph_eliminate(nvd_graph_t g, nvd_elim_info *info, nvd_stream_t stream);

/*
 * nvd_eliminate_host -- the same elimination on a host CSR (symmetric, no GPU
 * work), for checking it: writes the kept nodes (increasing ids) and the reduced
 * graph's CSR on their indices.  keep [n], red_rowptr [n + 1], red_colidx and
 * red_w [rowptr[n]] (the reduced graph has at most as many entries); any output
 * array may be NULL.  Errors: NVD_ERR_INVALID_ARG (n < 1, NULL rowptr or n_kept,
 * NULL colidx / w with entries), NVD_ERR_OOM.
 */
int nvd_eliminate_host(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *w,
                       int64_t *n_kept, int32_t *keep, int64_t *red_rowptr, int32_t *red_colidx,
                       double *red_w, int32_t *rounds);

/*
 * nvd_eliminate_host_program -- the per-solve program of the same elimination, for
 * checking it on the host: counts[5] = {records R, kept nodes K, record gather
 * entries, kept-node gather entries, rounds}.  Record r eliminates node rec_v[r]
 * (weighted degree rec_d[r]); records of round t are [round_ptr[t], round_ptr[t+1]);
 * the forward pass computes b_r = b[rec_v[r]] + sum_{e in [rin_ptr[r], rin_ptr[r+1])}
 * rin_f[e] b_{rin_src[e]} round by round, the reduced right-hand side of kept
 * node i = b[keep[i]] + the same sum over kin_*, and d^2 = reduced d^2 + sum_r
 * b_r^2 / rec_d[r].  The back-substitution (z_out) takes the records in reverse
 * round order: z[rec_v[r]] = b_r / rec_d[r] + rec_f0[r] z[rec_t0[r]] + rec_f1[r]
 * z[rec_t1[r]] (rec_t1 = -1: none), from the reduced solution on the kept nodes,
 * then mean-zero per component.  With any array NULL only counts is written
 * (sizes: R, R, rounds + 1, R + 1, counts[2] x2, K, K + 1, counts[3] x2, R x4).
 */
int nvd_eliminate_host_program(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *w,
                               int64_t *counts, int32_t *rec_v, double *rec_d, int64_t *round_ptr,
                               int64_t *rin_ptr, int32_t *rin_src, double *rin_f, int32_t *keep,
                               int64_t *kin_ptr, int32_t *kin_src, double *kin_f, int32_t *rec_t0,
                               int32_t *rec_t1, double *rec_f0, double *rec_f1);

/*
 * nvd_ge_distance_warm -- nvd_ge_distance started from a saved solution z0
 * instead of z = 0 (a warm start, e.g. the z_out of an earlier call when the
 * vectors or the weights have changed a little).  CG runs on L c = P(delta - L z0)
 * from z0; the residual test stays relative to |P delta|, so the same rtol gives
 * the same accuracy in fewer iterations when z0 is close.  d^2 is the variational
 * 2 delta^T z - z^T L z (error quadratic in the error of z); constants per
 * component in z0 have no effect.
 *
 *   z0      [k][n] device array of xdtype (the layout of z_out; may be the same
 *           buffer as z_out).
 * Other arguments as nvd_ge_distance.  FP64 mode and device inputs only; the
 * solve runs host-driven (NVD_SOLVE_PERSISTENT and a tuned persistent launch are
 * not used).
 * Errors: NVD_ERR_INVALID_ARG (z0 NULL with k > 0, FP32 or MIXED mode,
 * NVD_SOLVE_HOST_INPUTS), otherwise as nvd_ge_distance.
 */
int nvd_ge_distance_warm(nvd_graph_t g, int32_t k, const void *x, const void *y, int32_t xdtype,
                         const void *z0, const nvd_solve_opts *opts, double *d2_out, void *z_out,
                         nvd_solve_stats *stats, nvd_stream_t stream);

/*
 * nvd_effective_resistance -- R(u_j, v_j) = (e_u - e_v)^T L^+ (e_u - e_v) for j < k:
 * the GE distance (Section 3.1) of two indicator vectors, which on a graph with
 * conductances w is the effective resistance between the two nodes (the
 * L^+ quadratic forms of Section 2.1).  Solved like nvd_ge_distance, with the
 * right-hand sides built on the device from the ids (no [k][n] input).
 *
 *   u, v    [k] host int32 node ids in [0, n).
 *   r_out   [k] host doubles: R for u, v in one component; 0 for u = v; +inf
 *           for u != v in different components (or an isolated node), which
 *           are not solved.
 *   stats   optional [k] host array (iters 0 for pairs that were not solved).
 * opts as for nvd_ge_distance (NVD_SOLVE_ELIMINATE: on the handle's reduced
 * graph); NVD_SOLVE_D2_DEVICE and NVD_SOLVE_HOST_INPUTS are invalid here.
 * Synchronous.
 * Errors: NVD_ERR_INVALID_ARG (NULL pointer, k < 0, an id outside [0, n), bad
 * opts), NVD_ERR_NOT_CONVERGED / NVD_ERR_NUMERIC (every output still written),
 * NVD_ERR_OOM, NVD_ERR_CUDA.
 */
int nvd_effective_resistance(nvd_graph_t g, int32_t k, const int32_t *u, const int32_t *v,
                             const nvd_solve_opts *opts, double *r_out, nvd_solve_stats *stats,
                             nvd_stream_t stream);

/*
 * nvd_resistance_matrix -- the effective-resistance matrix of a node subset,
 * R[i][j] = R(nodes[i], nodes[j]) (the L^+ quadratic forms of Section 2.1 on
 * indicator vectors, GE equation of Section 3.1).  Per component, one node of
 * the subset is the reference r and each other distinct node d gets one solve
 * z_d = L^+ (e_d - e_r); then R(a, b) = z_a[a] - z_a[b] - z_b[a] + z_b[b]
 * (z_r = 0), so s nodes in one component cost s - 1 solves, not s(s-1)/2.
 *
 *   nodes   [s] host int32 node ids in [0, n); repeats allowed.
 *   R_out   [s][s] host doubles, row-major, symmetric up to rounding: 0 where
 *           nodes[i] = nodes[j]; +inf across components or to an isolated node.
 *   stats   optional [s] host array: entry i describes the solve of nodes[i]
 *           (iters 0 for reference nodes and nodes without a solve).
 * opts as for nvd_effective_resistance.  Device memory: up to 2 GiB of z per
 * batch of solves (columns are processed in batches of at most 2^28 / n).
 * Synchronous.
 * Errors: NVD_ERR_INVALID_ARG (NULL pointer, s < 0, an id outside [0, n), bad
 * opts), NVD_ERR_NOT_CONVERGED / NVD_ERR_NUMERIC (every output still written),
 * NVD_ERR_OOM, NVD_ERR_CUDA.
 */
int nvd_resistance_matrix(nvd_graph_t g, int32_t s, const int32_t *nodes, const nvd_solve_opts *opts,
                          double *R_out, nvd_solve_stats *stats, nvd_stream_t stream);

/*
 * nvd_network_variance -- the network variance of non-negative node weights p
 * (a distribution on the graph; the variance of distributions on graphs cited in
 * Section 2): var = (1/2) sum_ij p_i p_j R(nodes[i], nodes[j]), R the effective
 * resistance, from nvd_resistance_matrix on the nodes with p_i > 0.  +inf when
 * two nodes with positive weight lie in different components.  p is not
 * normalised (for a distribution it sums to 1).
 *
 *   nodes   [s] host int32 node ids in [0, n); p [s] host doubles >= 0.
 *   var_out host double.
 * opts as for nvd_effective_resistance.  Synchronous.
 * Errors: NVD_ERR_INVALID_ARG (NULL pointer, s < 0, an id outside [0, n), a
 * negative or non-finite weight, bad opts), NVD_ERR_NOT_CONVERGED /
 * NVD_ERR_NUMERIC (var_out still written), NVD_ERR_OOM, NVD_ERR_CUDA.
 */
int nvd_network_variance(nvd_graph_t g, int32_t s, const int32_t *nodes, const double *p,
                         const nvd_solve_opts *opts, double *var_out, nvd_stream_t stream);

/*
 * nvd_ge_distance_batched -- many graphs in one solve: the G graphs are treated as
 * the diagonal blocks of one block-diagonal Laplacian and every (graph, pair)
 * keeps its own CG scalars and convergence test, so the result equals G
 * independent nvd_ge_distance calls.  The PCG iterations are driven from the
 * host, one launch per phase over all graphs (the kernels of nvd_ge_distance at
 * full occupancy; convergence polled one batch behind), or, with
 * NVD_SOLVE_PERSISTENT, run inside one persistent cooperative kernel captured in
 * a CUDA graph (replayed when the same arguments come again).  Measured on the
 * 64-graph workload (1.7e6 nodes) the host-driven form takes 23 ms per FP32 step
 * against 45 ms; the persistent kernel (two CTAs per SM at its register count,
 * three grid barriers per iteration) is ahead by at most ~10% on batches of a few
 * graphs or a few tens of thousands of nodes.
 *
 *   graphs  [G] handles (same device).
 *   k_per   [G] pairs per graph.
 *   x, y    [G] device pointers, x[g] and y[g] of shape [k_per[g]][n_g].
 *   d2_out  [sum k_per] host doubles, graph after graph.
 *   stats   optional [sum k_per].
 */
int nvd_ge_distance_batched(const nvd_graph_t *graphs, int32_t G, const int32_t *k_per,
                            const void *const *x, const void *const *y, int32_t xdtype,
                            const nvd_solve_opts *opts, double *d2_out, nvd_solve_stats *stats,
                            nvd_stream_t stream);

/*
 * nvd_ge_grad -- adjoint of d^2 (no new solve; reuses z from nvd_ge_distance).
 * With upstream weights gbar_j = dLoss/d(d_j^2):
 *
 *   grad_x[j] =  2 gbar_j z_j,   grad_y[j] = -2 gbar_j z_j        (L^+ symmetric)
 *   grad_w[e] = -1/2 sum_j gbar_j (z_j[u] - z_j[v])^2             per stored entry e = (u, v)
 *
 * The weight gradient follows from dL^+ = -L^+ dL L^+ with the operator built
 * from W_sym = (W + W^T)/2, so the two stored entries of an undirected edge
 * together receive -(z_u - z_v)^2 -- the derivative with respect to the edge
 * weight.  Self-loop entries receive 0.
 *
 *   z       [k][n] device array of zdtype (z_out of nvd_ge_distance).
 *   gbar    [k] device doubles.
 *   grad_w  [nnz] device array in the entry order given to nvd_graph_create, of
 *           the graph's weight dtype, or NULL.
 *   grad_x, grad_y  [k][n] device arrays of zdtype, or NULL.
 */
int nvd_ge_grad(nvd_graph_t g, int32_t k, const void *z, int32_t zdtype, const double *gbar,
                void *grad_w, void *grad_x, void *grad_y, nvd_stream_t stream);

/*
 * nvd_laplacian_apply -- y_j = L x_j for j < k ([k][n] device arrays of dtype),
 * the operator the solver uses (exposed for testing and benchmarking; FP64
 * arithmetic for NVD_F64, FP32 for NVD_F32).
 */
int nvd_laplacian_apply(nvd_graph_t g, int32_t k, const void *x, void *y, int32_t dtype,
                        nvd_stream_t stream);

/*
 * nvd_dot_f32 -- sum_i a_i b_i of two FP32 device vectors of length n into *out
 * (one device double), with the reduction the FP32-mode PCG uses for its inner
 * products (Section 3.2 solver, FP32 vectors): each thread accumulates the exact
 * products a_i b_i (a float product fits a double-float pair) in a double-float
 * pair, the per-thread values are added in FP64 within each block and the block
 * totals in block order, so the result does not depend on timing.  Its error is
 * about 1e-13 * sum_i |a_i b_i| (FP64 sums of at most 1,280 partials), where an
 * FP32 accumulation would give about 1e-7 times that.  Stream-ordered on `stream`
 * (8 KB of scratch from the stream-ordered allocator).
 * Errors: NVD_ERR_INVALID_ARG (n < 0, NULL out, NULL a or b with n > 0),
 * NVD_ERR_CUDA.
 */
int nvd_dot_f32(const float *a, const float *b, int64_t n, double *out, nvd_stream_t stream);

/*
 * nvd_laplacian_quadform_noalloc -- y_j = L x_j and q_j = x_j^T L x_j for j < k,
 * without allocating any memory.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory when they call, e.g. a
 * process whose device memory is already held by another framework's caching
 * allocator, or a time-critical loop that must not allocate (an allocation can
 * synchronise the device).  It is a variant of the SpMV with fused inner
 * product that the solver runs every iteration; the handle must exist already
 * (nvd_graph_create allocates, this call does not: no cudaMalloc, no cudaFree,
 * no allocating library routine).
 *
 *   x  [k][n] device doubles (caller's node order); y [k][n] device doubles or
 *   NULL; q [k] device doubles.  1 <= k <= 32 (larger k: NVD_ERR_INVALID_ARG).
 *
 * Scratch: the cross-block partial sums live in one file-scope device array of
 * 262,400 bytes (1024 blocks x 32 columns of doubles plus a counter), which every
 * GPU that loads the library keeps until the process exits.  Every call shares
 * that array and it keeps the last call's contents; calls that overlap on the GPU
 * (different streams, or several threads) race on it and must be serialised by
 * the caller.  The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make that
 * first call before any stream capture.  A device reset (cudaDeviceReset)
 * releases the array with the context: after one, this entry point must not be
 * called again in that process (the kept address would point at freed memory).
 * The work is ordered on `stream` and the call returns without waiting for it.
 */
int nvd_laplacian_quadform_noalloc(nvd_graph_t g, int32_t k, const double *x, double *y, double *q,
                                   nvd_stream_t stream);

/* ------------------------------------------------------------------ diagnostics */

/* nvd_status_string -- static name of a status code. */
const char *nvd_status_string(int status);

/* nvd_last_error -- detail of the last failure on this thread ("" if none). */
const char *nvd_last_error(void);

/*
 * Kernel timing.  While enabled (on = 1), every launch of the Laplacian SpMV/SpMM
 * kernel made by nvd_ge_distance is bracketed by CUDA events on its stream
 * (on = 2: the vector passes too, class 1);
 * nvd_profile_read returns the launch count, summed event time in ms and summed
 * algorithmic bytes of those launches since the last read (and resets them).
 * Class 0 = the SpMV/SpMM kernel of the CG iterations, class 1 = the streaming
 * vector passes (bytes not tracked), class 2 = the FP64 residual SpMM of the
 * MIXED refinement steps and of warm starts (every launch, no sampling).  SpMV
 * launches issued after every pair of a tile had converged
 * (they find nothing to do) are dropped from the count.  Bits 8..15 of `on`
 * give a sampling period s (0 or 1 = every launch): only every s-th SpMV launch
 * is bracketed, so the events disturb the launch sequence less (a bracketed
 * launch cannot overlap its neighbours' start-up).  Enabling forces the
 * host-driven loop (no persistent kernel) so launches can be bracketed.
 */
int nvd_profile_enable(int32_t on);
int nvd_profile_read(int32_t kernel_class, int64_t *launches, double *total_ms,
                     double *bytes);

/* nvd_kernel_launches -- number of kernels this library has launched in the
 * process so far (all entry points, all devices). */
int64_t nvd_kernel_launches(void);

/* nvd_version -- library version string. */
const char *nvd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NVD_H_ */
