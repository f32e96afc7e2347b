// Shared host/device definitions of the GE-distance library (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nvd {

constexpr int NT = 256;          // threads per CTA for every work kernel
constexpr int NWARP = NT / 32;

// Work decomposition of the SpMV/SpMM for KT right-hand sides with vector/accumulator
// element sizes szv/sza (shared by the host planner and the kernels).
//   Light rows (at most sp_row_max entries) are stored a second time in a sliced
//   layout: a slice holds sp_slice_rows rows (one per lane group of a warp), sorted
//   by length inside their block, with entry j of all its rows side by side, so one
//   warp load fetches entry j of every row and every lane of an arithmetic
//   instruction does useful work.
//   KT = 1: a row with more entries, up to sp_long_max, is a sub-item of its own for
//           a whole warp; longer rows are split into chunks of sp_chunk entries,
//           one warp each.
//   KT > 1: heavy rows are split into chunks of sp_chunk entries, one CTA each.
constexpr int sp_row_max(int KT, int szv) { return KT == 1 ? 128 : 32768 / (KT * szv); }
constexpr int sp_long_max(int KT) { return KT == 1 ? 8192 : 0; }
constexpr int sp_chunk(int KT, int szv) { return KT == 1 ? 4096 : 32768 / (KT * szv); }
// Rows (first to last) one single-column light SpMV block may span: its row sums
// are staged in shared memory by row so the row epilogue runs in row order.
constexpr int sp_span_max() { return 1024; }
// d^2 stop: the gap estimate takes the largest of the last d2_window ratios of
// consecutive d^2 increments (window and safety factor chosen on recorded CG
// traces of ER, BA, WS and SBM graphs of mean degree 2..32, paths and cycles).
constexpr int d2_window() { return 6; }
constexpr double d2_safety() { return 0.03; }
// Columns one lane owns (16-byte vectors where the row is that wide), lanes per
// row, and rows per slice (one row per lane group of a warp).
constexpr int sp_vec(int KT, int szv) { return KT * szv >= 16 ? 16 / szv : KT; }
constexpr int sp_lanes_per_row(int KT, int szv) { return KT / sp_vec(KT, szv); }
constexpr int sp_slice_rows(int KT, int szv) { return 32 / sp_lanes_per_row(KT, szv); }
// doubles of reduction scratch per CTA (KT = 1: every thread's partial of up to 4
// sums, added by one warp per sum)
constexpr int red_doubles(int KT) {
    return KT == 1 ? 4 * NT : (NWARP * 4 * KT) > 256 ? NWARP * 4 * KT : 256;
}
constexpr int vec_smem_bytes(int KT) { return (red_doubles(KT) + 4 * KT) * 8; }
// Stream plans of multi-column tiles (stream.cuh): light rows of at most
// 256 / H entries (longer slices would unbalance the warps of a block), heavy rows cut
// into chunks of 64 steps (64 * H entries), one warp each.  Tiles whose rows are 64 or
// 128 bytes (8 or 4 rows per slice, 512 bytes per step) can also gather with TMA.
constexpr int sp_row_max_stream(int KT, int szv) { return 256 / sp_slice_rows(KT, szv); }
constexpr int sp_chunk_stream(int KT, int szv) { return 64 * sp_slice_rows(KT, szv); }
constexpr bool tma_tile(int KT, int szv) { return KT > 1 && (KT * szv == 64 || KT * szv == 128); }

// Heavy sub-item of the Laplacian SpMV/SpMM (rows above the light-row limit; the
// light rows are in the sliced layout).
//   kind 2: one long row r0, entries [e0, e1), processed whole by a warp (KT = 1).
//   kind 1: entries [e0, e1) of a very long row r0 split over several sub-items
//           (merge-path style row splitting); this is chunk `hchunk` of `nchunk`;
//           its partial row sum goes to hsum[hbase + hchunk] and the chunk that
//           finishes last (counter hcount[hrow]) adds the chunks in chunk order,
//           applies the row epilogue and owns partial slot (n_blocks + hrow).
struct SpItem {
    int32_t r0, r1, kind, hrow;
    int64_t e0, e1;
    int32_t hbase, hchunk, nchunk, pad;
};
static_assert(sizeof(SpItem) == 48, "SpItem layout");

// A CTA block: a contiguous run of work inside one segment.
//   SpMV light blocks (pad = 0): slices [i0, i1) (rows r0 .. r0 + nr - 1 for one
//   column).  SpMV heavy blocks (pad = 1): sub-items [i0, i1).  Vector blocks:
//   rows [i0, i1).
struct Block {
    int64_t i0, i1;
    int32_t seg, pad;
    int32_t r0, nr;   // single-column light SpMV blocks: first row, rows spanned (<= sp_span_max)
};
static_assert(sizeof(Block) == 32, "Block layout");

// Where one user graph's pairs live: x, y, z of shape [k][n_o] already offset to
// the first column of the tile; the graph's nodes are internal nodes
// [base, base + n_o) and its segments [seg0, seg1).
struct Owner {
    const void *x, *y;
    void *z;
    int64_t base, ld;
    int32_t kc;        // valid columns of this tile (pairs beyond k are padding)
    int32_t seg0, seg1;
    int32_t idx;       // 1: x, y are int32 node ids, column j is e_x[j] - e_y[j]
};

// Everything a work kernel needs, passed by value.  Pointers whose element type
// depends on the solve precision are void* and cast by the kernel templates.
struct Ctx {
    // ---- graph (internal node order; components are contiguous node ranges)
    int64_t n;
    const int64_t *rowptr;
    const int32_t *colidx;   // padded to a multiple of 4 entries
    const void *w;           // TW, padded like colidx
    const double *deg64, *dinv64;
    const float *deg32, *dinv32;
    // ---- segments = connected components with >= 2 nodes
    int32_t nseg;
    const int64_t *seg_begin, *seg_end;
    const int32_t *seg_owner;
    // ---- SpMV work decomposition
    const SpItem *items;
    const Block *sblk;              // [n_sblk]
    int64_t n_sblk;
    const int32_t *seg_sblk_off;    // [nseg+1]
    const int32_t *seg_heavy_off;   // [nseg+1] heavy (split) rows of each segment
    int32_t *hcount;                // [n_heavy] chunk arrival counters (self-resetting)
    double *hsum;                   // [n_chunks][KT] partial row sums of split rows
    // ---- vector-pass work decomposition
    const Block *vblk;              // [n_vblk]
    int64_t n_vblk;
    const int32_t *seg_vblk_off;    // [nseg+1]
    // ---- deterministic two-level reductions
    double *part;                   // [ND][part_stride][KT]
    int64_t part_stride;            // >= max(n_sblk + n_heavy, n_vblk)
    unsigned *counter;              // [nseg] arrival counters (self-resetting)
    double *gpart;                  // [ND][part_stride][KT] sums of slot groups, at each group's first slot
    unsigned *gcount;               // [part_stride] group arrival counters, at each group's first slot (self-resetting)
    // ---- per (segment, column) scalar state, [nseg][KT]
    double *rho, *rr, *rr0, *alpha, *beta, *mean, *meanx, *d2, *dz, *zr;
    double *hs_sum, *hs_hist;       // d^2 stop: sum of alpha_k rho_k; [nseg*KT][d2_window] last terms
    int32_t *active, *iters, *status;
    int32_t *n_active;              // number of (segment, column) pairs still iterating
    int32_t *err;                   // sticky device error code (a bounded wait that gave up)
    double rtol2;
    double d2stop;                  // > 0: also stop when the estimated d^2 error <= d2stop * d^2
    int32_t max_iter;
    // ---- sources and destinations: one "owner" per user graph (one for single-graph
    //      solves, passed inline in own0; G for batched solves, in the owners table)
    const struct Owner *owners;     // [n_owner] device table, or NULL = use own0
    int32_t n_owner;
    const int32_t *perm;            // internal -> user node (NULL = identity)
    // ---- sliced copy of the light rows: slice s holds H = sp_slice_rows rows
    //      sl_row[s*H + r] (-1 = empty lane group); entry j of row r sits at
    //      sl_base[s] + j*H + r of sl_col / sl_w (TW); rows shorter than the slice's
    //      longest are padded with zero weights on their own column
    const int64_t *sl_base;         // [n_slices + 1]
    const int32_t *sl_row;          // [n_slices * H]
    const int32_t *sl_col;
    const void *sl_w;
    int32_t sl_h;                   // H of the plan the pointers above belong to
    int32_t sl_stream;              // 1: stream plan (stream.cuh): sl_* hold every warp's steps
    int32_t sl_tma;                 // stream plan engine: 1 TMA gathers, 2 per-lane asynchronous copies (tma.cuh)
    const int32_t *sl_wsplit;       // [n_sblk][NWARP + 1] first slice of each warp, relative to the block's
    const longlong2 *sl_wrun;       // stream plans: [n_sblk][NWARP] {first entry, steps} of each warp
    // ---- L2 residency of the gathered vector's hot rows (degree-ordered graphs)
    int64_t hot_begin, hot_rows;    // rows [hot_begin, hot_begin + hot_rows) of the gathered vector
    int32_t l2_hot;                 // 1: multi-column SpMMs keep those rows persisting in L2
    // ---- persistent-kernel grid barrier
    unsigned *bar_count, *bar_gen;
    int32_t bar_extra;              // arrivals awaited beyond the grid (0; 1 only to test the timeout)
    Owner own0;
};

// Per (owner, column) result collected at the end of a tile.
struct ColResult {
    double d2;
    double rr;
    double rr0;
    int32_t iters;
    int32_t status;
};

// Buffers of one persistent (single-launch) tile solve.
struct PersistArgs {
    double *delta;
    void *x, *r, *p, *q;
    void *u;             // D^-1 r (stored by the update phase)
    int fold;            // 1: two phases per iteration (direction folded into the SpMV), 0: three
    ColResult *res;      // [n_owner][KT]
    int n_owner;
    int write_z;
};

}  // namespace nvd
