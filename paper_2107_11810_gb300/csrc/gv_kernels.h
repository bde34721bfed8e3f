// gv_kernels.h -- launch interface between the host engine and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gv_device.cuh"

namespace gv {

// Records of one level.  A record is one canonical surface in one cell, packed as
// NFP fields [q_f (ND), q_t (LE), padding]: 16-bit fields biased by 2^15 (two per
// 32-bit word) on levels whose value bounds allow it, plain 32-bit fields
// otherwise.  The records of a cell start at a multiple of 32 (a tile); a tile's
// owning cell is tile_cell[tile].  mult (originals merged into a record) is NULL
// when every multiplicity is 1 (no grouping): it is then neither stored nor read.
struct RecView {
    uint32_t *rec;           // packed records
    uint32_t *mult;          // [records] or NULL
    uint32_t *tile_cell;     // [records / 32] cell index (as stored in the level's cell arrays)
};

// Cells of one level: packed leaf-aligned key, first record (a multiple of 32),
// record count, UB.
struct CellView {
    uint64_t *key;
    uint64_t *rbeg;
    uint32_t *rcnt;
    uint32_t *ub;
};

// Device-resident scalars of one solve.
struct Scalars {
    unsigned int best_lb;            // largest lower bound seen
    unsigned int pad;
    unsigned long long best_key;     // (UB << coord_bits) | ~leaf key (max = best leaf)
    unsigned long long n_cells;      // cells written to the next level
    unsigned long long n_recs;       // record slots (32-aligned per cell) of the next level
    unsigned long long tests;        // predicate calls
    unsigned long long records;      // records tested
    unsigned long long rechecks;     // FP64 rechecks of the FP32 screen
    unsigned long long trace_n;      // trace entries
    unsigned long long replay_ub;    // replay: surfaces reaching the target cell
    unsigned long long replay_lb;    // replay: ... passing its lower-bound test
    unsigned int err;                // nonzero: input out of range
    unsigned int pad2;
    unsigned int qmax[GV_MAXD + GV_MAXT];  // lift: largest |q_f,j|, |q_t,m| of the root records
    unsigned long long rechecks_df;  // snaps the double-float tier decided (FP32 screen undecided)
};

struct Trace {
    unsigned long long cap;
    int32_t *level;
    uint64_t *key;
    uint32_t *ub, *lb;
};

// Everything one expansion step (a chunk of cells of one level) needs.
struct Chunk {
    Problem P;
    Level lev;
    CellView cells;          // cells of level l (key, ub: absolute index c0 + cl)
    int64_t c0;              // first cell of the chunk
    int nc;                  // number of cells in the chunk
    RecView in;              // records of the chunk (tile_cell values: in_c0 + cl)
    const uint64_t *in_rbeg; // first record of chunk cell cl at in_rbeg[in_c0 + cl]
    const uint32_t *in_rcnt; // its record count
    int64_t in_c0;
    int64_t t0, t1;          // tile range of the chunk
    uint8_t *alive;          // [nc]   cell still above the pruning threshold
    double *geo64;           // [nc][2^k][NB]          basis change per free child slot
    float *geo32;            // [nc][2^k * ND * LE + ND * LE + 1] screen coefficients G, max |G|, exponent
    float *geo32lo;          // [nc][2^k * ND * LE]   G64 - G rounded to FP32 (double-float tier)
    uint32_t *cnt;           // [nc][2^d][3]      UB, LB, records per child
    int2 *tinfo;             // [t1 - t0]         per tile: chunk-local cell (-1: pruned), valid lanes
    uint32_t *ballot;        // [t1 - t0][2^d]    per tile and child: UB-pass lanes
    unsigned long long *tdst;// [t1 - t0][2^d]    per tile and child: first output slot (~0: none)
    int32_t *child_idx;      // [nc][2^d]         index of the child cell or -1
    uint32_t *cursor;        // [nc][2^d]         next free record of the child
    CellView next_cells;     // cells of level l+1
    RecView out;             // records of level l+1
    Scalars *sc;
    Trace trace;
    int prune;
    int precision;           // 0 = FP64, 1 = FP32 screen + FP64 recheck
    unsigned spin;           // polls of a bounded wait for a bulk copy before giving up
};

// Size in floats of one cell's screen geometry: G[2^k][ND][LE], per (j, m) the
// largest |G| over the free slots (rounded up), and the cell's exactness exponent e
// (every G is FP32-exact and a multiple of 2^e; kNoExp when not).
__host__ __device__ constexpr int geo32_floats(int nfs, int nd, int le) { return nfs * nd * le + nd * le + 1; }
constexpr int kNoExp = -1000;

// Path geometry for replaying surfaces along the root-to-cell path.
struct PathStep {
    int slot;
    double dpsi[GV_MAXT];
};

void launch_lift(const Problem &P, const Level &lev0, const double *prm, int64_t n, RecView out, Scalars *sc,
                 cudaStream_t st);
void launch_cell_geo(const Chunk &c, cudaStream_t st);
// launch a persistent kernel taking one Chunk: one block per resident slot on the
// device, at most `groups` blocks, 256 threads, smem bytes of dynamic shared memory
void launch_persistent(const void *kern, size_t smem, int64_t groups, const Chunk &c, cudaStream_t st);
// per tile of the chunk: tinfo (after k_cell_geo has set alive)
void launch_tile_info(const Chunk &c, cudaStream_t st);
void launch_count(const Chunk &c, cudaStream_t st);
// the count and emit passes of families with 64 child slots (gv_wide.cu)
void launch_count_wide(const Chunk &c, cudaStream_t st);
bool launch_emit_wide(const Chunk &c, cudaStream_t st);
// after the children are laid out: the next level's tile -> cell table for cells
// [0, ncells) and every tile's output positions (tdst)
void launch_next_tiles(const Chunk &c, int64_t ncells, cudaStream_t st);
void launch_tile_dst(const Chunk &c, cudaStream_t st);
// false if the level's record formats have no emit pass (never chosen by the engine)
bool launch_emit(const Chunk &c, cudaStream_t st);
void launch_child_lbmax(const Chunk &c, cudaStream_t st);
// keepflag, recn: [nc * 2^d]; bsums: 2 * ceil(nc * 2^d / 256)
void launch_child_alloc(const Chunk &c, uint32_t *keepflag, uint32_t *recn, unsigned long long *bsums,
                        cudaStream_t st);
void launch_path_geo(const Problem &P, const Level *levs_dev, int lam, uint64_t key, PathStep *path,
                     cudaStream_t st);
void launch_replay(const Problem &P, const Level *levs_dev, const PathStep *path, int lam, const double *prm,
                   int64_t n, uint32_t *reach, Scalars *sc, cudaStream_t st);

// Grouping of a chunk's records (c.in, tiles [c.t0, c.t1), cells c.in_rbeg/in_rcnt)
// into out (cells indexed 0..nc-1 by chunk-local index): table [tmask + 1] zeroed;
// owner, newpos [32 (t1 - t0)]; ccount, ccur [nc] zeroed; grbeg [nc] receives the
// canonical records' first slots (32-aligned), ccount their counts; total[0] = slots
// used, total[1] = canonical records, total[2] = records that entered the grouping.
void launch_group(const Chunk &c, uint32_t *table, uint32_t tmask, uint32_t *owner, uint32_t *ccount,
                  uint32_t *ccur, uint32_t *newpos, uint64_t *grbeg, unsigned long long *total, RecView out,
                  cudaStream_t st);

// soft inlier score (gv_softscore.cu): forward writes out[0] = S; backward writes
// out[0..d) = grad_out * dS/dp and, if grad_prm, grad_out * dS/dparams [P][n].
// partial: softscore_partial_doubles() doubles of scratch.
void launch_softscore(int fam, bool bwd, const double *prm, int64_t n, const uint32_t *mask, const double *p,
                      const double *inv_tol2, int nd, const double *grad_out, double *grad_prm, double *partial,
                      double *out, cudaStream_t st);
int softscore_partial_doubles();
bool softscore_supported(int fam);

// words of one record of a family in the 16- or 32-bit format
__host__ __device__ constexpr int rec_words(int nfp, bool q16) { return q16 ? nfp / 2 : nfp; }

}  // namespace gv
