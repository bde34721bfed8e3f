// gv_kernels.h -- launch interface between the host engine and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gv_device.cuh"

namespace gv {

// Records of one level, structure of arrays.  A record is one canonical surface
// in one cell: q_f (free parameter, multiple of s_f), q_t (essential parameters,
// multiples of the level's s_t), mult (originals merged into it), cell (index of
// its cell in the level's cell arrays).  mult is NULL when every multiplicity
// is 1 (no grouping): it is then neither stored nor read.
struct RecView {
    int32_t *qf[GV_MAXD];
    int32_t *qt[GV_MAXT];
    uint32_t *mult;
    uint32_t *cell;
};

// Cells of one level: packed leaf-aligned key, first record, record count, UB.
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
    unsigned long long n_recs;       // records written to the next level
    unsigned long long tests;        // predicate calls
    unsigned long long rechecks;     // FP64 rechecks of the FP32 screen
    unsigned long long trace_n;      // trace entries
    unsigned long long replay_ub;    // replay: surfaces reaching the target cell
    unsigned long long replay_lb;    // replay: ... passing its lower-bound test
    unsigned int err;                // nonzero: input out of range
    unsigned int pad2;
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
    CellView cells;          // cells of level l
    int64_t c0;              // first cell of the chunk
    int nc;                  // number of cells in the chunk
    RecView in;              // records of level l
    int64_t r0, r1;          // record range of the chunk
    uint8_t *alive;          // [nc]   cell still above the pruning threshold
    double *geo64;           // [nc][2^d][NB]     basis change per child
    float *geo32;            // [nc][2^d + 1][NB] FP32 copy + max |.| over children
    uint32_t *cnt;           // [nc][2^d][3]      UB, LB, records per child
    uint8_t *passmask;       // [r1 - r0]         children whose UB test passed
    int32_t *child_idx;      // [nc][2^d]         index of the child cell or -1
    uint32_t *cursor;        // [nc][2^d]         next free record of the child
    CellView next_cells;     // cells of level l+1
    RecView out;             // records of level l+1
    Scalars *sc;
    Trace trace;
    int prune;
    int precision;           // 0 = FP64, 1 = FP32 screen + FP64 recheck
};

// Path geometry for replaying surfaces along the root-to-cell path.
struct PathStep {
    int slot;
    double dpsi[GV_MAXT];
};

void launch_lift(const Problem &P, const Level &lev0, const double *prm, int64_t n, RecView out, Scalars *sc,
                 cudaStream_t st);
void launch_cell_geo(const Chunk &c, cudaStream_t st);
void launch_test(const Chunk &c, bool emit, cudaStream_t st);
void launch_child_lbmax(const Chunk &c, cudaStream_t st);
// two levels per record read: c = level-l chunk, c1 = its level-(l+1) children
// (pm2: grandchild pass masks, [r1 - r0][2^d] bytes)
void launch_test2(const Chunk &c, const Chunk &c1, bool emit, const uint8_t *pm2_in, uint8_t *pm2_out,
                  cudaStream_t st);
// keepflag, recn: [nc * 2^d]; bsums: 2 * ceil(nc * 2^d / 256)
void launch_child_alloc(const Chunk &c, uint32_t *keepflag, uint32_t *recn, unsigned long long *bsums,
                        cudaStream_t st);
void launch_path_geo(const Problem &P, const Level *levs_dev, int lam, uint64_t key, PathStep *path,
                     cudaStream_t st);
void launch_replay(const Problem &P, const Level *levs_dev, const PathStep *path, int lam, const double *prm,
                   int64_t n, uint32_t *reach, Scalars *sc, cudaStream_t st);

// grouping of a chunk's records [r0, r0 + nr) (cells [c0, c0 + nc)) into out:
// table [tmask + 1] zeroed; ccount, ccur [nc] zeroed; owner, newpos [nr];
// *total = number of canonical records
void launch_group(const Problem &P, RecView in, int64_t r0, int64_t nr, int64_t c0, int nc, uint32_t *table,
                  uint32_t tmask, uint32_t *owner, uint32_t *ccount, uint32_t *ccur, uint32_t *newpos,
                  unsigned long long *total, RecView out, Scalars *sc, cudaStream_t st);

// soft inlier score (gv_softscore.cu): forward writes out[0] = S; backward writes
// out[0..d) = grad_out * dS/dp and, if grad_prm, grad_out * dS/dparams [P][n].
// partial: softscore_partial_doubles() doubles of scratch.
void launch_softscore(int fam, bool bwd, const double *prm, int64_t n, const uint32_t *mask, const double *p,
                      const double *inv_tol2, int nd, const double *grad_out, double *grad_prm, double *partial,
                      double *out, cudaStream_t st);
int softscore_partial_doubles();

}  // namespace gv
