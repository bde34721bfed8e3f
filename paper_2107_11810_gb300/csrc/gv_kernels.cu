// gv_kernels.cu -- kernels of the level-wise voting search (Algorithm 2 of
// arXiv 2107.11810 with canonization, Sec. 3.2, and B&B pruning, Sec. 3.3).
//
//   k_lift        root records of the original surfaces (Eq. 1 in the frame of the
//                 domain centre), snapped for level 0
//   k_cell_geo    per cell of a chunk: pruning re-check and the change of the
//                 family's basis functions from the cell centre to each child
//                 centre (own sin/cos, FP64)
//   (k_count, k_emit: the proximity test itself, in gv_count.cu and gv_emit.cu)
//   k_child_*     best lower bound, pruning, allocation of surviving children,
//                 leaf argmax as a packed 64-bit atomicMax
//   k_path_geo,   replay of every original surface along one root-to-cell path:
//   k_replay      inlier mask of the best leaf and per-cell counts
#include <cstdio>
#include <map>
#include <mutex>

#include "gv_tile.cuh"

namespace gv {

__device__ __forceinline__ unsigned prune_threshold(const Problem &P, const Scalars *sc, int prune) {
    if (!prune) return 1u;
    unsigned lb = *(volatile const unsigned *)&sc->best_lb;
    unsigned long long bk = *(volatile const unsigned long long *)&sc->best_key;
    unsigned leaf = (unsigned)(bk >> P.coord_bits);
    unsigned t = lb > leaf ? lb : leaf;
    return t > 1u ? t : 1u;
}

// ---------------------------------------------------------------------------
// A0 lift
// ---------------------------------------------------------------------------
template <int FAM>
__global__ void k_lift(Problem P, Level lev0, const double *__restrict__ prm, int64_t n, RecView out,
                       Scalars *sc) {
    using F = Fam<FAM>;
    constexpr int NW = rec_words(F::NFP, false);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    unsigned qa[F::ND + F::LE];
#pragma unroll
    for (int x = 0; x < F::ND + F::LE; ++x) qa[x] = 0u;
    bool bad = false;
    if (i < n) {
        double c[F::D], psi[F::NB], f[F::ND], t[F::LE];
#pragma unroll
        for (int j = 0; j < F::D; ++j) c[j] = cell_center(P, lev0.h, j, 0);
        F::basis(P, c, psi);
        F::lift(prm, n, i, c, psi, f, t);
        uint32_t w[NW];
#pragma unroll
        for (int x = 0; x < NW; ++x) w[x] = 0u;
#pragma unroll
        for (int j = 0; j < F::ND; ++j) {
            double q = rint(dmul(f[j], P.inv_s_f[j]));
            bad |= !(fabs(q) < 1073741824.0);
            int qi = bad ? 0 : (int)q;
            w[j] = (uint32_t)qi;
            qa[j] = (unsigned)abs(qi);
        }
#pragma unroll
        for (int m = 0; m < F::LE; ++m) {
            double q = rint(dmul(t[m], lev0.inv_s_t[m]));
            bad |= !(fabs(q) < 1073741824.0);
            int qi = bad ? 0 : (int)q;
            w[F::ND + m] = (uint32_t)qi;
            qa[F::ND + m] = (unsigned)abs(qi);
        }
        store_words<NW>(out.rec, i, w);
        if (out.mult) out.mult[i] = 1u;
        if ((i & 31) == 0) out.tile_cell[i >> 5] = 0u;
    }
    // largest |q| per field (it sets the screen's band and the record formats)
#pragma unroll
    for (int x = 0; x < F::ND + F::LE; ++x) {
        unsigned m = __reduce_max_sync(kFull, qa[x]);
        if (lane == 0 && m) atomicMax(&sc->qmax[x], m);
    }
    if (bad) atomicOr(&sc->err, 1u);
}

// ---------------------------------------------------------------------------
// A1 cell geometry: basis change from the parent centre to each child centre
// ---------------------------------------------------------------------------
template <int FAM>
__device__ __forceinline__ void child_dpsi(const Problem &P, const Level &lev, uint64_t key, int fs,
                                           const double *psi_par, double *dpsi) {
    using F = Fam<FAM>;
    if constexpr (F::LINEAR_BASIS) {
        // psi is the free coordinates themselves: their changes are the exact child shifts
#pragma unroll
        for (int m = 0; m < F::NB; ++m) {
            const bool split = (lev.split_mask >> m) & 1;
            dpsi[m] = split ? (((fs >> m) & 1) ? lev.h1[m] : -lev.h1[m]) : 0.0;
        }
        return;
    } else {
    double cch[F::D];
#pragma unroll
    for (int j = 0; j < F::K; ++j) {
        int64_t i = cell_coord(P, key, lev.l, j);
        bool split = (lev.split_mask >> j) & 1;
        int64_t ic = split ? 2 * i + ((fs >> j) & 1) : i;
        cch[j] = cell_center(P, lev.h1, j, ic);
    }
    double psi_ch[F::NB];
    F::basis(P, cch, psi_ch);
#pragma unroll
    for (int m = 0; m < F::NB; ++m) dpsi[m] = dsub(psi_ch[m], psi_par[m]);
    if constexpr (F::LINEAR_TAIL) {
        // the last basis value is the last free coordinate: its change is the exact shift
        constexpr int j = F::K - 1;
        const bool split = (lev.split_mask >> j) & 1;
        dpsi[F::NB - 1] = split ? (((fs >> j) & 1) ? lev.h1[j] : -lev.h1[j]) : 0.0;
    }
    }
}

template <int FAM>
__device__ __forceinline__ void parent_psi(const Problem &P, const Level &lev, uint64_t key, double *psi) {
    using F = Fam<FAM>;
    double cpar[F::D];
#pragma unroll
    for (int j = 0; j < F::K; ++j) cpar[j] = cell_center(P, lev.h, j, cell_coord(P, key, lev.l, j));
    if (!F::LINEAR_BASIS) F::basis(P, cpar, psi);
}

// One thread per (cell, free-coordinate child slot fs); the 2^k threads of a cell
// are consecutive lanes.  Writes the FP64 basis changes (for the exact recheck) and
// the screen's coefficients G[fs][j][m] = coef_jm(dpsi) * s_t,m / s_f,j rounded to
// FP32, their remainders (G64 - G, rounded to FP32: the double-float tier's low
// parts; G64 is exact, coef only copies or negates and s_t / s_f is a power of two),
// per (j, m) the largest |G| over the child slots (rounded up), which bounds the
// magnitudes the screen's band scales with, and the cell's exactness exponent: the
// least e with every G a multiple of 2^e (at most 0), or kNoExp when some G is not
// exactly an FP32 value.
template <int FAM>
__global__ void k_cell_geo(Chunk c) {
    using F = Fam<FAM>;
    constexpr int NF = 1 << F::K;
    constexpr int GF = geo32_floats(NF, F::ND, F::LE);
    static_assert(32 % NF == 0, "a cell's threads must lie in one warp");
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int cell = gid / NF, fs = gid % NF;
    const bool in = cell < c.nc;
    const Problem &P = c.P;
    const Level &lev = c.lev;
    float ga[F::ND * F::LE];
#pragma unroll
    for (int x = 0; x < F::ND * F::LE; ++x) ga[x] = 0.0f;
    int ge = 0;                                      // exactness exponent (<= 0) of this thread's G
    if (in) {
        if (fs == 0) {
            unsigned thr = prune_threshold(P, c.sc, c.prune);
            c.alive[cell] = c.cells.ub[c.c0 + cell] >= thr ? 1 : 0;
        }
        double dpsi[F::NB];
#pragma unroll
        for (int m = 0; m < F::NB; ++m) dpsi[m] = 0.0;
        if (!(fs & ~lev.split_mask & (NF - 1))) {
            uint64_t key = c.cells.key[c.c0 + cell];
            double psi_par[F::NB];
            parent_psi<FAM>(P, lev, key, psi_par);
            child_dpsi<FAM>(P, lev, key, fs, psi_par, dpsi);
        }
#pragma unroll
        for (int m = 0; m < F::NB; ++m) c.geo64[((size_t)cell * NF + fs) * F::NB + m] = dpsi[m];
        double g[F::ND * F::LE];
        F::coef(dpsi, g);
#pragma unroll
        for (int x = 0; x < F::ND * F::LE; ++x) {
            const double gx = g[x] * lev.gscale[x / F::LE][x % F::LE];
            const float gh = (float)gx;
            c.geo32[(size_t)cell * GF + fs * F::ND * F::LE + x] = gh;
            c.geo32lo[((size_t)cell * NF + fs) * F::ND * F::LE + x] = (float)(gx - (double)gh);
            ga[x] = __double2float_ru(fabs(gx));
            if ((double)gh != gx) ge = kNoExp;
            else if (gx != 0.0 && ge > kNoExp) ge = min(ge, lowbit_exp(gx));
        }
    }
#pragma unroll
    for (int o = 1; o < NF; o <<= 1) {
#pragma unroll
        for (int x = 0; x < F::ND * F::LE; ++x) ga[x] = fmaxf(ga[x], __shfl_xor_sync(kFull, ga[x], o));
        ge = min(ge, __shfl_xor_sync(kFull, ge, o));
    }
    if (in && fs == 0) {
#pragma unroll
        for (int x = 0; x < F::ND * F::LE; ++x) c.geo32[(size_t)cell * GF + NF * F::ND * F::LE + x] = ga[x];
        c.geo32[(size_t)cell * GF + GF - 1] = (float)ge;
    }
}

// Block-wide exclusive scan of one 64-bit value per thread (blockDim = 256).
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long *total) {
    __shared__ unsigned long long warp_tot[8];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = lane < 8 ? warp_tot[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            unsigned long long y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < 8) warp_tot[lane] = t;   // inclusive warp prefix
    }
    __syncthreads();
    unsigned long long before = w ? warp_tot[w - 1] : 0ull;
    *total = warp_tot[7];
    __syncthreads();
    return before + x - v;
}

// ---------------------------------------------------------------------------
// A5 best lower bound, pruning, allocation of surviving children, leaf argmax
// ---------------------------------------------------------------------------
template <int NS>
__global__ void k_child_lbmax(Chunk c) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int cl = idx / NS, s = idx % NS;
    unsigned v = 0;
    if (cl < c.nc && !(s & ~c.lev.split_mask) && c.alive[cl]) v = c.cnt[(size_t)idx * 3 + 1];
    v = __reduce_max_sync(kFull, v);
    if ((threadIdx.x & 31) == 0 && v) atomicMax(&c.sc->best_lb, v);
}

// Phase A: per child of the chunk -- trace, pruning decision, leaf argmax, and
// per-block totals of surviving children and their records.
template <int NS>
__global__ void __launch_bounds__(256) k_child_mark(Chunk c, uint32_t *keepflag, uint32_t *recn,
                                                    unsigned long long *bs_cells, unsigned long long *bs_recs) {
    const Problem &P = c.P;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int cl = idx / NS, s = idx % NS;
    bool exists = cl < c.nc && !(s & ~c.lev.split_mask) && c.alive[cl];
    unsigned ub = 0, lb = 0, nrec = 0;
    uint64_t key = 0;
    if (exists) {
        ub = c.cnt[(size_t)idx * 3];
        lb = c.cnt[(size_t)idx * 3 + 1];
        nrec = c.cnt[(size_t)idx * 3 + 2];
        key = child_key(P, c.cells.key[c.c0 + cl], c.lev.l, s);
        if (c.trace.cap) {
            unsigned long long t = atomicAdd(&c.sc->trace_n, 1ull);
            if (t < c.trace.cap) {
                c.trace.level[t] = c.lev.l + 1;
                c.trace.key[t] = key;
                c.trace.ub[t] = ub;
                c.trace.lb[t] = lb;
            }
        }
    }
    unsigned thr = prune_threshold(P, c.sc, c.prune);
    bool keep = exists && ub >= thr;
    if (c.lev.leaf_children) {
        if (keep) {
            unsigned long long kmask = (1ull << P.coord_bits) - 1ull;
            unsigned long long cand = ((unsigned long long)ub << P.coord_bits) | (~key & kmask);
            atomicMax(&c.sc->best_key, cand);
        }
        return;
    }
    // a child's records start at a multiple of 32 (whole tiles)
    const unsigned slots = keep ? (nrec + 31u) & ~31u : 0u;
    if (idx < c.nc * NS) {
        keepflag[idx] = keep ? 1u : 0u;
        recn[idx] = slots;
    }
    unsigned long long tc, tr;
    block_excl_scan(keep ? 1ull : 0ull, &tc);
    block_excl_scan((unsigned long long)slots, &tr);
    if (threadIdx.x == 0) {
        bs_cells[blockIdx.x] = tc;
        bs_recs[blockIdx.x] = tr;
    }
}

// Phase B: exclusive scan of the per-block totals (one block of 256 threads).
__global__ void __launch_bounds__(256) k_scan_sums(unsigned long long *a, unsigned long long *b, int nb, Scalars *sc) {
    unsigned long long ca = 0, cb = 0;
    for (int base = 0; base < nb; base += 256) {
        int i = base + threadIdx.x;
        unsigned long long va = i < nb ? a[i] : 0ull, vb = i < nb ? b[i] : 0ull;
        unsigned long long ta, tb;
        unsigned long long ea = block_excl_scan(va, &ta);
        unsigned long long eb = block_excl_scan(vb, &tb);
        if (i < nb) {
            a[i] = ca + ea;
            b[i] = cb + eb;
        }
        ca += ta;
        cb += tb;
    }
    if (threadIdx.x == 0) {
        sc->n_cells = ca;
        sc->n_recs = cb;
    }
}

// Phase C: surviving children get consecutive cell indices and record ranges in
// (parent, slot) order; recn holds the slots (record count rounded up to 32).
template <int NS>
__global__ void __launch_bounds__(256) k_child_write(Chunk c, const uint32_t *keepflag, const uint32_t *recn,
                                                     const unsigned long long *bs_cells,
                                                     const unsigned long long *bs_recs) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    bool in = idx < c.nc * NS;
    unsigned keep = in ? keepflag[idx] : 0u;
    unsigned nrec = in ? recn[idx] : 0u;
    unsigned long long tc, tr;
    unsigned long long ec = block_excl_scan(keep, &tc);
    unsigned long long er = block_excl_scan(nrec, &tr);
    if (!in) return;
    if (keep) {
        int cl = idx / NS, s = idx % NS;
        unsigned long long ci = bs_cells[blockIdx.x] + ec;
        c.next_cells.key[ci] = child_key(c.P, c.cells.key[c.c0 + cl], c.lev.l, s);
        c.next_cells.rbeg[ci] = bs_recs[blockIdx.x] + er;
        c.next_cells.rcnt[ci] = c.cnt[(size_t)idx * 3 + 2];
        c.next_cells.ub[ci] = c.cnt[(size_t)idx * 3];
        c.child_idx[idx] = (int32_t)ci;
    } else {
        c.child_idx[idx] = -1;
    }
}

// ---------------------------------------------------------------------------
// Per-tile bookkeeping of the proximity test, so that the count and emit passes
// stream their inputs with bulk copies and never chase a pointer per tile.
// ---------------------------------------------------------------------------

// per tile: the chunk-local cell (-1 if it was pruned) and how many of its 32 lanes
// hold records
__global__ void k_tile_info(Chunk c) {
    const int64_t t = c.t0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= c.t1) return;
    const int64_t cell = (int64_t)c.in.tile_cell[t];
    const int cl = (int)(cell - c.in_c0);
    const int64_t left = (int64_t)c.in_rbeg[cell] + (int64_t)c.in_rcnt[cell] - 32 * t;
    c.tinfo[t - c.t0] = make_int2(c.alive[cl] ? cl : -1, left < 32 ? (int)left : 32);
}

// the next level's tile -> cell table: one warp per new cell writes its tiles
__global__ void k_next_tiles(CellView next, RecView out, int64_t ncells) {
    const int64_t cell = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (cell >= ncells) return;
    const int64_t t0 = (int64_t)(next.rbeg[cell] >> 5), nt = ((int64_t)next.rcnt[cell] + 31) >> 5;
    for (int64_t i = lane; i < nt; i += 32) out.tile_cell[t0 + i] = (uint32_t)cell;
}

// Output positions of the emit pass.  A block takes 32 consecutive tiles;
// warp w handles child slots w, w + 8, ... with one lane per tile: a segmented scan over the
// tiles (segments = runs of one cell) gives every tile its offset inside the run,
// the run's last lane reserves the run's records in the child with one atomic on
// the child's cursor, and the run's base is broadcast back.  tdst[tile][s] = first
// slot of the tile's records in child s, or ~0 when the tile writes none there.
template <int NS>
__global__ void __launch_bounds__(256) k_tile_dst(Chunk c) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NWARP = NS < 8 ? NS : 8;
    if (w >= NWARP) return;
    const int64_t t = c.t0 + (int64_t)blockIdx.x * 32 + lane;
    const bool in = t < c.t1;
    const int cl = in ? c.tinfo[t - c.t0].x : -1;
    // segments: maximal runs of lanes with the same cell
    const int prev = __shfl_up_sync(kFull, cl, 1);
    const unsigned heads = __ballot_sync(kFull, lane == 0 || prev != cl);
    const int next = __shfl_down_sync(kFull, cl, 1);
    const unsigned tails = __ballot_sync(kFull, lane == 31 || next != cl);
    const int head = 31 - __clz(heads & ((2u << lane) - 1u));          // this lane's segment head
    const int tail = __ffs(tails & ~((1u << lane) - 1u)) - 1;          // this lane's segment tail
#pragma unroll 1
    for (int s = w; s < NS; s += NWARP) {
        unsigned n = 0;
        int ci = -1;
        if (cl >= 0) {
            ci = c.child_idx[(size_t)cl * NS + s];
            if (ci >= 0) n = __popc(c.ballot[(size_t)(t - c.t0) * NS + s]);
        }
        // inclusive scan of n inside the segment
        unsigned x = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(kFull, x, o);
            if (lane - o >= head) x += y;
        }
        unsigned long long base = 0;
        if (((tails >> lane) & 1) && cl >= 0 && ci >= 0 && x)
            base = c.next_cells.rbeg[ci] + atomicAdd(&c.cursor[(size_t)cl * NS + s], x);
        base = __shfl_sync(kFull, base, tail);
        if (in) c.tdst[(size_t)(t - c.t0) * NS + s] = n ? base + (x - n) : ~0ull;
    }
}

// ---------------------------------------------------------------------------
// A7 replay of the original surfaces along one root-to-cell path
// ---------------------------------------------------------------------------
template <int FAM>
__global__ void k_path_geo(Problem P, const Level *__restrict__ levs, int lam, uint64_t key, PathStep *path) {
    using F = Fam<FAM>;
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= lam) return;
    const Level &lev = levs[l];
    int slot = 0;
    for (int j = 0; j < F::D; ++j)
        if (l < P.Lj[j]) slot |= (int)(cell_coord(P, key, l + 1, j) & 1) << j;
    double psi_par[F::NB], dpsi[F::NB];
    parent_psi<FAM>(P, lev, key, psi_par);
    child_dpsi<FAM>(P, lev, key, slot & ((1 << F::K) - 1), psi_par, dpsi);
    path[l].slot = slot;
#pragma unroll
    for (int m = 0; m < F::NB; ++m) path[l].dpsi[m] = dpsi[m];
}

template <int FAM>
__global__ void __launch_bounds__(256) k_replay(Problem P, const Level *__restrict__ levs,
                                               const PathStep *__restrict__ path, int lam,
                                               const double *__restrict__ prm, int64_t n, uint32_t *reach,
                                               Scalars *sc) {
    using F = Fam<FAM>;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    bool reached = false, lbp = false;
    if (i < n) {
        double c[F::D], psi[F::NB], f[F::ND], t[F::LE];
#pragma unroll
        for (int j = 0; j < F::D; ++j) c[j] = cell_center(P, levs[0].h, j, 0);
        F::basis(P, c, psi);
        F::lift(prm, n, i, c, psi, f, t);
        reached = true;
        for (int l = 0; l < lam; ++l) {
            const Level &lev = levs[l];
#pragma unroll
            for (int j = 0; j < F::ND; ++j) f[j] = dmul(rint(dmul(f[j], P.inv_s_f[j])), P.s_f[j]);
#pragma unroll
            for (int m = 0; m < F::LE; ++m) t[m] = dmul(rint(dmul(t[m], lev.inv_s_t[m])), lev.s_t[m]);
            double R[F::ND], fo[F::ND];
            radius64<FAM>(lev, t, R);
            int res = test64<FAM>(lev, f, t, R, path[l].dpsi, path[l].slot, fo);
            if (!(res & 1)) {
                reached = false;
                break;
            }
            if (l == lam - 1) lbp = (res >> 1) & 1;
#pragma unroll
            for (int j = 0; j < F::ND; ++j) f[j] = fo[j];
        }
    }
    unsigned b = __ballot_sync(kFull, reached);
    unsigned bl = __ballot_sync(kFull, lbp);
    if (lane == 0 && i < n) {
        if (reach) reach[i >> 5] = b;
        if (b) atomicAdd(&sc->replay_ub, (unsigned long long)__popc(b));
        if (bl) atomicAdd(&sc->replay_lb, (unsigned long long)__popc(bl));
    }
}

// ---------------------------------------------------------------------------
// A3 grouping: merge records of a chunk with equal (cell, q_f, q_t) (the
// canonization's grouping, Sec. 3.2).  An open-addressing table of record
// indices: each record claims its home slot by atomicCAS of (its index + 1); a
// record that finds the slot taken compares its full key with the owner's
// (immutable) record and either adopts it or probes on.  Exact: different keys
// are never merged.  Canonical records are then laid out per cell (scan of
// per-cell counts) and their multiplicities summed with integer atomics, so the
// grouped records are deterministic up to their order inside a cell.
// ---------------------------------------------------------------------------
// A record slot of the chunk: its chunk-local cell, or -1 for the padding after a
// cell's last record.
__device__ __forceinline__ int slot_cell(const Chunk &c, int64_t r) {
    int64_t cell = (int64_t)c.in.tile_cell[r >> 5];
    int cl = (int)(cell - c.in_c0);
    return r < (int64_t)c.in_rbeg[cell] + (int64_t)c.in_rcnt[cell] ? cl : -1;
}

template <int NW>
__device__ __forceinline__ uint64_t key_hash(int cl, const uint32_t *w) {
    uint64_t h = 0x9E3779B97F4A7C15ull ^ (uint32_t)cl;
#pragma unroll
    for (int i = 0; i < NW; ++i) h = (h ^ w[i]) * 0xff51afd7ed558ccdull;
    return h ^ (h >> 29);
}

template <int FAM, bool Q16>
__global__ void k_group_insert(Chunk c, uint32_t *table, uint32_t tmask, uint32_t *owner, uint32_t *ccount) {
    constexpr int NW = rec_words(Fam<FAM>::NFP, Q16);
    const int64_t nr = (c.t1 - c.t0) * 32;
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nr) return;
    const int64_t r = c.t0 * 32 + x;
    const int cl = slot_cell(c, r);
    if (cl < 0) {
        owner[x] = 0xffffffffu;
        return;
    }
    uint32_t w[NW];
    load_words<NW>(c.in.rec, r, w);
    uint32_t slot = (uint32_t)key_hash<NW>(cl, w) & tmask;
    for (uint32_t probe = 0; probe <= tmask; ++probe) {
        uint32_t prev = atomicCAS(&table[slot], 0u, (uint32_t)(x + 1));
        if (prev == 0u) {                                   // new canonical record
            owner[x] = (uint32_t)x;
            atomicAdd(&ccount[cl], 1u);
            return;
        }
        const int64_t r2 = c.t0 * 32 + (int64_t)(prev - 1);
        bool same = slot_cell(c, r2) == cl;
        if (same) {
            uint32_t w2[NW];
            load_words<NW>(c.in.rec, r2, w2);
#pragma unroll
            for (int i = 0; i < NW; ++i) same &= w2[i] == w[i];
        }
        if (same) {
            owner[x] = prev - 1;
            return;
        }
        slot = (slot + 1) & tmask;
    }
    atomicOr(&c.sc->err, 4u);                               // table full (cannot happen at load <= 1/2)
    owner[x] = (uint32_t)x;
}

// exclusive scan of per-cell record counts rounded up to whole tiles (one block of
// 256 threads): start[i]; total[0] = slots used, total[1] = sum of cnt, total[2] =
// sum of in_cnt (the cells' record counts before grouping)
__global__ void __launch_bounds__(256) k_scan_slots(const uint32_t *cnt, const uint32_t *in_cnt, uint64_t *start,
                                                    int64_t n, unsigned long long *total) {
    unsigned long long carry = 0, recs = 0, recs_in = 0;
    for (int64_t base = 0; base < n; base += 256) {
        int64_t i = base + threadIdx.x;
        unsigned long long v = i < n ? (cnt[i] + 31u) & ~31u : 0u, t;
        unsigned long long e = block_excl_scan(v, &t);
        if (i < n) start[i] = carry + e;
        carry += t;
        if (i < n) {
            recs += cnt[i];
            recs_in += in_cnt[i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        recs += __shfl_xor_sync(0xffffffffu, recs, o);
        recs_in += __shfl_xor_sync(0xffffffffu, recs_in, o);
    }
    __shared__ unsigned long long s_r[8], s_ri[8];
    if ((threadIdx.x & 31) == 0) {
        s_r[threadIdx.x >> 5] = recs;
        s_ri[threadIdx.x >> 5] = recs_in;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0;
        for (int w = 0; w < 8; ++w) a += s_r[w], b += s_ri[w];
        total[0] = carry;
        total[1] = a;
        total[2] = b;
    }
}

template <int FAM, bool Q16>
__global__ void k_group_place(Chunk c, const uint32_t *owner, const uint64_t *grbeg, uint32_t *ccur,
                              uint32_t *newpos, RecView out) {
    constexpr int NW = rec_words(Fam<FAM>::NFP, Q16);
    const int64_t nr = (c.t1 - c.t0) * 32;
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nr || owner[x] != (uint32_t)x) return;
    const int64_t r = c.t0 * 32 + x;
    const int cl = slot_cell(c, r);
    const uint64_t pos = grbeg[cl] + atomicAdd(&ccur[cl], 1u);
    newpos[x] = (uint32_t)pos;
    uint32_t w[NW];
    load_words<NW>(c.in.rec, r, w);
    store_words<NW>(out.rec, (int64_t)pos, w);
    out.mult[pos] = 0u;
    if ((pos & 31u) == 0) out.tile_cell[pos >> 5] = (uint32_t)cl;
}

__global__ void k_group_mult(Chunk c, const uint32_t *owner, const uint32_t *newpos, RecView out) {
    const int64_t nr = (c.t1 - c.t0) * 32;
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nr || owner[x] == 0xffffffffu) return;
    atomicAdd(&out.mult[newpos[owner[x]]], c.in.mult ? c.in.mult[c.t0 * 32 + x] : 1u);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

#define GV_DISPATCH(fam, CALL)                                      \
    switch (fam) {                                                  \
    case FAM_LINE2D: { constexpr int FAMV = FAM_LINE2D; CALL; } break;           \
    case FAM_PLANE3D_SPH: { constexpr int FAMV = FAM_PLANE3D_SPH; CALL; } break; \
    case FAM_POSE3DOF: { constexpr int FAMV = FAM_POSE3DOF; CALL; } break;       \
    case FAM_RAYS3D: { constexpr int FAMV = FAM_RAYS3D; CALL; } break;           \
    case FAM_POSE6DOF: { constexpr int FAMV = FAM_POSE6DOF; CALL; } break;       \
    case FAM_POINTSET2D: { constexpr int FAMV = FAM_POINTSET2D; CALL; } break;   \
    case FAM_AFFINE4D: { constexpr int FAMV = FAM_AFFINE4D; CALL; } break;       \
    case FAM_RADIAL5DOF: { constexpr int FAMV = FAM_RADIAL5DOF; CALL; } break;   \
    default: break;                                                 \
    }

void launch_lift(const Problem &P, const Level &lev0, const double *prm, int64_t n, RecView out, Scalars *sc,
                 cudaStream_t st) {
    if (n <= 0) return;
    GV_DISPATCH(P.fam, (k_lift<FAMV><<<blocks_for(n, 256), 256, 0, st>>>(P, lev0, prm, n, out, sc)));
}

void launch_cell_geo(const Chunk &c, cudaStream_t st) {
    if (c.nc <= 0) return;
    GV_DISPATCH(c.P.fam, (k_cell_geo<FAMV><<<blocks_for((int64_t)c.nc << Fam<FAMV>::K, 64), 64, 0, st>>>(c)));
}

// Persistent grid: as many blocks as fit on the device at once (the kernel's
// occupancy at its shared memory), at most one per group.  The occupancy of each
// kernel is looked up once.
void launch_persistent(const void *kern, size_t smem, int64_t groups, const Chunk &c, cudaStream_t st) {
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> occ;
    static int sms = 0;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (sms <= 0) sms = 1;
        }
        auto it = occ.find({kern, smem});
        if (it == occ.end()) {
            if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess || per_sm < 1)
                per_sm = 1;
            occ[{kern, smem}] = per_sm;
        } else {
            per_sm = it->second;
        }
    }
    int64_t g = (int64_t)sms * per_sm;
    if (g > groups) g = groups;
    void *args[] = {(void *)&c};
    cudaLaunchKernel(kern, dim3((unsigned)g), dim3(256), args, smem, st);
}

void launch_tile_info(const Chunk &c, cudaStream_t st) {
    const int64_t nt = c.t1 - c.t0;
    if (nt > 0) k_tile_info<<<blocks_for(nt, 256), 256, 0, st>>>(c);
}

void launch_next_tiles(const Chunk &c, int64_t ncells, cudaStream_t st) {
    if (ncells > 0) k_next_tiles<<<blocks_for(ncells * 32, 256), 256, 0, st>>>(c.next_cells, c.out, ncells);
}

void launch_tile_dst(const Chunk &c, cudaStream_t st) {
    const int64_t nt = c.t1 - c.t0;
    if (nt <= 0) return;
    const int ns = 1 << c.P.d;
    if (ns == 4) k_tile_dst<4><<<blocks_for(nt, 32), 32 * 4, 0, st>>>(c);
    else if (ns == 8) k_tile_dst<8><<<blocks_for(nt, 32), 32 * 8, 0, st>>>(c);
    else if (ns == 16) k_tile_dst<16><<<blocks_for(nt, 32), 32 * 8, 0, st>>>(c);
    else if (ns == 32) k_tile_dst<32><<<blocks_for(nt, 32), 32 * 8, 0, st>>>(c);
    else k_tile_dst<64><<<blocks_for(nt, 32), 32 * 8, 0, st>>>(c);
}

void launch_child_lbmax(const Chunk &c, cudaStream_t st) {
    int ns = 1 << c.P.d;
    int64_t n = (int64_t)c.nc * ns;
    if (n <= 0) return;
    if (ns == 4) k_child_lbmax<4><<<blocks_for(n, 256), 256, 0, st>>>(c);
    else if (ns == 8) k_child_lbmax<8><<<blocks_for(n, 256), 256, 0, st>>>(c);
    else if (ns == 16) k_child_lbmax<16><<<blocks_for(n, 256), 256, 0, st>>>(c);
    else if (ns == 32) k_child_lbmax<32><<<blocks_for(n, 256), 256, 0, st>>>(c);
    else k_child_lbmax<64><<<blocks_for(n, 256), 256, 0, st>>>(c);
}

void launch_child_alloc(const Chunk &c, uint32_t *keepflag, uint32_t *recn, unsigned long long *bsums,
                        cudaStream_t st) {
    int ns = 1 << c.P.d;
    int64_t n = (int64_t)c.nc * ns;
    if (n <= 0) return;
    unsigned nb = blocks_for(n, 256);
    unsigned long long *ba = bsums, *bb = bsums + nb;
    if (ns == 4) k_child_mark<4><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else if (ns == 8) k_child_mark<8><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else if (ns == 16) k_child_mark<16><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else if (ns == 32) k_child_mark<32><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else k_child_mark<64><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    if (c.lev.leaf_children) return;
    k_scan_sums<<<1, 256, 0, st>>>(ba, bb, (int)nb, c.sc);
    if (ns == 4) k_child_write<4><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else if (ns == 8) k_child_write<8><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else if (ns == 16) k_child_write<16><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else if (ns == 32) k_child_write<32><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else k_child_write<64><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
}

void launch_group(const Chunk &c, uint32_t *table, uint32_t tmask, uint32_t *owner, uint32_t *ccount,
                  uint32_t *ccur, uint32_t *newpos, uint64_t *grbeg, unsigned long long *total, RecView out,
                  cudaStream_t st) {
    const int64_t nr = (c.t1 - c.t0) * 32;
    if (nr <= 0) return;
    unsigned g = blocks_for(nr, 256);
    if (c.lev.q16) {
        GV_DISPATCH(c.P.fam, (k_group_insert<FAMV, true><<<g, 256, 0, st>>>(c, table, tmask, owner, ccount)));
    } else {
        GV_DISPATCH(c.P.fam, (k_group_insert<FAMV, false><<<g, 256, 0, st>>>(c, table, tmask, owner, ccount)));
    }
    k_scan_slots<<<1, 256, 0, st>>>(ccount, c.in_rcnt + c.in_c0, grbeg, c.nc, total);
    if (c.lev.q16) {
        GV_DISPATCH(c.P.fam, (k_group_place<FAMV, true><<<g, 256, 0, st>>>(c, owner, grbeg, ccur, newpos, out)));
    } else {
        GV_DISPATCH(c.P.fam, (k_group_place<FAMV, false><<<g, 256, 0, st>>>(c, owner, grbeg, ccur, newpos, out)));
    }
    k_group_mult<<<g, 256, 0, st>>>(c, owner, newpos, out);
}

void launch_path_geo(const Problem &P, const Level *levs_dev, int lam, uint64_t key, PathStep *path,
                     cudaStream_t st) {
    if (lam <= 0) return;
    GV_DISPATCH(P.fam, (k_path_geo<FAMV><<<blocks_for(lam, 64), 64, 0, st>>>(P, levs_dev, lam, key, path)));
}

void launch_replay(const Problem &P, const Level *levs_dev, const PathStep *path, int lam, const double *prm,
                   int64_t n, uint32_t *reach, Scalars *sc, cudaStream_t st) {
    if (n <= 0) return;
    GV_DISPATCH(P.fam, (k_replay<FAMV><<<blocks_for(n, 256), 256, 0, st>>>(P, levs_dev, path, lam, prm, n,
                                                                            reach, sc)));
}

}  // namespace gv
