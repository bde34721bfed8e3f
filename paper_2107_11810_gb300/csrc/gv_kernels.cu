// gv_kernels.cu -- kernels of the level-wise voting search (Algorithm 2 of
// arXiv 2107.11810 with canonization, Sec. 3.2, and B&B pruning, Sec. 3.3).
//
//   k_lift        root records of the original surfaces (Eq. 1 in the frame of the
//                 domain centre), snapped for level 0
//   k_cell_geo    per cell of a chunk: pruning re-check and the change of the
//                 family's basis functions from the cell centre to each child
//                 centre (own sin/cos, FP64)
//   k_test        the cell x surface proximity test ("eps plus the cell radius"),
//                 count pass (UB / LB / record count per child, warp-reduced) and
//                 emit pass (child records, snapped for the next level)
//   k_child_*     best lower bound, pruning, allocation of surviving children,
//                 leaf argmax as a packed 64-bit atomicMax
//   k_path_geo,   replay of every original surface along one root-to-cell path:
//   k_replay      inlier mask of the best leaf and per-cell counts
#include <cstdio>

#include "gv_kernels.h"

namespace gv {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned prune_threshold(const Problem &P, const Scalars *sc, int prune) {
    if (!prune) return 1u;
    unsigned lb = *(volatile const unsigned *)&sc->best_lb;
    unsigned long long bk = *(volatile const unsigned long long *)&sc->best_key;
    unsigned leaf = (unsigned)(bk >> P.coord_bits);
    unsigned t = lb > leaf ? lb : leaf;
    return t > 1u ? t : 1u;
}

// round-half-even of q/2: re-snap of an essential parameter when the step doubles
__device__ __forceinline__ int32_t resnap_half(int32_t q) {
    int32_t k = q >> 1;
    return k + ((q & 1) & (k & 1));
}

// ---------------------------------------------------------------------------
// A0 lift
// ---------------------------------------------------------------------------
template <int FAM>
__global__ void k_lift(Problem P, Level lev0, const double *__restrict__ prm, int64_t n, RecView out,
                       Scalars *sc) {
    using F = Fam<FAM>;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double c[F::D], psi[F::NB], f[F::ND], t[F::LE];
#pragma unroll
    for (int j = 0; j < F::D; ++j) c[j] = cell_center(P, lev0.h, j, 0);
    F::basis(c, psi);
    F::lift(prm, n, i, c, psi, f, t);
    bool bad = false;
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        double q = rint(dmul(f[j], P.inv_s_f[j]));
        bad |= !(fabs(q) < 1073741824.0);
        out.qf[j][i] = bad ? 0 : (int32_t)q;
    }
#pragma unroll
    for (int m = 0; m < F::LE; ++m) {
        double q = rint(dmul(t[m], lev0.inv_s_t[m]));
        bad |= !(fabs(q) < 1073741824.0);
        out.qt[m][i] = bad ? 0 : (int32_t)q;
    }
    if (out.mult) out.mult[i] = 1u;
    out.cell[i] = 0u;
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
        // psi is the free coordinate itself: its change is the exact child shift
        bool split = (lev.split_mask >> 0) & 1;
        dpsi[0] = split ? ((fs & 1) ? lev.h1[0] : -lev.h1[0]) : 0.0;
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
    F::basis(cch, psi_ch);
#pragma unroll
    for (int m = 0; m < F::NB; ++m) dpsi[m] = dsub(psi_ch[m], psi_par[m]);
    }
}

template <int FAM>
__device__ __forceinline__ void parent_psi(const Problem &P, const Level &lev, uint64_t key, double *psi) {
    using F = Fam<FAM>;
    double cpar[F::D];
#pragma unroll
    for (int j = 0; j < F::K; ++j) cpar[j] = cell_center(P, lev.h, j, cell_coord(P, key, lev.l, j));
    if (!F::LINEAR_BASIS) F::basis(cpar, psi);
}

// One thread per (cell, free-coordinate child slot fs); the 2^k threads of a cell
// are consecutive lanes and combine their max |dpsi| by shuffles.
template <int FAM>
__global__ void k_cell_geo(Chunk c) {
    using F = Fam<FAM>;
    constexpr int NS = 1 << F::D;
    constexpr int NF = 1 << F::K;
    static_assert(32 % NF == 0, "a cell's threads must lie in one warp");
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int cell = gid / NF, fs = gid % NF;
    const bool in = cell < c.nc;
    const Problem &P = c.P;
    const Level &lev = c.lev;
    float mx[F::NB];
#pragma unroll
    for (int m = 0; m < F::NB; ++m) mx[m] = 0.0f;
    if (in) {
        if (fs == 0) {
            unsigned thr = prune_threshold(P, c.sc, c.prune);
            c.alive[cell] = c.cells.ub[c.c0 + cell] >= thr ? 1 : 0;
        }
        if (!(fs & ~lev.split_mask & (NF - 1))) {
            uint64_t key = c.cells.key[c.c0 + cell];
            double psi_par[F::NB];
            parent_psi<FAM>(P, lev, key, psi_par);
            double dpsi[F::NB];
            child_dpsi<FAM>(P, lev, key, fs, psi_par, dpsi);
            for (int s = fs; s < NS; s += NF) {          // dependent-coordinate bits share psi
                if (s & ~lev.split_mask) continue;
#pragma unroll
                for (int m = 0; m < F::NB; ++m) {
                    c.geo64[((size_t)cell * NS + s) * F::NB + m] = dpsi[m];
                    c.geo32[((size_t)cell * (NS + 1) + s) * F::NB + m] = (float)dpsi[m];
                }
            }
#pragma unroll
            for (int m = 0; m < F::NB; ++m) mx[m] = fabsf((float)dpsi[m]);
        }
    }
#pragma unroll
    for (int o = 1; o < NF; o <<= 1)
#pragma unroll
        for (int m = 0; m < F::NB; ++m) mx[m] = fmaxf(mx[m], __shfl_xor_sync(kFull, mx[m], o));
    if (in && fs == 0)
#pragma unroll
        for (int m = 0; m < F::NB; ++m) c.geo32[((size_t)cell * (NS + 1) + NS) * F::NB + m] = mx[m];
}

// ---------------------------------------------------------------------------
// A4 proximity test (count pass and emit pass) and A6 emission
// ---------------------------------------------------------------------------
template <int FAM>
__device__ __forceinline__ void shifts64(const Level &lev, int s, double *sh) {
    using F = Fam<FAM>;
#pragma unroll
    for (int j = 0; j < F::D; ++j) {
        bool split = (lev.split_mask >> j) & 1;
        sh[j] = split ? (((s >> j) & 1) ? lev.h1[j] : -lev.h1[j]) : 0.0;
    }
}

template <int FAM>
__device__ __forceinline__ void shifts32(const Level &lev, int s, float *sh) {
    using F = Fam<FAM>;
#pragma unroll
    for (int j = 0; j < F::D; ++j) {
        bool split = (lev.split_mask >> j) & 1;
        sh[j] = split ? (((s >> j) & 1) ? lev.h1f[j] : -lev.h1f[j]) : 0.0f;
    }
}

// FP64 upper-bound radius of a record (Lipschitz test): R_j = ((eps_j + h1_j) +
// sum_i lam_ji h1_i) + A1_j, in this order.
template <int FAM>
__device__ __forceinline__ void radius64(const Level &lev, const double *t, double *R) {
    using F = Fam<FAM>;
    double lam[F::ND * F::K];
    F::lipschitz64(t, lam);
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        double r = lev.Rbase[j];
#pragma unroll
        for (int i = 0; i < F::K; ++i) r = dadd(r, dmul(lam[j * F::K + i], lev.h1[i]));
        R[j] = dadd(r, lev.A1[j]);
    }
}

// exact FP64 test of one (record, child): bit 0 UB pass, bit 1 LB pass
template <int FAM>
__device__ __forceinline__ int test64(const Level &lev, const double *f, const double *t, const double *R,
                                      const double *dpsi, int s, double *fo) {
    using F = Fam<FAM>;
    double sh[F::D];
    shifts64<FAM>(lev, s, sh);
    F::residual64(f, t, dpsi, sh, fo);
    int ub = 1, lb = 1;
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        double a = fabs(fo[j]);
        ub &= a <= R[j];
        lb &= a <= lev.rlb[j];
    }
    return ub | (lb << 1);
}

// Bits 0-3 of x moved to bits 0, 8, 16, 24 (the four shifted copies of x do not
// overlap, so the product has no carries).
__device__ __forceinline__ unsigned spread4(unsigned x) { return (x * 0x00204081u) & 0x01010101u; }

// Lanes of a warp hold consecutive records and a cell's records are contiguous, so
// the lanes of one cell form one run of lanes.  Returns the calling lane's run (key:
// the lane's cell, or -1 for a lane without a record).
__device__ __forceinline__ unsigned run_mask(int key, int lane) {
    int prev = __shfl_up_sync(kFull, key, 1);
    unsigned heads = __ballot_sync(kFull, lane == 0 || prev != key);
    unsigned upto = lane == 31 ? kFull : ((2u << lane) - 1u);     // lanes 0..lane
    int start = 31 - __clz(heads & upto);
    unsigned after = heads & ~upto;
    unsigned below_end = after ? ((1u << (__ffs(after) - 1)) - 1u) : kFull;
    return below_end & ~((1u << start) - 1u);
}

// Child slots that exist at this level (slots that split only unsplit coordinates do not).
template <int NS>
__device__ __forceinline__ unsigned valid_slots(int smask) {
    unsigned v = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (!(s & ~smask)) v |= 1u << s;
    return v;
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

// Per-record state of the proximity test: the canonical record in FP32 (screen)
// and, on demand, in FP64 (exact definition).
template <int FAM, int PREC>
struct RecState {
    using F = Fam<FAM>;
    int32_t qf[F::ND], qt[F::LE];
    uint32_t mult;
    float f32[F::ND], t32[F::LE], R32[F::ND], Eub[F::ND], Elb[F::ND];
    double f64[F::ND], t64[F::LE], R64[F::ND];
    bool have64;

    __device__ __forceinline__ void load(const RecView &in, int64_t r) {
#pragma unroll
        for (int j = 0; j < F::ND; ++j) qf[j] = in.qf[j][r];
#pragma unroll
        for (int m = 0; m < F::LE; ++m) qt[m] = in.qt[m][r];
        mult = in.mult ? in.mult[r] : 1u;
        have64 = false;
    }
    __device__ __forceinline__ void set(const int32_t *qf_, const int32_t *qt_, uint32_t mult_) {
#pragma unroll
        for (int j = 0; j < F::ND; ++j) qf[j] = qf_[j];
#pragma unroll
        for (int m = 0; m < F::LE; ++m) qt[m] = qt_[m];
        mult = mult_;
        have64 = false;
    }
    __device__ __forceinline__ void need64(const Problem &P, const Level &lev) {
        if (have64) return;
#pragma unroll
        for (int j = 0; j < F::ND; ++j) f64[j] = dmul((double)qf[j], P.s_f[j]);
#pragma unroll
        for (int m = 0; m < F::LE; ++m) t64[m] = dmul((double)qt[m], lev.s_t[m]);
        radius64<FAM>(lev, t64, R64);
        have64 = true;
    }
    // FP32 values and the screen's error margins; gmax = max |dpsi| over children
    __device__ __forceinline__ void prep32(const Problem &P, const Level &lev, const float *gmax) {
#pragma unroll
        for (int j = 0; j < F::ND; ++j) f32[j] = (float)qf[j] * P.s_ff[j];
#pragma unroll
        for (int m = 0; m < F::LE; ++m) t32[m] = (float)qt[m] * lev.s_tf[m];
        float lam[F::ND * F::K];
        F::lipschitz32(t32, lam);
        float shmax[F::D], err[F::ND];
#pragma unroll
        for (int j = 0; j < F::D; ++j) shmax[j] = ((lev.split_mask >> j) & 1) ? lev.h1f[j] : 0.0f;
        F::errmag32(f32, t32, gmax, shmax, err);
#pragma unroll
        for (int j = 0; j < F::ND; ++j) {
            float rr = lev.Rbasef[j];
#pragma unroll
            for (int i = 0; i < F::K; ++i) rr = rr + lam[j * F::K + i] * lev.h1f[i];
            R32[j] = rr + lev.A1f[j];
            Eub[j] = kScreenRel * (err[j] + R32[j]);
            Elb[j] = kScreenRel * (err[j] + fabsf(lev.rlbf[j]));
        }
    }
};

// Signed shift of dependent coordinate j (index k + j) for child slot s.
template <int FAM>
__device__ __forceinline__ double dep_shift64(const Level &lev, int j, int s) {
    constexpr int K = Fam<FAM>::K;
    bool split = (lev.split_mask >> (K + j)) & 1;
    return split ? (((s >> (K + j)) & 1) ? lev.h1[K + j] : -lev.h1[K + j]) : 0.0;
}
template <int FAM>
__device__ __forceinline__ float dep_shift32(const Level &lev, int j, int s) {
    constexpr int K = Fam<FAM>::K;
    bool split = (lev.split_mask >> (K + j)) & 1;
    return split ? (((s >> (K + j)) & 1) ? lev.h1f[K + j] : -lev.h1f[K + j]) : 0.0f;
}

// UB/LB decisions of one record against every child.  g32 / g64: the cell's basis
// changes per child slot ([slot][NB]; slots that differ only in dependent bits share
// them).  Returns the UB-pass and LB-pass slot masks; counts FP64 rechecks.
template <int FAM, int PREC>
__device__ __forceinline__ void eval_record(const Problem &P, const Level &lev, RecState<FAM, PREC> &st,
                                            const float *g32, const double *g64, unsigned &ubm, unsigned &lbm,
                                            unsigned &nrechk) {
    using F = Fam<FAM>;
    constexpr int NS = 1 << F::D;
    constexpr int NF = 1 << F::K;
    const int smask = lev.split_mask;
    ubm = 0;
    lbm = 0;
    unsigned unsure = 0;
#pragma unroll
    for (int fs = 0; fs < NF; ++fs) {
        if (fs & ~smask) continue;
        if (PREC == 0) {
            double pr[F::ND];
            F::partial64(st.f64, st.t64, g64 + fs * F::NB, pr);
#pragma unroll
            for (int s = fs; s < NS; s += NF) {
                if (s & ~smask) continue;
                int ub = 1, lb = 1;
#pragma unroll
                for (int j = 0; j < F::ND; ++j) {
                    double a = fabs(dsub(pr[j], dep_shift64<FAM>(lev, j, s)));
                    ub &= a <= st.R64[j];
                    lb &= a <= lev.rlb[j];
                }
                ubm |= (unsigned)ub << s;
                lbm |= (unsigned)lb << s;
            }
        } else {
            float pr[F::ND];
            F::partial32(st.f32, st.t32, g32 + fs * F::NB, pr);
#pragma unroll
            for (int s = fs; s < NS; s += NF) {
                if (s & ~smask) continue;
                // pass bits from the signs of |f'| - R; a slot is uncertain when a
                // margin is within the screen's error bound (the UB test's, or the
                // LB test's when the UB test passes)
                bool ub = true, lb = true, bu = false, bl = false;
#pragma unroll
                for (int j = 0; j < F::ND; ++j) {
                    float a = fabsf(pr[j] - dep_shift32<FAM>(lev, j, s));
                    float du = a - st.R32[j], dl = a - lev.rlbf[j];
                    ub &= du < 0.0f;
                    lb &= dl < 0.0f;
                    bu |= fabsf(du) <= st.Eub[j];
                    bl |= fabsf(dl) <= st.Elb[j];
                }
                ubm |= (unsigned)ub << s;
                lbm |= (unsigned)(ub & lb) << s;
                unsure |= (unsigned)(bu | (ub & bl)) << s;
            }
        }
    }
    if (PREC == 1 && unsure) {
        // the FP32 screen could not decide these children: exact FP64 test (one
        // copy of the code, not unrolled)
        ubm &= ~unsure;
        lbm &= ~unsure;
        st.need64(P, lev);
#pragma unroll 1
        for (unsigned u = unsure; u; u &= u - 1) {
            int s = __ffs(u) - 1;
            ++nrechk;
            double pr[F::ND];
            F::partial64(st.f64, st.t64, g64 + (s & (NF - 1)) * F::NB, pr);
            int ub = 1, lb = 1;
#pragma unroll
            for (int j = 0; j < F::ND; ++j) {
                double a = fabs(dsub(pr[j], dep_shift64<FAM>(lev, j, s)));
                ub &= a <= st.R64[j];
                lb &= a <= lev.rlb[j];
            }
            ubm |= (unsigned)ub << s;
            lbm |= (unsigned)lb << s;
        }
    }
}

// Exact FP64 snap of one child residual, out of line: the FP32 screen needs it
// rarely, and one shared copy keeps the emit kernels' instruction footprint small.
// Everything is passed by value (no reference to kernel parameters).
struct Snap64In {
    int32_t qf[2], qt[3];
    double sf[2], st[3], inv[2], sh[2];
    const double *g64;   // basis changes of the child ([NB] doubles)
};

template <int FAM>
__device__ __noinline__ void snap64(Snap64In a, int32_t *qn, Scalars *sc) {
    using F = Fam<FAM>;
    double f[2], t[3], pr[2];
#pragma unroll
    for (int j = 0; j < F::ND; ++j) f[j] = dmul((double)a.qf[j], a.sf[j]);
#pragma unroll
    for (int m = 0; m < F::LE; ++m) t[m] = dmul((double)a.qt[m], a.st[m]);
    F::partial64(f, t, a.g64, pr);
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        double q = rint(dmul(dsub(pr[j], a.sh[j]), a.inv[j]));
        if (!(fabs(q) < 1073741824.0)) {
            atomicOr(&sc->err, 2u);
            q = 0.0;
        }
        qn[j] = (int32_t)q;
    }
}

// Snapped free parameters of the record's surface at the centre of child s.
template <int FAM, int PREC>
__device__ __forceinline__ void child_qf(const Problem &P, const Level &lev, RecState<FAM, PREC> &st,
                                         const float *g32, const double *g64, int s, int32_t *qn, unsigned &nrechk,
                                         Scalars *sc) {
    using F = Fam<FAM>;
    constexpr int NF = 1 << F::K;
    const int fs = s & (NF - 1);
    bool done = false;
    if (PREC == 1) {
        float pr[F::ND];
        F::partial32(st.f32, st.t32, g32 + fs * F::NB, pr);
        done = true;
#pragma unroll
        for (int j = 0; j < F::ND; ++j) {
            float y = (pr[j] - dep_shift32<FAM>(lev, j, s)) * P.inv_s_ff[j];
            float q = rintf(y);
            float margin = 0.5f - fabsf(y - q);
            if (margin > st.Eub[j] * P.inv_s_ff[j] && fabsf(q) < 1.6e7f) qn[j] = (int32_t)q;
            else done = false;
        }
        if (!done) ++nrechk;
    }
    if (!done) {
        Snap64In a;
#pragma unroll
        for (int j = 0; j < F::ND; ++j) {
            a.qf[j] = st.qf[j];
            a.sf[j] = P.s_f[j];
            a.inv[j] = P.inv_s_f[j];
            a.sh[j] = dep_shift64<FAM>(lev, j, s);
        }
#pragma unroll
        for (int m = 0; m < F::LE; ++m) {
            a.qt[m] = st.qt[m];
            a.st[m] = lev.s_t[m];
        }
        a.g64 = g64 + fs * F::NB;
        snap64<FAM>(a, qn, sc);
    }
}

template <int FAM, int PREC>
__device__ __forceinline__ void write_child(const Chunk &c, const RecState<FAM, PREC> &st, const int32_t *qn,
                                            int ci, uint64_t at) {
    using F = Fam<FAM>;
#pragma unroll
    for (int j = 0; j < F::ND; ++j) c.out.qf[j][at] = qn[j];
#pragma unroll
    for (int m = 0; m < F::LE; ++m) c.out.qt[m][at] = c.lev.st_ratio_log2[m] ? resnap_half(st.qt[m]) : st.qt[m];
    if (c.out.mult) c.out.mult[at] = st.mult;
    c.out.cell[at] = (uint32_t)ci;
}

// Tile shape of the proximity kernels: 4 records per thread in the count pass, 2 in
// the emit pass, at least 5 blocks of 256 threads per SM (48 registers).  Measured
// fastest on GB300 among 2-4 records per thread and 4-6 blocks per SM.
#ifndef GV_KRPT
#define GV_KRPT 4
#endif
#ifndef GV_MINBLOCKS
#define GV_MINBLOCKS 5
#endif
constexpr int kRPT = GV_KRPT;        // records per thread in one tile (count pass, two-level)
#ifndef GV_KRPT_EMIT
#define GV_KRPT_EMIT 2
#endif
constexpr int kRPTEmit = GV_KRPT_EMIT;  // records per thread in one tile (emit pass)
constexpr int kTile = 256 * kRPT;    // records per block
constexpr int kSpanCells = 64;       // tiles spanning at most this many cells count in shared memory

// Proximity test of a chunk's records against all children of their cells.
// Count pass (EMIT = false): per child UB = sum of mult over UB-passing records,
// LB likewise, and the number of passing records; per record the UB-pass mask.
// Emit pass (EMIT = true): every UB-passing record of a surviving child is
// written into the child's record range, snapped for the next level.
// A block takes a tile of kTile consecutive records.  Records are sorted by cell,
// so a tile whose first and last record share a cell lies in one cell: then the
// cell's geometry is staged in shared memory, counts are reduced in registers
// and across the block (one global atomic per counter), and the emit pass
// reserves the child ranges with one atomic per child and a block scan.  Tiles
// spanning several cells fall back to warp-level aggregation.
template <int FAM, int PREC, bool EMIT>
__global__ void __launch_bounds__(256, GV_MINBLOCKS) k_test(Chunk c) {
    using F = Fam<FAM>;
    constexpr int NS = 1 << F::D;
    constexpr int RPT = EMIT ? kRPTEmit : kRPT;   // records per thread (tuned per pass)
    constexpr int TILE = 256 * RPT;
    const Problem &P = c.P;
    const Level &lev = c.lev;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int smask = lev.split_mask;
    __shared__ float s_g32[(NS + 1) * F::NB];
    __shared__ double s_g64[NS * F::NB];
    __shared__ unsigned s_red[8][3 * NS];
    __shared__ int s_ci[NS];
    __shared__ unsigned long long s_base[NS];
    __shared__ unsigned s_span[kSpanCells * NS * 3];
    __shared__ unsigned s_xw[2 * NS];
    const int64_t t0 = c.r0 + (int64_t)blockIdx.x * TILE;
    const int64_t t1 = t0 + TILE < c.r1 ? t0 + TILE : c.r1;
    // This thread's records (and, in the emit pass, their pass masks) are loaded
    // first, so that their latency overlaps the tile's classification and the
    // staging of the cell's geometry.
    int32_t pqf[RPT][F::ND], pqt[RPT][F::LE];
    uint32_t pmult[RPT], ppm[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        int64_t r = t0 + threadIdx.x + k * 256;
        ppm[k] = 0;
        if (r < t1) {
#pragma unroll
            for (int j = 0; j < F::ND; ++j) pqf[k][j] = c.in.qf[j][r];
#pragma unroll
            for (int m = 0; m < F::LE; ++m) pqt[k][m] = c.in.qt[m][r];
            pmult[k] = c.in.mult ? c.in.mult[r] : 1u;
            if (EMIT) ppm[k] = c.passmask[r - c.r0];
        }
    }
    const int cfirst = (int)((int64_t)c.in.cell[t0] - c.c0);
    const int clast = (int)((int64_t)c.in.cell[t1 - 1] - c.c0);
    unsigned nrechk = 0, ntest = 0;
    if (cfirst == clast) {
        // ------------------------------ one cell ------------------------------
        const int cl = cfirst;
        if (!c.alive[cl]) return;                        // uniform: whole block exits
        for (int i = threadIdx.x; i < (NS + 1) * F::NB; i += blockDim.x)
            s_g32[i] = c.geo32[(size_t)cl * (NS + 1) * F::NB + i];
        for (int i = threadIdx.x; i < NS * F::NB; i += blockDim.x) s_g64[i] = c.geo64[(size_t)cl * NS * F::NB + i];
        if (EMIT && threadIdx.x < NS) s_ci[threadIdx.x] = c.child_idx[(size_t)cl * NS + threadIdx.x];
        if (!EMIT && threadIdx.x < 2 * NS) s_xw[threadIdx.x] = 0u;
        __syncthreads();
        if (!EMIT) {
            // Per-slot pass counts packed one byte per slot (slots 0-3 in pu[0]/pl[0],
            // 4-7 in pu[1]/pl[1]): a thread adds at most RPT per byte and a warp at most
            // 32 * RPT < 256, so no byte carries into the next.  The weight of a record
            // beyond 1 (multiplicity after grouping) goes to shared counters.
            static_assert(32 * RPT < 256, "packed per-slot counters would overflow a byte");
            constexpr int NW = NS > 4 ? 2 : 1;
            unsigned pu[NW], pl[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) pu[w] = pl[w] = 0u;
            unsigned nrec = 0;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                int64_t r = t0 + threadIdx.x + k * 256;
                if (r < t1) {
                    RecState<FAM, PREC> st;
                    st.set(pqf[k], pqt[k], pmult[k]);
                    if (PREC == 1) st.prep32(P, lev, s_g32 + NS * F::NB);
                    else st.need64(P, lev);
                    unsigned ubm, lbm;
                    eval_record<FAM, PREC>(P, lev, st, s_g32, s_g64, ubm, lbm, nrechk);
                    c.passmask[r - c.r0] = (uint8_t)ubm;
                    ++nrec;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        pu[w] += spread4((ubm >> (4 * w)) & 15u);
                        pl[w] += spread4((lbm >> (4 * w)) & 15u);
                    }
                    if (st.mult != 1u) {
                        unsigned x = st.mult - 1u;
                        for (unsigned b = ubm; b; b &= b - 1) atomicAdd(&s_xw[2 * (__ffs(b) - 1)], x);
                        for (unsigned b = lbm; b; b &= b - 1) atomicAdd(&s_xw[2 * (__ffs(b) - 1) + 1], x);
                    }
                }
            }
            ntest = nrec * (unsigned)__popc(valid_slots<NS>(smask));
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                unsigned a = __reduce_add_sync(kFull, pu[w]);
                unsigned b = __reduce_add_sync(kFull, pl[w]);
                if (lane == 0) {
#pragma unroll
                    for (int q = 0; q < 4 && 4 * w + q < NS; ++q) {
                        unsigned na = (a >> (8 * q)) & 255u, nb = (b >> (8 * q)) & 255u;
                        s_red[warp][3 * (4 * w + q)] = na;
                        s_red[warp][3 * (4 * w + q) + 1] = nb;
                        s_red[warp][3 * (4 * w + q) + 2] = na;
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x < 3 * NS) {
                unsigned v = 0;
#pragma unroll
                for (int w = 0; w < 8; ++w) v += s_red[w][threadIdx.x];
                int s = threadIdx.x / 3, f = threadIdx.x % 3;
                if (f < 2) v += s_xw[2 * s + f];   // UB and LB sums are weighted by multiplicity
                if (v) atomicAdd(c.cnt + (size_t)cl * NS * 3 + threadIdx.x, v);
            }
        } else {
            // Positions in (k, warp, lane) order so that each warp's stores for one
            // child are contiguous: per k and slot, warp counts are scanned in smem.
            __shared__ unsigned s_wcnt[RPT][8][NS];
            unsigned em[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                int64_t r = t0 + threadIdx.x + k * 256;
                unsigned m = 0;
                if (r < t1) {
                    m = ppm[k];
#pragma unroll
                    for (int s = 0; s < NS; ++s)
                        if (s_ci[s] < 0) m &= ~(1u << s);
                }
                em[k] = m;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    unsigned b = __ballot_sync(kFull, (m >> s) & 1);
                    if (lane == 0) s_wcnt[k][warp][s] = __popc(b);
                }
            }
            __syncthreads();
            if (threadIdx.x < NS) {
                int s = threadIdx.x;
                unsigned run = 0;
                for (int k = 0; k < RPT; ++k)
                    for (int w = 0; w < 8; ++w) {
                        unsigned v = s_wcnt[k][w][s];
                        s_wcnt[k][w][s] = run;
                        run += v;
                    }
                s_base[s] = (run && s_ci[s] >= 0) ? atomicAdd(&c.cursor[(size_t)cl * NS + s], run) : 0;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                unsigned m = em[k];
                int64_t r = t0 + threadIdx.x + k * 256;
                RecState<FAM, PREC> st;
                if (m) {
                    st.set(pqf[k], pqt[k], pmult[k]);
                    if (PREC == 1) st.prep32(P, lev, s_g32 + NS * F::NB);
                }
                // only the slots some lane of the warp writes; one copy of the body
#pragma unroll 1
                for (unsigned u = __reduce_or_sync(kFull, m); u; u &= u - 1) {
                    const int s = __ffs(u) - 1;
                    unsigned b = __ballot_sync(kFull, (m >> s) & 1);
                    if (!((m >> s) & 1)) continue;
                    unsigned pos = (unsigned)s_base[s] + s_wcnt[k][warp][s] + __popc(b & ((1u << lane) - 1u));
                    int32_t qn[F::ND];
                    child_qf<FAM, PREC>(P, lev, st, s_g32, s_g64, s, qn, nrechk, c.sc);
                    int ci = s_ci[s];
                    write_child<FAM, PREC>(c, st, qn, ci, c.next_cells.rbeg[ci] + pos);
                }
            }
        }
    } else if (clast - cfirst < kSpanCells) {
        // ------------------ a few cells: shared-memory counters -------------------
        const int span = clast - cfirst + 1;
        for (int i = threadIdx.x; i < span * NS * 3; i += blockDim.x) s_span[i] = 0u;
        __syncthreads();
        if (!EMIT) {
#pragma unroll 1
            for (int k = 0; k < RPT; ++k) {
                int64_t r = t0 + threadIdx.x + k * 256;
                if (r >= t1) break;
                int cl = (int)((int64_t)c.in.cell[r] - c.c0);
                if (!c.alive[cl]) continue;
                RecState<FAM, PREC> st;
                st.load(c.in, r);
                if (PREC == 1) st.prep32(P, lev, c.geo32 + ((size_t)cl * (NS + 1) + NS) * F::NB);
                else st.need64(P, lev);
                unsigned ubm, lbm;
                eval_record<FAM, PREC>(P, lev, st, c.geo32 + (size_t)cl * (NS + 1) * F::NB,
                                       c.geo64 + (size_t)cl * NS * F::NB, ubm, lbm, nrechk);
                c.passmask[r - c.r0] = (uint8_t)ubm;
                unsigned *cnt = s_span + (cl - cfirst) * NS * 3;
                for (int s = 0; s < NS; ++s) {
                    if (s & ~smask) continue;
                    ++ntest;
                    if ((ubm >> s) & 1) {
                        atomicAdd(cnt + 3 * s, st.mult);
                        atomicAdd(cnt + 3 * s + 2, 1u);
                    }
                    if ((lbm >> s) & 1) atomicAdd(cnt + 3 * s + 1, st.mult);
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < span * NS * 3; i += blockDim.x)
                if (s_span[i]) atomicAdd(c.cnt + (size_t)cfirst * NS * 3 + i, s_span[i]);
        } else {
            // count this block's records per (cell, child), reserve each child's range
            // with one global atomic, then place records by shared-memory ranks
            unsigned em[RPT];
            int ck[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                int64_t r = t0 + threadIdx.x + k * 256;
                unsigned m = 0;
                ck[k] = -1;
                if (r < t1) {
                    int cl = (int)((int64_t)c.in.cell[r] - c.c0);
                    ck[k] = cl;
                    if (c.alive[cl]) {
                        m = ppm[k];
                        for (int s = 0; s < NS; ++s)
                            if (((m >> s) & 1) && c.child_idx[(size_t)cl * NS + s] < 0) m &= ~(1u << s);
                        unsigned *cnt = s_span + (cl - cfirst) * NS * 3;
                        for (int s = 0; s < NS; ++s)
                            if ((m >> s) & 1) atomicAdd(cnt + 3 * s, 1u);
                    }
                }
                em[k] = m;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < span * NS; i += blockDim.x) {
                unsigned v = s_span[3 * i];
                if (v) s_span[3 * i + 1] = atomicAdd(&c.cursor[(size_t)cfirst * NS + i], v);
                s_span[3 * i + 2] = 0u;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                unsigned m = em[k];
                unsigned wm = __reduce_or_sync(kFull, m);
                if (!wm) continue;                                  // uniform
                const unsigned run = run_mask(ck[k], lane);
                int cl = ck[k] < 0 ? cfirst : ck[k];
                const float *g32 = c.geo32 + (size_t)cl * (NS + 1) * F::NB;
                const double *g64 = c.geo64 + (size_t)cl * NS * F::NB;
                RecState<FAM, PREC> st;
                if (m) {
                    st.set(pqf[k], pqt[k], pmult[k]);
                    if (PREC == 1) st.prep32(P, lev, g32 + NS * F::NB);
                }
                unsigned *cnt = s_span + (cl - cfirst) * NS * 3;
#pragma unroll 1
                for (unsigned u = wm; u; u &= u - 1) {
                    const int s = __ffs(u) - 1;
                    bool want = (m >> s) & 1;
                    // lanes of one cell writing to the same child form a group: one
                    // shared atomic per group, contiguous positions inside it
                    unsigned grp = __ballot_sync(kFull, want) & run;
                    int leader = __ffs(grp) - 1;
                    unsigned base = 0;
                    if (want && lane == leader) base = atomicAdd(cnt + 3 * s + 2, (unsigned)__popc(grp));
                    base = __shfl_sync(kFull, base, want ? leader : lane);
                    if (!want) continue;
                    unsigned pos = cnt[3 * s + 1] + base + __popc(grp & ((1u << lane) - 1u));
                    int32_t qn[F::ND];
                    child_qf<FAM, PREC>(P, lev, st, g32, g64, s, qn, nrechk, c.sc);
                    int ci = c.child_idx[(size_t)cl * NS + s];
                    write_child<FAM, PREC>(c, st, qn, ci, c.next_cells.rbeg[ci] + pos);
                }
            }
        }
    } else {
        // --------------------------- many cells ----------------------------
#pragma unroll 1
        for (int k = 0; k < RPT; ++k) {
            int64_t r = t0 + threadIdx.x + k * 256;
            bool act = false;
            int cl = 0;
            RecState<FAM, PREC> st;
            if (r < t1) {
                cl = (int)((int64_t)c.in.cell[r] - c.c0);
                act = c.alive[cl] != 0;
                if (act) {
                    st.load(c.in, r);
                    if (PREC == 1) st.prep32(P, lev, c.geo32 + ((size_t)cl * (NS + 1) + NS) * F::NB);
                    else st.need64(P, lev);
                }
            }
            const float *g32 = c.geo32 + (size_t)cl * (NS + 1) * F::NB;
            const double *g64 = c.geo64 + (size_t)cl * NS * F::NB;
            unsigned actb = __ballot_sync(kFull, act);
            if (!actb) continue;
            int leader = __ffs(actb) - 1;
            int cl0 = __shfl_sync(kFull, cl, leader);
            if (!EMIT) {
                unsigned ubm = 0, lbm = 0;
                if (act) {
                    eval_record<FAM, PREC>(P, lev, st, g32, g64, ubm, lbm, nrechk);
                    c.passmask[r - c.r0] = (uint8_t)ubm;
                }
                bool uniform = __all_sync(kFull, !act || cl == cl0);
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    if (s & ~smask) continue;
                    if (act) ++ntest;
                    unsigned pu = act && ((ubm >> s) & 1);
                    unsigned vub = pu ? st.mult : 0u, vlb = (act && ((lbm >> s) & 1)) ? st.mult : 0u;
                    if (uniform) {
                        vub = __reduce_add_sync(kFull, vub);
                        vlb = __reduce_add_sync(kFull, vlb);
                        unsigned vn = __reduce_add_sync(kFull, pu);
                        if (lane == leader) {
                            uint32_t *b = c.cnt + ((size_t)cl0 * NS + s) * 3;
                            if (vub) atomicAdd(b, vub);
                            if (vlb) atomicAdd(b + 1, vlb);
                            if (vn) atomicAdd(b + 2, vn);
                        }
                    } else if (pu) {
                        uint32_t *b = c.cnt + ((size_t)cl * NS + s) * 3;
                        atomicAdd(b, vub);
                        if (vlb) atomicAdd(b + 1, vlb);
                        atomicAdd(b + 2, 1u);
                    }
                }
            } else {
                unsigned ubm = act ? c.passmask[r - c.r0] : 0u;
                const unsigned run = run_mask(r < t1 ? cl : -1, lane);
#pragma unroll 1
                for (unsigned u = __reduce_or_sync(kFull, ubm); u; u &= u - 1) {
                    const int s = __ffs(u) - 1;
                    bool want = (ubm >> s) & 1;
                    int ci = -1;
                    if (want) {
                        ci = c.child_idx[(size_t)cl * NS + s];
                        want = ci >= 0;
                    }
                    // one global atomic per (cell, child) group of lanes
                    unsigned grp = __ballot_sync(kFull, want) & run;
                    int ldr = __ffs(grp) - 1;
                    unsigned base = 0;
                    if (want && lane == ldr) base = atomicAdd(&c.cursor[(size_t)cl * NS + s], (unsigned)__popc(grp));
                    base = __shfl_sync(kFull, base, want ? ldr : lane);
                    if (!want) continue;
                    unsigned pos = base + __popc(grp & ((1u << lane) - 1u));
                    int32_t qn[F::ND];
                    child_qf<FAM, PREC>(P, lev, st, g32, g64, s, qn, nrechk, c.sc);
                    write_child<FAM, PREC>(c, st, qn, ci, c.next_cells.rbeg[ci] + pos);
                }
            }
        }
    }
    // counters (all threads of the block reach this point unless the block exited above)
    ntest = __reduce_add_sync(kFull, ntest);
    nrechk = __reduce_add_sync(kFull, nrechk);
    if (lane == 0) {
        if (!EMIT && ntest) atomicAdd(&c.sc->tests, (unsigned long long)ntest);
        if (nrechk) atomicAdd(&c.sc->rechecks, (unsigned long long)nrechk);
    }
}

// ---------------------------------------------------------------------------
// Two levels per record read.  c is a chunk of level-l cells whose counts, child
// cells (level l+1, in c1.cells) and UB-pass masks are known; c1 describes those
// child cells (their geometry, alive flags, grandchild counters, grandchild cells
// in c1.next_cells).  The level-(l+1) records are never written: each block takes a
// tile of level-l records and one child slot s, re-derives the child record of
// every record that passes child s (residual at the child centre, snapped for
// level l+1) and tests it against the grandchildren.  Count pass: grandchild
// UB/LB/record counts and the grandchild pass mask per (record, s).  Emit pass:
// the grandchild records, snapped for level l+2.
// ---------------------------------------------------------------------------
template <int FAM, int PREC>
__device__ __forceinline__ void derive_child(const Problem &P, const Level &lev, RecState<FAM, PREC> &st,
                                             const float *g32, const double *g64, int s, RecState<FAM, PREC> &ch,
                                             unsigned &nrechk, Scalars *sc) {
    using F = Fam<FAM>;
    int32_t qn[F::ND], qt[F::LE];
    child_qf<FAM, PREC>(P, lev, st, g32, g64, s, qn, nrechk, sc);
#pragma unroll
    for (int m = 0; m < F::LE; ++m) qt[m] = lev.st_ratio_log2[m] ? resnap_half(st.qt[m]) : st.qt[m];
    ch.set(qn, qt, st.mult);
}

template <int FAM, int PREC, bool EMIT>
__global__ void __launch_bounds__(256, GV_MINBLOCKS) k_test2(Chunk c, Chunk c1, const uint8_t *__restrict__ pm2_in,
                                                   uint8_t *pm2_out) {
    using F = Fam<FAM>;
    constexpr int NS = 1 << F::D;
    const Problem &P = c.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x % NS;
    const int64_t tile = blockIdx.x / NS;
    __shared__ float s_pg32[(NS + 1) * F::NB], s_cg32[(NS + 1) * F::NB];
    __shared__ double s_pg64[NS * F::NB], s_cg64[NS * F::NB];
    __shared__ unsigned s_red[8][3 * NS];
    __shared__ int s_gi[NS];
    __shared__ unsigned long long s_base[NS];
    __shared__ unsigned s_wcnt[kRPT][8][NS];
    __shared__ int s_list[kTile];
    __shared__ uint8_t s_em[kTile];
    __shared__ unsigned s_n;
    if (s & ~c.lev.split_mask) return;
    const int64_t t0 = c.r0 + tile * kTile;
    const int64_t t1 = t0 + kTile < c.r1 ? t0 + kTile : c.r1;
    const int cfirst = (int)((int64_t)c.in.cell[t0] - c.c0);
    const int clast = (int)((int64_t)c.in.cell[t1 - 1] - c.c0);
    unsigned nrechk = 0, ntest = 0;
    if (cfirst == clast) {
        const int cl = cfirst;
        if (!c.alive[cl]) return;
        const int ci = c.child_idx[(size_t)cl * NS + s];
        if (ci < 0 || !c1.alive[ci]) return;                   // uniform over the block
        for (int i = threadIdx.x; i < (NS + 1) * F::NB; i += blockDim.x) {
            s_pg32[i] = c.geo32[(size_t)cl * (NS + 1) * F::NB + i];
            s_cg32[i] = c1.geo32[(size_t)ci * (NS + 1) * F::NB + i];
        }
        for (int i = threadIdx.x; i < NS * F::NB; i += blockDim.x) {
            s_pg64[i] = c.geo64[(size_t)cl * NS * F::NB + i];
            s_cg64[i] = c1.geo64[(size_t)ci * NS * F::NB + i];
        }
        if (EMIT && threadIdx.x < NS) s_gi[threadIdx.x] = c1.child_idx[(size_t)ci * NS + threadIdx.x];
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        // Compact the tile's records that have work for child s (count pass: pass
        // child s; emit pass: also reach a surviving grandchild) so that every lane
        // of a warp works on one.
#pragma unroll
        for (int k = 0; k < kRPT; ++k) {
            int64_t r = t0 + threadIdx.x + k * 256;
            unsigned m = 0;
            if (r < t1 && ((c.passmask[r - c.r0] >> s) & 1)) {
                if (!EMIT) {
                    m = 1;
                } else {
                    m = pm2_in[(size_t)(r - c.r0) * NS + s];
#pragma unroll
                    for (int g = 0; g < NS; ++g)
                        if (s_gi[g] < 0) m &= ~(1u << g);
                }
            }
            unsigned b = __ballot_sync(kFull, m != 0);
            unsigned base = 0;
            if (lane == 0 && b) base = atomicAdd(&s_n, (unsigned)__popc(b));
            base = __shfl_sync(kFull, base, 0);
            if (m) {
                unsigned at = base + __popc(b & ((1u << lane) - 1u));
                s_list[at] = (int)(r - t0);
                s_em[at] = (uint8_t)m;
            }
        }
        __syncthreads();
        const int nlist = (int)s_n;
        if (!EMIT) {
            unsigned aub[NS], alb[NS], an[NS];
#pragma unroll
            for (int g = 0; g < NS; ++g) aub[g] = alb[g] = an[g] = 0;
#pragma unroll 1
            for (int i = threadIdx.x; i < nlist; i += 256) {
                int64_t r = t0 + s_list[i];
                RecState<FAM, PREC> st, ch;
                st.load(c.in, r);
                if (PREC == 1) st.prep32(P, c.lev, s_pg32 + NS * F::NB);
                derive_child<FAM, PREC>(P, c.lev, st, s_pg32, s_pg64, s, ch, nrechk, c.sc);
                if (PREC == 1) ch.prep32(P, c1.lev, s_cg32 + NS * F::NB);
                else ch.need64(P, c1.lev);
                unsigned ubm, lbm;
                eval_record<FAM, PREC>(P, c1.lev, ch, s_cg32, s_cg64, ubm, lbm, nrechk);
                pm2_out[(size_t)(r - c.r0) * NS + s] = (uint8_t)ubm;
#pragma unroll
                for (int g = 0; g < NS; ++g) {
                    if (g & ~c1.lev.split_mask) continue;
                    ++ntest;
                    aub[g] += ((ubm >> g) & 1) ? ch.mult : 0u;
                    alb[g] += ((lbm >> g) & 1) ? ch.mult : 0u;
                    an[g] += (ubm >> g) & 1;
                }
            }
#pragma unroll
            for (int g = 0; g < NS; ++g) {
                unsigned a = __reduce_add_sync(kFull, aub[g]);
                unsigned b = __reduce_add_sync(kFull, alb[g]);
                unsigned d = __reduce_add_sync(kFull, an[g]);
                if (lane == 0) {
                    s_red[warp][3 * g] = a;
                    s_red[warp][3 * g + 1] = b;
                    s_red[warp][3 * g + 2] = d;
                }
            }
            __syncthreads();
            if (threadIdx.x < 3 * NS) {
                unsigned v = 0;
#pragma unroll
                for (int w = 0; w < 8; ++w) v += s_red[w][threadIdx.x];
                if (v) atomicAdd(c1.cnt + (size_t)ci * NS * 3 + threadIdx.x, v);
            }
        } else {
            // positions in (iteration, warp, lane) order over the compacted list
#pragma unroll
            for (int k = 0; k < kRPT; ++k) {
                int i = threadIdx.x + k * 256;
                unsigned m = i < nlist ? s_em[i] : 0u;
#pragma unroll
                for (int g = 0; g < NS; ++g) {
                    unsigned b = __ballot_sync(kFull, (m >> g) & 1);
                    if (lane == 0) s_wcnt[k][warp][g] = __popc(b);
                }
            }
            __syncthreads();
            if (threadIdx.x < NS) {
                int g = threadIdx.x;
                unsigned run = 0;
                for (int k = 0; k < kRPT; ++k)
                    for (int w = 0; w < 8; ++w) {
                        unsigned v = s_wcnt[k][w][g];
                        s_wcnt[k][w][g] = run;
                        run += v;
                    }
                s_base[g] = (run && s_gi[g] >= 0) ? atomicAdd(&c1.cursor[(size_t)ci * NS + g], run) : 0;
            }
            __syncthreads();
#pragma unroll 1
            for (int k = 0; k < kRPT; ++k) {
                int i = threadIdx.x + k * 256;
                if (k * 256 >= nlist) break;                     // uniform
                unsigned m = i < nlist ? s_em[i] : 0u;
                RecState<FAM, PREC> st, ch;
                if (m) {
                    int64_t r = t0 + s_list[i];
                    st.load(c.in, r);
                    if (PREC == 1) st.prep32(P, c.lev, s_pg32 + NS * F::NB);
                    derive_child<FAM, PREC>(P, c.lev, st, s_pg32, s_pg64, s, ch, nrechk, c.sc);
                    if (PREC == 1) ch.prep32(P, c1.lev, s_cg32 + NS * F::NB);
                }
#pragma unroll
                for (int g = 0; g < NS; ++g) {
                    unsigned b = __ballot_sync(kFull, (m >> g) & 1);
                    if (!((m >> g) & 1)) continue;
                    unsigned pos = (unsigned)s_base[g] + s_wcnt[k][warp][g] + __popc(b & ((1u << lane) - 1u));
                    int32_t qn[F::ND];
                    child_qf<FAM, PREC>(P, c1.lev, ch, s_cg32, s_cg64, g, qn, nrechk, c.sc);
                    int gi = s_gi[g];
                    write_child<FAM, PREC>(c1, ch, qn, gi, c1.next_cells.rbeg[gi] + pos);
                }
            }
        }
    } else {
        // tile spans several level-l cells: per record, global atomics
#pragma unroll 1
        for (int k = 0; k < kRPT; ++k) {
            int64_t r = t0 + threadIdx.x + k * 256;
            if (r >= t1) break;
            int cl = (int)((int64_t)c.in.cell[r] - c.c0);
            if (!c.alive[cl] || !((c.passmask[r - c.r0] >> s) & 1)) continue;
            int ci = c.child_idx[(size_t)cl * NS + s];
            if (ci < 0 || !c1.alive[ci]) continue;
            const float *pg32 = c.geo32 + (size_t)cl * (NS + 1) * F::NB;
            const double *pg64 = c.geo64 + (size_t)cl * NS * F::NB;
            const float *cg32 = c1.geo32 + (size_t)ci * (NS + 1) * F::NB;
            const double *cg64 = c1.geo64 + (size_t)ci * NS * F::NB;
            RecState<FAM, PREC> st, ch;
            st.load(c.in, r);
            if (PREC == 1) st.prep32(P, c.lev, pg32 + NS * F::NB);
            derive_child<FAM, PREC>(P, c.lev, st, pg32, pg64, s, ch, nrechk, c.sc);
            if (PREC == 1) ch.prep32(P, c1.lev, cg32 + NS * F::NB);
            else ch.need64(P, c1.lev);
            if (!EMIT) {
                unsigned ubm, lbm;
                eval_record<FAM, PREC>(P, c1.lev, ch, cg32, cg64, ubm, lbm, nrechk);
                pm2_out[(size_t)(r - c.r0) * NS + s] = (uint8_t)ubm;
                for (int g = 0; g < NS; ++g) {
                    if (g & ~c1.lev.split_mask) continue;
                    ++ntest;
                    uint32_t *b = c1.cnt + ((size_t)ci * NS + g) * 3;
                    if ((ubm >> g) & 1) {
                        atomicAdd(b, ch.mult);
                        atomicAdd(b + 2, 1u);
                    }
                    if ((lbm >> g) & 1) atomicAdd(b + 1, ch.mult);
                }
            } else {
                unsigned m = pm2_in[(size_t)(r - c.r0) * NS + s];
                for (int g = 0; g < NS; ++g) {
                    if (!((m >> g) & 1)) continue;
                    int gi = c1.child_idx[(size_t)ci * NS + g];
                    if (gi < 0) continue;
                    unsigned pos = atomicAdd(&c1.cursor[(size_t)ci * NS + g], 1u);
                    int32_t qn[F::ND];
                    child_qf<FAM, PREC>(P, c1.lev, ch, cg32, cg64, g, qn, nrechk, c.sc);
                    write_child<FAM, PREC>(c1, ch, qn, gi, c1.next_cells.rbeg[gi] + pos);
                }
            }
        }
    }
    ntest = __reduce_add_sync(kFull, ntest);
    nrechk = __reduce_add_sync(kFull, nrechk);
    if (lane == 0) {
        if (!EMIT && ntest) atomicAdd(&c.sc->tests, (unsigned long long)ntest);
        if (nrechk) atomicAdd(&c.sc->rechecks, (unsigned long long)nrechk);
    }
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
    if (idx < c.nc * NS) {
        keepflag[idx] = keep ? 1u : 0u;
        recn[idx] = keep ? nrec : 0u;
    }
    unsigned long long tc, tr;
    block_excl_scan(keep ? 1ull : 0ull, &tc);
    block_excl_scan(keep ? (unsigned long long)nrec : 0ull, &tr);
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
// (parent, slot) order.
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
        c.next_cells.rcnt[ci] = nrec;
        c.next_cells.ub[ci] = c.cnt[(size_t)idx * 3];
        c.child_idx[idx] = (int32_t)ci;
    } else {
        c.child_idx[idx] = -1;
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
        F::basis(c, psi);
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
template <int ND, int LE>
__device__ __forceinline__ bool same_key(const RecView &in, int64_t a, int64_t b) {
    if (in.cell[a] != in.cell[b]) return false;
#pragma unroll
    for (int j = 0; j < ND; ++j)
        if (in.qf[j][a] != in.qf[j][b]) return false;
#pragma unroll
    for (int m = 0; m < LE; ++m)
        if (in.qt[m][a] != in.qt[m][b]) return false;
    return true;
}

template <int ND, int LE>
__device__ __forceinline__ uint64_t key_hash(const RecView &in, int64_t r) {
    uint64_t h = 0x9E3779B97F4A7C15ull ^ in.cell[r];
#pragma unroll
    for (int j = 0; j < ND; ++j) h = (h ^ (uint32_t)in.qf[j][r]) * 0xff51afd7ed558ccdull;
#pragma unroll
    for (int m = 0; m < LE; ++m) h = (h ^ (uint32_t)in.qt[m][r]) * 0xc4ceb9fe1a85ec53ull;
    return h ^ (h >> 29);
}

template <int FAM>
__global__ void k_group_insert(RecView in, int64_t r0, int64_t nr, int64_t c0, uint32_t *table, uint32_t tmask,
                               uint32_t *owner, uint32_t *ccount, Scalars *sc) {
    using F = Fam<FAM>;
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nr) return;
    int64_t r = r0 + x;
    uint32_t slot = (uint32_t)key_hash<F::ND, F::LE>(in, r) & tmask;
    for (uint32_t probe = 0; probe <= tmask; ++probe) {
        uint32_t prev = atomicCAS(&table[slot], 0u, (uint32_t)(x + 1));
        if (prev == 0u) {                                   // new canonical record
            owner[x] = (uint32_t)x;
            atomicAdd(&ccount[in.cell[r] - c0], 1u);
            return;
        }
        if (same_key<F::ND, F::LE>(in, r, r0 + (int64_t)(prev - 1))) {
            owner[x] = prev - 1;
            return;
        }
        slot = (slot + 1) & tmask;
    }
    atomicOr(&sc->err, 4u);                                 // table full (cannot happen at load <= 1/2)
    owner[x] = (uint32_t)x;
}

// exclusive scan of n u32 values in place (one block of 256 threads); *total = sum
__global__ void __launch_bounds__(256) k_scan_u32(uint32_t *a, int64_t n, unsigned long long *total) {
    unsigned long long carry = 0;
    for (int64_t base = 0; base < n; base += 256) {
        int64_t i = base + threadIdx.x;
        unsigned long long v = i < n ? a[i] : 0u, t;
        unsigned long long e = block_excl_scan(v, &t);
        if (i < n) a[i] = (uint32_t)(carry + e);
        carry += t;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <int FAM>
__global__ void k_group_place(RecView in, int64_t r0, int64_t nr, int64_t c0, const uint32_t *owner,
                              const uint32_t *coff, uint32_t *ccur, uint32_t *newpos, RecView out) {
    using F = Fam<FAM>;
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nr || owner[x] != (uint32_t)x) return;
    int64_t r = r0 + x;
    uint32_t cl = in.cell[r] - (uint32_t)c0;
    uint32_t pos = coff[cl] + atomicAdd(&ccur[cl], 1u);
    newpos[x] = pos;
#pragma unroll
    for (int j = 0; j < F::ND; ++j) out.qf[j][pos] = in.qf[j][r];
#pragma unroll
    for (int m = 0; m < F::LE; ++m) out.qt[m][pos] = in.qt[m][r];
    out.cell[pos] = in.cell[r];
    out.mult[pos] = 0u;
}

__global__ void k_group_mult(RecView in, int64_t r0, int64_t nr, const uint32_t *owner, const uint32_t *newpos,
                             RecView out) {
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nr) return;
    atomicAdd(&out.mult[newpos[owner[x]]], in.mult[r0 + x]);
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

void launch_test(const Chunk &c, bool emit, cudaStream_t st) {
    int64_t nr = c.r1 - c.r0;
    if (nr <= 0) return;
    unsigned g = blocks_for(nr, emit ? 256 * kRPTEmit : kTile);
    if (c.precision == 0) {
        if (emit) { GV_DISPATCH(c.P.fam, (k_test<FAMV, 0, true><<<g, 256, 0, st>>>(c))); }
        else      { GV_DISPATCH(c.P.fam, (k_test<FAMV, 0, false><<<g, 256, 0, st>>>(c))); }
    } else {
        if (emit) { GV_DISPATCH(c.P.fam, (k_test<FAMV, 1, true><<<g, 256, 0, st>>>(c))); }
        else      { GV_DISPATCH(c.P.fam, (k_test<FAMV, 1, false><<<g, 256, 0, st>>>(c))); }
    }
}

void launch_test2(const Chunk &c, const Chunk &c1, bool emit, const uint8_t *pm2_in, uint8_t *pm2_out,
                  cudaStream_t st) {
    int64_t nr = c.r1 - c.r0;
    if (nr <= 0) return;
    int ns = 1 << c.P.d;
    unsigned g = blocks_for(nr, kTile) * ns;
    if (c.precision == 0) {
        if (emit) { GV_DISPATCH(c.P.fam, (k_test2<FAMV, 0, true><<<g, 256, 0, st>>>(c, c1, pm2_in, pm2_out))); }
        else      { GV_DISPATCH(c.P.fam, (k_test2<FAMV, 0, false><<<g, 256, 0, st>>>(c, c1, pm2_in, pm2_out))); }
    } else {
        if (emit) { GV_DISPATCH(c.P.fam, (k_test2<FAMV, 1, true><<<g, 256, 0, st>>>(c, c1, pm2_in, pm2_out))); }
        else      { GV_DISPATCH(c.P.fam, (k_test2<FAMV, 1, false><<<g, 256, 0, st>>>(c, c1, pm2_in, pm2_out))); }
    }
}

void launch_child_lbmax(const Chunk &c, cudaStream_t st) {
    int ns = 1 << c.P.d;
    int64_t n = (int64_t)c.nc * ns;
    if (n <= 0) return;
    if (ns == 4) k_child_lbmax<4><<<blocks_for(n, 256), 256, 0, st>>>(c);
    else k_child_lbmax<8><<<blocks_for(n, 256), 256, 0, st>>>(c);
}

void launch_child_alloc(const Chunk &c, uint32_t *keepflag, uint32_t *recn, unsigned long long *bsums,
                        cudaStream_t st) {
    int ns = 1 << c.P.d;
    int64_t n = (int64_t)c.nc * ns;
    if (n <= 0) return;
    unsigned nb = blocks_for(n, 256);
    unsigned long long *ba = bsums, *bb = bsums + nb;
    if (ns == 4) k_child_mark<4><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else k_child_mark<8><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    if (c.lev.leaf_children) return;
    k_scan_sums<<<1, 256, 0, st>>>(ba, bb, (int)nb, c.sc);
    if (ns == 4) k_child_write<4><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
    else k_child_write<8><<<nb, 256, 0, st>>>(c, keepflag, recn, ba, bb);
}

void launch_group(const Problem &P, RecView in, int64_t r0, int64_t nr, int64_t c0, int nc, uint32_t *table,
                  uint32_t tmask, uint32_t *owner, uint32_t *ccount, uint32_t *ccur, uint32_t *newpos,
                  unsigned long long *total, RecView out, Scalars *sc, cudaStream_t st) {
    if (nr <= 0) return;
    unsigned g = blocks_for(nr, 256);
    GV_DISPATCH(P.fam, (k_group_insert<FAMV><<<g, 256, 0, st>>>(in, r0, nr, c0, table, tmask, owner, ccount, sc)));
    k_scan_u32<<<1, 256, 0, st>>>(ccount, nc, total);
    GV_DISPATCH(P.fam, (k_group_place<FAMV><<<g, 256, 0, st>>>(in, r0, nr, c0, owner, ccount, ccur, newpos, out)));
    k_group_mult<<<g, 256, 0, st>>>(in, r0, nr, owner, newpos, out);
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
