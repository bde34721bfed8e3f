// gv_engine.cu -- host engine and C ABI of libvote (see include/vote.h).
//
// The engine drives Algorithm 2 (SurfaceConsensus) of arXiv 2107.11810 level by
// level on the GPU.  Each level keeps a stack of cells and of their records
// (canonical surfaces).  One expansion step takes a chunk of cells from the top of
// the deepest non-empty level, tests all their children (k_test count pass),
// raises the best lower bound, drops children below it (B&B pruning, Sec. 3.3),
// lays out the survivors and writes their records, snapped for the next level
// (emit pass, canonization of Sec. 3.2).  Taking the deepest level first is a
// depth-first order over chunks: memory stays bounded by one chunk's expansion per
// level, and leaves are reached early, which raises the pruning bound early.  The
// result does not depend on this order.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gv_kernels.h"
#include "gv_tile.cuh"
#include "vote.h"

using namespace gv;

static thread_local char g_err[512] = "";

static void set_err(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_err("%s failed: %s", #call, cudaGetErrorString(e_));                    \
            return VOTE_ECUDA;                                                          \
        }                                                                               \
    } while (0)

#define TRY(x)                                                                          \
    do {                                                                                \
        vote_status s_ = (x);                                                           \
        if (s_ != VOTE_OK) return s_;                                                   \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct LevelStore {
    DevBuf rec, mult, tile_cell;       // packed records (whole tiles), multiplicities, owning cell per tile
    DevBuf key, rbeg, rcnt, ub;
    int64_t ncells = 0, nrecs = 0;     // nrecs: record slots in use (a multiple of 32)
};

struct vote_ctx {
    Problem P;
    Level lev[GV_MAXL];
    double h_leaf[GV_MAXD];
    int ns = 0;                // 2^d child slots
    int device = 0;
    cudaStream_t stream = 0;
    int precision = 1, prune = 1, group = 0;
    int64_t chunk_records = 1 << 25;
    uint32_t initial_lb = 0;
    int kernel_timing = 0;
    int log = 0;               // VOTE_LOG=1: per-level counters on stderr after each solve;
                               // 2: also one line per expansion step
    unsigned spin_limit = GV_SPIN_LIMIT;   // VOTE_OPT_SPIN_LIMIT
    int batch_workers = 4;
    int dive = 2;              // greedy dive: 0 off, 1 on, 2 on for n >= kDiveMinN
    int family = 0;
    double eps_in[GV_MAXD] = {}, bounds_in[2 * GV_MAXD] = {};
    std::vector<vote_ctx *> workers;   // sub-contexts of vote_solve_batched
    static const int kEv = 24;
    cudaEvent_t ev[kEv] = {};
    int ev_n = 0;              // events recorded since the last collection
    int ev_cls[kEv] = {};      // kernel class of the interval ending at event i
    double kms[VOTE_K_CLASSES] = {};
    int64_t klaunch[VOTE_K_CLASSES] = {};
    double kbytes[VOTE_K_CLASSES] = {};
    int64_t lv_cells[GV_MAXL] = {}, lv_recs[GV_MAXL] = {};
    int64_t lv_gin[GV_MAXL] = {}, lv_gout[GV_MAXL] = {};  // records into / out of grouping
    int64_t trace_cap = 0;
    int64_t fault_alloc_at = 0, alloc_count = 0;
    LevelStore ls[GV_MAXL + 1];
    DevBuf levs_dev, path, scal, alive, geo64, geo32, geo32lo, cnt, tinfo, ballot, tdst, child_idx, cursor, keepflag, recn, bsums;
    DevBuf tr_level, tr_key, tr_ub, tr_lb, surf_tmp, mask_tmp;
    DevBuf ss_partial, ss_io;  // soft score: block partials; point [d] + outputs [d] + grad_out [1]
    DevBuf g_table, g_owner, g_newpos, g_ccount, g_ccur, g_rbeg, g_rec, g_mult, g_tile;
    Scalars *h_sc = nullptr;   // pinned mirror of the device scalars
    uint64_t *h_tmp = nullptr; // pinned slot for single values
    // device slot for single values: 64 bytes after the scalars block
    void *h_tmp_dev() { return (char *)scal.p + ((sizeof(Scalars) + 63) / 64) * 64; }
    int64_t trace_written = 0;
    bool trace_overflow = false;
    vote_stats stats;
};

// ---------------------------------------------------------------------------
// problem constants (the same definition as the paper-derived oracle, written
// independently: per-coordinate levels, power-of-two snap steps, accumulated
// canonization error)
// ---------------------------------------------------------------------------
static int family_shape(int fam, int d, int k, int *le, int *np) {
    switch (fam) {
    case VOTE_LINE2D: if (d != 2 || k != 1) return 1; *le = 1; *np = 2; return 0;
    case VOTE_PLANE3D_SPH: if (d != 3 || k != 2) return 1; *le = 3; *np = 3; return 0;
    case VOTE_POSE3DOF: if (d != 3 || k != 1) return 1; *le = 2; *np = 4; return 0;
    case VOTE_POSE6DOF: if (d != 6 || k != 4) return 1; *le = 11; *np = 5; return 0;
    case VOTE_RAYS3D: if (d != 3 || k != 1) return 1; *le = 2; *np = 4; return 0;
    case VOTE_POINTSET2D: if (d != 4 || k != 2) return 1; *le = 2; *np = 4; return 0;
    case VOTE_AFFINE4D: if (d != 4 || k != 3) return 1; *le = 3; *np = 4; return 0;
    case VOTE_RADIAL5DOF: if (d != 5 || k != 4) return 1; *le = 7; *np = 5; return 0;
    default: return 1;
    }
}

// bound on the change of each basis function across a cell of half-widths h
static void family_sigma(int fam, const double *h, double *sigma) {
    switch (fam) {
    case VOTE_LINE2D: sigma[0] = h[0]; break;
    case VOTE_PLANE3D_SPH:
        sigma[0] = h[0] + h[1];
        sigma[1] = h[0] + h[1];
        sigma[2] = h[0];
        break;
    case VOTE_POSE3DOF:
        sigma[0] = h[0];
        sigma[1] = h[0];
        break;
    case VOTE_RAYS3D:       // a and c multiply x
        sigma[0] = h[0];
        sigma[1] = h[0];
        break;
    case VOTE_AFFINE4D:     // x_i multiplies a_i
        sigma[0] = h[0];
        sigma[1] = h[1];
        sigma[2] = h[2];
        break;
    case VOTE_POINTSET2D:   // u, v multiply c in one equation and d in the other
        sigma[0] = h[0] > h[1] ? h[0] : h[1];
        sigma[1] = sigma[0];
        break;
    case VOTE_POSE6DOF: {
        // an entry of the rotation moves by at most |d phi|_2 <= sum of the phi
        // half-widths (its gradient has norm <= 1); z is linear
        const double hr = (h[0] + h[1]) + h[2];
        for (int m = 0; m < 9; ++m) sigma[m] = hr;
        sigma[9] = h[3];
        sigma[10] = h[3];
        break;
    }
    case VOTE_RADIAL5DOF: {
        // the six entries of rows r1, r2 (as for 6DoF); y is linear
        const double hr = (h[0] + h[1]) + h[2];
        for (int m = 0; m < 6; ++m) sigma[m] = hr;
        sigma[6] = h[3];
        break;
    }
    }
}

static double pow2_floor(double x, int *e_out) {
    int e;
    std::frexp(x, &e);
    if (e_out) *e_out = e - 1;
    return std::ldexp(1.0, e - 1);
}

static vote_status problem_init(vote_ctx *c, int fam, int d, int k, const double *eps, const double *bounds) {
    int le, np;
    if (family_shape(fam, d, k, &le, &np)) {
        set_err("family %d does not take d=%d, k=%d", fam, d, k);
        return VOTE_EINVAL;
    }
    Problem &P = c->P;
    std::memset(&P, 0, sizeof(P));
    P.fam = fam; P.d = d; P.k = k; P.nd = d - k; P.le = le; P.np = np;
    P.inv_fact[0] = 1.0;
    for (int m = 1; m < 31; ++m) P.inv_fact[m] = P.inv_fact[m - 1] / (double)m;
    P.L = 0;
    for (int j = 0; j < d; ++j) {
        double lo = bounds[2 * j], hi = bounds[2 * j + 1];
        if (!(eps[j] > 0.0) || !std::isfinite(eps[j]) || !std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo)) {
            set_err("coordinate %d: need finite eps > 0 and lo < hi", j);
            return VOTE_EINVAL;
        }
        P.lo[j] = lo;
        P.W[j] = hi - lo;
        P.eps[j] = eps[j];
        int Lj = 0;
        while (std::ldexp(P.W[j], -Lj) > eps[j]) ++Lj;
        if (Lj > 30) {
            set_err("coordinate %d needs %d levels (> 30)", j, Lj);
            return VOTE_EUNSUPPORTED;
        }
        P.Lj[j] = Lj;
        if (Lj > P.L) P.L = Lj;
    }
    if (P.L > GV_MAXL - 1) {
        set_err("too many levels");
        return VOTE_EUNSUPPORTED;
    }
    int bits = 0;
    for (int j = d - 1; j >= 0; --j) {
        P.coord_shift[j] = bits;
        bits += P.Lj[j];
    }
    P.coord_bits = bits;
    if (bits > 44) {       // the best leaf packs (UB << bits) | leaf key into 64 bits
        set_err("leaf key needs %d bits (> 44)", bits);
        return VOTE_EUNSUPPORTED;
    }
    double h[GV_MAXL + 1][GV_MAXD];
    for (int l = 0; l <= P.L; ++l)
        for (int j = 0; j < d; ++j) {
            int e = l < P.Lj[j] ? l : P.Lj[j];
            h[l][j] = std::ldexp(P.W[j], -(e + 1));
        }
    for (int j = 0; j < d; ++j) c->h_leaf[j] = h[P.L][j];
    if (P.L == 0) return VOTE_OK;
    double epsp_min = INFINITY;
    for (int j = 0; j < P.nd; ++j) {
        double epsp = P.eps[k + j] / (double)P.L;
        if (epsp < epsp_min) epsp_min = epsp;
        P.s_f[j] = pow2_floor(epsp / (double)(le + 1), nullptr);
        P.inv_s_f[j] = 1.0 / P.s_f[j];
    }
    double s_t[GV_MAXL + 1][GV_MAXT];
    int s_te[GV_MAXL + 1][GV_MAXT];
    double A[GV_MAXL + 1][GV_MAXD];
    for (int j = 0; j < P.nd; ++j) A[0][j] = 0.0;
    for (int l = 0; l < P.L; ++l) {
        double sigma[GV_MAXT];
        family_sigma(fam, h[l], sigma);
        for (int m = 0; m < le; ++m) s_t[l][m] = pow2_floor(epsp_min / ((double)(le + 1) * sigma[m]), &s_te[l][m]);
        for (int j = 0; j < P.nd; ++j) {
            double delta = P.s_f[j] * 0.5;
            for (int m = 0; m < le; ++m) delta = delta + (s_t[l][m] * 0.5) * sigma[m];
            delta = delta + std::ldexp(P.eps[k + j], -32);
            A[l + 1][j] = A[l][j] + delta;
        }
    }
    for (int l = 0; l < P.L; ++l) {
        Level &v = c->lev[l];
        std::memset(&v, 0, sizeof(v));
        v.l = l;
        v.leaf_children = (l + 1 == P.L);
        for (int j = 0; j < d; ++j) {
            if (l < P.Lj[j]) v.split_mask |= 1 << j;
            v.h[j] = h[l][j];
            v.h1[j] = h[l + 1][j];
        }
        for (int m = 0; m < le; ++m) {
            v.s_t[m] = s_t[l][m];
            v.inv_s_t[m] = std::ldexp(1.0, -s_te[l][m]);
            if (l + 1 < P.L) {
                int r = s_te[l + 1][m] - s_te[l][m];
                if (r < 0 || r > 1) {
                    set_err("internal: snap step ratio 2^%d at level %d", r, l);
                    return VOTE_EINTERNAL;
                }
                v.st_ratio_log2[m] = r;
            }
        }
        for (int j = 0; j < P.nd; ++j) {
            v.Rbase[j] = P.eps[k + j] + h[l + 1][k + j];
            v.A1[j] = A[l + 1][j];
            v.rlb[j] = P.eps[k + j] - A[l + 1][j];
            // FP32 screen constants in steps of s_f,j (rounding is covered by its band)
            for (int m = 0; m < le; ++m) v.gscale[j][m] = s_t[l][m] / P.s_f[j];
            v.Hs[j] = (float)(h[l + 1][k + j] / P.s_f[j]);
            v.Hs_lo[j] = (float)(h[l + 1][k + j] / P.s_f[j] - (double)v.Hs[j]);
            if (l < P.Lj[k + j]) {              // the dependent coordinate splits: its shift enters
                const double hs = h[l + 1][k + j] / P.s_f[j];
                if ((double)v.Hs[j] != hs) v.hs_exp = kNoExp;
                else if (v.hs_exp > kNoExp && hs != 0.0) v.hs_exp = std::min(v.hs_exp, lowbit_exp(hs));
            }
            v.rc0[j] = (float)((v.Rbase[j] + v.A1[j]) / P.s_f[j]);
            v.Lc[j] = (float)(v.rlb[j] / P.s_f[j]);
        }
        // Lipschitz term of the radius from the essential parameters in steps
        switch (fam) {
        case VOTE_LINE2D:        // |t| h1_m
            v.lam_c[0] = (float)(h[l + 1][0] * s_t[l][0] / P.s_f[0]);
            break;
        case VOTE_PLANE3D_SPH:   // |q| h1_theta + |q_xy| h1_phi; s_t,x = s_t,y
            v.lam_c[0] = (float)(h[l + 1][0] * s_t[l][0] / P.s_f[0]);
            v.lam_c[1] = (float)(h[l + 1][1] * s_t[l][0] / P.s_f[0]);
            v.rho2 = (float)((s_t[l][2] / s_t[l][0]) * (s_t[l][2] / s_t[l][0]));
            break;
        case VOTE_POSE3DOF:      // sqrt(a^2 + b^2) h1_yaw; s_t,a = s_t,b
            for (int j = 0; j < P.nd; ++j) v.lam_c[j] = (float)(h[l + 1][0] * s_t[l][0] / P.s_f[j]);
            break;
        case VOTE_RAYS3D:        // |a| h1_x and |c| h1_x
            v.lam_c[0] = (float)(h[l + 1][0] * s_t[l][0] / P.s_f[0]);
            v.lam_c[1] = (float)(h[l + 1][0] * s_t[l][1] / P.s_f[1]);
            break;
        case VOTE_AFFINE4D:      // sum_i |x_i| h1_i
            for (int m = 0; m < 3; ++m) v.lam_c[m] = (float)(h[l + 1][m] * s_t[l][m] / P.s_f[0]);
            break;
        case VOTE_POINTSET2D:    // a: |u| h1_c + |v| h1_d; b: |v| h1_c + |u| h1_d
            v.lam_c[0] = (float)(h[l + 1][0] * s_t[l][0] / P.s_f[0]);
            v.lam_c[1] = (float)(h[l + 1][1] * s_t[l][1] / P.s_f[0]);
            v.lam_c[2] = (float)(h[l + 1][0] * s_t[l][1] / P.s_f[1]);
            v.lam_c[3] = (float)(h[l + 1][1] * s_t[l][0] / P.s_f[1]);
            break;
        case VOTE_POSE6DOF: {    // (|xi w| + |w|) sum h1_phi + |xi| h1_z (and y with eta)
            const double hphi = (h[l + 1][0] + h[l + 1][1]) + h[l + 1][2];
            v.lam_c[0] = (float)(hphi * s_t[l][0] / P.s_f[0]);
            v.lam_c[1] = (float)(h[l + 1][3] * s_t[l][9] / P.s_f[0]);
            v.lam_c[2] = (float)(hphi * s_t[l][0] / P.s_f[1]);
            v.lam_c[3] = (float)(h[l + 1][3] * s_t[l][10] / P.s_f[1]);
            break;
        }
        case VOTE_RADIAL5DOF: {  // (|rho w| + |w|) sum h1_phi + |rho| h1_y
            const double hphi = (h[l + 1][0] + h[l + 1][1]) + h[l + 1][2];
            v.lam_c[0] = (float)(hphi * s_t[l][0] / P.s_f[0]);
            v.lam_c[1] = (float)(h[l + 1][3] * s_t[l][6] / P.s_f[0]);
            break;
        }
        }
        bool equal = true;
        if (fam == VOTE_PLANE3D_SPH || fam == VOTE_POSE3DOF) equal = s_t[l][0] == s_t[l][1];
        if (fam == VOTE_POSE6DOF)
            for (int m = 1; m < 9; ++m) equal &= s_t[l][m] == s_t[l][0];
        if (fam == VOTE_RADIAL5DOF)
            for (int m = 1; m < 6; ++m) equal &= s_t[l][m] == s_t[l][0];
        if (!equal) {
            set_err("internal: unequal essential steps at level %d", l);
            return VOTE_EINTERNAL;
        }
    }
    return VOTE_OK;
}

// Upper bounds on the Lipschitz factors Lambda_ji from bounds T_m on |t_m|.
static void lambda_max(int fam, const double *T, double *lam) {
    switch (fam) {
    case VOTE_LINE2D: lam[0] = T[0]; break;
    case VOTE_PLANE3D_SPH:
        lam[0] = std::sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
        lam[1] = std::sqrt(T[0] * T[0] + T[1] * T[1]);
        break;
    case VOTE_POSE3DOF: lam[0] = lam[1] = std::sqrt(T[0] * T[0] + T[1] * T[1]); break;
    case VOTE_RAYS3D: lam[0] = T[0]; lam[1] = T[1]; break;
    case VOTE_POINTSET2D: lam[0] = T[0]; lam[1] = T[1]; lam[2] = T[1]; lam[3] = T[0]; break;
    case VOTE_AFFINE4D: lam[0] = T[0]; lam[1] = T[1]; lam[2] = T[2]; break;
    case VOTE_POSE6DOF: {
        const double nw = std::sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
        const double nxw = std::sqrt(T[3] * T[3] + T[4] * T[4] + T[5] * T[5]);
        const double nyw = std::sqrt(T[6] * T[6] + T[7] * T[7] + T[8] * T[8]);
        lam[0] = lam[1] = lam[2] = nxw + nw;
        lam[3] = T[9];
        lam[4] = lam[5] = lam[6] = nyw + nw;
        lam[7] = T[10];
        break;
    }
    case VOTE_RADIAL5DOF: {
        const double nrw = std::sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
        const double nw = std::sqrt(T[3] * T[3] + T[4] * T[4] + T[5] * T[5]);
        lam[0] = lam[1] = lam[2] = nrw + nw;
        lam[3] = T[6];
        break;
    }
    }
}

// Per-solve level constants, once the root records' largest |q| are known
// (qmax[j] for free, qmax[nd + m] for essential parameters): bounds on the records'
// fields at every level, and the record format of
// each level (16-bit fields where every bound stays below 32000; level 0, and
// every level in plain FP64 mode, 32-bit).  A level-l record (l >= 1) passed the
// UB test of level l-1, so |f| <= that radius; |q_t| only shrinks as steps double.
static void finalize_levels(vote_ctx *c, const unsigned *qmax) {
    const Problem &P = c->P;
    double rprev[GV_MAXD] = {};
    for (int l = 0; l < P.L; ++l) {
        Level &v = c->lev[l];
        double T[GV_MAXT], lam[GV_MAXD * GV_MAXD], qtb[GV_MAXT];
        bool fits = c->precision == 1 && l >= 1;
        for (int m = 0; m < P.le; ++m) {
            double ratio = v.s_t[m] / c->lev[0].s_t[m];                 // a power of two >= 1
            qtb[m] = std::floor((double)qmax[P.nd + m] / ratio) + 1.0;
            T[m] = (qtb[m] + 1.0) * v.s_t[m];
            v.qt_max[m] = (float)qtb[m];
            fits &= qtb[m] <= 32000.0;
        }
        lambda_max(P.fam, T, lam);
        for (int j = 0; j < P.nd; ++j) {
            double R = v.Rbase[j];
            for (int i = 0; i < P.k; ++i) R += lam[j * P.k + i] * v.h1[i];
            R = (R + v.A1[j]) * 1.001;
            double qfb = l == 0 ? (double)qmax[j] + 1.0 : std::ceil(rprev[j] / P.s_f[j]) + 1.0;
            fits &= qfb <= 32000.0;
            rprev[j] = R;
        }
        v.q16 = fits ? 1 : 0;
    }
    // a level keeps 16-bit records only if every deeper level does (the bounds shrink
    // with depth, so this only guards the format sequence the emit pass supports)
    for (int l = P.L - 2; l >= 0; --l) c->lev[l].q16 &= c->lev[l + 1].q16;
    for (int l = 0; l < P.L; ++l) c->lev[l].q16_next = l + 1 < P.L ? c->lev[l + 1].q16 : 0;
}

// ---------------------------------------------------------------------------
// device memory
// ---------------------------------------------------------------------------
static vote_status ensure(vote_ctx *c, DevBuf &b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return VOTE_OK;
    size_t want = bytes + bytes / 4 + 256;
    if (b.p) {
        CK(cudaFreeAsync(b.p, c->stream));
        b.p = nullptr;
        b.bytes = 0;
    }
    ++c->alloc_count;
    if (c->fault_alloc_at && c->alloc_count == c->fault_alloc_at) {
        set_err("injected allocation failure (allocation %lld)", (long long)c->alloc_count);
        return VOTE_ENOMEM;
    }
    cudaError_t e = cudaMallocAsync(&b.p, want, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        set_err("device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
        return VOTE_ENOMEM;
    }
    b.bytes = want;
    return VOTE_OK;
}

static void release(vote_ctx *c, DevBuf &b) {
    if (b.p) cudaFreeAsync(b.p, c->stream);
    b.p = nullptr;
    b.bytes = 0;
}

// record fields and basis values of a family, from its device definition
static int family_nfp(int fam) {
    switch (fam) {
    case VOTE_LINE2D: return Fam<FAM_LINE2D>::NFP;
    case VOTE_PLANE3D_SPH: return Fam<FAM_PLANE3D_SPH>::NFP;
    case VOTE_POSE3DOF: return Fam<FAM_POSE3DOF>::NFP;
    case VOTE_RAYS3D: return Fam<FAM_RAYS3D>::NFP;
    case VOTE_POINTSET2D: return Fam<FAM_POINTSET2D>::NFP;
    case VOTE_AFFINE4D: return Fam<FAM_AFFINE4D>::NFP;
    case VOTE_RADIAL5DOF: return Fam<FAM_RADIAL5DOF>::NFP;
    default: return Fam<FAM_POSE6DOF>::NFP;
    }
}
static int family_nb(int fam) {
    switch (fam) {
    case VOTE_LINE2D: return Fam<FAM_LINE2D>::NB;
    case VOTE_PLANE3D_SPH: return Fam<FAM_PLANE3D_SPH>::NB;
    case VOTE_POSE3DOF: return Fam<FAM_POSE3DOF>::NB;
    case VOTE_RAYS3D: return Fam<FAM_RAYS3D>::NB;
    case VOTE_POINTSET2D: return Fam<FAM_POINTSET2D>::NB;
    case VOTE_AFFINE4D: return Fam<FAM_AFFINE4D>::NB;
    case VOTE_RADIAL5DOF: return Fam<FAM_RADIAL5DOF>::NB;
    default: return Fam<FAM_POSE6DOF>::NB;
    }
}
static_assert((int)VOTE_LINE2D == FAM_LINE2D && (int)VOTE_PLANE3D_SPH == FAM_PLANE3D_SPH &&
                  (int)VOTE_POSE3DOF == FAM_POSE3DOF && (int)VOTE_POSE6DOF == FAM_POSE6DOF &&
                  (int)VOTE_RAYS3D == FAM_RAYS3D && (int)VOTE_POINTSET2D == FAM_POINTSET2D &&
                  (int)VOTE_AFFINE4D == FAM_AFFINE4D && (int)VOTE_RADIAL5DOF == FAM_RADIAL5DOF,
              "family numbers");

// bytes of one record of level l (its format is fixed per solve by finalize_levels)
static int rec_bytes_at(const vote_ctx *c, int l) {
    return 4 * rec_words(family_nfp(c->P.fam), l < c->P.L && c->lev[l].q16);
}

// Every array is checked against its own allocated size (ensure returns at once
// when it is large enough), so no separate capacity figure can drift from the
// allocations.  slots: record slots (a multiple of 32).
static vote_status ensure_level(vote_ctx *c, int l, size_t slots, size_t cells) {
    LevelStore &s = c->ls[l];
    if (slots > 0) {
        TRY(ensure(c, s.rec, slots * rec_bytes_at(c, l)));
        if (c->group) TRY(ensure(c, s.mult, slots * 4));   // without grouping every mult is 1
        TRY(ensure(c, s.tile_cell, (slots / 32) * 4));
    }
    if (cells > 0) {
        TRY(ensure(c, s.key, cells * 8));
        TRY(ensure(c, s.rbeg, cells * 8));
        TRY(ensure(c, s.rcnt, cells * 4));
        TRY(ensure(c, s.ub, cells * 4));
    }
    return VOTE_OK;
}

static RecView rec_view(vote_ctx *c, int l) {
    RecView v;
    v.rec = (uint32_t *)c->ls[l].rec.p;
    v.mult = c->group ? (uint32_t *)c->ls[l].mult.p : nullptr;
    v.tile_cell = (uint32_t *)c->ls[l].tile_cell.p;
    return v;
}

static CellView cell_view(vote_ctx *c, int l) {
    CellView v;
    v.key = (uint64_t *)c->ls[l].key.p;
    v.rbeg = (uint64_t *)c->ls[l].rbeg.p;
    v.rcnt = (uint32_t *)c->ls[l].rcnt.p;
    v.ub = (uint32_t *)c->ls[l].ub.p;
    return v;
}

static Scalars *dsc(vote_ctx *c) { return (Scalars *)c->scal.p; }

static vote_status read_scalars(vote_ctx *c) {
    CK(cudaMemcpyAsync(c->h_sc, c->scal.p, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return VOTE_OK;
}

// ---------------------------------------------------------------------------
// kernel timing (CUDA events on the context's stream, read after the stream has
// passed them)
// ---------------------------------------------------------------------------
// Events are recorded in sequence; the interval ending at event i is charged to
// class ev_cls[i] (-1: not charged).  They are read once the stream has passed
// them (at the next synchronisation).
static void ev_mark(vote_ctx *c, int cls) {
    if (!c->kernel_timing || c->ev_n >= vote_ctx::kEv) return;
    cudaEventRecord(c->ev[c->ev_n], c->stream);
    c->ev_cls[c->ev_n] = cls;
    ++c->ev_n;
}

static void ev_collect(vote_ctx *c) {
    if (!c->kernel_timing) return;
    for (int i = 1; i < c->ev_n; ++i) {
        float ms;
        int cls = c->ev_cls[i];
        if (cls >= 0 && cudaEventElapsedTime(&ms, c->ev[i - 1], c->ev[i]) == cudaSuccess) {
            c->kms[cls] += ms;
            c->klaunch[cls] += 1;
        }
    }
    c->ev_n = 0;
}

// ---------------------------------------------------------------------------
// search
// ---------------------------------------------------------------------------

// Expand a chunk of level-l cells taken from the top of the level's stack.  With
// only >= 0, the single cell `only` is expanded where it sits instead (greedy
// dive); its UB is then set to 0, so the sweep later finds it below every
// threshold and gives it no children.
static vote_status expand_chunk(vote_ctx *c, int l, int64_t only = -1) {
    const Problem &P = c->P;
    LevelStore &S = c->ls[l];
    const int ns = c->ns;
    const Level &lev = c->lev[l];
    int nvalid = 0;
    for (int s = 0; s < ns; ++s)
        if (!(s & ~lev.split_mask)) ++nvalid;
    // chunk: cells [c0, c1) from the top of the stack, about chunk_records records
    int64_t c1 = only >= 0 ? only + 1 : S.ncells, r1 = S.nrecs;
    int64_t avg = S.nrecs / (S.ncells > 0 ? S.ncells : 1);
    int64_t K = c->chunk_records / (avg > 0 ? avg : 1);
    if (K < 1 || only >= 0) K = 1;
    if (K > (1 << 22)) K = 1 << 22;
    int64_t c0, r0;
    for (;;) {
        c0 = c1 - K > 0 ? c1 - K : 0;
        CK(cudaMemcpyAsync(c->h_tmp, (uint64_t *)S.rbeg.p + c0, 8, cudaMemcpyDeviceToHost, c->stream));
        if (only >= 0)
            CK(cudaMemcpyAsync(c->h_tmp + 1, (uint32_t *)S.rcnt.p + only, 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        ev_collect(c);
        r0 = (int64_t)c->h_tmp[0];
        if (only >= 0) {
            r1 = r0 + (((int64_t)(uint32_t)c->h_tmp[1] + 31) & ~(int64_t)31);
            break;
        }
        if (r1 - r0 <= 2 * c->chunk_records || K == 1) break;
        K = K / 2;
    }
    nvtxRangePushA("expand_chunk");
    const int nc = (int)(c1 - c0);
    const int nfs = 1 << P.k;
    const int NB = family_nb(P.fam);
    const int gf = geo32_floats(nfs, P.nd, P.le);
    const size_t nch = (size_t)nc * ns;
    TRY(ensure(c, c->alive, nc));
    TRY(ensure(c, c->geo64, (size_t)nc * nfs * NB * 8));
    TRY(ensure(c, c->geo32, (size_t)nc * gf * 4));
    TRY(ensure(c, c->geo32lo, (size_t)nc * nfs * P.nd * P.le * 4));
    TRY(ensure(c, c->cnt, nch * 12));
    TRY(ensure(c, c->child_idx, nch * 4));
    TRY(ensure(c, c->cursor, nch * 4));
    TRY(ensure(c, c->keepflag, nch * 4));
    TRY(ensure(c, c->recn, nch * 4));
    TRY(ensure(c, c->bsums, ((nch + 255) / 256) * 16 + 16));
    if (!lev.leaf_children) TRY(ensure_level(c, l + 1, 0, nch));    // records: sized below, exactly
    CK(cudaMemsetAsync(c->cnt.p, 0, nch * 12, c->stream));
    CK(cudaMemsetAsync(c->cursor.p, 0, nch * 4, c->stream));
    CK(cudaMemsetAsync(&dsc(c)->n_cells, 0, 16, c->stream));

    Chunk ch;
    std::memset(&ch, 0, sizeof(ch));
    ch.P = P;
    ch.lev = lev;
    ch.cells = cell_view(c, l);
    ch.c0 = c0;
    ch.nc = nc;
    ch.in = rec_view(c, l);
    ch.in_rbeg = (const uint64_t *)S.rbeg.p;
    ch.in_rcnt = (const uint32_t *)S.rcnt.p;
    ch.in_c0 = c0;
    ch.t0 = r0 / 32;
    ch.t1 = r1 / 32;
    ch.alive = (uint8_t *)c->alive.p;
    ch.geo64 = (double *)c->geo64.p;
    ch.geo32 = (float *)c->geo32.p;
    ch.geo32lo = (float *)c->geo32lo.p;
    ch.cnt = (uint32_t *)c->cnt.p;
    ch.child_idx = (int32_t *)c->child_idx.p;
    ch.cursor = (uint32_t *)c->cursor.p;
    ch.sc = dsc(c);
    if (c->trace_cap > 0) {
        ch.trace.cap = (unsigned long long)c->trace_cap;
        ch.trace.level = (int32_t *)c->tr_level.p;
        ch.trace.key = (uint64_t *)c->tr_key.p;
        ch.trace.ub = (uint32_t *)c->tr_ub.p;
        ch.trace.lb = (uint32_t *)c->tr_lb.p;
    }
    ch.prune = c->prune;
    ch.precision = c->precision;
    ch.spin = c->spin_limit;

    const int rb = rec_bytes_at(c, l);
    if (c->group && r1 - r0 > 32) {
        // canonization's grouping: merge records with equal (cell, q_f, q_t)
        const size_t nr = (size_t)(r1 - r0);
        size_t cap = 1;
        while (cap < nr * 2) cap <<= 1;
        TRY(ensure(c, c->g_table, cap * 4));
        TRY(ensure(c, c->g_owner, nr * 4));
        TRY(ensure(c, c->g_newpos, nr * 4));
        TRY(ensure(c, c->g_ccount, (size_t)nc * 4));
        TRY(ensure(c, c->g_ccur, (size_t)nc * 4));
        TRY(ensure(c, c->g_rbeg, (size_t)nc * 8));
        // canonical records need at most the slots of the originals plus one tile per cell
        const size_t gslots = nr + 32 * (size_t)nc;
        TRY(ensure(c, c->g_rec, gslots * rb));
        TRY(ensure(c, c->g_mult, gslots * 4));
        TRY(ensure(c, c->g_tile, (gslots / 32) * 4));
        CK(cudaMemsetAsync(c->g_table.p, 0, cap * 4, c->stream));
        CK(cudaMemsetAsync(c->g_ccount.p, 0, (size_t)nc * 4, c->stream));
        CK(cudaMemsetAsync(c->g_ccur.p, 0, (size_t)nc * 4, c->stream));
        RecView gv;
        gv.rec = (uint32_t *)c->g_rec.p;
        gv.mult = (uint32_t *)c->g_mult.p;
        gv.tile_cell = (uint32_t *)c->g_tile.p;
        ev_mark(c, -1);
        launch_group(ch, (uint32_t *)c->g_table.p, (uint32_t)(cap - 1), (uint32_t *)c->g_owner.p,
                     (uint32_t *)c->g_ccount.p, (uint32_t *)c->g_ccur.p, (uint32_t *)c->g_newpos.p,
                     (uint64_t *)c->g_rbeg.p, (unsigned long long *)c->h_tmp_dev(), gv, c->stream);
        ev_mark(c, VOTE_K_GROUP);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(c->h_tmp, c->h_tmp_dev(), 24, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const int64_t gs = (int64_t)c->h_tmp[0];
        c->stats.launches += 4;
        c->kbytes[VOTE_K_GROUP] += (double)nr * (rb + 4) * 2;
        c->lv_gout[l] += (int64_t)c->h_tmp[1];
        c->lv_gin[l] += (int64_t)c->h_tmp[2];
        ch.in = gv;
        ch.in_rbeg = (const uint64_t *)c->g_rbeg.p;
        ch.in_rcnt = (const uint32_t *)c->g_ccount.p;
        ch.in_c0 = 0;
        ch.t0 = 0;
        ch.t1 = gs / 32;
    }
    const int64_t nt = ch.t1 - ch.t0;
    TRY(ensure(c, c->tinfo, (size_t)(nt > 0 ? nt : 1) * 8 + 16));
    TRY(ensure(c, c->ballot, (size_t)(nt > 0 ? nt : 1) * ns * 4));
    ch.tinfo = (int2 *)c->tinfo.p;
    ch.ballot = (uint32_t *)c->ballot.p;
    if (!lev.leaf_children) {
        ch.next_cells = cell_view(c, l + 1);
        ch.out = rec_view(c, l + 1);
    }
    ev_mark(c, -1);
    launch_cell_geo(ch, c->stream);
    launch_tile_info(ch, c->stream);
    ev_mark(c, VOTE_K_CELL_GEO);
    launch_count(ch, c->stream);
    ev_mark(c, VOTE_K_TEST_COUNT);
    launch_child_lbmax(ch, c->stream);
    launch_child_alloc(ch, (uint32_t *)c->keepflag.p, (uint32_t *)c->recn.p, (unsigned long long *)c->bsums.p,
                       c->stream);
    ev_mark(c, VOTE_K_CHILDREN);
    // algorithmic bytes: the records of whole tiles read, the ballots written
    c->kbytes[VOTE_K_TEST_COUNT] += (double)nt * 32 * rb + (double)nt * ns * 4;
    c->kbytes[VOTE_K_CELL_GEO] += (double)nc * (8 + 4);
    CK(cudaGetLastError());
    c->stats.chunks++;
    c->stats.launches += lev.leaf_children ? 5 : 7;
    c->stats.cells += nc;
    c->lv_cells[l] += nc;
    c->lv_recs[l] += nt * 32;
    if (only >= 0) {
        CK(cudaMemsetAsync((uint32_t *)S.ub.p + only, 0, 4, c->stream));
    } else {
        S.ncells = c0;
        S.nrecs = r0;
    }
    if (lev.leaf_children) {
        if (c->log >= 2)
            std::fprintf(stderr, "[vote] step %lld level %d: %lld cells, %lld tiles, count %.0f B, leaves\n",
                         (long long)c->stats.chunks - 1, l, (long long)nc, (long long)nt,
                         (double)nt * 32 * rb + (double)nt * ns * 4);
        c->stats.leaves += (int64_t)nc * nvalid;
        nvtxRangePop();
        return VOTE_OK;
    }
    CK(cudaMemcpyAsync(&c->h_sc->n_cells, &dsc(c)->n_cells, 16, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int64_t new_cells = (int64_t)c->h_sc->n_cells, new_slots = (int64_t)c->h_sc->n_recs;
    if (new_slots > 0) {
        TRY(ensure_level(c, l + 1, (size_t)new_slots, 0));
        TRY(ensure(c, c->tdst, (size_t)nt * ns * 8));
        ch.out = rec_view(c, l + 1);
        ch.tdst = (unsigned long long *)c->tdst.p;
        ev_mark(c, -1);
        launch_next_tiles(ch, new_cells, c->stream);
        launch_tile_dst(ch, c->stream);
        ev_mark(c, VOTE_K_CHILDREN);
        if (!launch_emit(ch, c->stream)) {
            set_err("internal: no emit pass for record formats %d -> %d", lev.q16, lev.q16_next);
            return VOTE_EINTERNAL;
        }
        c->stats.launches += 3;
        ev_mark(c, VOTE_K_TEST_EMIT);
        c->kbytes[VOTE_K_TEST_EMIT] += (double)nt * 32 * rb + (double)nt * ns * 4 +
                                       (double)new_slots * rec_bytes_at(c, l + 1);
    }
    CK(cudaGetLastError());
    if (c->log >= 2) {
        // the running FP64 recheck and test counters (a synchronisation per step: logging only)
        CK(cudaMemcpyAsync(&c->h_sc->tests, &dsc(c)->tests, 24, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(&c->h_sc->rechecks_df, &dsc(c)->rechecks_df, 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::fprintf(stderr, "[vote] step %lld level %d: %lld cells, %lld tiles, count %.0f B, emit %.0f B, "
                     "%lld child cells, %llu tests, %llu FP64 and %llu double-float rechecks so far\n",
                     (long long)c->stats.chunks - 1, l, (long long)nc, (long long)nt,
                     (double)nt * 32 * rb + (double)nt * ns * 4,
                     new_slots > 0 ? (double)nt * 32 * rb + (double)nt * ns * 4 +
                                         (double)new_slots * rec_bytes_at(c, l + 1) : 0.0,
                     (long long)new_cells, c->h_sc->tests, c->h_sc->rechecks, c->h_sc->rechecks_df);
    }
    c->ls[l + 1].ncells = new_cells;
    c->ls[l + 1].nrecs = new_slots;
    if (new_slots > c->stats.peak_records) c->stats.peak_records = new_slots;
    nvtxRangePop();
    return VOTE_OK;
}

static vote_status replay(vote_ctx *c, const double *surfaces, int64_t n, int lam, uint64_t key, uint32_t *reach,
                          int64_t *ub, int64_t *lb) {
    CK(cudaMemsetAsync(&dsc(c)->replay_ub, 0, 16, c->stream));
    ev_mark(c, -1);
    if (lam > 0) launch_path_geo(c->P, (const Level *)c->levs_dev.p, lam, key, (PathStep *)c->path.p, c->stream);
    launch_replay(c->P, (const Level *)c->levs_dev.p, (const PathStep *)c->path.p, lam, surfaces, n, reach,
                  dsc(c), c->stream);
    c->stats.launches += lam > 0 ? 2 : 1;
    ev_mark(c, VOTE_K_REPLAY);
    CK(cudaGetLastError());
    TRY(read_scalars(c));
    ev_collect(c);
    c->kbytes[VOTE_K_REPLAY] += (double)n * (8 * c->P.np) + (double)((n + 31) / 32) * 4;
    *ub = (int64_t)c->h_sc->replay_ub;
    *lb = (int64_t)c->h_sc->replay_lb;
    return VOTE_OK;
}

// Below this many surfaces the dive's per-level host round trips cost more than the
// pruning they buy (the whole search is then a few chunks).
static const int64_t kDiveMinN = 1 << 17;

static vote_status solve_inner(vote_ctx *c, const double *surfaces, int64_t n, double *best_point,
                               int64_t *best_leaf, int64_t *depth, uint32_t *mask);

// Per-level counters of the last solve on stderr (VOTE_LOG=1).
static void log_solve(const vote_ctx *c, vote_status st) {
    const vote_stats &x = c->stats;
    std::fprintf(stderr, "[vote] family %d L %d status %d: %.3f s, %lld tests, %lld FP64 rechecks, %lld chunks, "
                 "%lld launches, peak %lld record slots\n", c->P.fam, c->P.L, (int)st, x.seconds,
                 (long long)x.tests, (long long)x.rechecks, (long long)x.chunks, (long long)x.launches,
                 (long long)x.peak_records);
    for (int l = 0; l < c->P.L; ++l) {
        std::fprintf(stderr, "[vote]   level %2d: %lld cells expanded, %lld record slots tested, records %s", l,
                     (long long)c->lv_cells[l], (long long)c->lv_recs[l], c->lev[l].q16 ? "16-bit" : "32-bit");
        if (c->lv_gin[l])
            std::fprintf(stderr, ", grouping %lld -> %lld records (%.4f merged)", (long long)c->lv_gin[l],
                         (long long)c->lv_gout[l], 1.0 - (double)c->lv_gout[l] / (double)c->lv_gin[l]);
        std::fprintf(stderr, "\n");
    }
}

static vote_status solve_device(vote_ctx *c, const double *surfaces, int64_t n, double *best_point,
                                int64_t *best_leaf, int64_t *depth, uint32_t *mask) {
    nvtxRangePushA("vote_solve");
    vote_status st = solve_inner(c, surfaces, n, best_point, best_leaf, depth, mask);
    nvtxRangePop();
    if (c->log) log_solve(c, st);
    return st;
}

static vote_status solve_inner(vote_ctx *c, const double *surfaces, int64_t n, double *best_point,
                               int64_t *best_leaf, int64_t *depth, uint32_t *mask) {
    auto t0 = std::chrono::steady_clock::now();
    const Problem &P = c->P;
    std::memset(&c->stats, 0, sizeof(c->stats));
    for (int l = 0; l < GV_MAXL; ++l) c->lv_cells[l] = c->lv_recs[l] = c->lv_gin[l] = c->lv_gout[l] = 0;
    c->stats.levels = P.L;
    if (n < 0 || !best_point || !depth || (n > 0 && !surfaces)) {
        set_err("invalid arguments");
        return VOTE_EINVAL;
    }
    if (n >= (int64_t)1 << 31 || (P.coord_bits > 0 && (uint64_t)n >= (1ull << (64 - P.coord_bits)))) {
        set_err("n = %lld too large", (long long)n);
        return VOTE_EUNSUPPORTED;
    }
    CK(cudaMemsetAsync(c->scal.p, 0, sizeof(Scalars), c->stream));
    if (c->initial_lb) CK(cudaMemcpyAsync(&dsc(c)->best_lb, &c->initial_lb, 4, cudaMemcpyHostToDevice, c->stream));
    for (int i = 0; i < VOTE_K_CLASSES; ++i) c->kms[i] = c->kbytes[i] = 0, c->klaunch[i] = 0;
    c->ev_n = 0;
    c->trace_written = 0;
    c->trace_overflow = false;
    for (int l = 0; l <= P.L; ++l) c->ls[l].ncells = c->ls[l].nrecs = 0;
    uint64_t leafkey = 0;
    int64_t dep = 0;
    if (n > 0 && P.L == 0) {
        dep = n;                                   // the domain is a leaf: every surface counts
    } else if (n > 0) {
        const int64_t slots0 = (n + 31) & ~(int64_t)31;
        TRY(ensure_level(c, 0, (size_t)slots0, 1));
        ev_mark(c, -1);
        launch_lift(P, c->lev[0], surfaces, n, rec_view(c, 0), dsc(c), c->stream);
        c->stats.launches += 1;
        ev_mark(c, VOTE_K_LIFT);
        CK(cudaGetLastError());
        uint64_t key0 = 0, rb0 = 0;
        uint32_t cnt0 = (uint32_t)n;
        CK(cudaMemcpyAsync(c->ls[0].key.p, &key0, 8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->ls[0].rbeg.p, &rb0, 8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->ls[0].rcnt.p, &cnt0, 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->ls[0].ub.p, &cnt0, 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));    // host sources above live on this frame
        c->ls[0].ncells = 1;
        c->ls[0].nrecs = slots0;
        TRY(read_scalars(c));
        ev_collect(c);
        c->kbytes[VOTE_K_LIFT] += (double)n * (8 * P.np + rec_bytes_at(c, 0) + (c->group ? 4 : 0));
        if (c->h_sc->err) {
            set_err("surface parameters are not finite or out of the representable range");
            return VOTE_EINVAL;
        }
        finalize_levels(c, c->h_sc->qmax);
        if (c->dive == 1 || (c->dive == 2 && n >= kDiveMinN)) {
            // greedy dive: from the root, expand only the child with the largest UB
            // (the first on ties) down to the leaves, so the sweep starts with a
            // leaf's count as its pruning bound
            int64_t cell = 0;
            for (int l = 0; l < P.L; ++l) {
                TRY(expand_chunk(c, l, cell));
                int64_t m = l + 1 < P.L ? c->ls[l + 1].ncells : 0;
                if (m <= 0) break;
                uint32_t best = 0;
                cell = -1;
                for (int64_t i0 = 0; i0 < m; i0 += 16) {      // 16 UBs fit the pinned slot
                    int64_t k = m - i0 < 16 ? m - i0 : 16;
                    CK(cudaMemcpyAsync(c->h_tmp, (uint32_t *)c->ls[l + 1].ub.p + i0, 4 * (size_t)k,
                                       cudaMemcpyDeviceToHost, c->stream));
                    CK(cudaStreamSynchronize(c->stream));
                    const uint32_t *ub = (const uint32_t *)c->h_tmp;
                    for (int64_t i = 0; i < k; ++i)
                        if (cell < 0 || ub[i] > best) best = ub[i], cell = i0 + i;
                }
            }
        }
        for (;;) {
            int l = -1;
            for (int x = P.L - 1; x >= 0; --x)
                if (c->ls[x].ncells > 0) {
                    l = x;
                    break;
                }
            if (l < 0) break;
            TRY(expand_chunk(c, l));
        }
        TRY(read_scalars(c));
        ev_collect(c);
        if (c->h_sc->err & kErrTimeout) {
            set_err("a bounded device-side wait ran out (bulk copy not completed)");
            return VOTE_ETIMEOUT;
        }
        if (c->h_sc->err) {
            set_err("internal: residual out of range (err %u)", c->h_sc->err);
            return VOTE_EINTERNAL;
        }
        unsigned long long bk = c->h_sc->best_key;
        if (bk) {
            dep = (int64_t)(bk >> P.coord_bits);
            leafkey = ~bk & ((1ull << P.coord_bits) - 1ull);
        }
        c->stats.tests = (int64_t)c->h_sc->tests;
        c->stats.records = (int64_t)c->h_sc->records;
        c->stats.rechecks = (int64_t)c->h_sc->rechecks;
        c->trace_written = (int64_t)c->h_sc->trace_n;
        if (c->trace_cap && c->trace_written > c->trace_cap) c->trace_overflow = true;
    }
    *depth = dep;
    for (int j = 0; j < P.d; ++j) {
        int64_t i = (int64_t)((leafkey >> P.coord_shift[j]) & ((1ull << P.Lj[j]) - 1ull));
        if (best_leaf) best_leaf[j] = i;
        best_point[j] = P.lo[j] + (double)(2 * i + 1) * c->h_leaf[j];
    }
    if (mask && n > 0) {
        if (dep > 0) {
            int64_t ub = 0, lb = 0;
            TRY(replay(c, surfaces, n, P.L, leafkey, mask, &ub, &lb));
            if (ub != dep) {
                set_err("internal: replayed inlier count %lld != depth %lld", (long long)ub, (long long)dep);
                return VOTE_EINTERNAL;
            }
        } else {
            CK(cudaMemsetAsync(mask, 0, (size_t)((n + 31) / 32) * 4, c->stream));
        }
    }
    CK(cudaStreamSynchronize(c->stream));
    c->stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return VOTE_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *vote_last_error(void) { return g_err; }

vote_status vote_create(int family, int d, int k, const double *eps, const double *bounds, vote_ctx **out) {
    if (!out || !eps || !bounds) {
        set_err("null argument");
        return VOTE_EINVAL;
    }
    *out = nullptr;
    vote_ctx *c = new (std::nothrow) vote_ctx();
    if (!c) {
        set_err("out of host memory");
        return VOTE_ENOMEM;
    }
    vote_status s = problem_init(c, family, d, k, eps, bounds);
    if (s != VOTE_OK) {
        delete c;
        return s;
    }
    c->ns = 1 << d;
    // step size measured fastest on GB300 (1e6-surface workloads): planes keep almost
    // every cell above the bound, so larger steps only remove per-step overhead;
    // 3DoF prunes well and needs fine depth-first steps
    // a step's children can hold 2^d times its records: 64-child families take
    // smaller steps so that the next level's records stay within a few GB
    c->chunk_records = family == VOTE_PLANE3D_SPH ? (int64_t)1 << 27
                       : (d >= 6 ? (int64_t)1 << 21 : (d >= 4 ? (int64_t)1 << 23 : (int64_t)1 << 25));
    c->family = family;
    if (const char *lg = std::getenv("VOTE_LOG")) c->log = std::atoi(lg) > 0 ? std::atoi(lg) : 0;
    for (int j = 0; j < d; ++j) {
        c->eps_in[j] = eps[j];
        c->bounds_in[2 * j] = bounds[2 * j];
        c->bounds_in[2 * j + 1] = bounds[2 * j + 1];
    }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_sc, sizeof(Scalars));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_tmp, 64);
    if (e != cudaSuccess) {
        set_err("CUDA unavailable: %s", cudaGetErrorString(e));
        delete c;
        return VOTE_ECUDA;
    }
    s = ensure(c, c->scal, ((sizeof(Scalars) + 63) / 64) * 64 + 64);
    if (s == VOTE_OK) s = ensure(c, c->levs_dev, sizeof(Level) * (c->P.L > 0 ? c->P.L : 1));
    if (s == VOTE_OK) s = ensure(c, c->path, sizeof(PathStep) * (c->P.L > 0 ? c->P.L : 1));
    if (s == VOTE_OK && c->P.L > 0) {
        e = cudaMemcpyAsync(c->levs_dev.p, c->lev, sizeof(Level) * c->P.L, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            set_err("upload of level constants failed: %s", cudaGetErrorString(e));
            s = VOTE_ECUDA;
        }
    }
    if (s != VOTE_OK) {
        vote_destroy(c);
        return s;
    }
    *out = c;
    return VOTE_OK;
}

vote_status vote_set_option(vote_ctx *c, int key, double v) {
    if (!c) { set_err("null context"); return VOTE_EINVAL; }
    switch (key) {
    case VOTE_OPT_PRECISION:
        if (v != 0 && v != 1) break;
        c->precision = (int)v;
        return VOTE_OK;
    case VOTE_OPT_PRUNE:
        if (v != 0 && v != 1) break;
        c->prune = (int)v;
        return VOTE_OK;
    case VOTE_OPT_CHUNK_RECORDS:
        if (!(v >= 1 && v <= 1e10)) break;
        c->chunk_records = (int64_t)v;
        return VOTE_OK;
    case VOTE_OPT_TRACE_CAP: {
        if (!(v >= 0 && v <= 1e9)) break;
        c->trace_cap = (int64_t)v;
        if (c->trace_cap > 0) {
            size_t m = (size_t)c->trace_cap;
            TRY(ensure(c, c->tr_level, m * 4));
            TRY(ensure(c, c->tr_key, m * 8));
            TRY(ensure(c, c->tr_ub, m * 4));
            TRY(ensure(c, c->tr_lb, m * 4));
        }
        return VOTE_OK;
    }
    case VOTE_OPT_GROUP:
        if (v != 0 && v != 1) break;
        c->group = (int)v;
        return VOTE_OK;
    case VOTE_OPT_FAULT_ALLOC_AT:
        if (!(v >= 0)) break;
        c->fault_alloc_at = (int64_t)v;
        c->alloc_count = 0;
        return VOTE_OK;
    case VOTE_OPT_INITIAL_LB:
        if (!(v >= 0 && v < 4294967295.0)) break;
        c->initial_lb = (uint32_t)v;
        return VOTE_OK;
    case VOTE_OPT_KERNEL_TIMING:
        if (v != 0 && v != 1) break;
        if (v == 1 && !c->ev[0])
            for (int i = 0; i < vote_ctx::kEv; ++i) CK(cudaEventCreate(&c->ev[i]));
        c->kernel_timing = (int)v;
        return VOTE_OK;
    case VOTE_OPT_BATCH_WORKERS:
        if (!(v >= 1 && v <= 32)) break;
        c->batch_workers = (int)v;
        return VOTE_OK;
    case VOTE_OPT_DIVE:
        if (v != 0 && v != 1 && v != 2) break;
        c->dive = (int)v;
        return VOTE_OK;
    case VOTE_OPT_SPIN_LIMIT:
        if (!(v >= 0 && v <= 4294967295.0)) break;
        c->spin_limit = (unsigned)v;
        return VOTE_OK;

    default:
        set_err("unknown option %d", key);
        return VOTE_EINVAL;
    }
    set_err("option %d: value %g out of range", key, v);
    return VOTE_EINVAL;
}

vote_status vote_set_stream(vote_ctx *c, void *stream) {
    if (!c) { set_err("null context"); return VOTE_EINVAL; }
    c->stream = (cudaStream_t)stream;
    return VOTE_OK;
}

vote_status vote_solve(vote_ctx *c, const double *surfaces, int64_t n, double *best_point, int64_t *best_leaf,
                       int64_t *depth, uint32_t *inlier_mask) {
    if (!c) { set_err("null context"); return VOTE_EINVAL; }
    return solve_device(c, surfaces, n, best_point, best_leaf, depth, inlier_mask);
}

vote_status vote_solve_host(vote_ctx *c, const double *surfaces, int64_t n, double *best_point, int64_t *best_leaf,
                            int64_t *depth, uint32_t *inlier_mask) {
    if (!c) { set_err("null context"); return VOTE_EINVAL; }
    if (n < 0 || (n > 0 && !surfaces)) { set_err("invalid arguments"); return VOTE_EINVAL; }
    size_t in_bytes = (size_t)n * c->P.np * 8, words = (size_t)(n + 31) / 32;
    TRY(ensure(c, c->surf_tmp, in_bytes > 0 ? in_bytes : 8));
    TRY(ensure(c, c->mask_tmp, words > 0 ? words * 4 : 4));
    if (n > 0) CK(cudaMemcpyAsync(c->surf_tmp.p, surfaces, in_bytes, cudaMemcpyHostToDevice, c->stream));
    TRY(solve_device(c, (const double *)c->surf_tmp.p, n, best_point, best_leaf, depth,
                     inlier_mask ? (uint32_t *)c->mask_tmp.p : nullptr));
    if (inlier_mask && words) {
        CK(cudaMemcpyAsync(inlier_mask, c->mask_tmp.p, words * 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return VOTE_OK;
}

vote_status vote_solve_batched(vote_ctx *c, const double *surfaces, const int64_t *offsets, int B,
                               double *best_points, int64_t *best_leaves, int64_t *depths, uint32_t *masks,
                               double *latency_ms) {
    if (!c || !offsets || B < 0 || !best_points || !depths) { set_err("invalid arguments"); return VOTE_EINVAL; }
    std::memset(&c->stats, 0, sizeof(c->stats));     // this batch's counters, even when it is empty
    if (offsets[0] != 0) { set_err("offsets[0] must be 0"); return VOTE_EINVAL; }
    for (int b = 0; b < B; ++b)
        if (offsets[b + 1] < offsets[b]) { set_err("offsets must be non-decreasing"); return VOTE_EINVAL; }
    if (B == 0) return VOTE_OK;
    if (offsets[B] > 0 && !surfaces) { set_err("null surfaces"); return VOTE_EINVAL; }
    const int d = c->P.d, np = c->P.np;
    int nw = c->batch_workers < B ? c->batch_workers : B;
    CK(cudaSetDevice(c->device));
    while ((int)c->workers.size() < nw) {     // sub-contexts with their own streams
        vote_ctx *w = nullptr;
        TRY(vote_create(c->family, d, c->P.k, c->eps_in, c->bounds_in, &w));
        cudaStream_t ws;
        cudaError_t e = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
        if (e != cudaSuccess) { vote_destroy(w); set_err("stream creation failed"); return VOTE_ECUDA; }
        w->stream = ws;
        c->workers.push_back(w);
    }
    for (int i = 0; i < nw; ++i) {
        vote_ctx *w = c->workers[i];
        w->precision = c->precision;
        w->prune = c->prune;
        w->chunk_records = c->chunk_records;
        w->dive = c->dive;
        w->group = c->group;
        w->spin_limit = c->spin_limit;
        w->fault_alloc_at = 0;
    }
    std::vector<int64_t> wordoff(B + 1, 0);
    for (int b = 0; b < B; ++b) wordoff[b + 1] = wordoff[b] + (offsets[b + 1] - offsets[b] + 31) / 32;
    CK(cudaStreamSynchronize(c->stream));     // inputs written on the caller's stream are visible
    std::atomic<int> next(0);
    std::atomic<int> failed(0);
    std::vector<vote_status> wst(nw, VOTE_OK);
    std::vector<std::string> wmsg(nw);
    std::vector<vote_stats> wsum((size_t)nw);   // per worker: totals over its problems
    for (auto &x : wsum) std::memset(&x, 0, sizeof(x));
    auto t0 = std::chrono::steady_clock::now();
    auto work = [&](int wi) {
        vote_ctx *w = c->workers[wi];
        cudaSetDevice(c->device);
        for (;;) {
            int b = next.fetch_add(1);
            if (b >= B || failed.load()) break;
            int64_t n = offsets[b + 1] - offsets[b];
            vote_status st = solve_device(w, surfaces + np * offsets[b], n, best_points + (size_t)b * d,
                                          best_leaves ? best_leaves + (size_t)b * d : nullptr, depths + b,
                                          masks ? masks + wordoff[b] : nullptr);
            if (st != VOTE_OK) {
                wst[wi] = st;
                wmsg[wi] = g_err;
                failed.store(1);
                break;
            }
            if (latency_ms)
                latency_ms[b] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            vote_stats &a = wsum[wi];
            const vote_stats &e = w->stats;
            a.levels = e.levels > a.levels ? e.levels : a.levels;
            a.cells += e.cells;
            a.records += e.records;
            a.tests += e.tests;
            a.rechecks += e.rechecks;
            a.chunks += e.chunks;
            a.leaves += e.leaves;
            a.peak_records = e.peak_records > a.peak_records ? e.peak_records : a.peak_records;
            a.launches += e.launches;
        }
    };
    std::vector<std::thread> th;
    for (int i = 1; i < nw; ++i) th.emplace_back(work, i);
    work(0);
    for (auto &t : th) t.join();
    std::memset(&c->stats, 0, sizeof(c->stats));
    for (int i = 0; i < nw; ++i) {
        if (wst[i] != VOTE_OK) {
            set_err("%s", wmsg[i].c_str());
            return wst[i];
        }
    }
    for (int i = 0; i < nw; ++i) {                  // statistics of the whole batch
        const vote_stats &a = wsum[i];
        c->stats.levels = a.levels > c->stats.levels ? a.levels : c->stats.levels;
        c->stats.cells += a.cells;
        c->stats.records += a.records;
        c->stats.tests += a.tests;
        c->stats.rechecks += a.rechecks;
        c->stats.chunks += a.chunks;
        c->stats.leaves += a.leaves;
        c->stats.peak_records = a.peak_records > c->stats.peak_records ? a.peak_records : c->stats.peak_records;
        c->stats.launches += a.launches;
    }
    c->stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return VOTE_OK;
}

vote_status vote_cell_counts(vote_ctx *c, const double *surfaces, int64_t n, int level, const int64_t *coords,
                             int64_t *ub, int64_t *lb, uint32_t *reach) {
    if (!c || !coords || !ub || !lb || n < 0 || (n > 0 && !surfaces)) { set_err("invalid arguments"); return VOTE_EINVAL; }
    const Problem &P = c->P;
    if (level < 0 || level > P.L) { set_err("level %d outside [0, %d]", level, P.L); return VOTE_EINVAL; }
    uint64_t key = 0;
    for (int j = 0; j < P.d; ++j) {
        int e = level < P.Lj[j] ? level : P.Lj[j];
        if (coords[j] < 0 || coords[j] >= ((int64_t)1 << e)) { set_err("coordinate %d out of range", j); return VOTE_EINVAL; }
        key |= (uint64_t)coords[j] << (P.coord_shift[j] + P.Lj[j] - e);
    }
    if (n == 0) { *ub = 0; *lb = 0; return VOTE_OK; }
    TRY(replay(c, surfaces, n, level, key, reach, ub, lb));
    return VOTE_OK;
}

static vote_status ss_prepare(vote_ctx *c, const double *tol, double *inv_tol2) {
    const Problem &P = c->P;
    if (!softscore_supported(P.fam)) {
        set_err("the soft score is not available for family %d", P.fam);
        return VOTE_EUNSUPPORTED;
    }
    for (int j = 0; j < P.nd; ++j) {
        double t = tol ? tol[j] : P.eps[P.k + j];
        if (!(t > 0.0) || !std::isfinite(t)) { set_err("tol must be finite and > 0"); return VOTE_EINVAL; }
        inv_tol2[j] = 1.0 / (t * t);
    }
    TRY(ensure(c, c->ss_partial, sizeof(double) * softscore_partial_doubles()));
    TRY(ensure(c, c->ss_io, sizeof(double) * (2 * GV_MAXD + 2)));
    return VOTE_OK;
}

vote_status vote_softscore_fwd(vote_ctx *c, const double *surfaces, int64_t n, const uint32_t *mask,
                               const double *point, const double *tol, double *score) {
    if (!c || n < 0 || (n > 0 && !surfaces) || !point || !score) { set_err("invalid arguments"); return VOTE_EINVAL; }
    double inv_tol2[GV_MAXD];
    TRY(ss_prepare(c, tol, inv_tol2));
    if (n == 0) { CK(cudaMemsetAsync(score, 0, sizeof(double), c->stream)); return VOTE_OK; }
    launch_softscore(c->P.fam, false, surfaces, n, mask, point, inv_tol2, c->P.nd, nullptr, nullptr,
                     (double *)c->ss_partial.p, score, c->stream);
    CK(cudaGetLastError());
    return VOTE_OK;
}

vote_status vote_softscore_bwd(vote_ctx *c, const double *surfaces, int64_t n, const uint32_t *mask,
                               const double *point, const double *tol, const double *grad_score,
                               double *grad_point, double *grad_surfaces) {
    if (!c || n < 0 || (n > 0 && !surfaces) || !point || !grad_score) { set_err("invalid arguments"); return VOTE_EINVAL; }
    double inv_tol2[GV_MAXD];
    TRY(ss_prepare(c, tol, inv_tol2));
    double *gp = grad_point ? grad_point : (double *)c->ss_io.p + GV_MAXD;
    if (n == 0) { CK(cudaMemsetAsync(gp, 0, sizeof(double) * c->P.d, c->stream)); return VOTE_OK; }
    launch_softscore(c->P.fam, true, surfaces, n, mask, point, inv_tol2, c->P.nd, grad_score, grad_surfaces,
                     (double *)c->ss_partial.p, gp, c->stream);
    CK(cudaGetLastError());
    return VOTE_OK;
}

vote_status vote_refine(vote_ctx *c, const double *surfaces, int64_t n, const uint32_t *mask, const double *cell_lo,
                        const double *cell_hi, const double *tol, int iters, double *point_inout,
                        double *score_out) {
    if (!c || n < 0 || (n > 0 && !surfaces) || !cell_lo || !cell_hi || !point_inout || iters < 0) {
        set_err("invalid arguments");
        return VOTE_EINVAL;
    }
    const int d = c->P.d;
    for (int j = 0; j < d; ++j)
        if (!(cell_hi[j] >= cell_lo[j])) { set_err("empty cell in coordinate %d", j); return VOTE_EINVAL; }
    double inv_tol2[GV_MAXD];
    TRY(ss_prepare(c, tol, inv_tol2));
    double *dio = (double *)c->ss_io.p;       // [0, d): point, [d, 2d): outputs, [2 MAXD]: 1.0
    double host[2 * GV_MAXD + 2];
    auto eval = [&](const double *pt, bool grad, double *res) -> vote_status {
        std::memcpy(host, pt, sizeof(double) * d);
        host[2 * GV_MAXD] = 1.0;
        CK(cudaMemcpyAsync(dio, host, sizeof(double) * d, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(dio + 2 * GV_MAXD, host + 2 * GV_MAXD, sizeof(double), cudaMemcpyHostToDevice, c->stream));
        launch_softscore(c->P.fam, grad, surfaces, n, mask, dio, inv_tol2, c->P.nd, dio + 2 * GV_MAXD, nullptr,
                         (double *)c->ss_partial.p, dio + GV_MAXD, c->stream);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(res, dio + GV_MAXD, sizeof(double) * (grad ? d : 1), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return VOTE_OK;
    };
    double p[GV_MAXD], q[GV_MAXD], g[GV_MAXD], D[GV_MAXD], S = 0.0, Sq = 0.0;
    for (int j = 0; j < d; ++j) {
        p[j] = std::fmin(std::fmax(point_inout[j], cell_lo[j]), cell_hi[j]);
        D[j] = (cell_hi[j] - cell_lo[j]) * (cell_hi[j] - cell_lo[j]);
    }
    if (n > 0) {
        TRY(eval(p, false, &S));
        for (int it = 0; it < iters; ++it) {
            TRY(eval(p, true, g));
            double gdg = 0.0;
            for (int j = 0; j < d; ++j) gdg += g[j] * g[j] * D[j];
            if (!(gdg > 0.0)) break;
            bool moved = false;
            for (double t = 1.0 / std::sqrt(gdg); t > 1e-14; t *= 0.5) {
                for (int j = 0; j < d; ++j) q[j] = std::fmin(std::fmax(p[j] + t * D[j] * g[j], cell_lo[j]), cell_hi[j]);
                TRY(eval(q, false, &Sq));
                if (Sq >= S + 1e-4 * t * gdg) {
                    std::memcpy(p, q, sizeof(double) * d);
                    S = Sq;
                    moved = true;
                    break;
                }
            }
            if (!moved) break;
        }
    }
    std::memcpy(point_inout, p, sizeof(double) * d);
    if (score_out) *score_out = S;
    return VOTE_OK;
}

vote_status vote_leaf_box(vote_ctx *c, const int64_t *leaf, double *lo, double *hi) {
    if (!c || !leaf || !lo || !hi) { set_err("invalid arguments"); return VOTE_EINVAL; }
    const Problem &P = c->P;
    for (int j = 0; j < P.d; ++j) {
        if (leaf[j] < 0 || leaf[j] >= ((int64_t)1 << P.Lj[j])) { set_err("leaf coordinate %d out of range", j); return VOTE_EINVAL; }
        double w = 2.0 * c->h_leaf[j];
        lo[j] = P.lo[j] + (double)leaf[j] * w;
        hi[j] = lo[j] + w;
    }
    return VOTE_OK;
}

vote_status vote_levels(vote_ctx *c, int *L, int *Lj) {
    if (!c || !L) { set_err("invalid arguments"); return VOTE_EINVAL; }
    *L = c->P.L;
    if (Lj) for (int j = 0; j < c->P.d; ++j) Lj[j] = c->P.Lj[j];
    return VOTE_OK;
}

vote_status vote_level_constants(int family, int d, int k, const double *eps, const double *bounds, int *L,
                                 int *Lj, double *s_f, double *s_t, double *A) {
    if (!eps || !bounds || !L) { set_err("invalid arguments"); return VOTE_EINVAL; }
    vote_ctx tmp;                        // host-side constants only (no device memory)
    TRY(problem_init(&tmp, family, d, k, eps, bounds));
    const Problem &P = tmp.P;
    *L = P.L;
    if (Lj) for (int j = 0; j < P.d; ++j) Lj[j] = P.Lj[j];
    if (s_f) for (int j = 0; j < P.nd; ++j) s_f[j] = P.s_f[j];
    for (int l = 0; l < P.L; ++l) {
        if (s_t) for (int m = 0; m < P.le; ++m) s_t[(size_t)l * P.le + m] = tmp.lev[l].s_t[m];
        if (A) for (int j = 0; j < P.nd; ++j) A[(size_t)l * P.nd + j] = tmp.lev[l].A1[j];
    }
    return VOTE_OK;
}

vote_status vote_get_trace(vote_ctx *c, int64_t cap, int32_t *level, int64_t *coords, int64_t *ub, int64_t *lb,
                           int64_t *count) {
    if (!c || !count || cap < 0) { set_err("invalid arguments"); return VOTE_EINVAL; }
    int64_t m = c->trace_written < c->trace_cap ? c->trace_written : c->trace_cap;
    if (m > cap) m = cap;
    *count = m;
    if (m > 0) {
        int32_t *lv = new int32_t[m];
        uint64_t *ky = new uint64_t[m];
        uint32_t *u = new uint32_t[m], *b = new uint32_t[m];
        cudaError_t e = cudaMemcpy(lv, c->tr_level.p, m * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(ky, c->tr_key.p, m * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(u, c->tr_ub.p, m * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(b, c->tr_lb.p, m * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            const Problem &P = c->P;
            for (int64_t i = 0; i < m; ++i) {
                if (level) level[i] = lv[i];
                if (ub) ub[i] = u[i];
                if (lb) lb[i] = b[i];
                if (coords)
                    for (int j = 0; j < P.d; ++j) {
                        int ex = lv[i] < P.Lj[j] ? lv[i] : P.Lj[j];
                        coords[i * P.d + j] = (int64_t)((ky[i] >> (P.coord_shift[j] + P.Lj[j] - ex)) & ((1ull << ex) - 1ull));
                    }
            }
        }
        delete[] lv; delete[] ky; delete[] u; delete[] b;
        if (e != cudaSuccess) { set_err("trace copy failed: %s", cudaGetErrorString(e)); return VOTE_ECUDA; }
    }
    if (c->trace_overflow) { set_err("trace overflowed (%lld entries)", (long long)c->trace_written); return VOTE_ECAPACITY; }
    return VOTE_OK;
}

vote_status vote_get_kernel_times(vote_ctx *c, double *ms, int64_t *launches, double *bytes) {
    if (!c) { set_err("null context"); return VOTE_EINVAL; }
    for (int i = 0; i < VOTE_K_CLASSES; ++i) {
        if (ms) ms[i] = c->kms[i];
        if (launches) launches[i] = c->klaunch[i];
        if (bytes) bytes[i] = c->kbytes[i];
    }
    return VOTE_OK;
}

vote_status vote_get_level_stats(vote_ctx *c, int64_t *cells, int64_t *records, int64_t *grouped_in,
                                 int64_t *grouped_out) {
    if (!c) { set_err("null context"); return VOTE_EINVAL; }
    for (int l = 0; l < c->P.L; ++l) {
        if (cells) cells[l] = c->lv_cells[l];
        if (records) records[l] = c->lv_recs[l];
        if (grouped_in) grouped_in[l] = c->lv_gin[l];
        if (grouped_out) grouped_out[l] = c->lv_gout[l];
    }
    return VOTE_OK;
}

vote_status vote_get_stats(vote_ctx *c, vote_stats *out) {
    if (!c || !out) { set_err("invalid arguments"); return VOTE_EINVAL; }
    *out = c->stats;
    return VOTE_OK;
}

void vote_destroy(vote_ctx *c) {
    if (!c) return;
    for (vote_ctx *w : c->workers) {
        cudaStream_t ws = w->stream;
        vote_destroy(w);
        if (ws) cudaStreamDestroy(ws);
    }
    c->workers.clear();
    for (int l = 0; l <= GV_MAXL; ++l) {
        LevelStore &s = c->ls[l];
        release(c, s.rec); release(c, s.mult); release(c, s.tile_cell);
        release(c, s.key); release(c, s.rbeg); release(c, s.rcnt); release(c, s.ub);
    }
    DevBuf *bufs[] = {&c->levs_dev, &c->path, &c->scal, &c->alive, &c->geo64, &c->geo32, &c->geo32lo, &c->cnt, &c->tinfo,
                      &c->ballot, &c->tdst,
                      &c->child_idx, &c->cursor, &c->keepflag, &c->recn, &c->bsums, &c->tr_level, &c->tr_key,
                      &c->tr_ub, &c->tr_lb, &c->surf_tmp, &c->mask_tmp, &c->ss_partial,
                      &c->ss_io, &c->g_table, &c->g_owner, &c->g_newpos, &c->g_ccount, &c->g_ccur,
                      &c->g_rbeg, &c->g_rec, &c->g_mult, &c->g_tile};
    for (DevBuf *b : bufs) release(c, *b);
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < vote_ctx::kEv; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->h_tmp) cudaFreeHost(c->h_tmp);
    delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Entry point without allocation (vote_cell_counts_noalloc).  Its scratch is this
// file-scope device array; host code must not use the symbol as an address (in
// host code it names a host-side stand-in), so the device address is looked up
// once per device with cudaGetSymbolAddress and passed to the kernels.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[VOTE_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr size_t kNaLevels = 0;
constexpr size_t kNaPath = kNaLevels + sizeof(Level) * GV_MAXL;
constexpr size_t kNaScalars = (kNaPath + sizeof(PathStep) * GV_MAXL + 255) / 256 * 256;
constexpr size_t kNaEnd = kNaScalars + sizeof(Scalars);
static_assert(kNaEnd <= VOTE_NOALLOC_SCRATCH_BYTES, "no-alloc scratch too small");

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char *g_na_ptr[kNaMaxDevices] = {};
}  // namespace

static vote_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_err("device %d out of range", dev);
        return VOTE_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));   // once per device, this device current
        g_na_ptr[dev] = (unsigned char *)p;
    }
    *out = g_na_ptr[dev];
    return VOTE_OK;
}

extern "C" vote_status vote_cell_counts_noalloc(int family, int d, int k, const double *eps, const double *bounds,
                                                const double *surfaces, int64_t n, int level,
                                                const int64_t *coords, int64_t *ub, int64_t *lb, uint32_t *reach,
                                                void *cuda_stream) {
    if (!eps || !bounds || !coords || !ub || !lb || n < 0 || (n > 0 && !surfaces)) {
        set_err("invalid arguments");
        return VOTE_EINVAL;
    }
    vote_ctx tmp;                        // host-side constants only (no device memory)
    TRY(problem_init(&tmp, family, d, k, eps, bounds));
    const Problem &P = tmp.P;
    if (P.L > GV_MAXL - 1) {
        set_err("%d levels exceed the no-alloc scratch (%d)", P.L, GV_MAXL - 1);
        return VOTE_EUNSUPPORTED;
    }
    if (level < 0 || level > P.L) { set_err("level %d outside [0, %d]", level, P.L); return VOTE_EINVAL; }
    uint64_t key = 0;
    for (int j = 0; j < P.d; ++j) {
        int e = level < P.Lj[j] ? level : P.Lj[j];
        if (coords[j] < 0 || coords[j] >= ((int64_t)1 << e)) { set_err("coordinate %d out of range", j); return VOTE_EINVAL; }
        key |= (uint64_t)coords[j] << (P.coord_shift[j] + P.Lj[j] - e);
    }
    if (n == 0) { *ub = 0; *lb = 0; return VOTE_OK; }
    unsigned char *base = nullptr;
    TRY(noalloc_scratch(&base));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Level *levs = (Level *)(base + kNaLevels);
    PathStep *path = (PathStep *)(base + kNaPath);
    Scalars *sc = (Scalars *)(base + kNaScalars);
    if (P.L > 0) CK(cudaMemcpyAsync(levs, tmp.lev, sizeof(Level) * P.L, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(sc, 0, sizeof(Scalars), st));        // the counters must start at zero
    if (level > 0) launch_path_geo(P, levs, level, key, path, st);
    launch_replay(P, levs, path, level, surfaces, n, reach, sc, st);
    CK(cudaGetLastError());
    unsigned long long cnt[2] = {0, 0};
    CK(cudaMemcpyAsync(cnt, &sc->replay_ub, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *ub = (int64_t)cnt[0];
    *lb = (int64_t)cnt[1];
    return VOTE_OK;
}
