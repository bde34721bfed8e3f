// gv_device.cuh -- device-side definitions of the general-voting hot path.
//
// Surfaces follow Sec. 3, Eq. 1 of Aiger et al. (arXiv 2107.11810):
// x_j = F_j(x_free; t) + f_j.  A record holds one canonical surface in the frame of
// its cell: the free parameter as an integer multiple q_f of the snap step s_f
// (its vertical residual at the cell centre) and the essential parameters as
// integer multiples q_t of the level's step s_t (canonization, Sec. 3.2).
//
// Every FP64 operation that decides a count is issued as one explicitly rounded
// IEEE operation (__dadd_rn, __dmul_rn, ...), in a fixed order, so the compiler
// cannot fuse or reorder it; the results are bit-identical to the definition.
// The FP32 screen works in units of the free-parameter step: a record's residual
// at a child centre is u_j = q_f,j + sum_m q_t,m G_jm - H_j, with G_jm the
// coefficient of t_m in that residual scaled by s_t,m / s_f,j (exact power-of-two
// scaling of an FP64 value rounded once to FP32) and H_j the child shift in steps.
#pragma once
#include <cstdint>
#include <cstring>

#define GV_MAXD 6
#define GV_MAXT 11
#define GV_MAXL 32

namespace gv {

// ---------------------------------------------------------------------------
// Problem and level constants (computed once on the host, passed by value).
// ---------------------------------------------------------------------------
struct Problem {
    int fam, d, k, nd, le, np, L;
    int Lj[GV_MAXD];
    int coord_shift[GV_MAXD];  // bit offset of coordinate j in a packed leaf key
    int coord_bits;            // sum of Lj
    double lo[GV_MAXD], W[GV_MAXD], eps[GV_MAXD];
    double s_f[GV_MAXD], inv_s_f[GV_MAXD];  // per dependent coordinate
    double inv_fact[31];       // 1/m!, from m! = m (m-1)! in FP64 (the 6DoF rotation's series)
};

struct Level {                 // tests of the children of a level-l cell
    int l;
    int split_mask;            // bit j: coordinate j splits at this level
    int leaf_children;         // children are leaves (l + 1 == L)
    int st_ratio_log2[GV_MAXT];// log2(s_t(l+1) / s_t(l)), 0 or 1
    double h[GV_MAXD];         // half-widths at level l
    double h1[GV_MAXD];        // half-widths at level l+1
    double s_t[GV_MAXT];       // essential-parameter snap step at level l
    double inv_s_t[GV_MAXT];
    double Rbase[GV_MAXD];     // eps_j + h1_j            (dependent index)
    double A1[GV_MAXD];        // accumulated canonization error at level l+1
    double rlb[GV_MAXD];       // eps_j - A1_j             (lower-bound radius)
    double gscale[GV_MAXD][GV_MAXT];  // s_t,m / s_f,j (a power of two)
    // FP32 screen constants, in units of s_f,j (dependent coordinate j)
    float Hs[GV_MAXD];         // h1 of dependent coordinate j
    float Hs_lo[GV_MAXD];      // h1 / s_f,j - Hs rounded to FP32 (the double-float tier's low part)
    int hs_exp;                // every split Hs is FP32-exact and a multiple of 2^hs_exp (<= 0), else
                               // -1000
    float rc0[GV_MAXD];        // (eps_j + h1_j + A1_j): the radius without its Lipschitz term
    float lam_c[4];            // family-specific scale of the Lipschitz term (see Fam::radius32)
    float rho2;                // family-specific ratio of essential steps (planes: (s_t,z / s_t,x)^2)
    float Lc[GV_MAXD];         // eps_j - A1_j (lower-bound radius)
    // set per solve, once the input's parameter ranges are known
    float qt_max[GV_MAXT];     // bound on |q_t,m| of this level's records
    int q16;                   // this level's records hold 16-bit fields
    int q16_next;              // the next level's records hold 16-bit fields
};
// ---------------------------------------------------------------------------
// Explicitly rounded FP64 operations.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// ---------------------------------------------------------------------------
// sin / cos of cell-centre angles: Cody-Waite reduction by pi/2 with a three-part
// constant (two 33-bit parts, so k*part is exact for small k), then the Taylor
// series of sin (to r^19) and cos (to r^20) with coefficients (-1)^n/n! rounded to
// double, evaluated by Horner's rule in explicitly rounded steps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double taylor_sin(double r) {
    const double c[9] = {-0x1.5555555555555p-3, 0x1.1111111111111p-7, -0x1.a01a01a01a01ap-13,
                         0x1.71de3a556c734p-19, -0x1.ae64567f544e4p-26, 0x1.6124613a86d09p-33,
                         -0x1.ae7f3e733b81fp-41, 0x1.952c77030ad4ap-49, -0x1.2f49b46814157p-57};
    double s = dmul(r, r);
    double p = c[8];
#pragma unroll
    for (int n = 7; n >= 0; --n) p = dadd(dmul(p, s), c[n]);
    return dadd(r, dmul(r, dmul(s, p)));
}

__device__ __forceinline__ double taylor_cos(double r) {
    const double c[10] = {-0x1.0000000000000p-1, 0x1.5555555555555p-5, -0x1.6c16c16c16c17p-10,
                          0x1.a01a01a01a01ap-16, -0x1.27e4fb7789f5cp-22, 0x1.1eed8eff8d898p-29,
                          -0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-45, -0x1.6827863b97d97p-53,
                          0x1.e542ba4020225p-62};
    double s = dmul(r, r);
    double p = c[9];
#pragma unroll
    for (int n = 8; n >= 0; --n) p = dadd(dmul(p, s), c[n]);
    return dadd(1.0, dmul(s, p));
}

__device__ __forceinline__ void vsincos(double x, double *sn, double *cs) {
    const double pio2_hi = 0x1.921fb544p+0, pio2_mid = 0x1.0b4611a6p-34,
                 pio2_lo = 0x1.3198a2e037073p-69, two_over_pi = 0x1.45f306dc9c883p-1;
    double k = rint(dmul(x, two_over_pi));
    double r = dsub(x, dmul(k, pio2_hi));
    r = dsub(r, dmul(k, pio2_mid));
    r = dsub(r, dmul(k, pio2_lo));
    long long ki = (long long)k;
    int q = (int)(((ki % 4) + 4) % 4);
    double ts = taylor_sin(r), tc = taylor_cos(r);
    switch (q) {
    case 0: *sn = ts; *cs = tc; break;
    case 1: *sn = tc; *cs = -ts; break;
    case 2: *sn = -ts; *cs = -tc; break;
    default: *sn = -tc; *cs = ts; break;
    }
}

// Exponent of the lowest set bit of a finite nonzero x: x is an odd multiple of
// 2^lowbit_exp(x).
__host__ __device__ __forceinline__ int lowbit_exp(double x) {
    unsigned long long b;
    memcpy(&b, &x, 8);
    const int e = (int)((b >> 52) & 0x7ff);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e) m |= 1ull << 52;
    int z = 0;
    while (!(m & 1ull)) {
        m >>= 1;
        ++z;
    }
    return (e ? e : 1) - 1075 + z;
}

// ---------------------------------------------------------------------------
// Cell geometry.  Cells are keyed by their leaf-aligned packed coordinates:
// coordinate j of a level-l cell occupies the top e_j = min(l, L_j) bits of its
// L_j-bit field; coordinate 0 sits in the most significant field, so the packed
// key orders leaves lexicographically.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int splits_at(const Problem &P, int l, int j) { return l < P.Lj[j] ? l : P.Lj[j]; }

__device__ __forceinline__ int64_t cell_coord(const Problem &P, uint64_t key, int l, int j) {
    int e = splits_at(P, l, j);
    return (int64_t)((key >> (P.coord_shift[j] + P.Lj[j] - e)) & ((1ull << e) - 1ull));
}

__device__ __forceinline__ double cell_center(const Problem &P, const double *h, int j, int64_t i) {
    return dadd(P.lo[j], dmul((double)(2 * i + 1), h[j]));
}

__device__ __forceinline__ uint64_t child_key(const Problem &P, uint64_t key, int l, int slot) {
    for (int j = 0; j < P.d; ++j)
        if (l < P.Lj[j] && ((slot >> j) & 1)) key |= 1ull << (P.coord_shift[j] + P.Lj[j] - (l + 1));
    return key;
}

// ---------------------------------------------------------------------------
// Families.  For each: D, K (free coords), ND (dependent), LE (essential params),
// NP (input rows), NB (basis values), NFP (record fields, padded so that a record
// is 1, 2 or a multiple of 4 words); basis(), lift(), residual64(), partial64(),
// lipschitz64() (the exact FP64 definition), and for the FP32 screen coef()
// (coefficient of t_m in dependent residual j for a basis change), uses(j, m)
// (whether t_m enters residual j at all) and radius32() (the UB radius in steps).
// LINEAR_BASIS: the basis is the free coordinate itself; LINEAR_TAIL: the last
// basis value is the last free coordinate (its change is the exact child shift).
// ---------------------------------------------------------------------------
enum { FAM_LINE2D = 1, FAM_PLANE3D_SPH = 2, FAM_POSE3DOF = 3, FAM_POSE6DOF = 4, FAM_RAYS3D = 5, FAM_POINTSET2D = 6,
       FAM_AFFINE4D = 7, FAM_RADIAL5DOF = 8 };

template <int FAM> struct Fam;

// LINE2D: coords (m, b); b = y - x m.  t = x, psi = m (linear: its change across a
// child shift is the shift itself).
template <> struct Fam<FAM_LINE2D> {
    static constexpr int D = 2, K = 1, ND = 1, LE = 1, NP = 2, NB = 1, NFP = 2;
    static constexpr bool LINEAR_BASIS = true, LINEAR_TAIL = false;
    __host__ __device__ static constexpr bool uses(int, int) { return true; }
    __device__ static void basis(const Problem &, const double *c, double *psi) { psi[0] = c[0]; }
    __device__ static void lift(const double *prm, int64_t n, int64_t i, const double *c, const double *psi,
                                double *f, double *t) {
        double x = prm[i], y = prm[n + i];
        t[0] = x;
        f[0] = dsub(dsub(y, dmul(x, c[0])), c[1]);
        (void)psi;
    }
    __device__ static void residual64(const double *f, const double *t, const double *dpsi, const double *sh,
                                      double *fo) {
        fo[0] = dsub(dsub(f[0], dmul(t[0], dpsi[0])), sh[1]);
    }
    __device__ static void lipschitz64(const double *t, double *lam) { lam[0] = fabs(t[0]); }
    // residual before subtracting the dependent-coordinate shift (same op order)
    __device__ static void partial64(const double *f, const double *t, const double *dpsi, double *p) {
        p[0] = dsub(f[0], dmul(t[0], dpsi[0]));
    }
    __device__ static void coef(const double *dpsi, double *g) { g[0] = -dpsi[0]; }
    // |t| = s_t |q_t|: radius = rc0 + lam_c[0] |q_t|
    __device__ static void radius32(const Level &lev, const float *qt, float *R) {
        R[0] = __fmaf_rn(lev.lam_c[0], fabsf(qt[0]), lev.rc0[0]);
    }
};

// PLANE3D_SPH: coords (theta, phi, d); d = q . n(theta, phi).  t = q; psi = n.
template <> struct Fam<FAM_PLANE3D_SPH> {
    static constexpr int D = 3, K = 2, ND = 1, LE = 3, NP = 3, NB = 3, NFP = 4;
    static constexpr bool LINEAR_BASIS = false, LINEAR_TAIL = false;
    __host__ __device__ static constexpr bool uses(int, int) { return true; }
    __device__ static void basis(const Problem &, const double *c, double *psi) {
        double st, ct, sp, cp;
        vsincos(c[0], &st, &ct);
        vsincos(c[1], &sp, &cp);
        psi[0] = dmul(st, cp);
        psi[1] = dmul(st, sp);
        psi[2] = ct;
    }
    __device__ static void lift(const double *prm, int64_t n, int64_t i, const double *c, const double *psi,
                                double *f, double *t) {
        double qx = prm[i], qy = prm[n + i], qz = prm[2 * n + i];
        t[0] = qx; t[1] = qy; t[2] = qz;
        f[0] = dsub(dadd(dadd(dmul(qx, psi[0]), dmul(qy, psi[1])), dmul(qz, psi[2])), c[2]);
    }
    __device__ static void residual64(const double *f, const double *t, const double *dpsi, const double *sh,
                                      double *fo) {
        double s = dadd(dadd(dmul(t[0], dpsi[0]), dmul(t[1], dpsi[1])), dmul(t[2], dpsi[2]));
        fo[0] = dsub(dadd(f[0], s), sh[2]);
    }
    __device__ static void partial64(const double *f, const double *t, const double *dpsi, double *p) {
        p[0] = dadd(f[0], dadd(dadd(dmul(t[0], dpsi[0]), dmul(t[1], dpsi[1])), dmul(t[2], dpsi[2])));
    }
    __device__ static void lipschitz64(const double *t, double *lam) {
        double xy = dadd(dmul(t[0], t[0]), dmul(t[1], t[1]));
        lam[0] = dsqrt(dadd(xy, dmul(t[2], t[2])));
        lam[1] = dsqrt(xy);
    }
    __device__ static void coef(const double *dpsi, double *g) { g[0] = dpsi[0]; g[1] = dpsi[1]; g[2] = dpsi[2]; }
    // s_t,x = s_t,y (their sigma bounds are equal) and s_t,z = s_t,x sqrt(rho2):
    // |q| = s_t,x sqrt(qx^2 + qy^2 + rho2 qz^2), |q_xy| = s_t,x sqrt(qx^2 + qy^2)
    __device__ static void radius32(const Level &lev, const float *qt, float *R) {
        float xy = __fmaf_rn(qt[1], qt[1], qt[0] * qt[0]);
        float all = __fmaf_rn(qt[2] * lev.rho2, qt[2], xy);
        R[0] = __fmaf_rn(lev.lam_c[0], sqrtf(all), __fmaf_rn(lev.lam_c[1], sqrtf(xy), lev.rc0[0]));
    }
};

// POSE3DOF: coords (yaw, x, y); x = w1 - (a cos yaw - b sin yaw),
// y = w2 - (a sin yaw + b cos yaw).  t = (a, b); psi = (cos yaw, sin yaw).
template <> struct Fam<FAM_POSE3DOF> {
    static constexpr int D = 3, K = 1, ND = 2, LE = 2, NP = 4, NB = 2, NFP = 4;
    static constexpr bool LINEAR_BASIS = false, LINEAR_TAIL = false;
    __host__ __device__ static constexpr bool uses(int, int) { return true; }
    __device__ static void basis(const Problem &, const double *c, double *psi) {
        double s, co;
        vsincos(c[0], &s, &co);
        psi[0] = co;
        psi[1] = s;
    }
    __device__ static void lift(const double *prm, int64_t n, int64_t i, const double *c, const double *psi,
                                double *f, double *t) {
        double w1 = prm[i], w2 = prm[n + i], a = prm[2 * n + i], b = prm[3 * n + i];
        t[0] = a; t[1] = b;
        f[0] = dsub(dsub(w1, dsub(dmul(a, psi[0]), dmul(b, psi[1]))), c[1]);
        f[1] = dsub(dsub(w2, dadd(dmul(a, psi[1]), dmul(b, psi[0]))), c[2]);
    }
    __device__ static void residual64(const double *f, const double *t, const double *dpsi, const double *sh,
                                      double *fo) {
        fo[0] = dsub(dsub(f[0], dsub(dmul(t[0], dpsi[0]), dmul(t[1], dpsi[1]))), sh[1]);
        fo[1] = dsub(dsub(f[1], dadd(dmul(t[0], dpsi[1]), dmul(t[1], dpsi[0]))), sh[2]);
    }
    __device__ static void partial64(const double *f, const double *t, const double *dpsi, double *p) {
        p[0] = dsub(f[0], dsub(dmul(t[0], dpsi[0]), dmul(t[1], dpsi[1])));
        p[1] = dsub(f[1], dadd(dmul(t[0], dpsi[1]), dmul(t[1], dpsi[0])));
    }
    __device__ static void lipschitz64(const double *t, double *lam) {
        double r = dsqrt(dadd(dmul(t[0], t[0]), dmul(t[1], t[1])));
        lam[0] = r;
        lam[1] = r;
    }
    // x residual: -a dcos + b dsin; y residual: -a dsin - b dcos
    __device__ static void coef(const double *dpsi, double *g) {
        g[0] = -dpsi[0]; g[1] = dpsi[1];
        g[2] = -dpsi[1]; g[3] = -dpsi[0];
    }
    // s_t,a = s_t,b: sqrt(a^2 + b^2) = s_t sqrt(qa^2 + qb^2)
    __device__ static void radius32(const Level &lev, const float *qt, float *R) {
        float r = sqrtf(__fmaf_rn(qt[1], qt[1], qt[0] * qt[0]));
        R[0] = __fmaf_rn(lev.lam_c[0], r, lev.rc0[0]);
        R[1] = __fmaf_rn(lev.lam_c[1], r, lev.rc0[1]);
    }
};

// RAYS3D: rays in 3-space (Sec. 4.3); coords (x, y, z); y = a x + b, z = c x + d.
// t = (a, c); psi = x (linear: its change across a child shift is the shift itself).
template <> struct Fam<FAM_RAYS3D> {
    static constexpr int D = 3, K = 1, ND = 2, LE = 2, NP = 4, NB = 1, NFP = 4;
    static constexpr bool LINEAR_BASIS = true, LINEAR_TAIL = false;
    __host__ __device__ static constexpr bool uses(int j, int m) { return j == m; }
    __device__ static void basis(const Problem &, const double *c, double *psi) { psi[0] = c[0]; }
    __device__ static void lift(const double *prm, int64_t n, int64_t i, const double *c, const double *psi,
                                double *f, double *t) {
        const double a = prm[i], b = prm[n + i], cc = prm[2 * n + i], dd = prm[3 * n + i];
        t[0] = a;
        t[1] = cc;
        f[0] = dsub(dadd(dmul(a, psi[0]), b), c[1]);
        f[1] = dsub(dadd(dmul(cc, psi[0]), dd), c[2]);
    }
    __device__ static void residual64(const double *f, const double *t, const double *dpsi, const double *sh,
                                      double *fo) {
        fo[0] = dsub(dadd(f[0], dmul(t[0], dpsi[0])), sh[1]);
        fo[1] = dsub(dadd(f[1], dmul(t[1], dpsi[0])), sh[2]);
    }
    __device__ static void partial64(const double *f, const double *t, const double *dpsi, double *p) {
        p[0] = dadd(f[0], dmul(t[0], dpsi[0]));
        p[1] = dadd(f[1], dmul(t[1], dpsi[0]));
    }
    __device__ static void lipschitz64(const double *t, double *lam) {
        lam[0] = fabs(t[0]);
        lam[1] = fabs(t[1]);
    }
    __device__ static void coef(const double *dpsi, double *g) {
        g[0] = dpsi[0]; g[1] = 0.0;
        g[2] = 0.0; g[3] = dpsi[0];
    }
    // |a| h1_x = lam_c[0] |q_a|, |c| h1_x = lam_c[1] |q_c|
    __device__ static void radius32(const Level &lev, const float *qt, float *R) {
        R[0] = __fmaf_rn(lev.lam_c[0], fabsf(qt[0]), lev.rc0[0]);
        R[1] = __fmaf_rn(lev.lam_c[1], fabsf(qt[1]), lev.rc0[1]);
    }
};

// AFFINE4D: hyperplanes x4 = a . (x1, x2, x3) + b in the affine form (Sec. 4.1,
// d = 4); coords (a1, a2, a3, b), dual surface b = x4 - a . x.  t = (x1, x2, x3);
// psi = (a1, a2, a3) (linear: their changes across a child shift are the shifts).
template <> struct Fam<FAM_AFFINE4D> {
    static constexpr int D = 4, K = 3, ND = 1, LE = 3, NP = 4, NB = 3, NFP = 4;
    static constexpr bool LINEAR_BASIS = true, LINEAR_TAIL = false;
    __host__ __device__ static constexpr bool uses(int, int) { return true; }
    __device__ static void basis(const Problem &, const double *c, double *psi) {
        psi[0] = c[0];
        psi[1] = c[1];
        psi[2] = c[2];
    }
    __device__ static void lift(const double *prm, int64_t n, int64_t i, const double *c, const double *psi,
                                double *f, double *t) {
        const double x1 = prm[i], x2 = prm[n + i], x3 = prm[2 * n + i], x4 = prm[3 * n + i];
        t[0] = x1;
        t[1] = x2;
        t[2] = x3;
        f[0] = dsub(dsub(dsub(dsub(x4, dmul(x1, psi[0])), dmul(x2, psi[1])), dmul(x3, psi[2])), c[3]);
    }
    __device__ static double tsum(const double *t, const double *dpsi) {
        return dadd(dadd(dmul(t[0], dpsi[0]), dmul(t[1], dpsi[1])), dmul(t[2], dpsi[2]));
    }
    __device__ static void residual64(const double *f, const double *t, const double *dpsi, const double *sh,
                                      double *fo) {
        fo[0] = dsub(dsub(f[0], tsum(t, dpsi)), sh[3]);
    }
    __device__ static void partial64(const double *f, const double *t, const double *dpsi, double *p) {
        p[0] = dsub(f[0], tsum(t, dpsi));
    }
    __device__ static void lipschitz64(const double *t, double *lam) {
        lam[0] = fabs(t[0]);
        lam[1] = fabs(t[1]);
        lam[2] = fabs(t[2]);
    }
    __device__ static void coef(const double *dpsi, double *g) {
        g[0] = -dpsi[0];
        g[1] = -dpsi[1];
        g[2] = -dpsi[2];
    }
    // sum_i |x_i| h1_i = sum_i lam_c[i] |q_i|
    __device__ static void radius32(const Level &lev, const float *qt, float *R) {
        R[0] = __fmaf_rn(lev.lam_c[0], fabsf(qt[0]),
                         __fmaf_rn(lev.lam_c[1], fabsf(qt[1]), __fmaf_rn(lev.lam_c[2], fabsf(qt[2]), lev.rc0[0])));
    }
};

// POINTSET2D: point-set similarity alignment (Sec. 4.4); coords (c, d, a, b) with
// q_x = a p_x + b p_y + c, q_y = -b p_x + a p_y + d.  A correspondence p -> q gives
// a = g_a - u c - v d and b = g_b - v c + u d, u = p_x/|p|^2, v = p_y/|p|^2; t = (u, v),
// psi = (c, d) (linear: their changes across a child shift are the shifts).
template <> struct Fam<FAM_POINTSET2D> {
    static constexpr int D = 4, K = 2, ND = 2, LE = 2, NP = 4, NB = 2, NFP = 4;
    static constexpr bool LINEAR_BASIS = true, LINEAR_TAIL = false;
    __host__ __device__ static constexpr bool uses(int, int) { return true; }
    __device__ static void basis(const Problem &, const double *c, double *psi) {
        psi[0] = c[0];
        psi[1] = c[1];
    }
    __device__ static void lift(const double *prm, int64_t n, int64_t i, const double *c, const double *psi,
                                double *f, double *t) {
        const double px = prm[i], py = prm[n + i], qx = prm[2 * n + i], qy = prm[3 * n + i];
        const double n2 = dadd(dmul(px, px), dmul(py, py));
        const double u = ddiv(px, n2), v = ddiv(py, n2);
        const double ga = ddiv(dadd(dmul(px, qx), dmul(py, qy)), n2);
        const double gb = ddiv(dsub(dmul(py, qx), dmul(px, qy)), n2);
        t[0] = u;
        t[1] = v;
        f[0] = dsub(dsub(dsub(ga, dmul(u, psi[0])), dmul(v, psi[1])), c[2]);
        f[1] = dsub(dadd(dsub(gb, dmul(v, psi[0])), dmul(u, psi[1])), c[3]);
    }
    __device__ static void residual64(const double *f, const double *t, const double *dpsi, const double *sh,
                                      double *fo) {
        fo[0] = dsub(dsub(f[0], dadd(dmul(t[0], dpsi[0]), dmul(t[1], dpsi[1]))), sh[2]);
        fo[1] = dsub(dsub(f[1], dsub(dmul(t[1], dpsi[0]), dmul(t[0], dpsi[1]))), sh[3]);
    }
    __device__ static void partial64(const double *f, const double *t, const double *dpsi, double *p) {
        p[0] = dsub(f[0], dadd(dmul(t[0], dpsi[0]), dmul(t[1], dpsi[1])));
        p[1] = dsub(f[1], dsub(dmul(t[1], dpsi[0]), dmul(t[0], dpsi[1])));
    }
    // da/dc = -u, da/dd = -v, db/dc = -v, db/dd = u
    __device__ static void lipschitz64(const double *t, double *lam) {
        lam[0] = fabs(t[0]);
        lam[1] = fabs(t[1]);
        lam[2] = fabs(t[1]);
        lam[3] = fabs(t[0]);
    }
    __device__ static void coef(const double *dpsi, double *g) {
        g[0] = -dpsi[0]; g[1] = -dpsi[1];      // a: -(u dc + v dd)
        g[2] = dpsi[1]; g[3] = -dpsi[0];       // b: -(v dc - u dd)
    }
    // lam_c: [a with |u|, a with |v|, b with |v|, b with |u|]
    __device__ static void radius32(const Level &lev, const float *qt, float *R) {
        const float au = fabsf(qt[0]), av = fabsf(qt[1]);
        R[0] = __fmaf_rn(lev.lam_c[0], au, __fmaf_rn(lev.lam_c[1], av, lev.rc0[0]));
        R[1] = __fmaf_rn(lev.lam_c[2], av, __fmaf_rn(lev.lam_c[3], au, lev.rc0[1]));
    }
};

// POSE6DOF: calibrated camera (Sec. 4.2.3: the 7DoF surfaces of Sec. 4.2.2 with
// f = 1); coords (phi1, phi2, phi3, z, x, y), X = R(phi) w + (x, y, z).  A match
// (w, xi, eta) gives x = xi (r3 . w + z) - r1 . w and y = eta (r3 . w + z) - r2 . w,
// affine in the basis psi = (rows of R(phi), z) with coefficients
// t = (w, xi w, eta w, xi, eta).  R by Rodrigues' formula with its three scalar
// functions as power series in theta^2 (no division by theta, no sin/cos).
template <> struct Fam<FAM_POSE6DOF> {
    static constexpr int D = 6, K = 4, ND = 2, LE = 11, NP = 5, NB = 10, NFP = 16;
    static constexpr bool LINEAR_BASIS = false, LINEAR_TAIL = true;
    // x uses w (with r1), xi w (r3), xi (z); y uses w (r2), eta w (r3), eta (z)
    __host__ __device__ static constexpr bool uses(int j, int m) {
        return m < 3 || (j == 0 ? ((m >= 3 && m < 6) || m == 9) : ((m >= 6 && m < 9) || m == 10));
    }
    __device__ static void rotation(const Problem &P, const double *ph, double *R) {
        const double s = dadd(dadd(dmul(ph[0], ph[0]), dmul(ph[1], ph[1])), dmul(ph[2], ph[2]));
        double C = 0.0, A = 0.0, B = 0.0;
#pragma unroll
        for (int n = 14; n >= 0; --n) {
            const double sg = (n & 1) ? -1.0 : 1.0;
            C = dadd(dmul(C, s), sg * P.inv_fact[2 * n]);
            A = dadd(dmul(A, s), sg * P.inv_fact[2 * n + 1]);
            B = dadd(dmul(B, s), sg * P.inv_fact[2 * n + 2]);
        }
        const double a0 = dmul(A, ph[0]), a1 = dmul(A, ph[1]), a2 = dmul(A, ph[2]);
        const double b0 = dmul(B, ph[0]), b1 = dmul(B, ph[1]), b2 = dmul(B, ph[2]);
        R[0] = dadd(C, dmul(b0, ph[0])); R[1] = dsub(dmul(b0, ph[1]), a2); R[2] = dadd(dmul(b0, ph[2]), a1);
        R[3] = dadd(dmul(b1, ph[0]), a2); R[4] = dadd(C, dmul(b1, ph[1])); R[5] = dsub(dmul(b1, ph[2]), a0);
        R[6] = dsub(dmul(b2, ph[0]), a1); R[7] = dadd(dmul(b2, ph[1]), a0); R[8] = dadd(C, dmul(b2, ph[2]));
    }
    __device__ static void basis(const Problem &P, const double *c, double *psi) {
        rotation(P, c, psi);
        psi[9] = c[3];
    }
    // the t-dependent parts of x and y for basis values (or their changes) p
    __device__ static void tpart(const double *t, const double *p, double *gx, double *gy) {
        const double sx3 = dadd(dadd(dmul(t[3], p[6]), dmul(t[4], p[7])), dmul(t[5], p[8]));
        const double sx1 = dadd(dadd(dmul(t[0], p[0]), dmul(t[1], p[1])), dmul(t[2], p[2]));
        const double sy3 = dadd(dadd(dmul(t[6], p[6]), dmul(t[7], p[7])), dmul(t[8], p[8]));
        const double sy2 = dadd(dadd(dmul(t[0], p[3]), dmul(t[1], p[4])), dmul(t[2], p[5]));
        *gx = dsub(dadd(sx3, dmul(t[9], p[9])), sx1);
        *gy = dsub(dadd(sy3, dmul(t[10], p[9])), sy2);
    }
    __device__ static void lift(const double *prm, int64_t n, int64_t i, const double *c, const double *psi,
                                double *f, double *t) {
        const double xi = prm[3 * n + i], eta = prm[4 * n + i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double w = prm[j * n + i];
            t[j] = w;
            t[3 + j] = dmul(xi, w);
            t[6 + j] = dmul(eta, w);
        }
        t[9] = xi;
        t[10] = eta;
        double gx, gy;
        tpart(t, psi, &gx, &gy);
        f[0] = dsub(gx, c[4]);
        f[1] = dsub(gy, c[5]);
    }
    __device__ static void residual64(const double *f, const double *t, const double *dpsi, const double *sh,
                                      double *fo) {
        double gx, gy;
        tpart(t, dpsi, &gx, &gy);
        fo[0] = dsub(dadd(f[0], gx), sh[4]);
        fo[1] = dsub(dadd(f[1], gy), sh[5]);
    }
    __device__ static void partial64(const double *f, const double *t, const double *dpsi, double *p) {
        double gx, gy;
        tpart(t, dpsi, &gx, &gy);
        p[0] = dadd(f[0], gx);
        p[1] = dadd(f[1], gy);
    }
    // |dx/dphi_a| <= |xi w| + |w|, |dx/dz| = |xi| (and y with eta), lam[j * K + a]
    __device__ static void lipschitz64(const double *t, double *lam) {
        const double nw = dsqrt(dadd(dadd(dmul(t[0], t[0]), dmul(t[1], t[1])), dmul(t[2], t[2])));
        const double nxw = dsqrt(dadd(dadd(dmul(t[3], t[3]), dmul(t[4], t[4])), dmul(t[5], t[5])));
        const double nyw = dsqrt(dadd(dadd(dmul(t[6], t[6]), dmul(t[7], t[7])), dmul(t[8], t[8])));
        const double lx = dadd(nxw, nw), ly = dadd(nyw, nw);
        lam[0] = lx; lam[1] = lx; lam[2] = lx; lam[3] = fabs(t[9]);
        lam[4] = ly; lam[5] = ly; lam[6] = ly; lam[7] = fabs(t[10]);
    }
    // g[j * LE + m]: coefficient of t_m in residual j for basis changes dpsi
    __device__ static void coef(const double *dpsi, double *g) {
#pragma unroll
        for (int x = 0; x < ND * LE; ++x) g[x] = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            g[i] = -dpsi[i];                 // x: -r1 . w
            g[3 + i] = dpsi[6 + i];          // x: xi w . r3
            g[LE + i] = -dpsi[3 + i];        // y: -r2 . w
            g[LE + 6 + i] = dpsi[6 + i];     // y: eta w . r3
        }
        g[9] = dpsi[9];                      // x: xi z
        g[LE + 10] = dpsi[9];                // y: eta z
    }
    // s_t equal for the nine rotation coefficients and for xi, eta:
    // |w| + |xi w| = s_t (|q_w| + |q_xiw|); lam_c: [x rotation, x z, y rotation, y z]
    __device__ static void radius32(const Level &lev, const float *qt, float *R) {
        const float nw = sqrtf(__fmaf_rn(qt[2], qt[2], __fmaf_rn(qt[1], qt[1], qt[0] * qt[0])));
        const float nxw = sqrtf(__fmaf_rn(qt[5], qt[5], __fmaf_rn(qt[4], qt[4], qt[3] * qt[3])));
        const float nyw = sqrtf(__fmaf_rn(qt[8], qt[8], __fmaf_rn(qt[7], qt[7], qt[6] * qt[6])));
        R[0] = __fmaf_rn(lev.lam_c[0], nxw + nw, __fmaf_rn(lev.lam_c[1], fabsf(qt[9]), lev.rc0[0]));
        R[1] = __fmaf_rn(lev.lam_c[2], nyw + nw, __fmaf_rn(lev.lam_c[3], fabsf(qt[10]), lev.rc0[1]));
    }
};

// RADIAL5DOF: radial camera with unknown focal length (Sec. 4.2.4); coords (phi1, phi2,
// phi3, y, x), the camera's rows (r1, -y) and (r2, x).  A match (w, xi, eta) gives
// eta (r1 . w - y) = xi (r2 . w + x): with rho = eta / xi, x = rho (r1 . w) - r2 . w -
// rho y, affine in the basis psi = (rows of R(phi), y) (r3 unused) with coefficients
// t = (rho w, w, rho).
template <> struct Fam<FAM_RADIAL5DOF> {
    static constexpr int D = 5, K = 4, ND = 1, LE = 7, NP = 5, NB = 10, NFP = 8;
    static constexpr bool LINEAR_BASIS = false, LINEAR_TAIL = true;
    __host__ __device__ static constexpr bool uses(int, int) { return true; }
    __device__ static void basis(const Problem &P, const double *c, double *psi) {
        Fam<FAM_POSE6DOF>::rotation(P, c, psi);
        psi[9] = c[3];
    }
    // the t-dependent part of x for basis values (or their changes) p
    __device__ static double tpart(const double *t, const double *p) {
        const double s1 = dadd(dadd(dmul(t[0], p[0]), dmul(t[1], p[1])), dmul(t[2], p[2]));
        const double s2 = dadd(dadd(dmul(t[3], p[3]), dmul(t[4], p[4])), dmul(t[5], p[5]));
        return dsub(dsub(s1, s2), dmul(t[6], p[9]));
    }
    __device__ static void lift(const double *prm, int64_t n, int64_t i, const double *c, const double *psi,
                                double *f, double *t) {
        const double xi = prm[3 * n + i], eta = prm[4 * n + i];
        const double rho = ddiv(eta, xi);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double w = prm[j * n + i];
            t[j] = dmul(rho, w);
            t[3 + j] = w;
        }
        t[6] = rho;
        f[0] = dsub(tpart(t, psi), c[4]);
    }
    __device__ static void residual64(const double *f, const double *t, const double *dpsi, const double *sh,
                                      double *fo) {
        fo[0] = dsub(dadd(f[0], tpart(t, dpsi)), sh[4]);
    }
    __device__ static void partial64(const double *f, const double *t, const double *dpsi, double *p) {
        p[0] = dadd(f[0], tpart(t, dpsi));
    }
    // |dx/dphi_a| <= |rho w| + |w| (as for 6DoF), dx/dy = -rho
    __device__ static void lipschitz64(const double *t, double *lam) {
        const double nrw = dsqrt(dadd(dadd(dmul(t[0], t[0]), dmul(t[1], t[1])), dmul(t[2], t[2])));
        const double nw = dsqrt(dadd(dadd(dmul(t[3], t[3]), dmul(t[4], t[4])), dmul(t[5], t[5])));
        const double lx = dadd(nrw, nw);
        lam[0] = lx; lam[1] = lx; lam[2] = lx; lam[3] = fabs(t[6]);
    }
    // g[m]: coefficient of t_m in x for basis changes dpsi
    __device__ static void coef(const double *dpsi, double *g) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            g[i] = dpsi[i];                  // rho w . r1
            g[3 + i] = -dpsi[3 + i];         // -w . r2
        }
        g[6] = -dpsi[9];                     // -rho y
    }
    // s_t equal for the six rotation coefficients: |rho w| + |w| = s_t (|q_rw| + |q_w|);
    // lam_c: [rotation, y]
    __device__ static void radius32(const Level &lev, const float *qt, float *R) {
        const float nrw = sqrtf(__fmaf_rn(qt[2], qt[2], __fmaf_rn(qt[1], qt[1], qt[0] * qt[0])));
        const float nw = sqrtf(__fmaf_rn(qt[5], qt[5], __fmaf_rn(qt[4], qt[4], qt[3] * qt[3])));
        R[0] = __fmaf_rn(lev.lam_c[0], nrw + nw, __fmaf_rn(lev.lam_c[1], fabsf(qt[6]), lev.rc0[0]));
    }
};

// Width of the FP32 screen's band, from the magnitudes of one record (in steps):
// M_j = |q_f,j| + sum_m |q_t,m| Gmax_jm + |H_j|.  The FP32 residual y takes one fused
// multiply-add per essential parameter that enters it (at most 7), one add and
// coefficients rounded once from FP64, so |y - y_exact| <= 10 u M_j (u = 2^-24; the
// FP64 definition's own error is below 2^-48 M_j); the FP32 radius (at most three
// approximate square roots of at most 4 ulp, a few multiply-adds, constants rounded
// once) is within 13 u R of the exact radius.
// A comparison of |y| with R (or with the lower-bound radius) is decided in FP32
// only when it clears kBandTest (M_j + R); a snap only when y is kBandSnap M_j away
// from a rounding tie: both about twice the bound.
constexpr float kU32 = 5.9604645e-08f;
constexpr float kBandTest = 24.0f * kU32;
constexpr float kBandSnap = 12.0f * kU32;
// The double-float tier (a residual the FP32 screen left undecided, recomputed as
// an unevaluated sum hi + lo of FP32 values with error-free products and sums,
// Dekker 1971 / Knuth TAOCP 4.2.2): coefficients G64 = G + G_lo to 2^-48 relative,
// at most 2 (LE + 1) roundings of a low part bounded by (LE + 6) u M_j, so its
// value is within 2^-39 M_j + 2^-25 of the exact residual; the FP64 definition is
// within 24 * 2^-53 M_j of it.  A snap is taken from the double-float value when it
// is kBandDF M_j + kBandDFAbs away from a rounding tie (about 8 times both bounds;
// kBandDFAbs also covers FP32 underflow of G_lo and of the product errors).
constexpr float kBandDF = 1.4551915e-11f;      // 2^-36
constexpr float kBandDFAbs = 9.5367432e-07f;   // 2^-20

}  // namespace gv
