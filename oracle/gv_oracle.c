/*
 * gv_oracle.c -- plain, slow reference implementation of approximate max-depth
 * general voting (Aiger, Lynen, Hosang, Zeisl, "Efficient Large Scale Inlier
 * Voting for Geometric Vision Problems", ICCV 2021, arXiv 2107.11810).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file.  It shares no code, header, table or
 * constant with the CUDA library; the two meet only through the seeded input
 * arrays.
 *
 * What it computes (every step in FP64, one IEEE operation at a time, in the
 * written order; build with -ffp-contract=off so no multiply-add is fused):
 *
 *   Surfaces (Sec. 3, Eq. 1): x_j = F_j(x_free; t) + f_j for each dependent
 *   coordinate j.  A record stores the surface in the frame of the current cell:
 *   f_j is its vertical residual at the cell centre, t its essential parameters.
 *
 *   Search (Algorithm 2, SurfaceConsensus): a box whose width is <= eps in every
 *   coordinate is a leaf; otherwise canonize the surfaces for the box, split it
 *   into 2^d sub-boxes, keep for each sub-box the surfaces that come near it,
 *   recurse, and return the best sub-result.
 *
 *   Canonization (Sec. 3.2, "Canonization"): each free parameter is rounded to a
 *   multiple of eps'/(l+1), each essential parameter to a multiple of
 *   eps'/((l+1) delta); identical rounded surfaces are merged (multiplicities
 *   add up).  The rounding error of one level is bounded; it accumulates over the
 *   log(1/eps) levels and is compensated by enlarging eps ("update eps slightly").
 *
 *   Surface-box predicate (Sec. 3.2, "Surface-Box intersection"; the paper uses
 *   a subset of the exact conditions): the conservative Lipschitz test
 *   |residual at child centre| <= eps + child half-width + Lipschitz * free
 *   half-widths + accumulated canonization error.
 *
 *   Pruning (Sec. 3.3, Branch&Bound combined with canonization): a lower bound
 *   LB(cell) counts surfaces within eps - accumulated error of the cell centre;
 *   a cell whose upper bound UB is below the best lower bound seen is dropped.
 *   The result does not depend on pruning or visiting order.
 *
 * Readings of points the paper leaves open (all of them are listed in the
 * design notes of the repository):
 *   - per-coordinate eps; coordinate j stops splitting after
 *     L_j = ceil(log2(W_j/eps_j)) levels; L = max_j L_j;
 *   - snap steps are powers of two rounded down: s_f = 2^floor(log2(eps'/(l+1))),
 *     s_t = 2^floor(log2(eps'/((l+1) sigma))) with sigma a bound on how much the
 *     surface's basis functions change across the cell; eps' = eps / L;
 *   - snapping is round-half-even of value/step (exact, since steps are powers
 *     of two);
 *   - the frame is anchored at the cell centre, not at the lowest vertex;
 *   - ties between leaves of equal depth go to the lexicographically smallest
 *     integer leaf coordinates;
 *   - the reported point is the centre of the best leaf, the inlier set is every
 *     original surface whose own record reaches that leaf;
 *   - per family (stated where each family is defined below): its coordinates and
 *     dependent/free split, the affine form used for canonization (6DoF, 7DoF and
 *     the radial camera: more coefficients than the paper's essential parameters),
 *     its margin bounds sigma and Lambda, and a constant tolerance on the dependent
 *     coordinates of the camera families.
 *
 * Transcendentals: sin/cos come from gvo_vsin/gvo_vcos below (Cody-Waite argument
 * reduction by pi/2 with a three-part constant, then the Taylor series of sin and
 * cos, coefficients (-1)^n/n! rounded to double, evaluated by Horner's rule).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GVO_MAXD 7
#define GVO_MAXT 11
#define GVO_MAXL 40

enum { GVO_LINE2D = 1, GVO_PLANE3D_SPH = 2, GVO_POSE3DOF = 3, GVO_POSE6DOF = 4, GVO_RAYS3D = 5,
       GVO_POINTSET2D = 6, GVO_AFFINE4D = 7, GVO_RADIAL5DOF = 8, GVO_POSE7DOF = 9 };
enum { GVO_NO_MERGE = 1, GVO_NO_PRUNE = 2, GVO_REVERSE = 4 };

/* ------------------------------------------------------------------------- */
/* sin / cos from their Taylor series.                                        */
/* ------------------------------------------------------------------------- */

/* pi/2 = PIO2_1 + PIO2_2 + PIO2_3: the first two parts carry 33 significant
 * bits each, so k * PIO2_1 and k * PIO2_2 are exact for |k| < 2^20. */
static const double PIO2_1 = 0x1.921fb544p+0;
static const double PIO2_2 = 0x1.0b4611a6p-34;
static const double PIO2_3 = 0x1.3198a2e037073p-69;
static const double TWO_OVER_PI = 0x1.45f306dc9c883p-1;

/* 1/(2n+1)! with alternating signs, n = 1..9 */
static const double SIN_C[9] = {
    -0x1.5555555555555p-3,  /* -1/3!  */
    0x1.1111111111111p-7,   /* 1/5!   */
    -0x1.a01a01a01a01ap-13, /* -1/7!  */
    0x1.71de3a556c734p-19,  /* 1/9!   */
    -0x1.ae64567f544e4p-26, /* -1/11! */
    0x1.6124613a86d09p-33,  /* 1/13!  */
    -0x1.ae7f3e733b81fp-41, /* -1/15! */
    0x1.952c77030ad4ap-49,  /* 1/17!  */
    -0x1.2f49b46814157p-57, /* -1/19! */
};
/* 1/(2n)! with alternating signs, n = 1..10 */
static const double COS_C[10] = {
    -0x1.0000000000000p-1,  /* -1/2!  */
    0x1.5555555555555p-5,   /* 1/4!   */
    -0x1.6c16c16c16c17p-10, /* -1/6!  */
    0x1.a01a01a01a01ap-16,  /* 1/8!   */
    -0x1.27e4fb7789f5cp-22, /* -1/10! */
    0x1.1eed8eff8d898p-29,  /* 1/12!  */
    -0x1.93974a8c07c9dp-37, /* -1/14! */
    0x1.ae7f3e733b81fp-45,  /* 1/16!  */
    -0x1.6827863b97d97p-53, /* -1/18! */
    0x1.e542ba4020225p-62,  /* 1/20!  */
};

static double taylor_sin(double r)
{
    double s = r * r;
    double p = SIN_C[8];
    for (int n = 7; n >= 0; --n) p = p * s + SIN_C[n];
    return r + r * (s * p);
}

static double taylor_cos(double r)
{
    double s = r * r;
    double p = COS_C[9];
    for (int n = 8; n >= 0; --n) p = p * s + COS_C[n];
    return 1.0 + s * p;
}

/* reduce x to r in [-pi/4, pi/4] with x = k*pi/2 + r; returns k mod 4 */
static int reduce_pio2(double x, double *r)
{
    double k = rint(x * TWO_OVER_PI);
    double y = x - k * PIO2_1;
    y = y - k * PIO2_2;
    y = y - k * PIO2_3;
    *r = y;
    long long ki = (long long)k;
    return (int)(((ki % 4) + 4) % 4);
}

double gvo_vsin(double x)
{
    double r;
    int q = reduce_pio2(x, &r);
    switch (q) {
    case 0: return taylor_sin(r);
    case 1: return taylor_cos(r);
    case 2: return -taylor_sin(r);
    default: return -taylor_cos(r);
    }
}

double gvo_vcos(double x)
{
    double r;
    int q = reduce_pio2(x, &r);
    switch (q) {
    case 0: return taylor_cos(r);
    case 1: return -taylor_sin(r);
    case 2: return -taylor_cos(r);
    default: return taylor_sin(r);
    }
}

/* ------------------------------------------------------------------------- */
/* Problem set-up: levels, snap steps, accumulated canonization error.        */
/* ------------------------------------------------------------------------- */

typedef struct {
    int fam, d, k, nd, le, np, nb;   /* nb: basis values psi (Sec. 3.2's canonization frame) */
    int L, Lj[GVO_MAXD];
    double lo[GVO_MAXD], W[GVO_MAXD], eps[GVO_MAXD];
    double h[GVO_MAXL + 1][GVO_MAXD];     /* half-width of a level-l cell      */
    double s_f[GVO_MAXD];                 /* snap step of free param j (dep.)  */
    double s_t[GVO_MAXL + 1][GVO_MAXT];   /* snap step of essential param m    */
    double A[GVO_MAXL + 2][GVO_MAXD];     /* accumulated error, dependent j    */
    double inv_fact[31];                  /* 1/m!, m! = m (m-1)! in FP64 (Rodrigues) */
} gvo_problem;

typedef struct {
    double f[GVO_MAXD];   /* residual at the cell centre, per dependent coord */
    double t[GVO_MAXT];   /* essential parameters                             */
    int64_t mult;         /* number of original surfaces it stands for        */
    int64_t orig;         /* original index (only when records are not merged) */
} gvo_rec;

/* number of essential parameters and of input parameters per family */
static int family_shape(int fam, int d, int k, int *le, int *np)
{
    switch (fam) {
    case GVO_LINE2D:      if (d != 2 || k != 1) return 1; *le = 1; *np = 2; return 0;
    case GVO_PLANE3D_SPH: if (d != 3 || k != 2) return 1; *le = 3; *np = 3; return 0;
    case GVO_POSE3DOF:    if (d != 3 || k != 1) return 1; *le = 2; *np = 4; return 0;
    case GVO_POSE6DOF:    if (d != 6 || k != 4) return 1; *le = 11; *np = 5; return 0;
    case GVO_RAYS3D:      if (d != 3 || k != 1) return 1; *le = 2; *np = 4; return 0;
    case GVO_POINTSET2D:  if (d != 4 || k != 2) return 1; *le = 2; *np = 4; return 0;
    case GVO_AFFINE4D:    if (d != 4 || k != 3) return 1; *le = 3; *np = 4; return 0;
    case GVO_RADIAL5DOF:  if (d != 5 || k != 4) return 1; *le = 7; *np = 5; return 0;
    case GVO_POSE7DOF:    if (d != 7 || k != 5) return 1; *le = 11; *np = 5; return 0;
    default: return 1;
    }
}

/* sigma_m: bound on |psi_m(x) - psi_m(c)| for x anywhere in a cell of the given
 * half-widths, psi_m being the basis function that multiplies essential
 * parameter m in F. */
static void family_sigma(const gvo_problem *p, const double *h, double *sigma)
{
    switch (p->fam) {
    case GVO_LINE2D:      /* F = -x * m: psi = m */
        sigma[0] = h[0];
        break;
    case GVO_PLANE3D_SPH: /* F = q . n(theta, phi) */
        sigma[0] = h[0] + h[1];
        sigma[1] = h[0] + h[1];
        sigma[2] = h[0];
        break;
    case GVO_POSE3DOF:    /* F = -R(yaw) (a, b) */
        sigma[0] = h[0];
        sigma[1] = h[0];
        break;
    case GVO_RAYS3D:      /* y = a x + b, z = c x + d: a and c multiply x */
        sigma[0] = h[0];
        sigma[1] = h[0];
        break;
    case GVO_POINTSET2D:  /* u, v multiply c in one equation and d in the other */
        sigma[0] = h[0] > h[1] ? h[0] : h[1];
        sigma[1] = sigma[0];
        break;
    case GVO_AFFINE4D:    /* b = x4 - sum_i x_i a_i: x_i multiplies a_i */
        sigma[0] = h[0];
        sigma[1] = h[1];
        sigma[2] = h[2];
        break;
    case GVO_POSE6DOF: {  /* F = sum_m t_m psi_m with psi = entries of R(phi) and z */
        /* An entry R_ki of R(phi) has gradient e_k . (J e_a x R e_i) along phi_a, J the
         * rotation's Jacobian (operator norm 1), so |grad R_ki| <= 1 and the entry moves
         * by at most |d phi|_2 <= h_phi1 + h_phi2 + h_phi3 across the cell; z is linear. */
        double hr = (h[0] + h[1]) + h[2];
        for (int m = 0; m < 9; ++m) sigma[m] = hr;
        sigma[9] = h[3];
        sigma[10] = h[3];
        break;
    }
    case GVO_RADIAL5DOF: {  /* entries of the rows r1, r2 of R(phi) (as for 6DoF), and y */
        double hphi = (h[0] + h[1]) + h[2];
        for (int m = 0; m < 6; ++m) sigma[m] = hphi;
        sigma[6] = h[3];
        break;
    }
    case GVO_POSE7DOF: {
        /* basis (r1, r2, r3 / f, z / f) with f >= f_lo > 0 on the domain: an entry of R
         * moves by at most hr (as for 6DoF), |1/f(x) - 1/f(c)| <= h_f / f_lo^2, so
         * r3_i / f moves by at most hr / f_lo + h_f / f_lo^2 and z / f by at most
         * h_z / f_lo + z_max h_f / f_lo^2 (|r3_i| <= 1, |z| <= z_max) */
        double hr7 = (h[0] + h[1]) + h[2];
        double flo = p->lo[4], zmax = fmax(fabs(p->lo[3]), fabs(p->lo[3] + p->W[3]));
        double inv2 = 1.0 / (flo * flo);
        double s3 = hr7 / flo + h[4] * inv2;
        double sz = h[3] / flo + (zmax * h[4]) * inv2;
        for (int m = 0; m < 3; ++m) sigma[m] = hr7;
        for (int m = 3; m < 9; ++m) sigma[m] = s3;
        sigma[9] = sz;
        sigma[10] = sz;
        break;
    }
    }
}

/* number of basis values psi of a family */
static int family_nb(int fam, int le)
{
    /* 6DoF and radial 5DoF: the nine entries of R(phi) and the last free coordinate;
     * rays: x; point sets: (c, d), le = 2 */
    return (fam == GVO_POSE6DOF || fam == GVO_RADIAL5DOF || fam == GVO_POSE7DOF) ? 10
                                                                                : (fam == GVO_RAYS3D ? 1 : le);
}

static double pow2_floor(double x)  /* 2^floor(log2 x), exact */
{
    int e;
    frexp(x, &e);
    return ldexp(1.0, e - 1);
}

static int problem_init(gvo_problem *p, int fam, int d, int k, const double *eps,
                        const double *bounds)
{
    memset(p, 0, sizeof(*p));
    int le, np;
    if (family_shape(fam, d, k, &le, &np)) return 1;
    p->fam = fam; p->d = d; p->k = k; p->nd = d - k; p->le = le; p->np = np;
    p->nb = family_nb(fam, le);
    p->inv_fact[0] = 1.0;
    for (int m = 1; m < 31; ++m) p->inv_fact[m] = p->inv_fact[m - 1] / (double)m;
    p->L = 0;
    for (int j = 0; j < d; ++j) {
        double lo = bounds[2 * j], hi = bounds[2 * j + 1];
        if (!(eps[j] > 0.0) || !(hi > lo) || !isfinite(lo) || !isfinite(hi) || !isfinite(eps[j]))
            return 1;
        p->lo[j] = lo;
        p->W[j] = hi - lo;
        p->eps[j] = eps[j];
        int Lj = 0;   /* smallest L_j with W_j 2^-L_j <= eps_j */
        while (ldexp(p->W[j], -Lj) > eps[j]) ++Lj;
        if (Lj > GVO_MAXL) return 1;
        p->Lj[j] = Lj;
        if (Lj > p->L) p->L = Lj;
    }
    for (int l = 0; l <= p->L; ++l)
        for (int j = 0; j < d; ++j) {
            int e = l < p->Lj[j] ? l : p->Lj[j];
            p->h[l][j] = ldexp(p->W[j], -(e + 1));
        }
    if (fam == GVO_POSE7DOF && !(p->lo[4] > 0.0)) return 1;   /* the focal length must stay positive */
    if (p->L == 0) return 0;
    /* eps' = eps / L per dependent coordinate */
    double epsp_min = INFINITY;
    for (int j = 0; j < p->nd; ++j) {
        double epsp = p->eps[k + j] / (double)p->L;
        if (epsp < epsp_min) epsp_min = epsp;
        p->s_f[j] = pow2_floor(epsp / (double)(le + 1));
    }
    for (int j = 0; j < p->nd; ++j) p->A[0][j] = 0.0;
    for (int l = 0; l < p->L; ++l) {
        double sigma[GVO_MAXT];
        family_sigma(p, p->h[l], sigma);
        for (int m = 0; m < le; ++m)
            p->s_t[l][m] = pow2_floor(epsp_min / ((double)(le + 1) * sigma[m]));
        for (int j = 0; j < p->nd; ++j) {
            double delta = p->s_f[j] * 0.5;
            for (int m = 0; m < le; ++m) delta = delta + (p->s_t[l][m] * 0.5) * sigma[m];
            delta = delta + ldexp(p->eps[k + j], -32);   /* FP64 rounding allowance */
            p->A[l + 1][j] = p->A[l][j] + delta;
        }
    }
    return 0;
}

static double cell_center(const gvo_problem *p, int l, int j, int64_t i)
{
    return p->lo[j] + (double)(2 * i + 1) * p->h[l][j];
}

/* ------------------------------------------------------------------------- */
/* Families (Sec. 3 Eq. 2 line duality; Sec. 4.1 plane fitting; 3DoF posing;   */
/* Sec. 4.2.3 calibrated 6DoF posing; Sec. 4.3 rays in 3-space; Sec. 4.4      */
/* point-set similarity alignment; Sec. 4.1 affine hyperplanes in 4-space;    */
/* Sec. 4.2.4 radial camera; Sec. 4.2.2 7DoF posing with unknown focal).      */
/* ------------------------------------------------------------------------- */

/* Rotation matrix (row-major) of the axis-angle vector ph, theta = |ph|, by
 * Rodrigues' formula R = cos(theta) I + (sin(theta)/theta) [ph]x
 * + ((1 - cos(theta))/theta^2) ph ph^T.  The three scalar functions are even in
 * theta, so each is a power series in s = theta^2: cos = sum_n (-1)^n s^n/(2n)!,
 * sin(theta)/theta = sum_n (-1)^n s^n/(2n+1)!, (1 - cos)/theta^2 = sum_n (-1)^n
 * s^n/(2n+2)!, evaluated by Horner's rule with 15 terms (for theta <= 2 the first
 * omitted term is below 1e-21), coefficients 1/m! from m! = m (m-1)! as divisions
 * in FP64.  No division by theta and no sin/cos: the formula holds at theta = 0. */
static void rodrigues(const double *inv_fact, const double *ph, double *R)
{
    double s = (ph[0] * ph[0] + ph[1] * ph[1]) + ph[2] * ph[2];
    double C = 0.0, A = 0.0, B = 0.0;
    for (int n = 14; n >= 0; --n) {
        double sg = (n & 1) ? -1.0 : 1.0;
        C = C * s + sg * inv_fact[2 * n];
        A = A * s + sg * inv_fact[2 * n + 1];
        B = B * s + sg * inv_fact[2 * n + 2];
    }
    double a0 = A * ph[0], a1 = A * ph[1], a2 = A * ph[2];
    double b0 = B * ph[0], b1 = B * ph[1], b2 = B * ph[2];
    R[0] = C + b0 * ph[0];  R[1] = b0 * ph[1] - a2;  R[2] = b0 * ph[2] + a1;
    R[3] = b1 * ph[0] + a2; R[4] = C + b1 * ph[1];  R[5] = b1 * ph[2] - a0;
    R[6] = b2 * ph[0] - a1; R[7] = b2 * ph[1] + a0; R[8] = C + b2 * ph[2];
}

/* Basis values psi(c) at the centre of the level-l cell with coords i. */
static void family_basis(const gvo_problem *p, int l, const int64_t *i, double *psi)
{
    switch (p->fam) {
    case GVO_LINE2D:
        psi[0] = cell_center(p, l, 0, i[0]);                  /* m */
        break;
    case GVO_RAYS3D:
        psi[0] = cell_center(p, l, 0, i[0]);                  /* x */
        break;
    case GVO_POINTSET2D:
        psi[0] = cell_center(p, l, 0, i[0]);                  /* c */
        psi[1] = cell_center(p, l, 1, i[1]);                  /* d */
        break;
    case GVO_AFFINE4D:
        for (int j = 0; j < 3; ++j) psi[j] = cell_center(p, l, j, i[j]);   /* a_1, a_2, a_3 */
        break;
    case GVO_PLANE3D_SPH: {
        double th = cell_center(p, l, 0, i[0]);
        double ph = cell_center(p, l, 1, i[1]);
        double st = gvo_vsin(th), ct = gvo_vcos(th);
        double sp = gvo_vsin(ph), cp = gvo_vcos(ph);
        psi[0] = st * cp;                                     /* n_x */
        psi[1] = st * sp;                                     /* n_y */
        psi[2] = ct;                                          /* n_z */
        break;
    }
    case GVO_POSE3DOF: {
        double yaw = cell_center(p, l, 0, i[0]);
        psi[0] = gvo_vcos(yaw);
        psi[1] = gvo_vsin(yaw);
        break;
    }
    case GVO_POSE6DOF:                                        /* rows of R(phi), then z */
    case GVO_RADIAL5DOF: {                                    /* rows of R(phi), then y */
        double ph[3];
        for (int j = 0; j < 3; ++j) ph[j] = cell_center(p, l, j, i[j]);
        rodrigues(p->inv_fact, ph, psi);
        psi[9] = cell_center(p, l, 3, i[3]);
        break;
    }
    case GVO_POSE7DOF: {                                      /* r1, r2, r3 / f, z / f */
        double ph[3];
        for (int j = 0; j < 3; ++j) ph[j] = cell_center(p, l, j, i[j]);
        rodrigues(p->inv_fact, ph, psi);
        double z = cell_center(p, l, 3, i[3]), f = cell_center(p, l, 4, i[4]);
        psi[6] = psi[6] / f;
        psi[7] = psi[7] / f;
        psi[8] = psi[8] / f;
        psi[9] = z / f;
        break;
    }
    }
}

/* Root record of original surface i: its essential parameters and its vertical
 * residual at the centre of the whole domain. */
static void family_lift(const gvo_problem *p, const double *params, int64_t n, int64_t i,
                        gvo_rec *r)
{
    int64_t root[GVO_MAXD] = {0};
    double c[GVO_MAXD], psi[GVO_MAXT];
    for (int j = 0; j < p->d; ++j) c[j] = cell_center(p, 0, j, 0);
    family_basis(p, 0, root, psi);
    switch (p->fam) {
    case GVO_LINE2D: {                      /* point (x, y) -> dual line b = y - x m */
        double x = params[0 * n + i], y = params[1 * n + i];
        r->t[0] = x;
        r->f[0] = (y - x * c[0]) - c[1];
        break;
    }
    case GVO_PLANE3D_SPH: {                 /* point q -> d = q . n(theta, phi) */
        double qx = params[0 * n + i], qy = params[1 * n + i], qz = params[2 * n + i];
        r->t[0] = qx; r->t[1] = qy; r->t[2] = qz;
        r->f[0] = ((qx * psi[0] + qy * psi[1]) + qz * psi[2]) - c[2];
        break;
    }
    case GVO_POSE3DOF: {                    /* x = w1 - (a cos - b sin), y = w2 - (a sin + b cos) */
        double w1 = params[0 * n + i], w2 = params[1 * n + i];
        double a = params[2 * n + i], b = params[3 * n + i];
        r->t[0] = a; r->t[1] = b;
        r->f[0] = (w1 - (a * psi[0] - b * psi[1])) - c[1];
        r->f[1] = (w2 - (a * psi[1] + b * psi[0])) - c[2];
        break;
    }
    case GVO_RAYS3D: {                      /* ray y = a x + b, z = c x + d (Sec. 4.3) */
        double a = params[0 * n + i], b = params[1 * n + i];
        double cc = params[2 * n + i], dd = params[3 * n + i];
        r->t[0] = a; r->t[1] = cc;
        r->f[0] = (a * psi[0] + b) - c[1];
        r->f[1] = (cc * psi[0] + dd) - c[2];
        break;
    }
    case GVO_AFFINE4D: {                    /* point x -> dual hyperplane b = x4 - a . (x1, x2, x3) */
        double x1 = params[0 * n + i], x2 = params[1 * n + i], x3 = params[2 * n + i];
        double x4 = params[3 * n + i];
        r->t[0] = x1; r->t[1] = x2; r->t[2] = x3;
        r->f[0] = (((x4 - x1 * psi[0]) - x2 * psi[1]) - x3 * psi[2]) - c[3];
        break;
    }
    case GVO_POINTSET2D: {
        /* correspondence p -> q under q_x = a p_x + b p_y + c, q_y = -b p_x + a p_y + d
         * (Sec. 4.4): a = g_a - u c - v d, b = g_b - v c + u d with u = p_x/|p|^2,
         * v = p_y/|p|^2, g_a = (p . q)/|p|^2, g_b = (p_y q_x - p_x q_y)/|p|^2 */
        double px = params[0 * n + i], py = params[1 * n + i];
        double qx = params[2 * n + i], qy = params[3 * n + i];
        double n2 = px * px + py * py;
        double u = px / n2, v = py / n2;
        double ga = (px * qx + py * qy) / n2, gb = (py * qx - px * qy) / n2;
        r->t[0] = u; r->t[1] = v;
        r->f[0] = ((ga - u * psi[0]) - v * psi[1]) - c[2];
        r->f[1] = ((gb - v * psi[0]) + u * psi[1]) - c[3];
        break;
    }
    case GVO_POSE6DOF:
    case GVO_POSE7DOF: {
        /* match (w, xi, eta): x = xi (r3 . w + z) - r1 . w, y = eta (r3 . w + z) - r2 . w
         * (Sec. 4.2.2 with f = 1, Sec. 4.2.3).  Affine in the basis (rows of R, z) with
         * coefficients t = (w, xi w, eta w, xi, eta). */
        double w[3], xi = params[3 * n + i], eta = params[4 * n + i];
        for (int j = 0; j < 3; ++j) w[j] = params[j * n + i];
        for (int j = 0; j < 3; ++j) {
            r->t[j] = w[j];
            r->t[3 + j] = xi * w[j];
            r->t[6 + j] = eta * w[j];
        }
        r->t[9] = xi;
        r->t[10] = eta;
        const double *t = r->t;
        double sx3 = (t[3] * psi[6] + t[4] * psi[7]) + t[5] * psi[8];
        double sx1 = (t[0] * psi[0] + t[1] * psi[1]) + t[2] * psi[2];
        double sy3 = (t[6] * psi[6] + t[7] * psi[7]) + t[8] * psi[8];
        double sy2 = (t[0] * psi[3] + t[1] * psi[4]) + t[2] * psi[5];
        /* 7DoF (Sec. 4.2.2): the same with the basis (r1, r2, r3 / f, z / f), x and y
         * being coordinates 5 and 6 */
        const int jx = p->fam == GVO_POSE7DOF ? 5 : 4;
        r->f[0] = ((sx3 + t[9] * psi[9]) - sx1) - c[jx];
        r->f[1] = ((sy3 + t[10] * psi[9]) - sy2) - c[jx + 1];
        break;
    }
    case GVO_RADIAL5DOF: {
        /* match (w, xi, eta) under the radial camera with rows p1 = (r1, -y), p2 = (r2, x)
         * (Sec. 4.2.4): eta (r1 . w - y) = xi (r2 . w + x), so with rho = eta / xi
         * x = rho (r1 . w) - r2 . w - rho y, affine in the basis (rows of R, y) with
         * coefficients t = (rho w, w, rho). */
        double w[3], xi = params[3 * n + i], eta = params[4 * n + i];
        for (int j = 0; j < 3; ++j) w[j] = params[j * n + i];
        double rho = eta / xi;
        for (int j = 0; j < 3; ++j) {
            r->t[j] = rho * w[j];
            r->t[3 + j] = w[j];
        }
        r->t[6] = rho;
        const double *t = r->t;
        double s1 = (t[0] * psi[0] + t[1] * psi[1]) + t[2] * psi[2];
        double s2 = (t[3] * psi[3] + t[4] * psi[4]) + t[5] * psi[5];
        r->f[0] = ((s1 - s2) - t[6] * psi[9]) - c[4];
        break;
    }
    }
    r->mult = 1;
    r->orig = i;
}

/* Geometry of one child: shifts of its centre and changes of the basis. */
typedef struct {
    int64_t ci[GVO_MAXD];   /* child integer coords            */
    double shift[GVO_MAXD]; /* child centre - parent centre     */
    double dpsi[GVO_MAXT];  /* psi(child centre) - psi(parent)  */
} gvo_child;

/* child slot b is valid iff it sets no bit of a coordinate that no longer splits */
static int child_valid(const gvo_problem *p, int l, int b)
{
    for (int j = 0; j < p->d; ++j)
        if (((b >> j) & 1) && l >= p->Lj[j]) return 0;
    return 1;
}

static void child_geometry(const gvo_problem *p, int l, const int64_t *i, const double *psi_parent,
                           int b, gvo_child *g)
{
    for (int j = 0; j < p->d; ++j) {
        if (l < p->Lj[j]) {
            int bit = (b >> j) & 1;
            g->ci[j] = 2 * i[j] + bit;
            g->shift[j] = bit ? p->h[l + 1][j] : -p->h[l + 1][j];
        } else {
            g->ci[j] = i[j];
            g->shift[j] = 0.0;
        }
    }
    if (p->fam == GVO_LINE2D || p->fam == GVO_RAYS3D || p->fam == GVO_POINTSET2D || p->fam == GVO_AFFINE4D) {
        for (int m = 0; m < p->nb; ++m) g->dpsi[m] = g->shift[m];   /* psi is linear: exact shift */
    } else {
        double psi_child[GVO_MAXT];
        family_basis(p, l + 1, g->ci, psi_child);
        for (int m = 0; m < p->nb; ++m) g->dpsi[m] = psi_child[m] - psi_parent[m];
        /* z (6DoF) and y (radial 5DoF) are linear: exact shifts */
        if (p->fam == GVO_POSE6DOF || p->fam == GVO_RADIAL5DOF) g->dpsi[9] = g->shift[3];
    }
}

/* residual of the canonical record (f, t) at the child centre */
static void family_residual(const gvo_problem *p, const double *f, const double *t,
                            const gvo_child *g, double *fo)
{
    switch (p->fam) {
    case GVO_LINE2D:
        fo[0] = (f[0] - t[0] * g->dpsi[0]) - g->shift[1];
        break;
    case GVO_PLANE3D_SPH:
        fo[0] = (f[0] + ((t[0] * g->dpsi[0] + t[1] * g->dpsi[1]) + t[2] * g->dpsi[2])) - g->shift[2];
        break;
    case GVO_POSE3DOF:
        fo[0] = (f[0] - (t[0] * g->dpsi[0] - t[1] * g->dpsi[1])) - g->shift[1];
        fo[1] = (f[1] - (t[0] * g->dpsi[1] + t[1] * g->dpsi[0])) - g->shift[2];
        break;
    case GVO_RAYS3D:
        fo[0] = (f[0] + t[0] * g->dpsi[0]) - g->shift[1];
        fo[1] = (f[1] + t[1] * g->dpsi[0]) - g->shift[2];
        break;
    case GVO_AFFINE4D:
        fo[0] = (f[0] - ((t[0] * g->dpsi[0] + t[1] * g->dpsi[1]) + t[2] * g->dpsi[2])) - g->shift[3];
        break;
    case GVO_POINTSET2D:
        fo[0] = (f[0] - (t[0] * g->dpsi[0] + t[1] * g->dpsi[1])) - g->shift[2];
        fo[1] = (f[1] - (t[1] * g->dpsi[0] - t[0] * g->dpsi[1])) - g->shift[3];
        break;
    case GVO_POSE6DOF:
    case GVO_POSE7DOF: {
        const double *d = g->dpsi;
        const int jx = p->fam == GVO_POSE7DOF ? 5 : 4;
        double sx3 = (t[3] * d[6] + t[4] * d[7]) + t[5] * d[8];
        double sx1 = (t[0] * d[0] + t[1] * d[1]) + t[2] * d[2];
        double sy3 = (t[6] * d[6] + t[7] * d[7]) + t[8] * d[8];
        double sy2 = (t[0] * d[3] + t[1] * d[4]) + t[2] * d[5];
        fo[0] = (f[0] + ((sx3 + t[9] * d[9]) - sx1)) - g->shift[jx];
        fo[1] = (f[1] + ((sy3 + t[10] * d[9]) - sy2)) - g->shift[jx + 1];
        break;
    }
    case GVO_RADIAL5DOF: {
        const double *d = g->dpsi;
        double s1 = (t[0] * d[0] + t[1] * d[1]) + t[2] * d[2];
        double s2 = (t[3] * d[3] + t[4] * d[4]) + t[5] * d[5];
        fo[0] = (f[0] + ((s1 - s2) - t[6] * d[9])) - g->shift[4];
        break;
    }
    }
}

/* Lipschitz bounds lam[j * k + i] of dependent coord j w.r.t. free coord i */
static void family_lipschitz(const gvo_problem *p, const double *t, double *lam)
{
    switch (p->fam) {
    case GVO_LINE2D:
        lam[0] = fabs(t[0]);
        break;
    case GVO_PLANE3D_SPH:
        lam[0] = sqrt((t[0] * t[0] + t[1] * t[1]) + t[2] * t[2]);   /* d/dtheta */
        lam[1] = sqrt(t[0] * t[0] + t[1] * t[1]);                   /* d/dphi   */
        break;
    case GVO_POSE3DOF: {
        double r = sqrt(t[0] * t[0] + t[1] * t[1]);
        lam[0] = r;
        lam[1] = r;
        break;
    }
    case GVO_RAYS3D:                        /* dy/dx = a, dz/dx = c */
        lam[0] = fabs(t[0]);
        lam[1] = fabs(t[1]);
        break;
    case GVO_AFFINE4D:                      /* db/da_i = -x_i */
        lam[0] = fabs(t[0]);
        lam[1] = fabs(t[1]);
        lam[2] = fabs(t[2]);
        break;
    case GVO_POINTSET2D:                    /* da/dc = -u, da/dd = -v, db/dc = -v, db/dd = u */
        lam[0] = fabs(t[0]);
        lam[1] = fabs(t[1]);
        lam[2] = fabs(t[1]);
        lam[3] = fabs(t[0]);
        break;
    case GVO_POSE6DOF: {
        /* d/dphi_a of e_k . R v is e_k . (J e_a x R v), at most |v| (J of norm 1):
         * |dx/dphi_a| <= |xi w| + |w|, |dy/dphi_a| <= |eta w| + |w|; dx/dz = xi, dy/dz = eta */
        double nw = sqrt((t[0] * t[0] + t[1] * t[1]) + t[2] * t[2]);
        double nxw = sqrt((t[3] * t[3] + t[4] * t[4]) + t[5] * t[5]);
        double nyw = sqrt((t[6] * t[6] + t[7] * t[7]) + t[8] * t[8]);
        double lx = nxw + nw, ly = nyw + nw;
        lam[0] = lx; lam[1] = lx; lam[2] = lx; lam[3] = fabs(t[9]);
        lam[4] = ly; lam[5] = ly; lam[6] = ly; lam[7] = fabs(t[10]);
        break;
    }
    case GVO_POSE7DOF: {
        /* x = xi (r3 . w + z) / f - r1 . w with f >= f_lo: |dx/dphi_a| <= |xi w| / f_lo + |w|,
         * |dx/dz| <= |xi| / f_lo, |dx/df| = |xi (r3 . w + z)| / f^2 <= (|xi w| + |xi| z_max) / f_lo^2
         * (and y with eta) */
        double flo = p->lo[4], zmax = fmax(fabs(p->lo[3]), fabs(p->lo[3] + p->W[3]));
        double nw = sqrt((t[0] * t[0] + t[1] * t[1]) + t[2] * t[2]);
        double nxw = sqrt((t[3] * t[3] + t[4] * t[4]) + t[5] * t[5]);
        double nyw = sqrt((t[6] * t[6] + t[7] * t[7]) + t[8] * t[8]);
        double inv2 = 1.0 / (flo * flo);
        double lx7 = nxw / flo + nw, ly7 = nyw / flo + nw;
        lam[0] = lx7; lam[1] = lx7; lam[2] = lx7; lam[3] = fabs(t[9]) / flo;
        lam[4] = (nxw + fabs(t[9]) * zmax) * inv2;
        lam[5] = ly7; lam[6] = ly7; lam[7] = ly7; lam[8] = fabs(t[10]) / flo;
        lam[9] = (nyw + fabs(t[10]) * zmax) * inv2;
        break;
    }
    case GVO_RADIAL5DOF: {
        /* |dx/dphi_a| <= |rho w| + |w| (rows r1, r2; the same bound as for 6DoF); dx/dy = -rho */
        double nrw = sqrt((t[0] * t[0] + t[1] * t[1]) + t[2] * t[2]);
        double nw = sqrt((t[3] * t[3] + t[4] * t[4]) + t[5] * t[5]);
        double lx = nrw + nw;
        lam[0] = lx; lam[1] = lx; lam[2] = lx; lam[3] = fabs(t[6]);
        break;
    }
    }
}

/* Upper- and lower-bound tests of one canonical record against one child at
 * level l+1.  Returns bit 0 = UB pass, bit 1 = LB pass; writes the residual. */
static int proximity_test(const gvo_problem *p, int l, const gvo_rec *r, const gvo_child *g,
                          double *fo)
{
    double lam[GVO_MAXD * GVO_MAXD];
    family_residual(p, r->f, r->t, g, fo);
    family_lipschitz(p, r->t, lam);
    int ub = 1, lb = 1;
    for (int j = 0; j < p->nd; ++j) {
        int jj = p->k + j;
        double R = p->eps[jj] + p->h[l + 1][jj];
        for (int i = 0; i < p->k; ++i) R = R + lam[j * p->k + i] * p->h[l + 1][i];
        R = R + p->A[l + 1][j];
        double rl = p->eps[jj] - p->A[l + 1][j];
        double a = fabs(fo[j]);
        if (!(a <= R)) ub = 0;
        if (!(a <= rl)) lb = 0;
    }
    return ub | (lb << 1);
}

/* Canonize one record at level l: snap f to s_f and t to s_t[l]. */
static void snap_record(const gvo_problem *p, int l, gvo_rec *r, int64_t *key)
{
    for (int j = 0; j < p->nd; ++j) {
        double q = rint(r->f[j] / p->s_f[j]);
        key[j] = (int64_t)q;
        r->f[j] = q * p->s_f[j];
    }
    for (int m = 0; m < p->le; ++m) {
        double q = rint(r->t[m] / p->s_t[l][m]);
        key[p->nd + m] = (int64_t)q;
        r->t[m] = q * p->s_t[l][m];
    }
}

/* ------------------------------------------------------------------------- */
/* Canonization with merging of identical rounded surfaces.                   */
/* ------------------------------------------------------------------------- */

static _Thread_local const int64_t *g_sort_keys;   /* per thread: gvo_solve_parallel */
static _Thread_local int g_sort_klen;

static int cmp_key_index(const void *a, const void *b)
{
    int64_t ia = *(const int64_t *)a, ib = *(const int64_t *)b;
    const int64_t *ka = g_sort_keys + ia * g_sort_klen;
    const int64_t *kb = g_sort_keys + ib * g_sort_klen;
    for (int x = 0; x < g_sort_klen; ++x) {
        if (ka[x] < kb[x]) return -1;
        if (ka[x] > kb[x]) return 1;
    }
    return (ia > ib) - (ia < ib);
}

/* Snap every record of the list in place; when merging, replace runs of equal
 * keys by one record whose multiplicity is their sum.  Returns the new count. */
static int64_t canonize(const gvo_problem *p, int l, gvo_rec *recs, int64_t n, int merge)
{
    if (n == 0) return 0;
    int klen = p->nd + p->le;
    int64_t *keys = (int64_t *)malloc((size_t)n * klen * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) snap_record(p, l, &recs[i], keys + i * klen);
    if (!merge) { free(keys); return n; }
    int64_t *idx = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    g_sort_keys = keys;
    g_sort_klen = klen;
    qsort(idx, (size_t)n, sizeof(int64_t), cmp_key_index);
    gvo_rec *out = (gvo_rec *)malloc((size_t)n * sizeof(gvo_rec));
    int64_t m = 0;
    for (int64_t a = 0; a < n;) {
        int64_t b = a + 1;
        while (b < n && memcmp(keys + idx[a] * klen, keys + idx[b] * klen, klen * sizeof(int64_t)) == 0) ++b;
        out[m] = recs[idx[a]];
        int64_t mult = 0;
        for (int64_t x = a; x < b; ++x) mult += recs[idx[x]].mult;
        out[m].mult = mult;
        if (b - a > 1) out[m].orig = -1;
        ++m;
        a = b;
    }
    memcpy(recs, out, (size_t)m * sizeof(gvo_rec));
    free(out);
    free(idx);
    free(keys);
    return m;
}

/* ------------------------------------------------------------------------- */
/* Depth-first SurfaceConsensus with bound-based pruning.                      */
/* ------------------------------------------------------------------------- */

/* A subtree handed to a worker thread by gvo_solve_parallel: one cell and the
 * records that reach it. */
typedef struct {
    int64_t ci[GVO_MAXD];
    gvo_rec *recs;
    int64_t n, ub;
} gvo_task;

typedef struct {
    const gvo_problem *p;
    int flags;
    int sink_level;        /* > 0: cells of this level become tasks instead of being visited */
    gvo_task *tasks;
    int64_t ntasks, cap_tasks;
    int64_t bestLB;
    int have_best;
    int64_t best_ub;
    int64_t best_leaf[GVO_MAXD];
    int64_t *best_members;
    int64_t tests, cells, leaves;
    int64_t trace_cap, trace_n;
    int32_t *trace_level;
    int64_t *trace_coords, *trace_ub, *trace_lb;
} gvo_search;

static int lex_less(const int64_t *a, const int64_t *b, int d)
{
    for (int j = 0; j < d; ++j) {
        if (a[j] < b[j]) return 1;
        if (a[j] > b[j]) return 0;
    }
    return 0;
}

static void visit(gvo_search *S, int l, const int64_t *ci, gvo_rec *recs, int64_t n)
{
    const gvo_problem *p = S->p;
    int d = p->d;
    if (S->sink_level > 0 && l == S->sink_level) {     /* collect the subtree as a task */
        if (S->ntasks == S->cap_tasks) {
            S->cap_tasks = S->cap_tasks ? 2 * S->cap_tasks : 64;
            S->tasks = (gvo_task *)realloc(S->tasks, (size_t)S->cap_tasks * sizeof(gvo_task));
        }
        gvo_task *t = &S->tasks[S->ntasks++];
        memcpy(t->ci, ci, d * sizeof(int64_t));
        t->recs = (gvo_rec *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gvo_rec));
        memcpy(t->recs, recs, (size_t)n * sizeof(gvo_rec));
        t->n = n;
        t->ub = 0;
        for (int64_t r = 0; r < n; ++r) t->ub += recs[r].mult;
        return;
    }
    if (l == p->L) {                                   /* leaf: Diam(B) <= eps */
        S->leaves++;
        int64_t ub = 0;
        for (int64_t r = 0; r < n; ++r) ub += recs[r].mult;
        if (ub == 0) return;
        if (!S->have_best || ub > S->best_ub || (ub == S->best_ub && lex_less(ci, S->best_leaf, d))) {
            S->have_best = 1;
            S->best_ub = ub;
            memcpy(S->best_leaf, ci, d * sizeof(int64_t));
            if (S->best_members) {
                int64_t x = 0;
                for (int64_t r = 0; r < n; ++r) S->best_members[x++] = recs[r].orig;
            }
        }
        return;
    }
    int64_t nc = canonize(p, l, recs, n, !(S->flags & GVO_NO_MERGE));
    S->cells++;
    double psi[GVO_MAXT];
    family_basis(p, l, ci, psi);
    int nslots = 1 << d;
    gvo_child geo[1 << GVO_MAXD];
    int64_t ub[1 << GVO_MAXD], lb[1 << GVO_MAXD];
    int order[1 << GVO_MAXD], nvalid = 0;
    for (int b = 0; b < nslots; ++b) {
        if (!child_valid(p, l, b)) continue;
        child_geometry(p, l, ci, psi, b, &geo[b]);
        ub[b] = 0;
        lb[b] = 0;
        for (int64_t r = 0; r < nc; ++r) {
            double fo[GVO_MAXD];
            int t = proximity_test(p, l, &recs[r], &geo[b], fo);
            S->tests++;
            if (t & 1) ub[b] += recs[r].mult;
            if (t & 2) lb[b] += recs[r].mult;
        }
        if (S->trace_n < S->trace_cap) {
            int64_t x = S->trace_n++;
            S->trace_level[x] = l + 1;
            for (int j = 0; j < d; ++j) S->trace_coords[x * d + j] = geo[b].ci[j];
            S->trace_ub[x] = ub[b];
            S->trace_lb[x] = lb[b];
        }
        if (lb[b] > S->bestLB) S->bestLB = lb[b];
        order[nvalid++] = b;
    }
    /* visiting order: UB descending, then slot ascending (descending if REVERSE) */
    for (int x = 1; x < nvalid; ++x) {
        int v = order[x], y = x;
        while (y > 0) {
            int u = order[y - 1];
            int before = ub[u] > ub[v] || (ub[u] == ub[v] && ((S->flags & GVO_REVERSE) ? u > v : u < v));
            if (before) break;
            order[y] = u;
            --y;
        }
        order[y] = v;
    }
    for (int x = 0; x < nvalid; ++x) {
        int b = order[x];
        int64_t thr = S->bestLB;
        if (S->have_best && S->best_ub > thr) thr = S->best_ub;
        if (S->flags & GVO_NO_PRUNE) thr = 1;
        if (ub[b] == 0 || ub[b] < thr) continue;
        gvo_rec *child = (gvo_rec *)malloc((size_t)nc * sizeof(gvo_rec));
        int64_t m = 0;
        for (int64_t r = 0; r < nc; ++r) {
            double fo[GVO_MAXD];
            int t = proximity_test(p, l, &recs[r], &geo[b], fo);
            if (!(t & 1)) continue;
            child[m] = recs[r];
            for (int j = 0; j < p->nd; ++j) child[m].f[j] = fo[j];
            ++m;
        }
        visit(S, l + 1, geo[b].ci, child, m);
        free(child);
    }
}

/* ------------------------------------------------------------------------- */
/* Replay of one original surface along the path to a given cell.             */
/* ------------------------------------------------------------------------- */

static int splits(const gvo_problem *p, int l, int j) { return l < p->Lj[j] ? l : p->Lj[j]; }

/* Returns 1 if the record of original i reaches the cell (level lam, coords ct)
 * by passing the upper-bound test at every level; *lb_pass tells whether it
 * also passes the lower-bound test at that cell. */
static int replay_one(const gvo_problem *p, const double *params, int64_t n, int64_t i, int lam,
                      const int64_t *ct, int *lb_pass)
{
    gvo_rec r;
    int64_t key[GVO_MAXD + GVO_MAXT];
    family_lift(p, params, n, i, &r);
    *lb_pass = 0;
    for (int l = 0; l < lam; ++l) {
        int64_t ci[GVO_MAXD];
        int b = 0;
        for (int j = 0; j < p->d; ++j) {
            ci[j] = ct[j] >> (splits(p, lam, j) - splits(p, l, j));
            if (l < p->Lj[j]) b |= (int)((ct[j] >> (splits(p, lam, j) - splits(p, l + 1, j))) & 1) << j;
        }
        snap_record(p, l, &r, key);
        double psi[GVO_MAXT];
        family_basis(p, l, ci, psi);
        gvo_child g;
        child_geometry(p, l, ci, psi, b, &g);
        double fo[GVO_MAXD];
        int t = proximity_test(p, l, &r, &g, fo);
        if (!(t & 1)) return 0;
        if (l == lam - 1) *lb_pass = (t >> 1) & 1;
        for (int j = 0; j < p->nd; ++j) r.f[j] = fo[j];
    }
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Public entry points (called from Python through ctypes).                   */
/* ------------------------------------------------------------------------- */

static int check_inputs(const gvo_problem *p, const double *params, int64_t n)
{
    if (n < 0) return 1;
    for (int64_t x = 0; x < (int64_t)p->np * n; ++x)
        if (!isfinite(params[x])) return 1;
    return 0;
}

/* Level structure: returns L (or -1 on invalid input) and fills Lj[d]; when the
 * arrays are given, h[(L+1)*d], s_f[d-k], s_t[L*le] and A[(L+1)*(d-k)]. */
int gvo_levels(int fam, int d, int k, const double *eps, const double *bounds, int32_t *Lj,
               double *h, double *s_f, double *s_t, double *A)
{
    gvo_problem p;
    if (problem_init(&p, fam, d, k, eps, bounds)) return -1;
    for (int j = 0; j < d; ++j) Lj[j] = p.Lj[j];
    if (h) for (int l = 0; l <= p.L; ++l) for (int j = 0; j < d; ++j) h[l * d + j] = p.h[l][j];
    if (s_f) for (int j = 0; j < p.nd; ++j) s_f[j] = p.s_f[j];
    if (s_t) for (int l = 0; l < p.L; ++l) for (int m = 0; m < p.le; ++m) s_t[l * p.le + m] = p.s_t[l][m];
    if (A) for (int l = 0; l <= p.L; ++l) for (int j = 0; j < p.nd; ++j) A[l * p.nd + j] = p.A[l][j];
    return p.L;
}

/* Root records: f[(d-k)*n] (SoA) and t[le*n] (SoA). */
int gvo_root_records(int fam, int d, int k, const double *eps, const double *bounds,
                     const double *params, int64_t n, double *f, double *t)
{
    gvo_problem p;
    if (problem_init(&p, fam, d, k, eps, bounds) || check_inputs(&p, params, n)) return 1;
    for (int64_t i = 0; i < n; ++i) {
        gvo_rec r;
        family_lift(&p, params, n, i, &r);
        for (int j = 0; j < p.nd; ++j) f[j * n + i] = r.f[j];
        for (int m = 0; m < p.le; ++m) t[m * n + i] = r.t[m];
    }
    return 0;
}

int gvo_solve(int fam, int d, int k, const double *eps, const double *bounds, const double *params,
              int64_t n, int flags, double *best_point, int64_t *best_leaf, int64_t *depth,
              uint32_t *mask, int64_t *stats, int64_t trace_cap, int32_t *trace_level,
              int64_t *trace_coords, int64_t *trace_ub, int64_t *trace_lb, int64_t *trace_n,
              int64_t *members)
{
    gvo_problem p;
    if (problem_init(&p, fam, d, k, eps, bounds) || check_inputs(&p, params, n)) return 1;
    gvo_search S;
    memset(&S, 0, sizeof(S));
    S.p = &p;
    S.flags = flags;
    S.trace_cap = trace_cap;
    S.trace_level = trace_level;
    S.trace_coords = trace_coords;
    S.trace_ub = trace_ub;
    S.trace_lb = trace_lb;
    if (members && (flags & GVO_NO_MERGE)) S.best_members = members;
    gvo_rec *root = (gvo_rec *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gvo_rec));
    for (int64_t i = 0; i < n; ++i) family_lift(&p, params, n, i, &root[i]);
    int64_t zero[GVO_MAXD] = {0};
    visit(&S, 0, zero, root, n);
    free(root);
    if (!S.have_best) {                        /* nothing reaches any leaf */
        S.best_ub = 0;
        memset(S.best_leaf, 0, sizeof(S.best_leaf));
    }
    *depth = S.best_ub;
    for (int j = 0; j < d; ++j) {
        best_leaf[j] = S.best_leaf[j];
        best_point[j] = cell_center(&p, p.L, j, S.best_leaf[j]);
    }
    if (mask) {
        memset(mask, 0, (size_t)((n + 31) / 32) * sizeof(uint32_t));
        if (S.best_ub > 0)
            for (int64_t i = 0; i < n; ++i) {
                int lbp;
                if (replay_one(&p, params, n, i, p.L, S.best_leaf, &lbp)) mask[i >> 5] |= 1u << (i & 31);
            }
    }
    if (stats) {
        stats[0] = S.tests;
        stats[1] = S.cells;
        stats[2] = S.leaves;
        stats[3] = p.L;
    }
    if (trace_n) *trace_n = S.trace_n;
    return 0;
}

/* UB and LB of one cell (level lam, coords[d]) by replaying every original
 * surface along the path from the root; reach (optional) gets the bit set of
 * originals whose records reach the cell. */
int gvo_cell_counts(int fam, int d, int k, const double *eps, const double *bounds,
                    const double *params, int64_t n, int lam, const int64_t *coords, int64_t *ub,
                    int64_t *lb, uint32_t *reach)
{
    gvo_problem p;
    if (problem_init(&p, fam, d, k, eps, bounds) || check_inputs(&p, params, n)) return 1;
    if (lam < 0 || lam > p.L) return 1;
    for (int j = 0; j < d; ++j)
        if (coords[j] < 0 || coords[j] >= ((int64_t)1 << splits(&p, lam, j))) return 1;
    *ub = 0;
    *lb = 0;
    if (reach) memset(reach, 0, (size_t)((n + 31) / 32) * sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i) {
        int lbp;
        if (replay_one(&p, params, n, i, lam, coords, &lbp)) {
            ++*ub;
            *lb += lbp;
            if (reach) reach[i >> 5] |= 1u << (i & 31);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Margin functions and canonical records along a path, exported so that the */
/* tests can check the bounds they rest on against the surface equations.    */
/* ------------------------------------------------------------------------- */

/* R[9] (row-major): the rotation matrix of axis-angle vector ph[3] that the
 * POSE6DOF family's basis uses. */
void gvo_rotation(const double *ph, double *R)
{
    gvo_problem p;
    memset(&p, 0, sizeof(p));
    p.inv_fact[0] = 1.0;
    for (int m = 1; m < 31; ++m) p.inv_fact[m] = p.inv_fact[m - 1] / (double)m;
    rodrigues(p.inv_fact, ph, R);
}

/* sigma[le]: the bound family_sigma gives for a cell of half-widths h[d]. */
static int margin_problem(gvo_problem *p, int fam, int d, int k, const double *bounds)
{
    memset(p, 0, sizeof(*p));
    if (family_shape(fam, d, k, &p->le, &p->np)) return 1;
    p->fam = fam; p->d = d; p->k = k; p->nd = d - k; p->nb = family_nb(fam, p->le);
    if (bounds)
        for (int j = 0; j < d; ++j) {
            p->lo[j] = bounds[2 * j];
            p->W[j] = bounds[2 * j + 1] - bounds[2 * j];
        }
    /* the 7DoF margins depend on the domain (its smallest focal length) */
    if (fam == GVO_POSE7DOF && !(bounds && p->lo[4] > 0.0)) return 1;
    return 0;
}

/* sigma[le] for half-widths h[d]; bounds[2d] (lo, hi per coordinate) may be NULL
 * for families whose bound does not depend on the domain. */
int gvo_sigma(int fam, int d, int k, const double *bounds, const double *h, double *sigma)
{
    gvo_problem p;
    if (margin_problem(&p, fam, d, k, bounds)) return 1;
    family_sigma(&p, h, sigma);
    return 0;
}

/* lam[(d-k)*k]: the Lipschitz bounds family_lipschitz gives for the essential
 * parameters t[le] (dependent coordinate j, free coordinate i at j*k + i). */
int gvo_lipschitz(int fam, int d, int k, const double *bounds, const double *t, double *lam)
{
    gvo_problem p;
    if (margin_problem(&p, fam, d, k, bounds)) return 1;
    family_lipschitz(&p, t, lam);
    return 0;
}

/* The canonical record of original surface i at every level of the path from the
 * root to the cell (level lam, coords ct), as replay_one forms it: f[l*(d-k)+j]
 * and t[l*le+m] after the snap at level l.  Returns the number of levels at which
 * the record exists (it reached the level-l cell of the path), or -1 on invalid
 * input. */
int gvo_path_records(int fam, int d, int k, const double *eps, const double *bounds, const double *params,
                     int64_t n, int64_t i, int lam, const int64_t *ct, double *f, double *t)
{
    gvo_problem p;
    if (problem_init(&p, fam, d, k, eps, bounds) || check_inputs(&p, params, n)) return -1;
    if (i < 0 || i >= n || lam < 0 || lam > p.L) return -1;
    for (int j = 0; j < d; ++j)
        if (ct[j] < 0 || ct[j] >= ((int64_t)1 << splits(&p, lam, j))) return -1;
    gvo_rec r;
    int64_t key[GVO_MAXD + GVO_MAXT];
    family_lift(&p, params, n, i, &r);
    for (int l = 0; l < lam; ++l) {
        int64_t ci[GVO_MAXD];
        int b = 0;
        for (int j = 0; j < p.d; ++j) {
            ci[j] = ct[j] >> (splits(&p, lam, j) - splits(&p, l, j));
            if (l < p.Lj[j]) b |= (int)((ct[j] >> (splits(&p, lam, j) - splits(&p, l + 1, j))) & 1) << j;
        }
        snap_record(&p, l, &r, key);
        for (int j = 0; j < p.nd; ++j) f[l * p.nd + j] = r.f[j];
        for (int m = 0; m < p.le; ++m) t[l * p.le + m] = r.t[m];
        double psi[GVO_MAXT];
        family_basis(&p, l, ci, psi);
        gvo_child g;
        child_geometry(&p, l, ci, psi, b, &g);
        double fo[GVO_MAXD];
        if (!(proximity_test(&p, l, &r, &g, fo) & 1)) return l + 1;
        for (int j = 0; j < p.nd; ++j) r.f[j] = fo[j];
    }
    return lam;
}

/* ------------------------------------------------------------------------- */
/* The same search on several host threads (the multi-core CPU baseline).     */
/* ------------------------------------------------------------------------- */

/* Runs the levels above a split level exactly as gvo_solve, turns every cell of the
 * split level that survives into a task, and visits the tasks' subtrees on
 * nthreads OpenMP threads with the serial visit().  Each task starts from the
 * best lower bound and best leaf known when it starts and merges its own at the
 * end; any valid bound may prune (Sec. 3.3), and the argmax keeps the same tie
 * rule, so depth, best leaf and mask equal gvo_solve's.  stats: tests, cells,
 * leaves, L, threads used, tasks. */
int gvo_solve_parallel(int fam, int d, int k, const double *eps, const double *bounds, const double *params,
                       int64_t n, int nthreads, double *best_point, int64_t *best_leaf, int64_t *depth,
                       uint32_t *mask, int64_t *stats)
{
    gvo_problem p;
    if (problem_init(&p, fam, d, k, eps, bounds) || check_inputs(&p, params, n)) return 1;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
    omp_set_num_threads(nthreads);
#else
    nthreads = 1;
#endif
    /* split level: the first level with at least 16 cells per thread */
    int split = 0;
    while (split < p.L) {
        int bits = 0;
        for (int j = 0; j < d; ++j) bits += splits(&p, split, j);
        if (bits >= 30 || ((int64_t)1 << bits) >= 16 * (int64_t)nthreads) break;
        ++split;
    }
    gvo_search top;
    memset(&top, 0, sizeof(top));
    top.p = &p;
    top.sink_level = split;
    gvo_rec *root = (gvo_rec *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gvo_rec));
    for (int64_t i = 0; i < n; ++i) family_lift(&p, params, n, i, &root[i]);
    int64_t zero[GVO_MAXD] = {0};
    if (split == 0) {
        top.sink_level = -1;
        visit(&top, 0, zero, root, n);
    } else {
        visit(&top, 0, zero, root, n);
    }
    free(root);
    /* largest upper bounds first: their leaves raise the bound early */
    for (int64_t x = 1; x < top.ntasks; ++x) {
        gvo_task v = top.tasks[x];
        int64_t y = x;
        while (y > 0 && top.tasks[y - 1].ub < v.ub) { top.tasks[y] = top.tasks[y - 1]; --y; }
        top.tasks[y] = v;
    }
    int64_t tests = top.tests, cells = top.cells, leaves = top.leaves;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : tests, cells, leaves)
    for (int64_t x = 0; x < top.ntasks; ++x) {
        gvo_task *t = &top.tasks[x];
        gvo_search S;
        memset(&S, 0, sizeof(S));
        S.p = &p;
        int64_t thr;
#pragma omp critical(gvo_best)
        {
            S.bestLB = top.bestLB;
            S.have_best = top.have_best;
            S.best_ub = top.best_ub;
            memcpy(S.best_leaf, top.best_leaf, sizeof(S.best_leaf));
        }
        thr = S.bestLB;
        if (S.have_best && S.best_ub > thr) thr = S.best_ub;
        if (t->ub > 0 && t->ub >= thr) {
            visit(&S, split, t->ci, t->recs, t->n);
            tests += S.tests;
            cells += S.cells;
            leaves += S.leaves;
#pragma omp critical(gvo_best)
            {
                if (S.bestLB > top.bestLB) top.bestLB = S.bestLB;
                if (S.have_best && (!top.have_best || S.best_ub > top.best_ub ||
                                    (S.best_ub == top.best_ub && lex_less(S.best_leaf, top.best_leaf, d)))) {
                    top.have_best = 1;
                    top.best_ub = S.best_ub;
                    memcpy(top.best_leaf, S.best_leaf, sizeof(top.best_leaf));
                }
            }
        }
        free(t->recs);
        t->recs = NULL;
    }
    free(top.tasks);
    if (!top.have_best) {
        top.best_ub = 0;
        memset(top.best_leaf, 0, sizeof(top.best_leaf));
    }
    *depth = top.best_ub;
    for (int j = 0; j < d; ++j) {
        best_leaf[j] = top.best_leaf[j];
        best_point[j] = cell_center(&p, p.L, j, top.best_leaf[j]);
    }
    if (mask) {
        int64_t words = (n + 31) / 32;
        memset(mask, 0, (size_t)words * sizeof(uint32_t));
        if (top.best_ub > 0) {
#pragma omp parallel for schedule(dynamic, 256)
            for (int64_t w = 0; w < words; ++w) {
                uint32_t bits = 0;
                for (int64_t i = 32 * w; i < n && i < 32 * w + 32; ++i) {
                    int lbp;
                    if (replay_one(&p, params, n, i, p.L, top.best_leaf, &lbp)) bits |= 1u << (i & 31);
                }
                mask[w] = bits;
            }
        }
    }
    if (stats) {
        stats[0] = tests;
        stats[1] = cells;
        stats[2] = leaves;
        stats[3] = p.L;
        stats[4] = nthreads;
        stats[5] = top.ntasks;
    }
    return 0;
}
