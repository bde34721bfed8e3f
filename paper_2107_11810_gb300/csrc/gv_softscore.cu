// gv_softscore.cu -- soft inlier score S(p) = sum_i w_i exp(-u_i^2 / 2),
// u_i^2 = sum_j (r_ij / tol_j)^2, r_ij the vertical residual of surface i at p in
// dependent coordinate j (Eq. 1 in global form), w_i = bit i of the inlier mask.
// Forward, backward (d S / d p and d S / d surface parameters, recomputing the
// residuals instead of storing them) and a projected gradient ascent that keeps p
// inside a cell.  This refines the voting result the way Sec. 4.2 suggests a
// "more accurate method" take over from the approximate pose.
//
// Reductions are deterministic: per-block partial sums in a fixed grid, then one
// block adds the partials in order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "gv_kernels.h"

namespace gv {

constexpr int kSsBlocks = 1024;
constexpr int kSsThreads = 256;

// Residuals r[j], d r / d p (dp[j][d]) and d r / d params (dq[j][P]) of surface i at p.
template <int FAM> struct SoftFam;

template <> struct SoftFam<FAM_LINE2D> {       // r = b - (y - x m)
    static constexpr int D = 2, ND = 1, NP = 2;
    __device__ static void eval(const double *prm, int64_t n, int64_t i, const double *p, double *r, double *dp,
                                double *dq) {
        double x = prm[i], y = prm[n + i];
        r[0] = p[1] - (y - x * p[0]);
        dp[0] = x; dp[1] = 1.0;
        dq[0] = p[0]; dq[1] = -1.0;
    }
};

template <> struct SoftFam<FAM_PLANE3D_SPH> {  // r = d - q . n(theta, phi)
    static constexpr int D = 3, ND = 1, NP = 3;
    __device__ static void eval(const double *prm, int64_t n, int64_t i, const double *p, double *r, double *dp,
                                double *dq) {
        double qx = prm[i], qy = prm[n + i], qz = prm[2 * n + i];
        double st, ct, sp, cp;
        sincos(p[0], &st, &ct);
        sincos(p[1], &sp, &cp);
        double nx = st * cp, ny = st * sp, nz = ct;
        r[0] = p[2] - (qx * nx + qy * ny + qz * nz);
        dp[0] = -(qx * ct * cp + qy * ct * sp - qz * st);
        dp[1] = -(-qx * st * sp + qy * st * cp);
        dp[2] = 1.0;
        dq[0] = -nx; dq[1] = -ny; dq[2] = -nz;
    }
};

template <> struct SoftFam<FAM_POSE3DOF> {     // r_x = x - (w1 - (a c - b s)), r_y = y - (w2 - (a s + b c))
    static constexpr int D = 3, ND = 2, NP = 4;
    __device__ static void eval(const double *prm, int64_t n, int64_t i, const double *p, double *r, double *dp,
                                double *dq) {
        double w1 = prm[i], w2 = prm[n + i], a = prm[2 * n + i], b = prm[3 * n + i];
        double s, c;
        sincos(p[0], &s, &c);
        r[0] = p[1] - (w1 - (a * c - b * s));
        r[1] = p[2] - (w2 - (a * s + b * c));
        dp[0] = -a * s - b * c; dp[1] = 1.0; dp[2] = 0.0;
        dp[3] = a * c - b * s;  dp[4] = 0.0; dp[5] = 1.0;
        dq[0] = -1.0; dq[1] = 0.0; dq[2] = c; dq[3] = -s;
        dq[4] = 0.0; dq[5] = -1.0; dq[6] = s; dq[7] = c;
    }
};

// r_x = x - (xi (r3 . w + z) - r1 . w), r_y = y - (eta (r3 . w + z) - r2 . w) with
// R = R(phi) (Rodrigues); d(R w)/d phi_a = (J e_a) x (R w), J = I + B [phi]x +
// C [phi]x^2 the rotation's left Jacobian, B = (1 - cos th)/th^2, C = (th - sin th)/th^3.
template <> struct SoftFam<FAM_POSE6DOF> {
    static constexpr int D = 6, ND = 2, NP = 5;
    __device__ static void eval(const double *prm, int64_t n, int64_t i, const double *p, double *r, double *dp,
                                double *dq) {
        const double w[3] = {prm[i], prm[n + i], prm[2 * n + i]};
        const double xi = prm[3 * n + i], eta = prm[4 * n + i];
        const double f0 = p[0], f1 = p[1], f2 = p[2];
        const double th2 = f0 * f0 + f1 * f1 + f2 * f2;
        double A, B, C;
        if (th2 < 1e-8) {            // series: the closed forms lose accuracy near 0
            A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
            B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
            C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
        } else {
            const double th = sqrt(th2);
            double sn, cs;
            sincos(th, &sn, &cs);
            A = sn / th;
            B = (1.0 - cs) / th2;
            C = (th - sn) / (th2 * th);
        }
        // R = I + A K + B K^2, K = [phi]x, K^2 = phi phi^T - th2 I
        double Rm[9];
        const double ph[3] = {f0, f1, f2};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Rm[3 * a + b] = B * ph[a] * ph[b] + (a == b ? 1.0 - B * th2 : 0.0);
        Rm[1] -= A * f2; Rm[2] += A * f1;
        Rm[3] += A * f2; Rm[5] -= A * f0;
        Rm[6] -= A * f1; Rm[7] += A * f0;
        double X[3];
        for (int a = 0; a < 3; ++a) X[a] = Rm[3 * a] * w[0] + Rm[3 * a + 1] * w[1] + Rm[3 * a + 2] * w[2];
        const double Dz = X[2] + p[3];
        r[0] = p[4] - (xi * Dz - X[0]);
        r[1] = p[5] - (eta * Dz - X[1]);
        for (int a = 0; a < 3; ++a) {
            // u = J e_a = e_a + B (phi x e_a) + C (phi x (phi x e_a))
            double e[3] = {0.0, 0.0, 0.0};
            e[a] = 1.0;
            const double c1[3] = {ph[1] * e[2] - ph[2] * e[1], ph[2] * e[0] - ph[0] * e[2], ph[0] * e[1] - ph[1] * e[0]};
            const double c2[3] = {ph[1] * c1[2] - ph[2] * c1[1], ph[2] * c1[0] - ph[0] * c1[2],
                                  ph[0] * c1[1] - ph[1] * c1[0]};
            double u[3];
            for (int b = 0; b < 3; ++b) u[b] = e[b] + B * c1[b] + C * c2[b];
            const double dX[3] = {u[1] * X[2] - u[2] * X[1], u[2] * X[0] - u[0] * X[2], u[0] * X[1] - u[1] * X[0]};
            dp[a] = -(xi * dX[2] - dX[0]);
            dp[D + a] = -(eta * dX[2] - dX[1]);
        }
        dp[3] = -xi; dp[4] = 1.0; dp[5] = 0.0;
        dp[D + 3] = -eta; dp[D + 4] = 0.0; dp[D + 5] = 1.0;
        for (int b = 0; b < 3; ++b) {
            dq[b] = -(xi * Rm[6 + b] - Rm[b]);
            dq[NP + b] = -(eta * Rm[6 + b] - Rm[3 + b]);
        }
        dq[3] = -Dz; dq[4] = 0.0;
        dq[NP + 3] = 0.0; dq[NP + 4] = -Dz;
    }
};

template <> struct SoftFam<FAM_RAYS3D> {       // r_y = y - (a x + b), r_z = z - (c x + d)
    static constexpr int D = 3, ND = 2, NP = 4;
    __device__ static void eval(const double *prm, int64_t n, int64_t i, const double *p, double *r, double *dp,
                                double *dq) {
        const double a = prm[i], b = prm[n + i], c = prm[2 * n + i], d = prm[3 * n + i];
        r[0] = p[1] - (a * p[0] + b);
        r[1] = p[2] - (c * p[0] + d);
        dp[0] = -a; dp[1] = 1.0; dp[2] = 0.0;
        dp[3] = -c; dp[4] = 0.0; dp[5] = 1.0;
        dq[0] = -p[0]; dq[1] = -1.0; dq[2] = 0.0; dq[3] = 0.0;
        dq[4] = 0.0; dq[5] = 0.0; dq[6] = -p[0]; dq[7] = -1.0;
    }
};

// r = b - (x4 - a . x)
template <> struct SoftFam<FAM_AFFINE4D> {
    static constexpr int D = 4, ND = 1, NP = 4;
    __device__ static void eval(const double *prm, int64_t n, int64_t i, const double *p, double *r, double *dp,
                                double *dq) {
        const double x1 = prm[i], x2 = prm[n + i], x3 = prm[2 * n + i], x4 = prm[3 * n + i];
        r[0] = p[3] - (x4 - ((p[0] * x1 + p[1] * x2) + p[2] * x3));
        dp[0] = x1; dp[1] = x2; dp[2] = x3; dp[3] = 1.0;
        dq[0] = p[0]; dq[1] = p[1]; dq[2] = p[2]; dq[3] = -1.0;
    }
};

// r_a = a - (p_x (q_x - c) + p_y (q_y - d)) / |p|^2, r_b = b - (p_y (q_x - c) - p_x (q_y - d)) / |p|^2
template <> struct SoftFam<FAM_POINTSET2D> {
    static constexpr int D = 4, ND = 2, NP = 4;
    __device__ static void eval(const double *prm, int64_t n, int64_t i, const double *p, double *r, double *dp,
                                double *dq) {
        const double px = prm[i], py = prm[n + i], qx = prm[2 * n + i], qy = prm[3 * n + i];
        const double N = px * px + py * py, ex = qx - p[0], ey = qy - p[1];
        const double A = px * ex + py * ey, B = py * ex - px * ey;
        r[0] = p[2] - A / N;
        r[1] = p[3] - B / N;
        dp[0] = px / N; dp[1] = py / N; dp[2] = 1.0; dp[3] = 0.0;
        dp[4] = py / N; dp[5] = -px / N; dp[6] = 0.0; dp[7] = 1.0;
        const double N2 = N * N;
        dq[0] = -(ex / N - A * 2.0 * px / N2);
        dq[1] = -(ey / N - A * 2.0 * py / N2);
        dq[2] = -(px / N);
        dq[3] = -(py / N);
        dq[4] = -(-ey / N - B * 2.0 * px / N2);
        dq[5] = -(ex / N - B * 2.0 * py / N2);
        dq[6] = -(py / N);
        dq[7] = -(-px / N);
    }
};

struct SoftArgs {
    const double *prm;
    int64_t n;
    const uint32_t *mask;     // NULL: every weight 1
    const double *p;          // device [d]
    double inv_tol2[GV_MAXD]; // 1 / tol_j^2
    const double *grad_out;   // device [1] (backward)
    double *grad_prm;         // device [P][n] or NULL (backward)
    double *partial;          // [kSsBlocks][1 + d]
};

__device__ __forceinline__ double block_sum(double v, double *sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kSsThreads / 32; ++i) t += sm[i];
    return t;                 // valid in thread 0
}

template <int FAM, bool BWD>
__global__ void __launch_bounds__(kSsThreads) k_softscore(SoftArgs a) {
    using S = SoftFam<FAM>;
    __shared__ double sm[kSsThreads / 32];
    double p[S::D];
#pragma unroll
    for (int j = 0; j < S::D; ++j) p[j] = a.p[j];
    double g0 = BWD ? a.grad_out[0] : 0.0;
    double acc = 0.0, accp[S::D];
#pragma unroll
    for (int j = 0; j < S::D; ++j) accp[j] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        double w = a.mask ? (double)((a.mask[i >> 5] >> (i & 31)) & 1u) : 1.0;
        double r[S::ND], dp[S::ND * S::D], dq[S::ND * S::NP];
        S::eval(a.prm, a.n, i, p, r, dp, dq);
        double u2 = 0.0;
#pragma unroll
        for (int j = 0; j < S::ND; ++j) u2 += r[j] * r[j] * a.inv_tol2[j];
        double k = w * exp(-0.5 * u2);
        if (!BWD) {
            acc += k;
        } else {
            // dS_i / dr_j = -k r_j / tol_j^2
            double gq[S::NP];
#pragma unroll
            for (int m = 0; m < S::NP; ++m) gq[m] = 0.0;
#pragma unroll
            for (int j = 0; j < S::ND; ++j) {
                double dr = -g0 * k * r[j] * a.inv_tol2[j];
#pragma unroll
                for (int q = 0; q < S::D; ++q) accp[q] += dr * dp[j * S::D + q];
#pragma unroll
                for (int m = 0; m < S::NP; ++m) gq[m] += dr * dq[j * S::NP + m];
            }
            if (a.grad_prm)
#pragma unroll
                for (int m = 0; m < S::NP; ++m) a.grad_prm[m * a.n + i] = gq[m];
        }
    }
    if (!BWD) {
        double t = block_sum(acc, sm);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = t;
    } else {
#pragma unroll
        for (int q = 0; q < S::D; ++q) {
            double t = block_sum(accp[q], sm);
            if (threadIdx.x == 0) a.partial[blockIdx.x * S::D + q] = t;
        }
    }
}

// out[q] = sum over blocks of partial[b * width + q], in block order
__global__ void k_softscore_final(const double *partial, int nb, int width, double *out) {
    int q = threadIdx.x;
    if (q >= width) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += partial[b * width + q];
    out[q] = t;
}

static int ss_blocks(int64_t n) {
    int64_t b = (n + kSsThreads - 1) / kSsThreads;
    return (int)(b < 1 ? 1 : (b > kSsBlocks ? kSsBlocks : b));
}

void launch_softscore(int fam, bool bwd, const double *prm, int64_t n, const uint32_t *mask, const double *p,
                      const double *inv_tol2, int nd, const double *grad_out, double *grad_prm, double *partial,
                      double *out, cudaStream_t st) {
    SoftArgs a;
    std::memset(&a, 0, sizeof(a));
    a.prm = prm; a.n = n; a.mask = mask; a.p = p; a.grad_out = grad_out; a.grad_prm = grad_prm;
    a.partial = partial;
    for (int j = 0; j < nd; ++j) a.inv_tol2[j] = inv_tol2[j];
    int nb = ss_blocks(n);
    int d = fam == FAM_LINE2D ? 2 : (fam == FAM_POSE6DOF ? 6 : ((fam == FAM_POINTSET2D || fam == FAM_AFFINE4D) ? 4 : 3));
    switch (fam) {
    case FAM_LINE2D:
        if (bwd) k_softscore<FAM_LINE2D, true><<<nb, kSsThreads, 0, st>>>(a);
        else k_softscore<FAM_LINE2D, false><<<nb, kSsThreads, 0, st>>>(a);
        break;
    case FAM_PLANE3D_SPH:
        if (bwd) k_softscore<FAM_PLANE3D_SPH, true><<<nb, kSsThreads, 0, st>>>(a);
        else k_softscore<FAM_PLANE3D_SPH, false><<<nb, kSsThreads, 0, st>>>(a);
        break;
    case FAM_POSE3DOF:
        if (bwd) k_softscore<FAM_POSE3DOF, true><<<nb, kSsThreads, 0, st>>>(a);
        else k_softscore<FAM_POSE3DOF, false><<<nb, kSsThreads, 0, st>>>(a);
        break;
    case FAM_AFFINE4D:
        if (bwd) k_softscore<FAM_AFFINE4D, true><<<nb, kSsThreads, 0, st>>>(a);
        else k_softscore<FAM_AFFINE4D, false><<<nb, kSsThreads, 0, st>>>(a);
        break;
    case FAM_POINTSET2D:
        if (bwd) k_softscore<FAM_POINTSET2D, true><<<nb, kSsThreads, 0, st>>>(a);
        else k_softscore<FAM_POINTSET2D, false><<<nb, kSsThreads, 0, st>>>(a);
        break;
    case FAM_RAYS3D:
        if (bwd) k_softscore<FAM_RAYS3D, true><<<nb, kSsThreads, 0, st>>>(a);
        else k_softscore<FAM_RAYS3D, false><<<nb, kSsThreads, 0, st>>>(a);
        break;
    case FAM_POSE6DOF:
        if (bwd) k_softscore<FAM_POSE6DOF, true><<<nb, kSsThreads, 0, st>>>(a);
        else k_softscore<FAM_POSE6DOF, false><<<nb, kSsThreads, 0, st>>>(a);
        break;
    }
    k_softscore_final<<<1, 32, 0, st>>>(partial, nb, bwd ? d : 1, out);
}

int softscore_partial_doubles() { return kSsBlocks * GV_MAXD; }

bool softscore_supported(int fam) {
    return fam == FAM_LINE2D || fam == FAM_PLANE3D_SPH || fam == FAM_POSE3DOF || fam == FAM_POSE6DOF ||
           fam == FAM_RAYS3D || fam == FAM_POINTSET2D || fam == FAM_AFFINE4D;
}

}  // namespace gv
