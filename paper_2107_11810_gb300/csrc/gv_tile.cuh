// gv_tile.cuh -- device code shared by the count and emit passes of the proximity
// test (the surface-box test of Sec. 3.2, "eps plus the cell radius", over every
// (canonical record, child cell) pair).
//
// Work unit: a tile of 32 consecutive records of one cell, one record per lane of
// a warp.  A block of kWarps warps takes groups of kBlockTiles consecutive tiles,
// warp w the kTW consecutive tiles w kTW .. w kTW + kTW - 1 of each group (so that
// a warp's run of tiles of one cell stays together and its counters are flushed
// once per run).
#pragma once
#include <type_traits>

#include "gv_kernels.h"

namespace gv {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;
#ifndef GV_TILES_PER_WARP
#define GV_TILES_PER_WARP 4
#endif
constexpr int kTW = GV_TILES_PER_WARP;           // tiles per warp
constexpr int kBlockTiles = kWarps * kTW;        // tiles per block
static_assert(32 * kTW < 256, "byte-packed per-slot counters would overflow");

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (global -> shared) completing on an mbarrier: the
// count and emit passes stream their records through shared memory, two groups
// of kBlockTiles tiles per block in flight.  Every wait is bounded: after
// kSpinLimit unsuccessful polls the kernel records VOTE_ETIMEOUT's error bit and
// stops (the host maps it to VOTE_ETIMEOUT).
// ---------------------------------------------------------------------------
constexpr unsigned kErrTimeout = 0x100u;
#ifndef GV_SPIN_LIMIT
#define GV_SPIN_LIMIT (1u << 22)
#endif

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the asynchronous (bulk copy) proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of a barrier; false (and the error bit set) if
// it did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit, unsigned *err) {
    for (unsigned it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(err, kErrTimeout);
    return false;
}

// 2^23 + 2^22: adding it to a float y with |y| < 2^22 rounds y to the nearest
// integer (ties to even) and leaves that integer in the low mantissa bits.
constexpr float kMagic = 12582912.0f;
// kMagic + 2^15: the same, with the integer biased by 2^15 (the 16-bit field format)
constexpr float kMagic16 = 12615680.0f;

template <int NW>
__device__ __forceinline__ void load_words(const uint32_t *base, int64_t r, uint32_t *w) {
    const uint32_t *p = base + r * NW;
    if constexpr (NW == 1) {
        w[0] = p[0];
    } else if constexpr (NW == 2) {
        uint2 v = *reinterpret_cast<const uint2 *>(p);
        w[0] = v.x; w[1] = v.y;
    } else {
        static_assert(NW % 4 == 0, "record words");
#pragma unroll
        for (int i = 0; i < NW; i += 4) {
            uint4 v = *reinterpret_cast<const uint4 *>(p + i);
            w[i] = v.x; w[i + 1] = v.y; w[i + 2] = v.z; w[i + 3] = v.w;
        }
    }
}

template <int NW>
__device__ __forceinline__ void store_words(uint32_t *base, int64_t r, const uint32_t *w) {
    uint32_t *p = base + r * NW;
    if constexpr (NW == 1) {
        p[0] = w[0];
    } else if constexpr (NW == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    } else {
#pragma unroll
        for (int i = 0; i < NW; i += 4) *reinterpret_cast<uint4 *>(p + i) = make_uint4(w[i], w[i + 1], w[i + 2], w[i + 3]);
    }
}

// Field i of a record as a float (exact: 16-bit fields always, 32-bit fields below 2^24).
template <bool Q16>
__device__ __forceinline__ float field_f(const uint32_t *w, int i) {
    if constexpr (Q16) {
        unsigned b = __byte_perm(w[i >> 1], 0x4B40u, (i & 1) ? 0x5432u : 0x5410u);
        return __int_as_float((int)b) - kMagic16;
    } else {
        return (float)(int32_t)w[i];
    }
}

template <bool Q16>
__device__ __forceinline__ int field_i(const uint32_t *w, int i) {
    if constexpr (Q16) return (int)((w[i >> 1] >> (16 * (i & 1))) & 0xffffu) - 32768;
    else return (int32_t)w[i];
}

// Pack NFP field values into record words.  fb[i]: for 16-bit records the low 16
// bits hold the biased field, for 32-bit records the field itself.
template <int NFP, bool Q16>
__device__ __forceinline__ void pack(const uint32_t *fb, uint32_t *w) {
    if constexpr (Q16) {
#pragma unroll
        for (int i = 0; i < NFP / 2; ++i) w[i] = __byte_perm(fb[2 * i], fb[2 * i + 1], 0x5410u);
    } else {
#pragma unroll
        for (int i = 0; i < NFP; ++i) w[i] = fb[i];
    }
}

// round half to even of q/2: re-snap of an essential parameter when its step doubles
__device__ __forceinline__ int32_t resnap_half(int32_t q) {
    int32_t k = q >> 1;
    return k + ((q & 1) & (k & 1));
}

// ---------------------------------------------------------------------------
// Exact FP64 definition (the recheck of the screen, and the plain FP64 mode).
// ---------------------------------------------------------------------------

// UB radius R_j = ((eps_j + h1_j) + sum_i lam_ji h1_i) + A1_j, in this order.
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

template <int FAM>
__device__ __forceinline__ double dep_shift64(const Level &lev, int j, int s) {
    constexpr int K = Fam<FAM>::K;
    bool split = (lev.split_mask >> (K + j)) & 1;
    return split ? (((s >> (K + j)) & 1) ? lev.h1[K + j] : -lev.h1[K + j]) : 0.0;
}

template <int FAM>
__device__ __forceinline__ void shifts64(const Level &lev, int s, double *sh) {
    using F = Fam<FAM>;
#pragma unroll
    for (int j = 0; j < F::D; ++j) {
        bool split = (lev.split_mask >> j) & 1;
        sh[j] = split ? (((s >> j) & 1) ? lev.h1[j] : -lev.h1[j]) : 0.0;
    }
}

// exact FP64 test of one (record, child): bit 0 UB pass, bit 1 LB pass; fo = the
// record's residual at the child centre
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

// pass masks: one bit per child slot
template <int FAM>
using SlotMask = typename std::conditional<((1 << Fam<FAM>::D) > 32), unsigned long long, unsigned>::type;

// UB/LB pass masks of one record (integer fields) against every child slot, exactly
// as the definition evaluates them.  g64: the cell's basis changes [2^k][NB].
template <int FAM>
__device__ __forceinline__ void eval64(const Problem &P, const Level &lev, const int *qf, const int *qt,
                                       const double *g64, SlotMask<FAM> &ubm, SlotMask<FAM> &lbm) {
    using F = Fam<FAM>;
    using Mask = SlotMask<FAM>;
    constexpr int NS = 1 << F::D, NFS = 1 << F::K;
    double f[F::ND], t[F::LE], R[F::ND];
#pragma unroll
    for (int j = 0; j < F::ND; ++j) f[j] = dmul((double)qf[j], P.s_f[j]);
#pragma unroll
    for (int m = 0; m < F::LE; ++m) t[m] = dmul((double)qt[m], lev.s_t[m]);
    radius64<FAM>(lev, t, R);
    ubm = 0;
    lbm = 0;
#pragma unroll
    for (int fs = 0; fs < NFS; ++fs) {
        if (fs & ~lev.split_mask) continue;
        double pr[F::ND];
        F::partial64(f, t, g64 + fs * F::NB, pr);
#pragma unroll
        for (int s = fs; s < NS; s += NFS) {
            if (s & ~lev.split_mask) continue;
            int ub = 1, lb = 1;
#pragma unroll
            for (int j = 0; j < F::ND; ++j) {
                double a = fabs(dsub(pr[j], dep_shift64<FAM>(lev, j, s)));
                ub &= a <= R[j];
                lb &= a <= lev.rlb[j];
            }
            ubm |= (Mask)ub << s;
            lbm |= (Mask)lb << s;
        }
    }
}

// Record words passed by value to the out-of-line FP64 helpers below (so that the
// caller's arrays stay in registers).
struct RecWords {
    uint32_t w[16];
};

template <int NW>
__device__ __forceinline__ RecWords rec_words_of(const uint32_t *w) {
    static_assert(NW <= 16, "record words");
    RecWords r;
#pragma unroll
    for (int i = 0; i < 16; ++i) r.w[i] = i < NW ? w[i] : 0u;
    return r;
}

// Exact UB/LB masks of one record from its words, out of line (the FP32 screen
// needs it rarely): x = UB mask, y = LB mask.
template <int FAM, bool Q16>
__device__ __noinline__ uint2 eval64_words(const Problem *P, const Level *lev, RecWords rw, const double *g64) {
    using F = Fam<FAM>;
    int qf[F::ND], qt[F::LE];
#pragma unroll
    for (int j = 0; j < F::ND; ++j) qf[j] = field_i<Q16>(rw.w, j);
#pragma unroll
    for (int m = 0; m < F::LE; ++m) qt[m] = field_i<Q16>(rw.w, F::ND + m);
    SlotMask<FAM> ubm, lbm;
    eval64<FAM>(*P, *lev, qf, qt, g64, ubm, lbm);
    if constexpr (sizeof(SlotMask<FAM>) == 8) {
        // families with more than 32 child slots use eval64_words_wide
        return make_uint2(0u, 0u);
    } else {
        return make_uint2(ubm, lbm);
    }
}

// The same for families with more than 32 child slots: x = UB mask, y = LB mask.
template <int FAM, bool Q16>
__device__ __noinline__ ulonglong2 eval64_words_wide(const Problem *P, const Level *lev, RecWords rw,
                                                    const double *g64) {
    using F = Fam<FAM>;
    int qf[F::ND], qt[F::LE];
#pragma unroll
    for (int j = 0; j < F::ND; ++j) qf[j] = field_i<Q16>(rw.w, j);
#pragma unroll
    for (int m = 0; m < F::LE; ++m) qt[m] = field_i<Q16>(rw.w, F::ND + m);
    SlotMask<FAM> ubm, lbm;
    eval64<FAM>(*P, *lev, qf, qt, g64, ubm, lbm);
    return make_ulonglong2((unsigned long long)ubm, (unsigned long long)lbm);
}

// Exact FP64 snap of one record's free parameters at the centre of child s, out of
// line (the FP32 path needs it rarely): the snapped values (x, y: dependent
// coordinates 0 and 1) and z != 0 if a value leaves the representable range.
template <int FAM, bool Q16>
__device__ __noinline__ int3 snap64_words(const Problem *P, const Level *lev, RecWords rw, const double *g64, int s) {
    using F = Fam<FAM>;
    static_assert(F::ND <= 2, "two dependent coordinates at most");
    constexpr int NFS = 1 << F::K;
    double f[F::ND], t[F::LE], pr[F::ND];
#pragma unroll
    for (int j = 0; j < F::ND; ++j) f[j] = dmul((double)field_i<Q16>(rw.w, j), P->s_f[j]);
#pragma unroll
    for (int m = 0; m < F::LE; ++m) t[m] = dmul((double)field_i<Q16>(rw.w, F::ND + m), lev->s_t[m]);
    F::partial64(f, t, g64 + (s & (NFS - 1)) * F::NB, pr);
    int bad = 0, qn[2] = {0, 0};
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        double q = rint(dmul(dsub(pr[j], dep_shift64<FAM>(*lev, j, s)), P->inv_s_f[j]));
        bad |= !(fabs(q) < 1073741824.0);
        qn[j] = bad ? 0 : (int)q;
    }
    return make_int3(qn[0], qn[1], bad);
}

// ---------------------------------------------------------------------------
// Double-float tier.  An integer field as an unevaluated sum hi + lo of two FP32
// values (exact for |q| < 2^31: |q - hi| <= 2^6), and Knuth's two-sum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_int(int q, float &hi, float &lo) {
    hi = __int2float_rn(q);
    lo = __int2float_rn(q - __float2int_rz(hi));
}

__device__ __forceinline__ float two_sum(float a, float b, float &err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// The snap of one record's dependent coordinates at the centre of child s, from
// the residual q_f,j + sum_m q_t,m G64[fs][j][m] -+ h1_j / s_f,j evaluated as a
// double-float (G64 = Gh + Gl, the cell's coefficients and their remainders):
// (x, y) the snapped values, z = 1 when both are decided (the value is more than
// bd_j away from a rounding tie and below lim in magnitude), else 0 (the FP64
// definition decides).  Out of line: the FP32 screen needs it rarely.
template <int FAM, bool Q16>
__device__ __noinline__ int3 snap_df_words(const Level *lev, RecWords rw, const float *Gh, const float *Gl, int s,
                                           float bd0, float bd1, float lim) {
    using F = Fam<FAM>;
    static_assert(F::ND <= 2, "two dependent coordinates at most");
    constexpr int NFS = 1 << F::K;
    const int fs = s & (NFS - 1);
    int qn[2] = {0, 0}, ok = 1;
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        float hi, lo;
        split_int(field_i<Q16>(rw.w, j), hi, lo);
#pragma unroll
        for (int m = 0; m < F::LE; ++m) {
            if (!F::uses(j, m)) continue;
            float th, tl;
            split_int(field_i<Q16>(rw.w, F::ND + m), th, tl);
            const int x = (fs * F::ND + j) * F::LE + m;
            const float gh = __ldg(Gh + x), gl = __ldg(Gl + x);
            const float p = __fmul_rn(th, gh);
            const float e = __fmaf_rn(th, gh, -p);                  // th gh = p + e exactly
            float err;
            hi = two_sum(hi, p, err);
            lo = __fadd_rn(lo, __fadd_rn(err, __fmaf_rn(tl, gl, __fmaf_rn(th, gl, __fmaf_rn(tl, gh, e)))));
        }
        if ((lev->split_mask >> (F::K + j)) & 1) {
            // the residual at the child centre: partial - h1 when the dependent bit is set
            const bool up = (s >> (F::K + j)) & 1;
            const float h = up ? -lev->Hs[j] : lev->Hs[j], hl = up ? -lev->Hs_lo[j] : lev->Hs_lo[j];
            float err;
            hi = two_sum(hi, h, err);
            lo = __fadd_rn(lo, __fadd_rn(err, hl));
        }
        const float r = rintf(hi);                                  // hi - r is exact
        const float w = __fadd_rn(__fsub_rn(hi, r), lo);
        const float k = rintf(w);
        const float fr = __fsub_rn(w, k);
        ok &= (int)(fabsf(hi) < lim) & (int)(0.5f - fabsf(fr) > (j ? bd1 : bd0));
        qn[j] = ok ? __float2int_rn(r) + __float2int_rn(k) : 0;
    }
    return make_int3(qn[0], qn[1], ok);
}

// ---------------------------------------------------------------------------
// FP32 screen (in steps of s_f): residual before the dependent shift for free
// slot fs, from the record's fields and the cell's coefficients G[fs][j][m].
// ---------------------------------------------------------------------------
template <int FAM>
__device__ __forceinline__ void partial32(const float *qf, const float *qt, const float *G, int fs, float *u) {
    using F = Fam<FAM>;
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        float v = qf[j];
#pragma unroll
        for (int m = 0; m < F::LE; ++m)
            if (F::uses(j, m)) v = __fmaf_rn(qt[m], G[(fs * F::ND + j) * F::LE + m], v);
        u[j] = v;
    }
}

// The magnitudes the screen's band scales with (steps): M_j = |q_f,j| + |H_j| +
// sum_m |q_t,m| Gmax_jm, Gmax = the cell's largest |G| per (j, m).
template <int FAM>
__device__ __forceinline__ void magnitudes(const float *qf, const float *qt, const float *Gmax, const float *hs,
                                           float *M) {
    using F = Fam<FAM>;
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        float v = fabsf(qf[j]) + hs[j];
#pragma unroll
        for (int m = 0; m < F::LE; ++m)
            if (F::uses(j, m)) v = __fmaf_ru(fabsf(qt[m]), Gmax[j * F::LE + m], v);
        M[j] = v;
    }
}

// One (record, child slot) decision of the screen.  hs: dependent shifts in steps
// (0 where the coordinate does not split); Rlo/Rhi = radius -+ band, Llo/Lhi the
// same for the lower-bound radius.  ub/lb: the decision if it is certain; uns: a
// comparison fell inside the band (the FP64 definition decides).
template <int FAM>
__device__ __forceinline__ void screen(int ds, const float *u, const float *hs, const float *Rlo, const float *Rhi,
                                       const float *Llo, const float *Lhi, bool &ub, bool &lb, bool &uns) {
    using F = Fam<FAM>;
    ub = true;
    lb = true;
#pragma unroll
    for (int j = 0; j < F::ND; ++j) {
        float a = fabsf(((ds >> j) & 1) ? u[j] - hs[j] : u[j] + hs[j]);
        bool um = a <= Rhi[j], us = a < Rlo[j];
        bool lm = a <= Lhi[j], ls = a < Llo[j];
        ub &= um;
        lb &= lm;
        uns |= (um != us) | (lm != ls);
    }
}

}  // namespace gv
