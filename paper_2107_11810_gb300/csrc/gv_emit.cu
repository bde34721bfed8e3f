// gv_emit.cu -- emit pass of the proximity test: every record of a chunk that
// passed the UB test of a surviving child (the ballots of the count pass) is
// written into that child's record range, with its free parameters snapped at the
// child's centre for the next level (canonization, Sec. 3.2: the residual at the
// child centre, rounded to the snap step; essential parameters re-snapped when
// their step doubles).
//
// Positions: every tile's first output slot per child comes from k_tile_dst;
// inside a tile a lane's position is the number of passing lanes below it.
//
// The snap is taken in FP32 (in steps) when the value is at least the screen's
// band away from a rounding tie, or when the residual is exact in FP32 (every term
// a multiple of 2^e and the magnitudes below 2^(24+e): a tie then rounds to even as
// the definition's exact FP64 value does); else by a double-float recomputation
// when that is far enough from a tie; else in FP64 by the definition.
#include "gv_tile.cuh"

namespace gv {

#ifndef GV_MINBLOCKS_EMIT
#define GV_MINBLOCKS_EMIT 3
#endif

// bit s set for the child slots s = ds << k of free slot 0 (ds over the dependent bits)
__host__ __device__ constexpr unsigned fs_slots(int k, int nd) {
    unsigned m = 0;
    for (int ds = 0; ds < (1 << nd); ++ds) m |= 1u << (ds << k);
    return m;
}

// Shared memory of one block: two buffers of one group (kBlockTiles tiles) of
// records, ballots and output positions.
template <int NW, int NS>
constexpr size_t emit_smem_bytes() {
    return 2 * (size_t)kBlockTiles * (32 * NW * 4 + NS * 4 + NS * 8);
}

// A persistent block takes a contiguous range of groups of kBlockTiles tiles;
// while one group is written, the next one's records, ballots and positions are
// copied into the other buffer.  Warp w writes the child records of tiles
// w * kTW .. w * kTW + kTW - 1 of each group.
template <int FAM, bool QI16, bool QO16, int PREC>
__global__ void __launch_bounds__(256, GV_MINBLOCKS_EMIT) k_emit(const __grid_constant__ Chunk c) {
    using F = Fam<FAM>;
    constexpr int NS = 1 << F::D, NFS = 1 << F::K, ND = F::ND, LE = F::LE, NFP = F::NFP;
    constexpr int NWI = rec_words(NFP, QI16), NWO = rec_words(NFP, QO16);
    constexpr int RW = 32 * NWI;
    constexpr int GT = kBlockTiles;
    constexpr int GF = geo32_floats(NFS, ND, LE);
    // child slots of free slot 0 (those of free slot fs: shifted left by fs)
    constexpr unsigned kFsSlots = fs_slots(F::K, ND);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Level &lev = c.lev;
    const int smask = lev.split_mask;
    extern __shared__ __align__(128) uint32_t s_dyn[];
    unsigned long long *s_dst = reinterpret_cast<unsigned long long *>(s_dyn);   // [2][GT * NS]
    uint32_t *s_rec = s_dyn + 2 * 2 * GT * NS;                                 // [2][GT * RW]
    uint32_t *s_bal = s_rec + 2 * GT * RW;                                     // [2][GT * NS]
    __shared__ __align__(8) uint64_t s_bar[2];

    const int64_t nt = c.t1 - c.t0;
    const int64_t ng = (nt + GT - 1) / GT;
    const int64_t g0 = (int64_t)blockIdx.x * ng / gridDim.x, g1 = (int64_t)(blockIdx.x + 1) * ng / gridDim.x;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int64_t g) {
        const int b = (int)((g - g0) & 1);
        const int64_t ta = g * GT;
        const int ntl = (int)((ta + GT < nt ? ta + GT : nt) - ta);
        const unsigned rbytes = (unsigned)ntl * RW * 4, bbytes = (unsigned)ntl * NS * 4, dbytes = (unsigned)ntl * NS * 8;
        mbar_expect_tx(&s_bar[b], rbytes + bbytes + dbytes);
        bulk_load(s_rec + b * GT * RW, c.in.rec + (c.t0 + ta) * RW, rbytes, &s_bar[b]);
        bulk_load(s_bal + b * GT * NS, c.ballot + ta * NS, bbytes, &s_bar[b]);
        bulk_load(s_dst + b * GT * NS, c.tdst + ta * NS, dbytes, &s_bar[b]);
    };
    if (threadIdx.x == 0 && g0 < g1) issue(g0);

    float hs[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) hs[j] = ((smask >> (F::K + j)) & 1) ? lev.Hs[j] : 0.0f;
    const unsigned below = (1u << lane) - 1u;
    int cur = -1;
    float G[GF];
#pragma unroll
    for (int i = 0; i < GF; ++i) G[i] = 0.0f;
    unsigned nrechk = 0, ndf = 0, bad = 0;
    int64_t gfail = -1;                                             // group whose copy did not arrive
#pragma unroll 1
    for (int64_t g = g0; g < g1; ++g) {
        const int b = (int)((g - g0) & 1);
        if (threadIdx.x == 0 && g + 1 < g1) issue(g + 1);
        const bool ok = mbar_wait(&s_bar[b], (unsigned)(((g - g0) >> 1) & 1), c.spin, &c.sc->err);
        if (__syncthreads_or(!ok)) {
            gfail = g;
            break;
        }
#pragma unroll 1
        for (int k = 0; k < kTW; ++k) {
            const int lt = warp * kTW + k;
            const int64_t tile = c.t0 + g * GT + lt;
            if (tile >= c.t1) break;                                    // uniform
            const uint32_t *bal = s_bal + b * GT * NS + lt * NS;
            const unsigned long long *dst = s_dst + b * GT * NS + lt * NS;
            unsigned vmask = 0;                                         // child slots this tile writes
#pragma unroll
            for (int s = 0; s < NS; ++s) vmask |= (unsigned)(dst[s] != ~0ull && bal[s] != 0u) << s;
            if (!vmask) continue;                                       // uniform: nothing to write
            const int cl = c.tinfo[tile - c.t0].x;                      // >= 0: something is written
            if (PREC == 1 && cl != cur) {
                const float *gp = c.geo32 + (size_t)cl * GF;
#pragma unroll
                for (int i = 0; i < GF; ++i) G[i] = __ldg(gp + i);
            }
            cur = cl;
            uint32_t w[NWI];
#pragma unroll
            for (int i = 0; i < NWI; ++i) w[i] = s_rec[b * GT * RW + lt * RW + lane * NWI + i];
            const int64_t r = tile * 32 + lane;
            const double *g64 = c.geo64 + (size_t)cl * NFS * F::NB;
            // the child's essential parameters (re-snapped when the step doubles)
            uint32_t fb[NFP];
#pragma unroll
            for (int i = 0; i < NFP; ++i) fb[i] = 0u;
            float qf[ND], qt[LE];
#pragma unroll
            for (int j = 0; j < ND; ++j) qf[j] = field_f<QI16>(w, j);
#pragma unroll
            for (int m = 0; m < LE; ++m) {
                qt[m] = field_f<QI16>(w, ND + m);
                if constexpr (QO16) {
                    // adding kMagic16 rounds to an integer, ties to even, biased by 2^15
                    float v = lev.st_ratio_log2[m] ? __fmaf_rn(qt[m], 0.5f, kMagic16) : qt[m] + kMagic16;
                    fb[ND + m] = __float_as_uint(v);
                } else {
                    const int q = field_i<QI16>(w, ND + m);
                    fb[ND + m] = (uint32_t)(lev.st_ratio_log2[m] ? resnap_half(q) : q);
                }
            }
            const uint32_t mult = c.out.mult ? c.in.mult[r] : 1u;
            float es[ND], bd[ND];                                       // the snaps' bands (steps)
            bool xs[ND];                                                // FP32 residual exact
            if (PREC == 1) {
                float M[ND];
                // every term a multiple of 2^ex and M below 2^(24 + ex): the FP32 residual, and
                // the definition's FP64 one, are exact, so a tie rounds to even in both
                const int ex = min(__float2int_rn(G[GF - 1]), lev.hs_exp);
                const float tq = ex > -100 ? __int_as_float((127 + 24 + ex) << 23) : 0.0f;
                magnitudes<FAM>(qf, qt, G + NFS * ND * LE, hs, M);
#pragma unroll
                for (int j = 0; j < ND; ++j) {
                    es[j] = 0.5f - kBandSnap * M[j];
                    bd[j] = __fmaf_ru(kBandDF, M[j], kBandDFAbs);
                    xs[j] = M[j] < tq;
                }
            }
#pragma unroll
            for (int fs = 0; fs < NFS; ++fs) {
                if (!(vmask & (kFsSlots << fs))) continue;             // uniform: no child of this free slot
                float u[ND];
#pragma unroll
                for (int j = 0; j < ND; ++j) u[j] = 0.0f;
                if (PREC == 1) partial32<FAM>(qf, qt, G, fs, u);
#pragma unroll
                for (int ds = 0; ds < (1 << ND); ++ds) {
                    const int s = fs | (ds << F::K);
                    if (!((vmask >> s) & 1)) continue;                  // uniform
                    const unsigned bs = bal[s];
                    if (!((bs >> lane) & 1)) continue;
                    const unsigned long long d0 = dst[s];
                    const unsigned long long pos = d0 + (unsigned)__popc(bs & below);
                    bool done = PREC == 1;
                    if (PREC == 1) {
#pragma unroll
                        for (int j = 0; j < ND; ++j) {
                            const float y = ((ds >> j) & 1) ? u[j] - hs[j] : u[j] + hs[j];
                            if constexpr (QO16) {
                                const float t = y + kMagic16;
                                done &= (fabsf(y - (t - kMagic16)) < es[j] || xs[j]) && fabsf(y) < 32767.0f;
                                fb[j] = __float_as_uint(t);
                            } else {
                                const float t = y + kMagic;
                                done &= (fabsf(y - (t - kMagic)) < es[j] || xs[j]) && fabsf(y) < 4.0e6f;
                                fb[j] = (uint32_t)(__float_as_int(t) - 0x4B400000);
                            }
                        }
                    }
                    if (!done) {
                        int3 q = make_int3(0, 0, 0);
                        if constexpr (PREC == 1) {                              // the double-float tier
                            q = snap_df_words<FAM, QI16>(&c.lev, rec_words_of<NWI>(w), c.geo32 + (size_t)cl * GF,
                                                         c.geo32lo + (size_t)cl * (NFS * ND * LE), s, bd[0],
                                                         bd[ND - 1], QO16 ? 32767.0f : 1.0e9f);
                            ++ndf;
                        }
                        if (!q.z) {                                             // the FP64 definition
                            q = snap64_words<FAM, QI16>(&c.P, &c.lev, rec_words_of<NWI>(w), g64, s);
                            bad |= (unsigned)(q.z != 0);
                            nrechk += PREC == 1;
                        }
                        const int qn[2] = {q.x, q.y};
#pragma unroll
                        for (int j = 0; j < ND; ++j) {
                            if constexpr (QO16) {
                                bad |= (unsigned)(qn[j] < -32768 || qn[j] > 32767) << 1;
                                fb[j] = (uint32_t)(qn[j] + 32768);
                            } else {
                                fb[j] = (uint32_t)qn[j];
                            }
                        }
                    }
                    uint32_t wo[NWO];
                    pack<NFP, QO16>(fb, wo);
                    store_words<NWO>(c.out.rec, (int64_t)pos, wo);
                    if (c.out.mult) c.out.mult[pos] = mult;
                }
            }
        }
        __syncthreads();                                                // buffer b is free again
    }
    if (gfail >= 0 && threadIdx.x == 0) {
        // the copies of groups gfail and gfail + 1 (no later one was issued) may still
        // be in flight: wait for them, bounded, before the block's shared memory is
        // released
        const int64_t ge = gfail + 2 < g1 ? gfail + 2 : g1;
        for (int64_t g = gfail; g < ge; ++g) {
            const int b = (int)((g - g0) & 1);
            if (!mbar_wait(&s_bar[b], (unsigned)(((g - g0) >> 1) & 1), GV_SPIN_LIMIT, &c.sc->err)) break;
        }
    }
    nrechk = __reduce_add_sync(kFull, nrechk);
    ndf = __reduce_add_sync(kFull, ndf);
    bad = __reduce_or_sync(kFull, bad);
    if (lane == 0) {
        if (nrechk) atomicAdd(&c.sc->rechecks, (unsigned long long)nrechk);
        if (ndf) atomicAdd(&c.sc->rechecks_df, (unsigned long long)ndf);
        if (bad) atomicOr(&c.sc->err, bad << 1);
    }
}

#define GV_DISPATCH(fam, CALL)                                                   \
    switch (fam) {                                                               \
    case FAM_LINE2D: { constexpr int FAMV = FAM_LINE2D; CALL; } break;           \
    case FAM_PLANE3D_SPH: { constexpr int FAMV = FAM_PLANE3D_SPH; CALL; } break; \
    case FAM_POSE3DOF: { constexpr int FAMV = FAM_POSE3DOF; CALL; } break;       \
    case FAM_RAYS3D: { constexpr int FAMV = FAM_RAYS3D; CALL; } break;           \
    default: break;                                                              \
    }


bool launch_emit(const Chunk &c, cudaStream_t st) {
    const int64_t nt = c.t1 - c.t0;
    if (nt <= 0) return true;
    if (c.P.d > 3) return launch_emit_wide(c, st);
    const int64_t ng = (nt + kBlockTiles - 1) / kBlockTiles;
    const int q = c.lev.q16, qn = c.lev.q16_next;
#define GV_EMIT(QI, QO, PREC)                                                                                 \
    {                                                                                                          \
        constexpr int NW = rec_words(Fam<FAMV>::NFP, QI), NS = 1 << Fam<FAMV>::D;                               \
        launch_persistent((const void *)k_emit<FAMV, QI, QO, PREC>, emit_smem_bytes<NW, NS>(), ng, c, st);                    \
    }
    if (c.precision == 0) {
        if (q || qn) return false;                  // plain FP64 mode keeps 32-bit records
        GV_DISPATCH(c.P.fam, GV_EMIT(false, false, 0));
    } else if (q && qn) {
        GV_DISPATCH(c.P.fam, GV_EMIT(true, true, 1));
    } else if (!q && qn) {
        GV_DISPATCH(c.P.fam, GV_EMIT(false, true, 1));
    } else if (!q && !qn) {
        GV_DISPATCH(c.P.fam, GV_EMIT(false, false, 1));
    } else {
        return false;                               // 16-bit to 32-bit: never chosen
    }
#undef GV_EMIT
    return true;
}

}  // namespace gv
