// gv_wide.cu -- the proximity test's count and emit passes for families whose
// cells split into 16, 32 or 64 children (d = 4, 5, 6: Algorithm 2's 2^d
// sub-boxes).  The same tests as gv_count.cu and gv_emit.cu (the surface-box test
// of Sec. 3.2 with the FP32 screen and FP64 recheck, and the snap of the child
// records for the next level), laid out for many child slots: lane s % 32 keeps the
// counters and the ballot of child slot s, and the screen's coefficients of the
// cell (the same for every lane of a warp) are staged in the warp's part of shared
// memory once per run of tiles of one cell.
//
// Each warp takes a contiguous range of the chunk's tiles (so runs of tiles of one
// cell stay together) and reads its records with plain loads; there are no
// device-side waits.
#include "gv_tile.cuh"

namespace gv {

template <int FAM, bool Q16, int PREC, bool WEIGHTED>
__global__ void __launch_bounds__(256) k_count_wide(const __grid_constant__ Chunk c) {
    using F = Fam<FAM>;
    using Mask = SlotMask<FAM>;
    constexpr int NS = 1 << F::D, NFS = 1 << F::K, NDS = 1 << F::ND, ND = F::ND, LE = F::LE;
    static_assert(NS >= 16 && NS <= 64, "16 to 64 child slots");
    constexpr int SPL = NS > 32 ? NS / 32 : 1;                     // child slots per lane
    constexpr int NW = rec_words(F::NFP, Q16);
    constexpr int GF = geo32_floats(NFS, ND, LE);
    const int lane = threadIdx.x & 31;
    // the current cell's screen coefficients, staged once per run of tiles of the
    // cell in the warp's part of shared memory (the per-free-slot loads then wait
    // on shared memory, not on the cache hierarchy); blocks of 8 warps
    __shared__ float s_g[8][GF];
    float *sg = s_g[threadIdx.x >> 5];
    int gcell = -1;
    auto stage = [&](int cell) {
        if (cell == gcell) return;                                  // uniform
        __syncwarp();                                               // the old cell's reads are done
        const float *src = c.geo32 + (size_t)cell * GF;
        for (int i = lane; i < GF; i += 32) sg[i] = src[i];
        __syncwarp();
        gcell = cell;
    };
    const int64_t nt = c.t1 - c.t0;
    const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t ta = gw * nt / nwarp, tb = (gw + 1) * nt / nwarp;        // chunk-relative tiles
    const Level &lev = c.lev;
    const int smask = lev.split_mask;
    float hs[ND], Lc[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
        hs[j] = ((smask >> (F::K + j)) & 1) ? lev.Hs[j] : 0.0f;
        Lc[j] = lev.Lc[j];
    }
    unsigned nvslot = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) nvslot += !(s & ~smask);

    // counters of the current run of tiles of one cell, for slots lane + 32 h
    unsigned cu[SPL], cl[SPL], cn[SPL];
#pragma unroll
    for (int h = 0; h < SPL; ++h) cu[h] = cl[h] = cn[h] = 0u;
    int run = -1;
    unsigned ntest = 0, nrechk = 0, nrec = 0;
    auto flush = [&]() {
        if (run < 0) return;
#pragma unroll
        for (int h = 0; h < SPL; ++h) {
            if (lane + 32 * h >= NS) break;
            uint32_t *bc = c.cnt + ((size_t)run * NS + lane + 32 * h) * 3;
            if (cu[h]) atomicAdd(bc, cu[h]);
            if (cl[h]) atomicAdd(bc + 1, cl[h]);
            if (cn[h]) atomicAdd(bc + 2, cn[h]);
            cu[h] = cl[h] = cn[h] = 0u;
        }
    };

#pragma unroll 1
    for (int64_t tt = ta; tt < tb; ++tt) {
        const int2 ti = c.tinfo[tt];
        const int cell = ti.x;
        if (cell < 0) continue;                                     // uniform: the cell was pruned
        if (cell != run) {                                          // uniform: a new cell
            flush();
            run = cell;
        }
        const int64_t tile = c.t0 + tt;
        const int nvalid = ti.y;
        const bool act = lane < nvalid;
        const int64_t r = tile * 32 + lane;
        ntest += (unsigned)nvalid * nvslot;
        nrec += (unsigned)nvalid;
        uint32_t w[NW];
        load_words<NW>(c.in.rec, r, w);                             // whole tiles are allocated
        const uint32_t mult = WEIGHTED ? (act ? c.in.mult[r] : 0u) : 1u;
        if constexpr (PREC == 1) stage(cell);
        const float *G = sg;
        const double *g64 = c.geo64 + (size_t)cell * NFS * F::NB;
        unsigned bw[SPL];                                           // ballots of slots lane + 32 h
#pragma unroll
        for (int h = 0; h < SPL; ++h) bw[h] = 0u;
        // child slot s: the warp's ballots and sums go to lane s % 32
        auto count = [&](int s, bool ub, bool lb) {
            const unsigned bu = __ballot_sync(kFull, ub);
            unsigned au, al;
            if constexpr (WEIGHTED) {
                au = __reduce_add_sync(kFull, ub ? mult : 0u);
                al = __reduce_add_sync(kFull, lb ? mult : 0u);
            } else {
                au = __popc(bu);
                al = __popc(__ballot_sync(kFull, lb));
            }
            if (lane == (s & 31)) {
                bw[s >> 5] = bu;
                cu[s >> 5] += au;
                cl[s >> 5] += al;
                cn[s >> 5] += (unsigned)__popc(bu);
            }
        };
        if constexpr (PREC == 1) {
            float qf[ND], qt[LE], R[ND], M[ND], Rlo[ND], Rhi[ND], Llo[ND], Lhi[ND];
#pragma unroll
            for (int j = 0; j < ND; ++j) qf[j] = field_f<Q16>(w, j);
#pragma unroll
            for (int m = 0; m < LE; ++m) qt[m] = field_f<Q16>(w, ND + m);
            F::radius32(lev, qt, R);
            magnitudes<FAM>(qf, qt, G + NFS * ND * LE, hs, M);
#pragma unroll
            for (int j = 0; j < ND; ++j) {
                const float e = kBandTest * (M[j] + R[j]);
                Rlo[j] = R[j] - e;
                Rhi[j] = R[j] + e;
                Llo[j] = Lc[j] - e;
                Lhi[j] = Lc[j] + e;
            }
            // a lane without a record fails every test (its residual is out of reach)
            if (!act) qf[0] = 1.0e30f;
            bool uns = false;
#pragma unroll 1
            for (int fs = 0; fs < NFS; ++fs) {
                float u[ND];
                partial32<FAM>(qf, qt, G, fs, u);
#pragma unroll
                for (int ds = 0; ds < NDS; ++ds) {
                    bool ub, lb;
                    screen<FAM>(ds, u, hs, Rlo, Rhi, Llo, Lhi, ub, lb, uns);
                    count(fs | (ds << F::K), ub, lb);
                }
            }
            const unsigned unsb = __ballot_sync(kFull, act && uns);
            if (unsb) {
                // rare: the lanes whose screen was unsure take the FP64 definition; the
                // difference to what was counted goes to the cell's counters directly
                Mask m64u = 0;
                if ((unsb >> lane) & 1) {
                    Mask m32u = 0, m32l = 0;
#pragma unroll 1
                    for (int fs = 0; fs < NFS; ++fs) {
                        float u[ND];
                        partial32<FAM>(qf, qt, G, fs, u);
#pragma unroll
                        for (int ds = 0; ds < NDS; ++ds) {
                            const int s = fs | (ds << F::K);
                            bool ub, lb, un = false;
                            screen<FAM>(ds, u, hs, Rlo, Rhi, Llo, Lhi, ub, lb, un);
                            m32u |= (Mask)ub << s;
                            m32l |= (Mask)lb << s;
                        }
                    }
                    const ulonglong2 m64 = eval64_words_wide<FAM, Q16>(&c.P, &c.lev, rec_words_of<NW>(w), g64);
                    m64u = (Mask)m64.x;
                    nrechk += nvslot;
                    for (Mask d = (m32u ^ (Mask)m64.x) | (m32l ^ (Mask)m64.y); d; d &= d - 1) {
                        const int s = __ffsll((long long)d) - 1;
                        const int du = (int)((m64.x >> s) & 1) - (int)((m32u >> s) & 1);
                        const int dl = (int)((m64.y >> s) & 1) - (int)((m32l >> s) & 1);
                        uint32_t *bc = c.cnt + ((size_t)cell * NS + s) * 3;
                        if (du) {
                            atomicAdd(bc, (unsigned)(du * (int)mult));
                            atomicAdd(bc + 2, (unsigned)du);
                        }
                        if (dl) atomicAdd(bc + 1, (unsigned)(dl * (int)mult));
                    }
                }
#pragma unroll 1
                for (int s = 0; s < NS; ++s) {
                    const unsigned fix = __ballot_sync(kFull, ((unsb >> lane) & 1) && ((m64u >> s) & 1));
                    if (lane == (s & 31)) bw[s >> 5] = (bw[s >> 5] & ~unsb) | fix;
                }
            }
        } else {
            // plain FP64: every record by the definition
            ulonglong2 m64 = make_ulonglong2(0ull, 0ull);
            if (act) m64 = eval64_words_wide<FAM, Q16>(&c.P, &c.lev, rec_words_of<NW>(w), g64);
#pragma unroll 1
            for (int s = 0; s < NS; ++s) count(s, (m64.x >> s) & 1, (m64.y >> s) & 1);
        }
        // the tile's ballots, one word per child slot
        uint32_t *bp = c.ballot + (size_t)tt * NS;
#pragma unroll
        for (int h = 0; h < SPL; ++h)
            if (lane + 32 * h < NS) bp[lane + 32 * h] = bw[h];
    }
    flush();
    ntest = __reduce_add_sync(kFull, lane == 0 ? ntest : 0u);
    nrec = __reduce_add_sync(kFull, lane == 0 ? nrec : 0u);
    nrechk = __reduce_add_sync(kFull, nrechk);
    if (lane == 0) {
        if (ntest) atomicAdd(&c.sc->tests, (unsigned long long)ntest);
        if (nrec) atomicAdd(&c.sc->records, (unsigned long long)nrec);
        if (nrechk) atomicAdd(&c.sc->rechecks, (unsigned long long)nrechk);
    }
}

template <int FAM, bool QI16, bool QO16, int PREC>
__global__ void __launch_bounds__(256) k_emit_wide(const __grid_constant__ Chunk c) {
    using F = Fam<FAM>;
    constexpr int NS = 1 << F::D, NFS = 1 << F::K, NDS = 1 << F::ND, ND = F::ND, LE = F::LE, NFP = F::NFP;
    static_assert(NS >= 16 && NS <= 64 && ND <= 2, "16 to 64 child slots, two dependent coordinates");
    constexpr int NWI = rec_words(NFP, QI16), NWO = rec_words(NFP, QO16);
    constexpr int GF = geo32_floats(NFS, ND, LE);
    const int lane = threadIdx.x & 31;
    // the current cell's screen coefficients, staged once per run of tiles of the
    // cell in the warp's part of shared memory (the per-free-slot loads then wait
    // on shared memory, not on the cache hierarchy); blocks of 8 warps
    __shared__ float s_g[8][GF];
    float *sg = s_g[threadIdx.x >> 5];
    int gcell = -1;
    auto stage = [&](int cell) {
        if (cell == gcell) return;                                  // uniform
        __syncwarp();                                               // the old cell's reads are done
        const float *src = c.geo32 + (size_t)cell * GF;
        for (int i = lane; i < GF; i += 32) sg[i] = src[i];
        __syncwarp();
        gcell = cell;
    };
    const unsigned below = (1u << lane) - 1u;
    const int64_t nt = c.t1 - c.t0;
    const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t ta = gw * nt / nwarp, tb = (gw + 1) * nt / nwarp;
    const Level &lev = c.lev;
    const int smask = lev.split_mask;
    float hs[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) hs[j] = ((smask >> (F::K + j)) & 1) ? lev.Hs[j] : 0.0f;
    unsigned nrechk = 0, ndf = 0, bad = 0;

#pragma unroll 1
    for (int64_t tt = ta; tt < tb; ++tt) {
        const int cell = c.tinfo[tt].x;
        if (cell < 0) continue;                                     // uniform
        const uint32_t *bp = c.ballot + (size_t)tt * NS;
        const unsigned long long *dp = c.tdst + (size_t)tt * NS;
        // slots lane (A) and lane + 32 (B)
        const bool hasA = lane < NS, hasB = lane + 32 < NS;
        const unsigned balA = hasA ? bp[lane] : 0u, balB = hasB ? bp[32 + lane] : 0u;
        const unsigned long long dA = hasA ? dp[lane] : ~0ull, dB = hasB ? dp[32 + lane] : ~0ull;
        // child slots this tile writes (bit s of vA: slot s, of vB: slot 32 + s)
        const unsigned vA = __ballot_sync(kFull, dA != ~0ull && balA != 0u);
        const unsigned vB = __ballot_sync(kFull, dB != ~0ull && balB != 0u);
        if (!(vA | vB)) continue;                                   // uniform
        const int64_t r = (c.t0 + tt) * 32 + lane;
        uint32_t w[NWI];
        load_words<NWI>(c.in.rec, r, w);
        if (PREC == 1) stage(cell);
        const float *G = sg;
        const double *g64 = c.geo64 + (size_t)cell * NFS * F::NB;
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
#pragma unroll 1
        for (int fs = 0; fs < NFS; ++fs) {
            unsigned any = 0;
#pragma unroll
            for (int ds = 0; ds < NDS; ++ds) {
                const int s = fs | (ds << F::K);
                any |= (s < 32 ? (vA >> s) : (vB >> (s - 32))) & 1u;
            }
            if (!any) continue;                                     // uniform
            float u[ND];
#pragma unroll
            for (int j = 0; j < ND; ++j) u[j] = 0.0f;
            if (PREC == 1) partial32<FAM>(qf, qt, G, fs, u);
#pragma unroll
            for (int ds = 0; ds < NDS; ++ds) {
                const int s = fs | (ds << F::K);
                if (!((s < 32 ? (vA >> s) : (vB >> (s - 32))) & 1u)) continue;    // uniform
                const unsigned bs = __shfl_sync(kFull, s < 32 ? balA : balB, s & 31);
                const unsigned long long d0 = __shfl_sync(kFull, s < 32 ? dA : dB, s & 31);
                if (!((bs >> lane) & 1)) continue;
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
                        q = snap_df_words<FAM, QI16>(&c.lev, rec_words_of<NWI>(w), c.geo32 + (size_t)cell * GF,
                                                     c.geo32lo + (size_t)cell * (NFS * ND * LE), s, bd[0],
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
    nrechk = __reduce_add_sync(kFull, nrechk);
    ndf = __reduce_add_sync(kFull, ndf);
    bad = __reduce_or_sync(kFull, bad);
    if (lane == 0) {
        if (nrechk) atomicAdd(&c.sc->rechecks, (unsigned long long)nrechk);
        if (ndf) atomicAdd(&c.sc->rechecks_df, (unsigned long long)ndf);
        if (bad) atomicOr(&c.sc->err, bad << 1);
    }
}

// a grid of 8-warp blocks: enough warps to fill the device, at most one per tile
static unsigned wide_blocks(int64_t nt) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int64_t want = (int64_t)sms * 8;                    // blocks of 8 warps, 8 blocks per SM
    int64_t need = (nt + 7) / 8;
    return (unsigned)(want < need ? want : need);
}

#define GV_DISPATCH_WIDE(fam, CALL)                                            \
    switch (fam) {                                                             \
    case FAM_POSE6DOF: { constexpr int FAMV = FAM_POSE6DOF; CALL; } break;     \
    case FAM_POINTSET2D: { constexpr int FAMV = FAM_POINTSET2D; CALL; } break; \
    case FAM_AFFINE4D: { constexpr int FAMV = FAM_AFFINE4D; CALL; } break;     \
    case FAM_RADIAL5DOF: { constexpr int FAMV = FAM_RADIAL5DOF; CALL; } break; \
    default: break;                                                            \
    }

void launch_count_wide(const Chunk &c, cudaStream_t st) {
    const int64_t nt = c.t1 - c.t0;
    if (nt <= 0) return;
    const unsigned g = wide_blocks(nt);
    const bool w = c.in.mult != nullptr;
#define GV_COUNT_WIDE(Q16, PREC)                                                         \
    {                                                                                   \
        if (w) k_count_wide<FAMV, Q16, PREC, true><<<g, 256, 0, st>>>(c);               \
        else k_count_wide<FAMV, Q16, PREC, false><<<g, 256, 0, st>>>(c);                \
    }
    if (c.precision == 0) {
        GV_DISPATCH_WIDE(c.P.fam, GV_COUNT_WIDE(false, 0));
    } else if (c.lev.q16) {
        GV_DISPATCH_WIDE(c.P.fam, GV_COUNT_WIDE(true, 1));
    } else {
        GV_DISPATCH_WIDE(c.P.fam, GV_COUNT_WIDE(false, 1));
    }
#undef GV_COUNT_WIDE
}

bool launch_emit_wide(const Chunk &c, cudaStream_t st) {
    const int64_t nt = c.t1 - c.t0;
    if (nt <= 0) return true;
    const unsigned g = wide_blocks(nt);
    const int q = c.lev.q16, qn = c.lev.q16_next;
    bool known = false;
    GV_DISPATCH_WIDE(c.P.fam, (known = FAMV > 0));
    if (!known) return false;
    if (c.precision == 0) {
        if (q || qn) return false;                  // plain FP64 mode keeps 32-bit records
        GV_DISPATCH_WIDE(c.P.fam, (k_emit_wide<FAMV, false, false, 0><<<g, 256, 0, st>>>(c)));
    } else if (q && qn) {
        GV_DISPATCH_WIDE(c.P.fam, (k_emit_wide<FAMV, true, true, 1><<<g, 256, 0, st>>>(c)));
    } else if (!q && qn) {
        GV_DISPATCH_WIDE(c.P.fam, (k_emit_wide<FAMV, false, true, 1><<<g, 256, 0, st>>>(c)));
    } else if (!q && !qn) {
        GV_DISPATCH_WIDE(c.P.fam, (k_emit_wide<FAMV, false, false, 1><<<g, 256, 0, st>>>(c)));
    } else {
        return false;                               // 16-bit to 32-bit: never chosen
    }
    return true;
}

}  // namespace gv
