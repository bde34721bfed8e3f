// gv_count.cu -- count pass of the proximity test (Algorithm 2's per-sub-box
// selection with the surface-box test of Sec. 3.2): for every record of a chunk and
// every child of its cell, the UB test (|residual| <= eps + cell radius + Lipschitz
// term + accumulated canonization error) and the LB test (|residual| <= eps -
// accumulated error); per child the multiplicity sums UB, LB and the number of
// UB-passing records; per tile and child the ballot of UB-passing lanes, which the
// emit pass uses to write the child records.
//
// FP32 screen + FP64 recheck: the decisions are taken in FP32 in units of the snap
// step; a lane whose comparison falls inside the screen's error band re-evaluates
// its record with the exact FP64 definition, and its counts and ballot bits are
// corrected (a rare path).  Plain FP64 mode evaluates every record exactly.
#include "gv_tile.cuh"

namespace gv {

#ifndef GV_MINBLOCKS_COUNT
#define GV_MINBLOCKS_COUNT 3
#endif

// Shared memory of one block: two buffers of one group (kBlockTiles tiles) of
// records and tile information.
template <int NW>
constexpr size_t count_smem_bytes() {
    return 2 * (size_t)kBlockTiles * 32 * NW * 4 + 2 * (size_t)kBlockTiles * sizeof(int2);
}

// A persistent block takes a contiguous range of groups of kBlockTiles tiles;
// while one group is tested, the next one's records and tile information are
// copied into the other buffer (bulk copies completing on an mbarrier).  Warp w
// tests tiles w * kTW .. w * kTW + kTW - 1 of each group.
template <int FAM, bool Q16, int PREC, bool WEIGHTED>
__global__ void __launch_bounds__(256, GV_MINBLOCKS_COUNT) k_count(const __grid_constant__ Chunk c) {
    using F = Fam<FAM>;
    constexpr int NS = 1 << F::D, NFS = 1 << F::K, ND = F::ND, LE = F::LE, NFP = F::NFP;
    constexpr int NW = rec_words(NFP, Q16);
    constexpr int RW = 32 * NW;                             // words per tile
    constexpr int GT = kBlockTiles;
    constexpr int NCW = (NS + 3) / 4;                      // byte-packed counter words
    constexpr int GF = geo32_floats(NFS, ND, LE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Level &lev = c.lev;
    const int smask = lev.split_mask;
    extern __shared__ __align__(128) uint32_t s_dyn[];
    uint32_t *s_rec = s_dyn;                                              // [2][GT * RW]
    int2 *s_ti = reinterpret_cast<int2 *>(s_dyn + 2 * GT * RW);           // [2][GT]
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
    // thread 0: copy group g into buffer (g - g0) & 1
    auto issue = [&](int64_t g) {
        const int b = (int)((g - g0) & 1);
        const int64_t ta = g * GT;                                        // chunk-relative first tile
        const int ntl = (int)((ta + GT < nt ? ta + GT : nt) - ta);
        const unsigned rbytes = (unsigned)ntl * RW * 4;
        const unsigned ibytes = (unsigned)((ntl + 1) & ~1) * (unsigned)sizeof(int2);   // 16-byte multiple
        mbar_expect_tx(&s_bar[b], rbytes + ibytes);
        bulk_load(s_rec + b * GT * RW, c.in.rec + (c.t0 + ta) * RW, rbytes, &s_bar[b]);
        bulk_load(s_ti + b * GT, c.tinfo + ta, ibytes, &s_bar[b]);
    };
    if (threadIdx.x == 0 && g0 < g1) issue(g0);

    // dependent shifts and lower-bound radii of this level (steps)
    float hs[ND], Lc[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
        hs[j] = ((smask >> (F::K + j)) & 1) ? lev.Hs[j] : 0.0f;
        Lc[j] = lev.Lc[j];
    }
    unsigned nvslot = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) nvslot += !(s & ~smask);

    // counts of the current run of tiles of one cell
    unsigned pu[NCW], pl[NCW];
    unsigned wu[WEIGHTED ? NS : 1], wl[WEIGHTED ? NS : 1], wn[WEIGHTED ? NS : 1];
#pragma unroll
    for (int x = 0; x < NCW; ++x) pu[x] = pl[x] = 0u;
#pragma unroll
    for (int s = 0; s < (WEIGHTED ? NS : 1); ++s) wu[s] = wl[s] = wn[s] = 0u;
    int run = -1;                 // chunk-local cell of the run
    float G[GF];
#pragma unroll
    for (int i = 0; i < GF; ++i) G[i] = 0.0f;
    unsigned ntest = 0, nrechk = 0, nrec = 0;

    // lane x < 3 NS accumulates counter x / NS (UB, LB, records) of child slot x % NS
    // for the current run; the byte-packed per-lane counters are drained into it
    // every kTW tiles (before a byte could carry) and it goes to the cell's global
    // counters when the run ends
    unsigned acc = 0;
    auto drain = [&]() {
        if constexpr (!WEIGHTED) {
            unsigned au[NCW], al[NCW];
#pragma unroll
            for (int x = 0; x < NCW; ++x) {
                au[x] = __reduce_add_sync(kFull, pu[x]);
                al[x] = __reduce_add_sync(kFull, pl[x]);
                pu[x] = pl[x] = 0u;
            }
            const int s = lane % NS, kind = lane / NS;
            unsigned word = kind == 1 ? al[0] : au[0];
#pragma unroll
            for (int x = 1; x < NCW; ++x)
                if ((s >> 2) == x) word = kind == 1 ? al[x] : au[x];
            if (lane < 3 * NS) acc += (word >> (8 * (s & 3))) & 255u;
        } else {
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (lane == s) acc += wu[s];
                if (lane == NS + s) acc += wl[s];
                if (lane == 2 * NS + s) acc += wn[s];
                wu[s] = wl[s] = wn[s] = 0u;
            }
        }
    };
    auto flush = [&]() {
        if (run < 0) return;
        drain();
        if (lane < 3 * NS && acc) atomicAdd(c.cnt + ((size_t)run * NS + lane % NS) * 3 + lane / NS, acc);
        acc = 0;
    };

    int64_t gfail = -1;                                             // group whose copy did not arrive
#pragma unroll 1
    for (int64_t g = g0; g < g1; ++g) {
        const int b = (int)((g - g0) & 1);
        if (threadIdx.x == 0 && g + 1 < g1) issue(g + 1);
        const bool ok = mbar_wait(&s_bar[b], (unsigned)(((g - g0) >> 1) & 1), c.spin, &c.sc->err);
        if (__syncthreads_or(!ok)) {                                // uniform: a copy did not arrive
            gfail = g;
            break;
        }
#pragma unroll 1
        for (int k = 0; k < kTW; ++k) {
            const int lt = warp * kTW + k;                          // tile within the group
            const int64_t tile = c.t0 + g * GT + lt;
            if (tile >= c.t1) break;                                // uniform
            const int2 ti = s_ti[b * GT + lt];
            const int cl = ti.x;
            if (cl < 0) continue;                                   // uniform: the cell was pruned
            if (cl != run) {                                        // uniform: a new cell
                flush();
                run = cl;
                if (PREC == 1) {
                    const float *gp = c.geo32 + (size_t)cl * GF;
#pragma unroll
                    for (int i = 0; i < GF; ++i) G[i] = __ldg(gp + i);
                }
            }
            uint32_t w[NW];
#pragma unroll
            for (int i = 0; i < NW; ++i) w[i] = s_rec[b * GT * RW + lt * RW + lane * NW + i];
            const int nvalid = ti.y;
            const bool act = lane < nvalid;
            const int64_t r = tile * 32 + lane;
            ntest += (unsigned)nvalid * nvslot;
            nrec += (unsigned)nvalid;
            const uint32_t mult = WEIGHTED ? (act ? c.in.mult[r] : 0u) : 1u;
            const double *g64 = c.geo64 + (size_t)cl * NFS * F::NB;
            unsigned bw[NS];                 // the tile's ballot per child slot
#pragma unroll
            for (int s = 0; s < NS; ++s) bw[s] = 0u;
            bool uns = false;
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
#pragma unroll
                for (int fs = 0; fs < NFS; ++fs) {
                    float u[ND];
                    partial32<FAM>(qf, qt, G, fs, u);
#pragma unroll
                    for (int ds = 0; ds < (1 << ND); ++ds) {
                        // every slot is tested, also those of coordinates that no longer
                        // split: their counts and ballots are never read, and testing them
                        // costs less than branching around them
                        const int s = fs | (ds << F::K);
                        bool ub, lb;
                        screen<FAM>(ds, u, hs, Rlo, Rhi, Llo, Lhi, ub, lb, uns);
                        const unsigned bb = __ballot_sync(kFull, ub);
                        bw[s] = bb;
                        if constexpr (!WEIGHTED) {
                            if (ub) pu[s >> 2] += 1u << (8 * (s & 3));
                            if (lb) pl[s >> 2] += 1u << (8 * (s & 3));
                        } else {
                            wu[s] += __reduce_add_sync(kFull, ub ? mult : 0u);
                            wl[s] += __reduce_add_sync(kFull, lb ? mult : 0u);
                            wn[s] += __popc(bb);
                        }
                    }
                }
                const unsigned unsb = __ballot_sync(kFull, act && uns);
                if (unsb) {
                    // rare: the lanes whose screen was unsure take the FP64 definition; the
                    // difference to what was counted is added directly to the cell's counters
                    unsigned m64u = 0;
                    if ((unsb >> lane) & 1) {
                        unsigned m32u = 0, m32l = 0;
#pragma unroll
                        for (int fs = 0; fs < NFS; ++fs) {
                            float u[ND];
                            partial32<FAM>(qf, qt, G, fs, u);
#pragma unroll
                            for (int ds = 0; ds < (1 << ND); ++ds) {
                                const int s = fs | (ds << F::K);
                                bool ub, lb, un = false;
                                screen<FAM>(ds, u, hs, Rlo, Rhi, Llo, Lhi, ub, lb, un);
                                m32u |= (unsigned)ub << s;
                                m32l |= (unsigned)lb << s;
                            }
                        }
                        const uint2 m64 = eval64_words<FAM, Q16>(&c.P, &c.lev, rec_words_of<NW>(w), g64);
                        m64u = m64.x;
                        nrechk += nvslot;
                        const unsigned valid = (1u << NS) - 1u;
                        for (unsigned d = ((m32u ^ m64.x) | (m32l ^ m64.y)) & valid; d; d &= d - 1) {
                            int s = __ffs(d) - 1;
                            int du = (int)((m64.x >> s) & 1) - (int)((m32u >> s) & 1);
                            int dl = (int)((m64.y >> s) & 1) - (int)((m32l >> s) & 1);
                            uint32_t *bc = c.cnt + ((size_t)cl * NS + s) * 3;
                            if (du) {
                                atomicAdd(bc, (unsigned)(du * (int)mult));
                                atomicAdd(bc + 2, (unsigned)du);
                            }
                            if (dl) atomicAdd(bc + 1, (unsigned)(dl * (int)mult));
                        }
                    }
#pragma unroll
                    for (int s = 0; s < NS; ++s)
                        bw[s] = (bw[s] & ~unsb) | __ballot_sync(kFull, ((unsb >> lane) & 1) && ((m64u >> s) & 1));
                }
            } else {
                // plain FP64: every record by the definition
                uint2 m64 = make_uint2(0u, 0u);
                if (act) m64 = eval64_words<FAM, Q16>(&c.P, &c.lev, rec_words_of<NW>(w), g64);
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    bool ub = (m64.x >> s) & 1, lb = (m64.y >> s) & 1;
                    const unsigned bb = __ballot_sync(kFull, ub);
                    bw[s] = bb;
                    if constexpr (!WEIGHTED) {
                        if (ub) pu[s >> 2] += 1u << (8 * (s & 3));
                        if (lb) pl[s >> 2] += 1u << (8 * (s & 3));
                    } else {
                        wu[s] += __reduce_add_sync(kFull, ub ? mult : 0u);
                        wl[s] += __reduce_add_sync(kFull, lb ? mult : 0u);
                        wn[s] += __popc(bb);
                    }
                }
            }
            // the tile's ballots, one word per child slot (0 for slots that do not exist)
            if (lane == 0) {
                uint4 *bp = reinterpret_cast<uint4 *>(c.ballot + (size_t)(tile - c.t0) * NS);
#pragma unroll
                for (int q = 0; q < NS / 4; ++q) bp[q] = make_uint4(bw[4 * q], bw[4 * q + 1], bw[4 * q + 2], bw[4 * q + 3]);
            }
        }
        // a warp's byte counters gain at most 32 per tile and group: drain them before
        // they could carry
        if (!WEIGHTED) drain();
        __syncthreads();                                            // buffer b is free again
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

#define GV_DISPATCH(fam, CALL)                                                   \
    switch (fam) {                                                               \
    case FAM_LINE2D: { constexpr int FAMV = FAM_LINE2D; CALL; } break;           \
    case FAM_PLANE3D_SPH: { constexpr int FAMV = FAM_PLANE3D_SPH; CALL; } break; \
    case FAM_POSE3DOF: { constexpr int FAMV = FAM_POSE3DOF; CALL; } break;       \
    case FAM_RAYS3D: { constexpr int FAMV = FAM_RAYS3D; CALL; } break;           \
    default: break;                                                              \
    }

// Persistent grid: as many blocks as fit on the device at once (kernel occupancy
// at the shared memory the records take), at most one per group.

void launch_count(const Chunk &c, cudaStream_t st) {
    const int64_t nt = c.t1 - c.t0;
    if (nt <= 0) return;
    if (c.P.d > 3) {
        launch_count_wide(c, st);
        return;
    }
    const int64_t ng = (nt + kBlockTiles - 1) / kBlockTiles;
    const bool w = c.in.mult != nullptr;
#define GV_COUNT(Q16, PREC)                                                                                   \
    {                                                                                                          \
        constexpr int NW = rec_words(Fam<FAMV>::NFP, Q16);                                                     \
        if (w) launch_persistent((const void *)k_count<FAMV, Q16, PREC, true>, count_smem_bytes<NW>(), ng, c, st);          \
        else launch_persistent((const void *)k_count<FAMV, Q16, PREC, false>, count_smem_bytes<NW>(), ng, c, st);           \
    }
    if (c.precision == 0) {
        GV_DISPATCH(c.P.fam, GV_COUNT(false, 0));
    } else if (c.lev.q16) {
        GV_DISPATCH(c.P.fam, GV_COUNT(true, 1));
    } else {
        GV_DISPATCH(c.P.fam, GV_COUNT(false, 1));
    }
#undef GV_COUNT
}

}  // namespace gv
