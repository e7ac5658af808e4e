// wect_cubical.cu -- stencil kernels for the WECT of full cubical grids (sm_103a).
//
// Lower-star values on a grid (Definition "Lower-Star Filtrations").  Along every grid axis
// the float64 height h = fma(x0,s0, fma(x1,s1, x2*s2)) is monotone in the vertex index, with
// the sign of s_a: each product is exact inside the fma, rounding is monotone, and each fma is
// monotone in its addend.  So the maximum height over a cell (a box of the grid) is attained
// at its "sign corner": the upper end on axes with s_a > 0, the lower end otherwise (ties give
// equal heights, hence equal bins).  Grouping the cells by their sign corner turns the
// per-cell scatter of Algorithm 1 into a per-vertex one:
//     c_o(v) = sum over the 2^n cells whose sign corner under octant o is v of (-1)^dim w(cell),
//     diff_p[bin_p(v)] += c_{o(p)}(v),
// which is exact (integer sums) and touches 2^n times fewer elements.  The c_o(v) come from
// each vertex's 3^n neighbourhood (the cell weight is the max of its vertex weights,
// Figure 1), computed per tile in shared memory and reused by every direction of the tile.
//
// Forward kernel layout: lanes <-> directions (1, 2 or 4 per lane), rows of the grid walked in
// order, per-CTA int32 histograms [T][Dt] in shared memory (a column per direction, so the 32
// lanes of a red.shared hit 32 distinct banks).  Wide weights use two int32 planes (low 16
// bits unsigned, high part signed) so that 65536 updates per entry cannot overflow.  Partial
// histograms are flushed into the int64 output with global atomics (exact, order-free).  When
// T x Dt int32 entries no longer fit shared memory (large T), the GH variant scatters every
// update straight into the int64 difference table in global memory instead (same bins, same
// integer sums; slower, but any T).  Rows longer than the shared row buffers are walked in
// segments (GridDesc::seg), each segment a unit of work with its own row of contributions.
#include <cuda.h>

#include <mutex>

#include "wect_cubical_common.cuh"
#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

constexpr int kFwdThreads = 512;

// Work item the CTA is on (its threshold tile is read back by the rare fix-ups, so that the hot
// row loop keeps no tile registers).
__shared__ int s_fwd_item;

// Threshold tile of the CTA's current item: the shared histogram's row of bin b is
// clamp(b - base, 0, HR - 1), and rows [rlo, rhi) carry the tile's bins (row 0 below and row
// HR - 1 above are discard rows, except at the ends of the range where they are the first and
// last bins).  Untiled: base 0, HR = T, rows [0, T).
__device__ __forceinline__ void fwd_tile(const CubicalFwdArgs &P, int &base, int &HR, int &rlo, int &rhi)
{
    const int T = P.T;
    base = 0;
    HR = T;
    rlo = 0;
    rhi = T;
    if (P.Tt > 0) {
        const int tt = P.items[s_fwd_item].tt;
        const int q0 = tt * P.Tt, q1 = min(T, q0 + P.Tt);
        base = (tt == 0) ? 0 : q0 - 1;
        rlo = q0 - base;
        rhi = q1 - base;
        HR = (q1 < T) ? rhi + 1 : rhi;
    }
}

// The float32 filter could not decide the bin of vertex (i0,i1,i2) in direction p: evaluate the
// float64 height, find its exact bin and move the contribution if the tentative bin was wrong.
// nr is the row filter's (real) integer offset; the histogram rows are those of the item's
// threshold tile (fwd_tile).
template <int N, int NSPLIT, bool GH>
__device__ __noinline__ void cubical_fixup(const CubicalFwdArgs &P, const GridDesc &g, int p, int i0, int i1, int i2,
                                           int thi, int nr, int col, uint32_t histAddr, int Dt, uint32_t HOFF,
                                           int cv, int hv, unsigned long long *oc)
{
    const int T = P.T;
    const int bt = clamp_bin(thi, nr, T);
    const double h = height3<N>(gcoord(g, 0, i0), gcoord(g, 1, i1), gcoord(g, 2, i2),
                                P.dirs + (int64_t)p * N);
    const int be = exact_bin_from(h, P.beta, T, bt);
    if (be == bt) return;
    if (GH) {            // global difference table of the complex (oc), row p
        if (p < P.d) {
            unsigned long long *row = oc + (int64_t)p * T;
            atomicAdd(row + bt, (unsigned long long)(-(long long)cv));
            atomicAdd(row + be, (unsigned long long)(long long)cv);
        }
        return;
    }
    int base, HR, rlo, rhi;
    fwd_tile(P, base, HR, rlo, rhi);
    const int rt = min(max(bt - base, 0), HR - 1), re = min(max(be - base, 0), HR - 1);
    if (rt == re) return;           // both in one discard row of the tile
    const uint32_t at = histAddr + ((uint32_t)rt * (uint32_t)Dt + (uint32_t)col) * 4u;
    const uint32_t ae = histAddr + ((uint32_t)re * (uint32_t)Dt + (uint32_t)col) * 4u;
    if (NSPLIT == 1) {
        red_shared_add(at, -cv);
        red_shared_add(ae, cv);
    } else {
        red_shared_add_u32(at, (uint32_t)(-cv));
        red_shared_add_u32(ae, (uint32_t)cv);
        red_shared_add(at + HOFF, -hv);
        red_shared_add(ae + HOFF, hv);
    }
}

// The undecided (vertex, direction) pairs of one block of U vertices, spread over the warp: every
// lane lists its pairs (bit u * DPL + j of pend) in a per-warp queue of 32 entries, and each lane
// then fixes one queued pair, whoever found it.  Lanes whose direction meets many exact ties
// (regular grids seen along axis or diagonal directions) no longer serialise the warp.
template <int N, int NSPLIT, int DPL, bool GH>
__device__ __noinline__ void cubical_fixup_block(const CubicalFwdArgs &P, const GridDesc &g, const int32_t *crow,
                                                 int CP, int i0, int x0, int i1, int i2, uint32_t pend, float k0,
                                                 const DirFilter *dirf, int colbase, int pbase, uint32_t histAddr,
                                                 int Dt, uint32_t HOFF, uint32_t *wq, unsigned long long *oc)
{
    constexpr int NOCT = 1 << N;
    const int lane = threadIdx.x & 31;
    const int cnt = __popc(pend);
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int first = incl - cnt;
    for (int base = 0; base < total; base += 32) {
        uint32_t rest = pend;
        for (int q = first; rest; ++q) {
            const int bit = __ffs(rest) - 1;
            rest &= rest - 1;
            if (q >= base && q < base + 32) wq[q - base] = ((uint32_t)lane << 8) | (uint32_t)bit;
        }
        __syncwarp();
        if (base + lane < total) {
            const uint32_t e = wq[lane];
            const int src = (int)(e >> 8), bit = (int)(e & 255u), u = bit / DPL, j = bit % DPL;
            const int col = colbase + j * 32 + src;
            const DirFilter f = dirf[col];
            const RowFilter rf = make_row_filter<N>(f, i1, i2, g.L);
            int tlo, thi;
            filter_ceil(k0 + 2.0f * (float)u, f.S0, rf.Glo, rf.Ghi, tlo, thi);
            const int cv = crow[f.oct * CP + i0 + u];
            const int hv = (NSPLIT == 2) ? crow[NOCT * CP + f.oct * CP + i0 + u] : 0;
            const int p = (pbase + col < P.d) ? P.perm[pbase + col] : P.d;
            cubical_fixup<N, NSPLIT, GH>(P, g, p, x0 + i0 + u, i1, i2, thi, rf.nr, col, histAddr, Dt, HOFF, cv, hv, oc);
        }
        __syncwarp();
    }
}

// One unit of a grid row (the whole row, or L0 vertices of it from x0 on when long rows are walked
// in segments; Lfull is the row's length) for the DPL directions of each lane.  CLAMP selects the
// variant whose bins may leave [0, T-1] (heights outside the threshold range); the other variant
// has been proven in range for the whole row and skips the clamp.  rf[j].nr arrives shifted by the
// item's threshold-tile base, so that thi + nr - kMagicBits is the histogram row, clamped to
// [0, HR - 1] (untiled: base 0, HR = T; the non-GEN instances are never tiled and take T).
template <int N, int NSPLIT, int DPL, bool CLAMP, bool GH, bool GEN>
__device__ __forceinline__ void fwd_row(const CubicalFwdArgs &P, const GridDesc &g, const int32_t *crow, int CP, int L0,
                                        int x0, int Lfull, int i1, int i2, const float (&S0)[DPL], const RowFilter (&rf)[DPL],
                                        const int (&oct)[DPL], const int (&col)[DPL], int pbase, uint32_t histAddr,
                                        int Dt, uint32_t HOFF, const DirFilter *dirf, int colbase, uint32_t *wq,
                                        unsigned long long *const (&orow)[DPL], unsigned long long *oc, int HR)
{
    constexpr int NOCT = 1 << N;
    constexpr int U = (NSPLIT == 1 && DPL <= 2) ? 8 : 4;
    const int T = P.T;
    const uint32_t D4 = (uint32_t)Dt * 4u;
    const uint32_t HIP = (uint32_t)(NOCT * CP) * 4u;        // byte offset of the high planes
    uint32_t cb[DPL], hb[DPL];
#pragma unroll
    for (int j = 0; j < DPL; ++j) {
        cb[j] = smem_addr(crow + oct[j] * CP);
        hb[j] = histAddr + (uint32_t)col[j] * 4u + (CLAMP ? 0u : (uint32_t)(rf[j].nr - kMagicBits) * D4);
    }
    const int LU = L0 - L0 % U;
    float k0 = (float)(2 * x0 + 1 - Lfull);            // k = 2 x - (Lfull - 1) of the unit's first vertex
    // packed copies of the per-row constants for the f32x2 path
    constexpr int NP = (DPL % 2 == 0) ? DPL / 2 : 1;
    F2 S0p[NP], Glop[NP], Ghip[NP];
    const F2 M2 = f2_pack(kMagic, kMagic);
    if (DPL % 2 == 0) {
#pragma unroll
        for (int j = 0; j + 1 < DPL; j += 2) {
            S0p[j / 2] = f2_pack(S0[j], S0[j + 1]);
            Glop[j / 2] = f2_pack(rf[j].Glo, rf[j + 1].Glo);
            Ghip[j / 2] = f2_pack(rf[j].Ghi, rf[j + 1].Ghi);
        }
    }
    F2 k02 = f2_pack(k0, k0);
    const F2 two2 = f2_pack(2.0f, 2.0f);
    // four blocks of U vertices per trip: the scheduler overlaps one block's shared-memory
    // scatter with the next block's filter arithmetic
#pragma unroll 4
    for (int i0 = 0; i0 < LU; i0 += U) {
        int cv[DPL][U], hv[DPL][U];
#pragma unroll
        for (int j = 0; j < DPL; ++j)
#pragma unroll
            for (int q = 0; q < U / 4; ++q) {
                const int4 t = lds128(cb[j] + (uint32_t)(i0 + 4 * q) * 4u);
                cv[j][4 * q] = t.x; cv[j][4 * q + 1] = t.y; cv[j][4 * q + 2] = t.z; cv[j][4 * q + 3] = t.w;
                if (NSPLIT == 2) {
                    const int4 h = lds128(cb[j] + HIP + (uint32_t)(i0 + 4 * q) * 4u);
                    hv[j][4 * q] = h.x; hv[j][4 * q + 1] = h.y; hv[j][4 * q + 2] = h.z; hv[j][4 * q + 3] = h.w;
                } else {
                    hv[j][4 * q] = hv[j][4 * q + 1] = hv[j][4 * q + 2] = hv[j][4 * q + 3] = 0;
                }
            }
        int bad = 0;
        F2 kk2 = k02;                           // k0 of vertex i0 + u, both halves (exact small integers)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int tlo[DPL], thi[DPL];
            if (DPL % 2 == 0) {
                // packed pairs of directions: one f32x2 instruction per step for two lanes' slots
#pragma unroll
                for (int j = 0; j < DPL; j += 2)
                    filter_ceil2(kk2, S0p[j / 2], Glop[j / 2], Ghip[j / 2], M2, tlo[j], thi[j], tlo[j + 1], thi[j + 1]);
                kk2 = f2_add_rn(kk2, two2);
            } else {
#pragma unroll
                for (int j = 0; j < DPL; ++j) filter_ceil(k0 + 2.0f * (float)u, S0[j], rf[j].Glo, rf[j].Ghi, tlo[j], thi[j]);
            }
#pragma unroll
            for (int j = 0; j < DPL; ++j) {
                bad |= tlo[j] ^ thi[j];
                if constexpr (GH) {
                    // int64 difference row of this lane's direction in global memory (null for
                    // an idle column)
                    if (orow[j]) atomicAdd(orow[j] + clamp_bin(thi[j], rf[j].nr, T), (unsigned long long)(long long)cv[j][u]);
                    continue;
                }
                uint32_t addr;
                if (!CLAMP) {
                    addr = (uint32_t)thi[j] * D4 + hb[j];
                } else {
                    const int b = clamp_bin(thi[j], rf[j].nr, GEN ? HR : T);
                    addr = hb[j] + (uint32_t)b * D4;
                }
                if (NSPLIT == 1) {
                    red_shared_add(addr, cv[j][u]);
                } else {
                    red_shared_add_u32(addr, (uint32_t)cv[j][u]);
                    red_shared_add(addr + HOFF, hv[j][u]);
                }
            }
        }
        if (__any_sync(0xffffffffu, bad != 0)) {
            uint32_t pend = 0;
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int j = 0; j < DPL; ++j) {
                    int tlo, thi;
                    filter_ceil(k0 + 2.0f * (float)u, S0[j], rf[j].Glo, rf[j].Ghi, tlo, thi);
                    if (tlo != thi) pend |= 1u << (u * DPL + j);
                }
            cubical_fixup_block<N, NSPLIT, DPL, GH>(P, g, crow, CP, i0, x0, i1, i2, pend, k0, dirf, colbase, pbase,
                                                    histAddr, Dt, HOFF, wq, oc);
        }
        k0 += 2.0f * (float)U;
        k02 = kk2;
    }
    // ragged tail of the row (fewer than U vertices), always clamped
    for (int i0 = LU; i0 < L0; ++i0) {
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            const int cvs = crow[oct[j] * CP + i0];
            const int hvs = (NSPLIT == 2) ? crow[NOCT * CP + oct[j] * CP + i0] : 0;
            int tlo, thi;
            filter_ceil(k0, S0[j], rf[j].Glo, rf[j].Ghi, tlo, thi);
            if constexpr (GH) {
                if (orow[j]) atomicAdd(orow[j] + clamp_bin(thi, rf[j].nr, T), (unsigned long long)(long long)cvs);
            } else {
                const int b = clamp_bin(thi, rf[j].nr, GEN ? HR : T);
                const uint32_t addr = histAddr + ((uint32_t)b * (uint32_t)Dt + (uint32_t)col[j]) * 4u;
                if (NSPLIT == 1) {
                    red_shared_add(addr, cvs);
                } else {
                    red_shared_add_u32(addr, (uint32_t)cvs);
                    red_shared_add(addr + HOFF, hvs);
                }
            }
            if (tlo != thi) {
                const int p = (pbase + col[j] < P.d) ? P.perm[pbase + col[j]] : P.d;
                int tb = 0, thr, t1, t2;                      // the real row offset: rf[j].nr + base
                if (GEN) fwd_tile(P, tb, thr, t1, t2);
                cubical_fixup<N, NSPLIT, GH>(P, g, p, x0 + i0, i1, i2, thi, rf[j].nr + tb, col[j], histAddr, Dt, HOFF,
                                             cvs, hvs, oc);
            }
        }
        k0 += 2.0f;
    }
}

// ------------------------------------------------------------------ forward

// GEN instances walk long rows in segments and threshold tiles; the others (whole rows, all T
// rows in the histogram) keep the row loop free of both.
template <int N, int NSPLIT, int DPL, bool GH, bool GEN>
__global__ void __launch_bounds__(kFwdThreads, 1) cubical_fwd_kernel(const CubicalFwdArgs P)
{
    constexpr int NOCT = 1 << N;
    constexpr int NROWS = (N >= 3) ? 9 : (N == 2 ? 3 : 1);      // neighbouring rows of a box
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) unsigned long long s_mbar[16][2];    // TMA completion, per row group
    const int T = P.T, Dt = P.Dt, CP = P.CP;
    // histogram rows: T, or a threshold tile of Tt bins and a discard row on each side
    const int HRmax = (GEN && P.Tt > 0) ? P.Tt + 2 : T;
    const int histWords = GH ? 0 : HRmax * Dt;  // GH: no shared histogram
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int WC = Dt / (32 * DPL);         // warps across the direction tile = warps of a row group
    const int RG = nwarps / WC;             // row groups, each walking its own rows
    const int wcol = wid % WC, rgroup = wid / WC;
    const int gtid = wcol * 32 + lane, gthreads = WC * 32;
    int32_t *hist = reinterpret_cast<int32_t *>(smem);                          // NSPLIT planes [HRmax][Dt]
    DirFilter *dirf = reinterpret_cast<DirFilter *>(hist + NSPLIT * histWords);  // [Dt]
    const int rowbuf = NSPLIT * NOCT * CP;                                       // words of one row buffer
    const int nbuf = (WC == 1) ? 1 : 2;     // a one-warp group needs no second buffer (warp-synchronous)
    int32_t *cgrp = reinterpret_cast<int32_t *>(dirf + Dt) + rgroup * nbuf * rowbuf;
    uint32_t *wq = reinterpret_cast<uint32_t *>(reinterpret_cast<int32_t *>(dirf + Dt) + RG * nbuf * rowbuf) + wid * 32;
    const uint32_t histAddr = smem_addr(hist);
    const uint32_t HOFF = (uint32_t)histWords * 4u;
    // TMA staging of the neighbouring rows: two boxes per row group, each NROWS rows of up to
    // L0s int32 (128-byte aligned), filled by the group's first thread one row ahead
    const uint32_t rawEnd = smem_addr(wq - wid * 32 + nwarps * 32);       // end of the fix-up queues
    const uint32_t stageAddr = (rawEnd + 127u) & ~127u;                      // 128-byte aligned in shared space
    int32_t *stage = reinterpret_cast<int32_t *>(smem + (stageAddr - smem_addr(smem))) +
                     (size_t)rgroup * 2 * NROWS * P.L0s;
    const uint32_t mbar0 = smem_addr(&s_mbar[rgroup][0]), mbar1 = smem_addr(&s_mbar[rgroup][1]);
    if (P.L0s > 0 && tid == 0) {
        for (int gi = 0; gi < RG; ++gi) {
            mbar_init(smem_addr(&s_mbar[gi][0]), 1);
            mbar_init(smem_addr(&s_mbar[gi][1]), 1);
        }
        mbar_fence_init();
    }
    unsigned krow = 0;                      // rows this group has staged (buffer krow & 1, phase krow >> 1)
    // the flush's transpose tiles: the shared memory past the histogram (direction filters, row
    // buffers, fix-up queues, staging boxes), idle between items
    const int flushTiles = (int)((dynamic_smem_bytes() - (uint32_t)(NSPLIT * histWords) * 4u) / (NSPLIT * 32u * 33u * 4u));

    for (int i = tid; i < NSPLIT * histWords; i += blockDim.x) hist[i] = 0;
    // launched as a programmatic dependent: the set-up above (shared memory only) overlapped the
    // preparation kernel; global memory is touched only from here on (its results and the
    // weights), and the scan may launch (items that store the final table themselves make this
    // the call's last kernel: no early signal)
    pdl_wait();
    if (!P.direct) pdl_trigger();
    // the range comes from the preparation kernel: read only after the wait
    const double lo = P.range[0], hi = P.range[1], step = P.range[2];

    for (;;) {
        __syncthreads();
        if (tid == 0) s_fwd_item = atomicAdd(P.counter, 1);
        __syncthreads();
        const int it = s_fwd_item;
        if (it >= P.n_items) break;
        const WorkItem W = P.items[it];
        const GridDesc g = P.grids[W.cx];
        const int L0 = g.L[0], L1 = g.L[1];
        const int pbase = W.dtile * Dt;
        // threshold tile of the item: the histogram row of bin b is clamp(b - base, 0, HR - 1), and
        // rows [rlo, rhi) carry the tile's bins (row 0 below and row HR - 1 above are discard
        // rows except at the ends of the range, where they are the first and last bins)
        int base = 0, HR = T, rlo = 0, rhi = T;
        if (GEN) fwd_tile(P, base, HR, rlo, rhi);

        // ---- float32 filter constants of the tile's directions, one per column
        for (int c = tid; c < Dt; c += blockDim.x) {
            const int p = (pbase + c < P.d) ? P.perm[pbase + c] : P.d;
            double s[3] = {0.0, 0.0, 0.0};
            DirFilter f;
            if (p < P.d) {
#pragma unroll
                for (int a = 0; a < N; ++a) s[a] = P.dirs[(int64_t)p * N + a];
                f = make_dir_filter<N>(s, g.L, lo, hi, step, T);
            } else {        // idle column: parked on bin 1, never flushed
                f.S0 = 0.f;
                f.B1 = f.B2 = DS{0.f, 0.f};
                f.C = DS{0.5f, 0.f};
                f.eta = 0x1p-8f;
                f.oct = 0;
            }
            dirf[c] = f;
        }
        __syncthreads();
        int col[DPL];
#pragma unroll
        for (int j = 0; j < DPL; ++j) col[j] = wcol * 32 * DPL + j * 32 + lane;
        // GH: the int64 difference rows of the lane's directions in the complex's output block
        unsigned long long *const oc = P.out + (int64_t)W.cx * P.d * T;
        unsigned long long *orow[DPL];
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            const int p = (pbase + col[j] < P.d) ? P.perm[pbase + col[j]] : P.d;
            orow[j] = (GH && p < P.d) ? oc + (int64_t)p * T : nullptr;
        }

        // ---- each row group walks rows r0 + rgroup, r0 + rgroup + RG, ... with a double-buffered
        // row of octant contributions (one group barrier per row, no block-wide barrier)
        // (a grid walked in segments is never staged: its box would not fit the stage)
        const bool tma = (N >= 2) && P.L0s > 0 && g.tmap != nullptr && (!GEN || g.nseg == 1);
        const uint32_t boxBytes = (uint32_t)(NROWS * L0) * 4u;
        // box of the rows around row r' (rows outside the grid come back as zeros)
        auto stage_row = [&](int rr, unsigned kb) {
            const uint32_t mb = (kb & 1u) ? mbar1 : mbar0;
            mbar_arrive_expect_tx(mb, boxBytes);
            tma_load_3d(smem_addr(stage + (size_t)(kb & 1u) * NROWS * P.L0s), g.tmap, 0, rr % L1 - 1,
                        N >= 3 ? rr / L1 - 1 : 0, mb);
        };
        if (tma && gtid == 0 && W.r0 + rgroup < W.r1) stage_row(W.r0 + rgroup, krow);
        int parity = 0;
        for (int r = W.r0 + rgroup; r < W.r1; r += RG, parity ^= 1) {
            int32_t *crow = cgrp + (nbuf == 2 ? parity : 0) * rowbuf;
            if (nbuf == 1) __syncwarp();        // the previous row's reads are done before the rewrite
            // unit r: grid row rr, or (GEN instances only) its segment of Lu vertices from x0 when
            // the grid's rows are walked in segments (such grids are not TMA-staged)
            const bool segd = GEN && g.nseg > 1;
            const int rr = segd ? r / g.nseg : r;
            const int x0 = segd ? (r - rr * g.nseg) * g.seg : 0;
            const int Lu = segd ? min(g.seg, L0 - x0) : L0;
            const int i1 = rr % L1, i2 = rr / L1;
            const unsigned k = krow;
            const int32_t *box = stage + (size_t)(k & 1u) * NROWS * P.L0s;
            if (tma) {
                ++krow;
                // the next row's box into the other buffer (its last reader finished before the
                // previous row's group barrier), then wait for this row's
                if (gtid == 0 && r + RG < W.r1) stage_row(r + RG, k + 1);
                if (!mbar_wait_bounded((k & 1u) ? mbar1 : mbar0, (k >> 1) & 1u)) atomicOr(g.status, kStatusTimeout);
            }
            for (int i0 = gtid; i0 < Lu; i0 += gthreads) {
                int32_t c[NOCT];
                if (tma)
                    octant_contribs_box<N>(box, g, i0, i1, i2, c);
                else
                    octant_contribs<N>(g, x0 + i0, i1, i2, c);
#pragma unroll
                for (int o = 0; o < NOCT; ++o) {
                    const int32_t v = c[o];
                    if (NSPLIT == 1) {
                        crow[o * CP + i0] = v;
                    } else {
                        crow[o * CP + i0] = v & 0xFFFF;
                        crow[NOCT * CP + o * CP + i0] = v >> 16;
                    }
                }
            }
            group_sync(rgroup, WC);

            RowFilter rf[DPL];
            float S0[DPL];
            int oct[DPL];
            bool clampRow = false;
#pragma unroll
            for (int j = 0; j < DPL; ++j) {
                const DirFilter f = dirf[col[j]];
                S0[j] = f.S0;
                oct[j] = f.oct;
                rf[j] = make_row_filter<N>(f, i1, i2, g.L);
                if (GEN) rf[j].nr -= base;          // histogram rows of the item's threshold tile
                // all rows of the row provably inside [0, HR-1]?  (NaN/inf compare false)
                const float A = __fmul_ru((float)(L0 - 1), fabsf(f.S0));
                const float lowf = __fadd_rd(__fsub_rd(rf[j].Glo, A), (float)(rf[j].nr - 1));
                const float highf = __fadd_ru(__fadd_ru(rf[j].Ghi, A), (float)(rf[j].nr + 1));
                clampRow |= !(lowf >= 0.0f) || !(highf <= (float)(HR - 1));
            }
            if constexpr (GH) {
                fwd_row<N, NSPLIT, DPL, true, true, GEN>(P, g, crow, CP, Lu, x0, L0, i1, i2, S0, rf, oct, col, pbase, histAddr, Dt,
                                                    HOFF, dirf, wcol * 32 * DPL, wq, orow, oc, HR);
            } else {
                if (__any_sync(0xffffffffu, clampRow))
                    fwd_row<N, NSPLIT, DPL, true, false, GEN>(P, g, crow, CP, Lu, x0, L0, i1, i2, S0, rf, oct, col, pbase, histAddr, Dt,
                                                         HOFF, dirf, wcol * 32 * DPL, wq, orow, oc, HR);
                else
                    fwd_row<N, NSPLIT, DPL, false, false, GEN>(P, g, crow, CP, Lu, x0, L0, i1, i2, S0, rf, oct, col, pbase, histAddr,
                                                          Dt, HOFF, dirf, wcol * 32 * DPL, wq, orow, oc, HR);
            }
        }
        __syncthreads();
        if constexpr (!GH) {
            if (P.direct)
                cubical_flush_direct<NSPLIT>(hist, T, Dt, W.dtile, P.d, P.perm, oc);
            else
                cubical_flush_coalesced<NSPLIT, GEN>(hist, HRmax, rlo, rhi, base, T, Dt, W.dtile, P.d, P.perm, oc,
                                                     hist + NSPLIT * histWords, flushTiles);
        }
    }
}

// ------------------------------------------------------------------ default range on a grid

// M = max over directions and grid corners of |h|: h is monotone along every axis, so its
// extremes over the grid are at corners.
template <int N>
__global__ void grid_max_abs_kernel(const GridDesc *grids, const double *dirs, int d, unsigned long long *Mbits)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d * (1 << N)) return;
    const int p = t >> N, corner = t & ((1 << N) - 1);
    const GridDesc g = grids[0];
    const double x0 = grid_coord((corner & 1) ? g.L[0] - 1 : 0, g.L[0]);
    const double x1 = grid_coord((corner & 2) ? g.L[1] - 1 : 0, g.L[1]);
    const double x2 = grid_coord((corner & 4) ? g.L[2] - 1 : 0, g.L[2]);
    const double h = fabs(height3<N>(x0, x1, x2, dirs + (int64_t)p * N));
    atomicMax(Mbits, (unsigned long long)__double_as_longlong(h));
}

// ------------------------------------------------------------------ launchers

// The dynamic shared-memory opt-in is set once per kernel instance and size (never inside a
// stream capture once a size has been seen).
template <int N, int NSPLIT, int DPL, bool GH, bool GEN>
static cudaError_t launch_fwd_s(const CubicalFwdArgs &a, int grid, size_t smem, cudaStream_t st, bool launch)
{
    static size_t done = 0;
    if (smem > done) {
        cudaError_t e = cudaFuncSetAttribute(cubical_fwd_kernel<N, NSPLIT, DPL, GH, GEN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        done = smem;
    }
    if (!launch) return cudaSuccess;
    const int threads = (a.threads > 0 && a.threads <= kFwdThreads) ? a.threads : kFwdThreads;
    return launch_kernel(cubical_fwd_kernel<N, NSPLIT, DPL, GH, GEN>, dim3(grid), dim3(threads), smem, st, a.pdl != 0, a);
}

// The general instance (segments of long rows, threshold tiles) only when the launch needs it;
// preparing sets up both.
template <int N, int NSPLIT, int DPL, bool GH>
static cudaError_t launch_fwd_t(const CubicalFwdArgs &a, int grid, size_t smem, cudaStream_t st, bool launch)
{
    if (!launch) {
        cudaError_t e = launch_fwd_s<N, NSPLIT, DPL, GH, false>(a, grid, smem, st, false);
        return e != cudaSuccess ? e : launch_fwd_s<N, NSPLIT, DPL, GH, true>(a, grid, smem, st, false);
    }
    return (a.segmented || a.Tt > 0) ? launch_fwd_s<N, NSPLIT, DPL, GH, true>(a, grid, smem, st, true)
                                     : launch_fwd_s<N, NSPLIT, DPL, GH, false>(a, grid, smem, st, true);
}

template <int N, int NSPLIT>
static cudaError_t launch_fwd_d(const CubicalFwdArgs &a, int dpl, int grid, size_t smem, cudaStream_t st, bool launch)
{
    switch (dpl) {
    case 1: return launch_fwd_t<N, NSPLIT, 1, false>(a, grid, smem, st, launch);
    case 2: return launch_fwd_t<N, NSPLIT, 2, false>(a, grid, smem, st, launch);
    default: return launch_fwd_t<N, NSPLIT, 4, false>(a, grid, smem, st, launch);
    }
}

// Global-histogram instances: one int32 row plane (the contributions are added as int64), one or
// two directions per lane.
template <int N>
static cudaError_t launch_fwd_gh(const CubicalFwdArgs &a, int dpl, int grid, size_t smem, cudaStream_t st, bool launch)
{
    return dpl == 1 ? launch_fwd_t<N, 1, 1, true>(a, grid, smem, st, launch)
                    : launch_fwd_t<N, 1, 2, true>(a, grid, smem, st, launch);
}

static cudaError_t cubical_fwd_dispatch(int n, int nsplit, int dpl, bool gh, const CubicalFwdArgs &a, int grid,
                                        size_t smem, cudaStream_t st, bool launch)
{
    if (gh) {
        if (dpl != 1 && dpl != 2) return cudaErrorInvalidValue;
        if (n == 1) return launch_fwd_gh<1>(a, dpl, grid, smem, st, launch);
        if (n == 2) return launch_fwd_gh<2>(a, dpl, grid, smem, st, launch);
        return launch_fwd_gh<3>(a, dpl, grid, smem, st, launch);
    }
    if (n == 1) return nsplit == 1 ? launch_fwd_d<1, 1>(a, dpl, grid, smem, st, launch) : launch_fwd_d<1, 2>(a, dpl, grid, smem, st, launch);
    if (n == 2) return nsplit == 1 ? launch_fwd_d<2, 1>(a, dpl, grid, smem, st, launch) : launch_fwd_d<2, 2>(a, dpl, grid, smem, st, launch);
    return nsplit == 1 ? launch_fwd_d<3, 1>(a, dpl, grid, smem, st, launch) : launch_fwd_d<3, 2>(a, dpl, grid, smem, st, launch);
}

cudaError_t launch_cubical_fwd(int n, int nsplit, int dpl, bool gh, const CubicalFwdArgs &a, int grid, size_t smem,
                               cudaStream_t st)
{
    return cubical_fwd_dispatch(n, nsplit, dpl, gh, a, grid, smem, st, true);
}

cudaError_t prepare_cubical_fwd(int n, int nsplit, int dpl, bool gh, size_t smem)
{
    CubicalFwdArgs a{};
    return cubical_fwd_dispatch(n, nsplit, dpl, gh, a, 1, smem, nullptr, false);
}

int cubical_fwd_pitch(int maxL0)
{
    const int L0p = (maxL0 + 3) & ~3;
    return ((L0p + 31) & ~31) + 4;        // words; = 4 mod 32: octant planes on distinct bank groups
}

// gh: no shared histogram (the global-histogram variant, one row plane).
int cubical_fwd_stage_len(int n, int maxL0)
{
    return (n >= 2 && maxL0 <= 256) ? (maxL0 + 31) & ~31 : 0;
}

size_t cubical_fwd_smem(int n, int nsplit, int dpl, int T, int Dt, int maxL0, bool gh, int threads, int L0s)
{
    if (threads <= 0 || threads > kFwdThreads) threads = kFwdThreads;
    if (gh) {
        nsplit = 1;
        T = 0;
    }
    const int noct = 1 << n;
    const int WC = Dt / (32 * dpl);
    const int RG = (threads / 32) / WC;
    const size_t rowbuf = (size_t)nsplit * noct * cubical_fwd_pitch(maxL0);
    const int nbuf = (WC == 1) ? 1 : 2;
    // + one 32-entry fix-up queue per warp
    size_t sz = (size_t)nsplit * T * Dt * 4u + (size_t)Dt * sizeof(DirFilter) + (size_t)RG * nbuf * rowbuf * 4u +
                (size_t)(threads / 32) * 32u * 4u;
    if (L0s > 0) {            // TMA staging: 128-byte aligned, two boxes of 3^(n-1) rows per row group
        const int nrows = n >= 3 ? 9 : (n == 2 ? 3 : 1);
        sz += 128u + (size_t)RG * 2u * nrows * L0s * 4u;      // + room to align the staging area
    }
    return sz;
}

int cubical_fwd_threads() { return kFwdThreads; }

// ------------------------------------------------------------------ TMA tensor maps

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link against libcuda).
static EncodeTiledFn encode_tiled()
{
    static std::mutex mu;
    static bool tried = false;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool encode_grid_tmap(int n, const int *dims, const int32_t *w, void *map)
{
    // rows of 16-byte multiples (x stays aligned at 0), a box of at most 256 along every axis,
    // at least three rows per axis the box spans
    if (n < 2 || dims[0] % 4 != 0 || dims[0] > 256 || dims[1] < 3 || (n >= 3 && dims[2] < 3)) return false;
    if (reinterpret_cast<uintptr_t>(w) & 15u) return false;
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t gdim[3] = {(cuuint64_t)dims[0], (cuuint64_t)dims[1], (cuuint64_t)(n >= 3 ? dims[2] : 1)};
    const cuuint64_t gstride[2] = {(cuuint64_t)dims[0] * 4u, (cuuint64_t)dims[0] * (cuuint64_t)dims[1] * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)dims[0], 3u, n >= 3 ? 3u : 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(reinterpret_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_INT32, 3,
                          const_cast<int32_t *>(w), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t launch_grid_max_abs(int n, const GridDesc *grids, const double *dirs, int d, unsigned long long *Mbits,
                                cudaStream_t st)
{
    const int tot = d * (1 << n);
    const int blocks = (tot + 255) / 256;
    if (n == 1) grid_max_abs_kernel<1><<<blocks, 256, 0, st>>>(grids, dirs, d, Mbits);
    else if (n == 2) grid_max_abs_kernel<2><<<blocks, 256, 0, st>>>(grids, dirs, d, Mbits);
    else grid_max_abs_kernel<3><<<blocks, 256, 0, st>>>(grids, dirs, d, Mbits);
    return cudaGetLastError();
}

}  // namespace wect
