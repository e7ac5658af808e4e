// wect_cubical_run.cu -- the run-based stencil kernel for the WECT of full cubical grids (sm_103a).
//
// The stencil kernel (wect_cubical.cu) adds each vertex's octant contribution c_o(v) into the
// histogram entry of its bin, one update per vertex and direction.  Along a grid row the float64
// height is monotone in the vertex index (with the sign of s_0), so the bins of a row form a
// monotone sequence of runs, and the updates of one run add up to a difference of prefix sums:
//     sum over v in the row of c_o(v) e_{bin(v)} = sum over runs [a, b) of (P_o[b] - P_o[a]) e_{bin},
// with P_o the prefix sums of c_o along the row (identical integers, added in another order).
// A row of L0 vertices spans about 2 |s_0| / step bins, so for long rows and moderate T the runs
// are far fewer than the vertices.  Each lane walks the bin boundaries of its direction instead of
// the vertices:
//   - the bins of the two ends of the row are exact (float32 filter, float64 where undecided);
//   - the first vertex whose bin reaches b is read off the threshold in vertex coordinates,
//         x(b) = ((b - 1) - G) / (2 S) + (L0 - 1) / 2        (walk direction: S = |S_0| > 0),
//     evaluated as a rigorous enclosure [x_lo, x_hi] from the filter's enclosure of G (directed
//     roundings, upper end strictly above).  When x_lo and x_hi have the same floor j, vertices
//     <= j certainly lie below the threshold and vertices > j certainly above, so the boundary is
//     j + 1.  Otherwise (a vertex within the filter's error of the threshold) the boundary is
//     found by bisection on exact float64 bins.
// Directions with s_0 < 0 walk the row from its far end.  Lanes map to directions sorted by
// |s_0|, so the lanes of a warp walk similar numbers of boundaries.
//
// Measured against the per-vertex kernel on the 128^3 u8 volume, 256 Fibonacci directions: the
// per-row set-up (octant contributions, prefix sums, end bins, enclosure constants) is a chain
// of dependent steps between row-group barriers and costs ~140 us in all, and each boundary
// costs more than a vertex update of the per-vertex kernel (the walks diverge across lanes and
// the warps of a row group wait for the longest walk).  So this kernel wins only with a few
// boundaries per long row (T = 8: 178 us against 267 us) and loses at T = 128 (827 us against
// 203 us); the host takes it only in that regime.
#include "wect_cubical_common.cuh"
#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

constexpr int kRunThreads = 512;

// Per column of the direction tile: reciprocal bounds of 2 |S_0| (A = 1 / (2 |S_0|)).
struct RunDir {
    float Alo, Aup;
};

// Exact bin of vertex (i0, i1, i2) in direction p (the float64 height against the thresholds).
template <int N>
__device__ __noinline__ int run_exact_bin(const CubicalFwdArgs &P, const GridDesc &g, int p, int i0, int i1, int i2,
                                          int cand)
{
    const double h = height3<N>(gcoord(g, 0, i0), gcoord(g, 1, i1), gcoord(g, 2, i2), P.dirs + (int64_t)p * N);
    return exact_bin_from(h, P.beta, P.T, cand);
}

// Exact bin of the vertex at walk position w (mirror: the row is walked from its far end), from
// the filter when it decides, else from the float64 height.
template <int N>
__device__ __forceinline__ int run_end_bin(const CubicalFwdArgs &P, const GridDesc &g, int p, int w, bool mirror,
                                           int L0, int i1, int i2, float S0, const RowFilter &rf)
{
    const int i0 = mirror ? L0 - 1 - w : w;
    int tlo, thi;
    filter_ceil((float)(2 * i0 - (L0 - 1)), S0, rf.Glo, rf.Ghi, tlo, thi);
    const int b = clamp_bin(thi, rf.nr, P.T);
    return (tlo == thi) ? b : run_exact_bin<N>(P, g, p, i0, i1, i2, b);
}

template <int N>
__global__ void __launch_bounds__(kRunThreads, 1) cubical_run_kernel(const CubicalFwdArgs P)
{
    constexpr int NOCT = 1 << N;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    const int T = P.T, Dt = P.Dt, CP = P.CP;
    const int histWords = T * Dt;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int WC = Dt / 32;                 // warps across the direction tile (one direction per lane)
    const int RG = nwarps / WC;             // row groups
    const int wcol = wid % WC, rgroup = wid / WC;
    const int gtid = wcol * 32 + lane, gthreads = WC * 32;
    int32_t *hist = reinterpret_cast<int32_t *>(smem);                       // [T][Dt]
    DirFilter *dirf = reinterpret_cast<DirFilter *>(hist + histWords);       // [Dt]
    RunDir *rdir = reinterpret_cast<RunDir *>(dirf + Dt);                    // [Dt]
    const int rowbuf = NOCT * CP;
    // per row group two row buffers: octant contributions, then in place their running sums
    int32_t *cgrp = reinterpret_cast<int32_t *>(rdir + Dt) + rgroup * 2 * rowbuf;
    const uint32_t histAddr = smem_addr(hist);
    const uint32_t D4 = (uint32_t)Dt * 4u;
    const double lo = P.range[0], hi = P.range[1], step = P.range[2];

    // the flush's transpose tiles: the shared memory past the histogram, idle between items
    const int flushTiles = (int)((dynamic_smem_bytes() - (uint32_t)histWords * 4u) / (32u * 33u * 4u));

    for (int i = tid; i < histWords; i += blockDim.x) hist[i] = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(P.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= P.n_items) break;
        const WorkItem W = P.items[it];
        const GridDesc g = P.grids[W.cx];
        const int L0 = g.L[0], L1 = g.L[1];
        const int pbase = W.dtile * Dt;

        // ---- filter constants and reciprocal bounds of the tile's directions
        for (int c = tid; c < Dt; c += blockDim.x) {
            const int p = (pbase + c < P.d) ? P.perm[pbase + c] : P.d;
            double s[3] = {0.0, 0.0, 0.0};
            DirFilter f;
            if (p < P.d) {
#pragma unroll
                for (int a = 0; a < N; ++a) s[a] = P.dirs[(int64_t)p * N + a];
                f = make_dir_filter<N>(s, g.L, lo, hi, step, T);
            } else {        // idle column: every vertex decided in bin 1, never flushed
                f.S0 = 0.f;
                f.B1 = f.B2 = DS{0.f, 0.f};
                f.C = DS{0.5f, 0.f};
                f.eta = 0x1p-8f;
                f.oct = 0;
            }
            dirf[c] = f;
            const float two = __fmul_rn(2.0f, fabsf(f.S0));      // exact
            rdir[c] = RunDir{__frcp_rd(two), __frcp_ru(two)};
        }
        __syncthreads();
        const int col = wcol * 32 + lane;
        const int p = (pbase + col < P.d) ? P.perm[pbase + col] : P.d;
        const DirFilter f = dirf[col];
        const RunDir rd = rdir[col];
        const uint32_t hcol = histAddr + (uint32_t)col * 4u;

        int parity = 0;
        for (int r = W.r0 + rgroup; r < W.r1; r += RG, parity ^= 1) {
            int32_t *crow = cgrp + parity * rowbuf;
            const int i1 = r % L1, i2 = r / L1;
            // ---- octant contributions of the row
            for (int i0 = gtid; i0 < L0; i0 += gthreads) {
                int32_t c[NOCT];
                octant_contribs<N>(g, i0, i1, i2, c);
#pragma unroll
                for (int o = 0; o < NOCT; ++o) {
                    const int32_t v = c[o];
                    crow[o * CP + i0] = v;
                }
            }
            group_sync(rgroup, WC);
            // ---- in place: I_o[i] = c_o[0] + ... + c_o[i] (each warp takes whole octants; a lane
            // sums a contiguous segment, the warp scans the segment sums, the lane rewrites it)
            const int seg = (L0 + 31) >> 5;
            for (int o = wcol; o < NOCT; o += WC) {
                int32_t *row = crow + o * CP;
                const int s0 = min(L0, lane * seg), s1 = min(L0, s0 + seg);
                int32_t tot = 0;
                for (int i = s0; i < s1; ++i) tot += row[i];
                int32_t inc = tot;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int32_t u = __shfl_up_sync(0xffffffffu, inc, off);
                    if (lane >= off) inc += u;
                }
                int32_t run = inc - tot;
                for (int i = s0; i < s1; ++i) {
                    run += row[i];
                    row[i] = run;
                }
            }
            group_sync(rgroup, WC);

            // ---- the lane's direction: walk the bin boundaries of the row
            const RowFilter rf = make_row_filter<N>(f, i1, i2, g.L);
            const int32_t *Irow = crow + f.oct * CP;             // running sums of the octant
            const int32_t tot = Irow[L0 - 1];
            // exact bins of the two ends; the exact bins are monotone along the row, so the walk
            // starts at the end with the lower bin (the far end when s_0 < 0)
            const bool live = p < P.d;                          // idle columns add nothing
            const int b0 = live ? run_end_bin<N>(P, g, p, 0, false, L0, i1, i2, f.S0, rf) : 0;
            const int b1 = live ? run_end_bin<N>(P, g, p, L0 - 1, false, L0, i1, i2, f.S0, rf) : 0;
            const bool mirror = b0 > b1;
            const int bs = min(b0, b1), be = max(b0, b1);
            // value of the walk prefix [0, a): forward I[a-1], mirrored tot - I[L0-1-a]; the code
            // keeps sign * I[...] and its start and end values (the differences are the same)
            const uint32_t ib = smem_addr(Irow);
            const uint32_t pb = mirror ? ib + (uint32_t)(L0 - 1) * 4u : ib - 4u;
            const int ps = mirror ? -4 : 4;
            int32_t prev = mirror ? -tot : 0;
            const int32_t vend = mirror ? 0 : tot;
            const int32_t sgn = mirror ? -1 : 1;
            uint32_t haddr = hcol + (uint32_t)bs * D4;
            if (live && be > bs) {
                // x(b) enclosure: x_lo = m A_lo + C_lo, x_hi = m A_up + C_hi with m = b - 1 >= 0
                const float half = 0.5f * (float)(L0 - 1);
                const float tl = __fadd_rd(rf.Glo, (float)rf.nr), th = __fadd_ru(rf.Ghi, (float)rf.nr);
                const float Chi0 = __fadd_ru(__fmul_ru(-tl, (-tl >= 0.0f) ? rd.Aup : rd.Alo), half);
                const float Chi = __fadd_ru(Chi0, fmaxf(fabsf(Chi0) * 0x1p-22f, 0x1p-100f));   // strictly above
                const float Clo = __fadd_rd(__fmul_rd(-th, (-th >= 0.0f) ? rd.Alo : rd.Aup), half);
                int aprev = 0;
                for (int b = bs + 1; b <= be; ++b) {
                    const float m = (float)(b - 1);
                    const int flo = __float_as_int(__fadd_rd(__fmaf_rd(m, rd.Alo, Clo), kMagic));
                    const int fhi = __float_as_int(__fadd_rd(__fmaf_ru(m, rd.Aup, Chi), kMagic));
                    const int j = fhi - kMagicBits;
                    int a;
                    if (flo == fhi && (unsigned)j <= (unsigned)(L0 - 2)) {
                        a = j + 1;
                    } else {
                        // bisection on exact bins: the first walk position in [aprev, L0 - 1]
                        // whose bin reaches b (position L0 - 1 has bin be >= b)
                        int l = max(aprev, 1), h = L0 - 1;
                        while (l < h) {
                            const int mid = (l + h) >> 1;
                            const int i0 = mirror ? L0 - 1 - mid : mid;
                            if (run_exact_bin<N>(P, g, p, i0, i1, i2, b) >= b) h = mid; else l = mid + 1;
                        }
                        a = l;
                    }
                    aprev = a;
                    const int32_t v = sgn * lds_s32(pb + (uint32_t)(a * ps));
                    red_shared_add(haddr, v - prev);
                    prev = v;
                    haddr += D4;
                }
            }
            if (live) red_shared_add(haddr, vend - prev);
        }
        __syncthreads();
        unsigned long long *oc = P.out + (int64_t)W.cx * P.d * T;
        if (P.direct)
            cubical_flush_direct<1>(hist, T, Dt, W.dtile, P.d, P.perm, oc);
        else
            cubical_flush_coalesced<1>(hist, T, 0, T, 0, T, Dt, W.dtile, P.d, P.perm, oc, hist + histWords, flushTiles);
    }
}

// ------------------------------------------------------------------ launchers

template <int N>
static cudaError_t launch_run_t(const CubicalFwdArgs &a, int grid, size_t smem, cudaStream_t st, bool launch)
{
    static size_t done = 0;
    if (smem > done) {
        cudaError_t e = cudaFuncSetAttribute(cubical_run_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        done = smem;
    }
    if (!launch) return cudaSuccess;
    cubical_run_kernel<N><<<grid, kRunThreads, smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t run_dispatch(int n, const CubicalFwdArgs &a, int grid, size_t smem, cudaStream_t st, bool launch)
{
    if (n == 1) return launch_run_t<1>(a, grid, smem, st, launch);
    if (n == 2) return launch_run_t<2>(a, grid, smem, st, launch);
    return launch_run_t<3>(a, grid, smem, st, launch);
}

cudaError_t launch_cubical_run(int n, const CubicalFwdArgs &a, int grid, size_t smem, cudaStream_t st)
{
    return run_dispatch(n, a, grid, smem, st, true);
}

cudaError_t prepare_cubical_run(int n, size_t smem)
{
    CubicalFwdArgs a{};
    return run_dispatch(n, a, 1, smem, nullptr, false);
}

// Row pitch of the run kernel's buffers: words, >= L0, = 4 mod 32 (octant rows on distinct banks).
int cubical_run_pitch(int maxL0)
{
    const int L0p = (maxL0 + 3) & ~3;
    return ((L0p + 31) & ~31) + 4;
}

size_t cubical_run_smem(int n, int T, int Dt, int maxL0)
{
    const int noct = 1 << n;
    const int WC = Dt / 32;
    const int RG = (kRunThreads / 32) / WC;
    return (size_t)T * Dt * 4u + (size_t)Dt * (sizeof(DirFilter) + sizeof(RunDir)) +
           (size_t)RG * 2u * noct * cubical_run_pitch(maxL0) * 4u;
}

int cubical_run_threads() { return kRunThreads; }

}  // namespace wect
