// wect_cubical_common.cuh -- pieces shared by the stencil kernels of full cubical grids: the
// per-vertex octant contributions, the row-group barrier and the histogram flushes.
#pragma once
#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

// ------------------------------------------------------------------ octant contributions

// c_o(v) for every octant o from the int32 fixed-point weights of v's 3^n neighbourhood (the
// accumulator modes bound 2^n max|w| below 2^31, checked when the weights are set, so |c_o| fits
// int32).  ld(dx, dy, dz) returns the weight of vertex (i0 + dx, i1 + dy, i2 + dz); it is called
// only inside the grid.
//
// c_o(v) = sum over the axis subsets e of (-1)^|e| w(cell spanned by v and its neighbours on the
// sides of o along the axes in e), the cell weight being the max over its vertices.  Vertices
// outside the grid stand in with weight S = 2^31 - 1, so the box maximum of every cell that leaves
// the grid is S, and the sum runs over all 2^n subsets without masks, in wrapping 32-bit
// arithmetic.  The S terms cancel: their signs sum to -[no side of o lies inside the grid] (the
// signed count of the subsets that meet the outside axes), so the plain sum is exact except at a
// grid corner of o, where the only cell is v itself and c_o = w(v).
template <int N, class Load>
__device__ __forceinline__ void octant_contribs_with(Load ld, int L0, int L1, int L2, int i0, int i1, int i2,
                                                     int32_t *c /* [1 << N] */)
{
    constexpr int NOCT = 1 << N;
    constexpr int NY = (N >= 2) ? 3 : 1;
    constexpr int NZ = (N >= 3) ? 3 : 1;
    constexpr int32_t S = 0x7fffffff;
    const bool ok0[3] = {i0 > 0, true, i0 < L0 - 1};
    const bool ok1[3] = {i1 > 0, true, i1 < L1 - 1};
    const bool ok2[3] = {i2 > 0, true, i2 < L2 - 1};
    // box maxima over the 3^n neighbourhood, axis by axis: A[z][y][x] = max over the box spanning
    // v and v + (x-1, y-1, z-1)
    int32_t A[NZ][NY][3];
#pragma unroll
    for (int z = 0; z < NZ; ++z)
#pragma unroll
        for (int y = 0; y < NY; ++y) {
            int32_t w[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const int dy = (N >= 2) ? y - 1 : 0, dz = (N >= 3) ? z - 1 : 0;
                const bool ok = ok0[x] && (N < 2 || ok1[y]) && (N < 3 || ok2[z]);
                w[x] = ok ? ld(x - 1, dy, dz) : S;
            }
            A[z][y][0] = max(w[0], w[1]);
            A[z][y][1] = w[1];
            A[z][y][2] = max(w[1], w[2]);
        }
    if (N >= 2) {
#pragma unroll
        for (int z = 0; z < NZ; ++z)
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const int32_t a0 = A[z][0][x], a1 = A[z][NY > 1 ? 1 : 0][x], a2 = A[z][NY > 2 ? 2 : 0][x];
                A[z][0][x] = max(a0, a1);
                if (NY > 2) A[z][2][x] = max(a1, a2);
            }
    }
    if (N >= 3) {
#pragma unroll
        for (int y = 0; y < NY; ++y)
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const int32_t a0 = A[0][y][x], a1 = A[NZ > 1 ? 1 : 0][y][x], a2 = A[NZ > 2 ? 2 : 0][y][x];
                A[0][y][x] = max(a0, a1);
                if (NZ > 2) A[2][y][x] = max(a1, a2);
            }
    }
    const int32_t wv = A[NZ / 2][NY / 2][1];
#pragma unroll
    for (int o = 0; o < NOCT; ++o) {
        uint32_t acc = 0;
        bool inside = false;                 // some side of o lies inside the grid
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const int side = ((o >> a) & 1) ? 0 : 2;     // sign corner at the upper end: the cells reach back
            inside = inside || (a == 0 ? ok0[side] : (a == 1 ? ok1[side] : ok2[side]));
        }
#pragma unroll
        for (int e = 0; e < NOCT; ++e) {
            int idx[3] = {1, 1, 1};
#pragma unroll
            for (int a = 0; a < N; ++a)
                if ((e >> a) & 1) idx[a] = ((o >> a) & 1) ? 0 : 2;
            const uint32_t wb = (uint32_t)A[N >= 3 ? idx[2] : 0][N >= 2 ? idx[1] : 0][idx[0]];
            acc = (__popc(e) & 1) ? acc - wb : acc + wb;
        }
        c[o] = inside ? (int32_t)acc : wv;
    }
}

// From the complex's int32 weights in global memory.
template <int N>
__device__ __forceinline__ void octant_contribs(const GridDesc &g, int i0, int i1, int i2, int32_t *c)
{
    const int L0 = g.L[0], L1 = g.L[1];
    const int32_t *w = g.w + (int64_t)i0 + (int64_t)L0 * ((int64_t)i1 + (int64_t)L1 * i2);
    octant_contribs_with<N>([&](int dx, int dy, int dz) { return __ldg(w + dx + (int64_t)L0 * (dy + (int64_t)L1 * dz)); },
                            L0, L1, g.L[2], i0, i1, i2, c);
}

// From a staged box of the neighbouring rows: row (i1 + y - 1, i2 + z - 1) of the grid at
// box + (z * NY + y) * L0 (rows outside the grid are zero and never read).
template <int N>
__device__ __forceinline__ void octant_contribs_box(const int32_t *box, const GridDesc &g, int i0, int i1, int i2,
                                                    int32_t *c)
{
    constexpr int NY = (N >= 2) ? 3 : 1;
    const int L0 = g.L[0];
    const int32_t *b = box + i0;
    octant_contribs_with<N>([&](int dx, int dy, int dz) { return b[((dz + (N >= 3 ? 1 : 0)) * NY + dy + (N >= 2 ? 1 : 0)) * L0 + dx]; },
                            L0, g.L[1], g.L[2], i0, i1, i2, c);
}

// ------------------------------------------------------------------ forward helpers

// Add the CTA's partial histograms into the int64 output block [d][T] and clear them.  The
// histogram has HR rows (the plane stride of the two-plane form); rows [rlo, rhi) hold the bins
// base + rlo .. base + rhi - 1 of the item's threshold tile, the others are discard rows (untiled:
// HR = T, rows [0, T), base 0; only TILED instances check the row range).
template <int NSPLIT, bool TILED = false>
__device__ __forceinline__ void cubical_flush(int32_t *hist, int HR, int rlo, int rhi, int base, int T, int Dt,
                                              int dtile, int d, const int *perm, unsigned long long *out)
{
    const int hw = HR * Dt;
    if (blockDim.x % Dt == 0) {
        // each thread keeps one column: no division and one perm load per thread
        const int col = threadIdx.x % Dt, bstep = blockDim.x / Dt;
        const int p = (dtile * Dt + col < d) ? perm[dtile * Dt + col] : d;
        unsigned long long *orow = out + (int64_t)min(p, d - 1) * T + base;
        for (int b = threadIdx.x / Dt; b < HR; b += bstep) {
            const int idx = b * Dt + col;
            int64_t v;
            if (NSPLIT == 1) {
                v = hist[idx];
            } else {
                v = ((int64_t)hist[hw + idx] << 16) + (int64_t)(uint32_t)hist[idx];
                hist[hw + idx] = 0;
            }
            hist[idx] = 0;
            if (p < d && v != 0 && (!TILED || (b >= rlo && b < rhi))) atomicAdd(orow + b, (unsigned long long)v);
        }
        return;
    }
    for (int idx = threadIdx.x; idx < hw; idx += blockDim.x) {
        const int b = idx / Dt, col = idx - b * Dt;
        const int p = (dtile * Dt + col < d) ? perm[dtile * Dt + col] : d;
        int64_t v;
        if (NSPLIT == 1) {
            v = hist[idx];
        } else {
            v = ((int64_t)hist[hw + idx] << 16) + (int64_t)(uint32_t)hist[idx];
            hist[hw + idx] = 0;
        }
        hist[idx] = 0;
        if (p < d && v != 0 && (!TILED || (b >= rlo && b < rhi)))
            atomicAdd(out + (int64_t)p * T + base + b, (unsigned long long)v);
    }
}

// The same flush with coalesced global atomics.  cubical_flush's warps add 32 directions of one
// bin, 32 rows of the output apart; here each warp moves a 32 x 32 block (32 bins x 32 columns)
// through a padded tile of its own in shared memory (conflict-free on both sides) and adds each
// column's 32 bins as one run of 32 consecutive int64, a quarter of the L2 sectors.  scratch
// holds ntiles tiles of NSPLIT x 32 x 33 words (the CTA's shared memory past the histogram, idle
// between items); warps beyond ntiles stay idle, and with no tile at all cubical_flush runs.  Dt
// is a multiple of 32.
template <int NSPLIT, bool TILED = false>
__device__ __forceinline__ void cubical_flush_coalesced(int32_t *hist, int HR, int rlo, int rhi, int base, int T,
                                                        int Dt, int dtile, int d, const int *perm,
                                                        unsigned long long *out, int32_t *scratch, int ntiles)
{
    if (ntiles <= 0) {
        cubical_flush<NSPLIT, TILED>(hist, HR, rlo, rhi, base, T, Dt, dtile, d, perm, out);
        return;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = min((int)(blockDim.x >> 5), ntiles);
    const int hw = HR * Dt, ncb = Dt >> 5, nblk = ncb * ((HR + 31) >> 5);
    if (wid < nw) {
        int32_t *sc = scratch + wid * (NSPLIT * 32 * 33);
        for (int blk = wid; blk < nblk; blk += nw) {
            const int cb = blk % ncb, rb = blk / ncb;
            const int c0 = cb * 32, b0 = rb * 32;
            // bins b0 + k, columns c0 + lane: row reads, cleared, into the tile's rows
            for (int k = 0; k < 32 && b0 + k < HR; ++k) {
                const int idx = (b0 + k) * Dt + c0 + lane;
                sc[k * 33 + lane] = hist[idx];
                hist[idx] = 0;
                if (NSPLIT == 2) {
                    sc[32 * 33 + k * 33 + lane] = hist[hw + idx];
                    hist[hw + idx] = 0;
                }
            }
            __syncwarp();
            // column c0 + k, bins b0 + lane: one run of 32 consecutive int64 of direction perm[c0 + k]
            const int pl = (dtile * Dt + c0 + lane < d) ? perm[dtile * Dt + c0 + lane] : d;
            const int b = b0 + lane;
            const bool rowok = b < HR && (!TILED || (b >= rlo && b < rhi));
            for (int k = 0; k < 32; ++k) {
                const int p = __shfl_sync(0xffffffffu, pl, k);
                int64_t v = 0;
                if (rowok) {
                    v = sc[lane * 33 + k];
                    if (NSPLIT == 2) v = ((int64_t)sc[32 * 33 + lane * 33 + k] << 16) + (int64_t)(uint32_t)v;
                }
                if (p < d && v != 0) atomicAdd(out + (int64_t)p * T + base + b, (unsigned long long)v);
            }
            __syncwarp();
        }
        fence_proxy_async_smem();           // the tiles may be TMA staging space of the next item
    }
}

// The item covered every row of its complex: the histogram is the complete difference table of
// its directions.  Scan it over the thresholds (Algorithm 1's cumulative sum) and store the
// transform directly (no atomics, no separate scan).
template <int NSPLIT>
__device__ __forceinline__ void cubical_flush_direct(int32_t *hist, int T, int Dt, int dtile, int d, const int *perm,
                                                     unsigned long long *out)
{
    const int hw = T * Dt;
    for (int col = threadIdx.x; col < Dt; col += blockDim.x) {
        const int p = (dtile * Dt + col < d) ? perm[dtile * Dt + col] : d;
        long long acc = 0;
        for (int q = 0; q < T; ++q) {
            const int idx = q * Dt + col;
            int64_t v;
            if (NSPLIT == 1) {
                v = hist[idx];
            } else {
                v = ((int64_t)hist[hw + idx] << 16) + (int64_t)(uint32_t)hist[idx];
                hist[hw + idx] = 0;
            }
            hist[idx] = 0;
            acc += v;
            if (p < d) out[(int64_t)p * T + q] = (unsigned long long)acc;
        }
    }
}

// Barrier of the WC warps of one row group (warp-synchronous when the group is one warp).
__device__ __forceinline__ void group_sync(int rgroup, int WC)
{
    if (WC == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + rgroup), "r"(WC * 32) : "memory");
    }
}

}  // namespace wect
