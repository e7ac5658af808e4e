// wect_simplicial.cu -- gather kernels for the WECT of simplicial complexes given as index lists
// (Section 3 "inputs": per dimension a [k_i][i+1] table of vertex ids and a weight per simplex).
//
// Per direction tile the vertex bins are computed once (float32 filter, exact float64 fallback)
// into a [nv][Dt] uint16 table; the simplex kernel then takes, for every simplex and direction,
// the max of its vertex bins (equal to the bin of the max height, Eq. "msi") and adds the
// signed simplex weight into a shared-memory histogram [T][Dt] (one column per lane, so a
// red.shared of a warp hits 32 distinct banks), flushed into the int64 output.
#include <climits>

#include <cmath>
#include <type_traits>

#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

constexpr int kSimplexThreads = 512;

// ------------------------------------------------------------------ vertex bins

// Per direction p, the float32 form u = sum_a x~_a A_a + C of the threshold coordinate
// (h - lo) / step, with x~_a = rn32(x_a), A_a = rn32(s_a / step), C = rn32(-lo / step), and a bound
// eta on |u - (h - lo) / step| (Sec. 3.2, the bin of a vertex height).  tab[p] = {A_0, A_1, A_2,
// A_3, C, eta, 0, 0} (A_a = 0 for a >= N).  A zero step (lo == hi) gives eta = inf, so every bin
// goes to the float64 path.
template <int N>
__global__ void dir_filter_kernel(const double *__restrict__ dirs, int d, int T, const double *__restrict__ range,
                                  float *__restrict__ tab)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d) return;
    const double lo = range[0], step = range[2];
    float Af[4] = {0.f, 0.f, 0.f, 0.f}, Cf = 0.f, eta = __int_as_float(0x7f800000);
    double U = 0.0;
    if (step > 0.0) {
        U = fabs(lo) / step;
        for (int a = 0; a < N; ++a) {
            const double A = __ddiv_rn(dirs[(int64_t)p * N + a], step);
            Af[a] = __double2float_rn(A);
            U += fabs(A) * range[3 + a];                      // range[3+a] = max |x_a| over the vertices
        }
        Cf = __double2float_rn(__ddiv_rn(-lo, step));
        // coordinate and coefficient roundings (2^-24 |x_a A_a| each) and N+1 fma/constant roundings
        // (2^-24 of a partial sum <= U): |u_f32 - u| <= 2^-24 (N+3) U; 25% margin
        eta = __double2float_ru(0x1p-24 * 1.25 * (double)(N + 3) * (U + 1.0) + 0x1p-40 * ((double)T + U));
    }
    // |u| <= U: beyond 2^21 (or a zero step) the magic-constant ceiling is not sound, so every
    // bin takes the exact path (u = 0, eta = inf)
    if (!(step > 0.0) || !(U + (double)T <= 0x1p21)) {
        Af[0] = Af[1] = Af[2] = Af[3] = Cf = 0.f;
        eta = __int_as_float(0x7f800000);
    }
    float4 *t = reinterpret_cast<float4 *>(tab + (int64_t)p * 8);
    t[0] = make_float4(Af[0], Af[1], Af[2], Af[3]);
    t[1] = make_float4(Cf, eta, 0.f, 0.f);
}

// Float32 copies of the vertex coordinates, rounded to nearest (the x~_a of the filter).
__global__ void coords_to_f32_kernel(const double *__restrict__ x, int64_t n, float *__restrict__ xf)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xf[i] = __double2float_rn(x[i]);
}

// bins[v][c] = bin of vertex v in direction dtile * Dt + c.  One warp row per vertex and
// direction column; a float32 filter decides the bin unless the interval u +- eta contains an
// integer, in which case the float64 height is compared with the threshold table.
template <int N>
__global__ void __launch_bounds__(256) vertex_bins_kernel(const double *__restrict__ coords,
                                                          const float *__restrict__ xf, int64_t nv,
                                                          const double *__restrict__ dirs,
                                                          const float *__restrict__ tab, int d, int dtile, int Dt,
                                                          int T, const double *__restrict__ beta,
                                                          uint16_t *__restrict__ bins)
{
    const int col = threadIdx.x % Dt;
    const int vpb = blockDim.x / Dt;                          // vertices per block pass
    const int p = dtile * Dt + col;
    const bool act = p < d;
    const int pc = act ? p : d - 1;
    const float4 t0 = __ldg(reinterpret_cast<const float4 *>(tab + (int64_t)pc * 8));
    const float Cf = __ldg(tab + (int64_t)pc * 8 + 4), eta = __ldg(tab + (int64_t)pc * 8 + 5);
    const float Af[4] = {t0.x, t0.y, t0.z, t0.w};
    for (int64_t v = (int64_t)blockIdx.x * vpb + threadIdx.x / Dt; v < nv; v += (int64_t)gridDim.x * vpb) {
        float u = Cf;
#pragma unroll
        for (int a = N - 1; a >= 0; --a) u = __fmaf_rn(__ldg(xf + v * N + a), Af[a], u);
        const int tlo = __float_as_int(__fadd_ru(__fsub_rd(u, eta), kMagic));
        const int thi = __float_as_int(__fadd_ru(__fadd_ru(u, eta), kMagic));
        int b = clamp_bin(thi, 0, T);
        if (tlo != thi) {
            const double h = heightv<N>(coords + v * N, dirs + (int64_t)pc * N);
            b = exact_bin_from(h, beta, T, b);
        }
        // every column gets a valid bin: a column past d (the last tile's padding) carries the
        // bin of direction d - 1, which the gathers read but never flush
        bins[v * Dt + col] = (uint16_t)b;
    }
}

// ------------------------------------------------------------------ simplex scatter

// One warp's share of GS consecutive simplices (n valid; n == GS when FULL) in a 32-direction
// tile, read from global memory.  All vertex ids, packed signed weights and vertex bins of the
// group are loaded before any is reduced, so GS dependent load chains are in flight.  Vertex ids
// are global int32 ids, or for M == 1 the simplex index itself (vbase + g).  bins and histLane
// already carry the lane's column; the max of the vertex bins (Eq. "msi") selects the histogram
// row.  With GH the signed weight goes straight to the lane's int64 difference row orow in global
// memory (null for a padding column) instead of the shared histogram.  (Staged chunks take
// gather_group_staged below.)
template <int NSPLIT, int M, int GS, bool FULL, bool GH = false>
__device__ __forceinline__ void gather_group(const int32_t *__restrict__ ids, int vbase, const int2 *__restrict__ wp,
                                             int n, const uint16_t *__restrict__ bins, uint32_t histLane,
                                             uint32_t HOFF, unsigned long long *orow = nullptr)
{
    int vid[GS][M];
    int2 w[GS];
    if (FULL) {
        // a full group is GS consecutive simplices whose ids and weights start on 16-byte
        // boundaries (chunks and groups are multiples of GS = 8 simplices): 128-bit loads
        static_assert(GS == 8, "vector loads assume groups of 8");
#pragma unroll
        for (int q = 0; q < GS / 2; ++q) {
            const int4 x = __ldg(reinterpret_cast<const int4 *>(wp) + q);
            w[2 * q] = make_int2(x.x, x.y);
            w[2 * q + 1] = make_int2(x.z, x.w);
        }
        if (M == 1) {
#pragma unroll
            for (int g = 0; g < GS; ++g) vid[g][0] = vbase + g;
        } else {
            int word[GS * M];
#pragma unroll
            for (int q = 0; q < GS * M / 4; ++q) {
                const int4 x = __ldg(reinterpret_cast<const int4 *>(ids) + q);
                word[4 * q] = x.x;
                word[4 * q + 1] = x.y;
                word[4 * q + 2] = x.z;
                word[4 * q + 3] = x.w;
            }
#pragma unroll
            for (int g = 0; g < GS; ++g)
#pragma unroll
                for (int j = 0; j < M; ++j) vid[g][j] = word[g * M + j];
        }
    } else {
#pragma unroll
        for (int g = 0; g < GS; ++g) {
            const int gi = min(g, n - 1);
#pragma unroll
            for (int j = 0; j < M; ++j) vid[g][j] = (M == 1) ? vbase + gi : __ldg(ids + gi * M + j);
            w[g] = (g < n) ? __ldg(wp + gi) : make_int2(0, 0);
        }
    }
    int bin[GS];
#pragma unroll
    for (int g = 0; g < GS; ++g) {
        int bm = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) bm = max(bm, (int)__ldg(bins + (int64_t)vid[g][j] * 32));
        bin[g] = bm;
    }
#pragma unroll
    for (int g = 0; g < GS; ++g) {
        if constexpr (GH) {
            // packed {v, 0} or {low 16 bits, v >> 16}: v = (w.y << 16) + w.x either way
            if (orow && (FULL || g < n))
                atomicAdd(orow + bin[g], (unsigned long long)(((long long)w[g].y << 16) + (long long)w[g].x));
        } else {
            const uint32_t addr = histLane + (uint32_t)bin[g] * 128u;
            red_shared_add(addr, w[g].x);
            if (NSPLIT == 2) red_shared_add(addr + HOFF, w[g].y);
        }
    }
}

__device__ __forceinline__ int lds_u16(uint32_t addr)
{
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return (int)v;
}

__device__ __forceinline__ int2 lds_v2s32(uint32_t addr)
{
    int2 v;
    asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

// gather_group for a staged chunk, every operand addressed in the shared window directly (32-bit
// shared addresses): ids is the address of the group's M * GS window-row offsets (u16 byte
// offsets), wts of its GS packed weights, winLane the window's address plus 2 * lane.
template <int NSPLIT, int M, int GS>
__device__ __forceinline__ void gather_group_staged(uint32_t ids, uint32_t wts, int n, uint32_t winLane,
                                                    uint32_t histLane, uint32_t HOFF)
{
    int off[GS][M];
    int2 w[GS];
    if (n == GS) {
        static_assert(GS == 8, "vector loads assume groups of 8");
        uint32_t word[GS * M / 2];
#pragma unroll
        for (int q = 0; q < GS * M / 8; ++q) {
            const int4 x = lds128(ids + 16u * q);
            word[4 * q] = (uint32_t)x.x;
            word[4 * q + 1] = (uint32_t)x.y;
            word[4 * q + 2] = (uint32_t)x.z;
            word[4 * q + 3] = (uint32_t)x.w;
        }
#pragma unroll
        for (int g = 0; g < GS; ++g)
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int e = g * M + j;
                off[g][j] = (int)((word[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
            }
#pragma unroll
        for (int q = 0; q < GS / 2; ++q) {
            const int4 x = lds128(wts + 16u * q);
            w[2 * q] = make_int2(x.x, x.y);
            w[2 * q + 1] = make_int2(x.z, x.w);
        }
    } else {
#pragma unroll
        for (int g = 0; g < GS; ++g) {
            const int gi = min(g, n - 1);
#pragma unroll
            for (int j = 0; j < M; ++j) off[g][j] = lds_u16(ids + 2u * (uint32_t)(gi * M + j));
            w[g] = (g < n) ? lds_v2s32(wts + 8u * (uint32_t)gi) : make_int2(0, 0);
        }
    }
    int bin[GS];
#pragma unroll
    for (int g = 0; g < GS; ++g) {
        int bm = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) bm = max(bm, lds_u16(winLane + (uint32_t)off[g][j]));
        bin[g] = bm;
    }
#pragma unroll
    for (int g = 0; g < GS; ++g) {
        const uint32_t addr = histLane + (uint32_t)bin[g] * 128u;
        red_shared_add(addr, w[g].x);
        if (NSPLIT == 2) red_shared_add(addr + HOFF, w[g].y);
    }
}

// Add a CTA's [NSPLIT][T][32] int32 histogram (low 16 bits unsigned + high part when NSPLIT = 2)
// into the int64 [d][T] difference table of the tile's directions, and clear it.
template <int NSPLIT>
__device__ __forceinline__ void simplex_flush(int32_t *hist, int T, int dtile, int d, unsigned long long *out)
{
    const int hw = T * 32;
    __syncthreads();
    for (int idx = threadIdx.x; idx < hw; idx += blockDim.x) {
        const int q = idx >> 5, c = idx & 31;
        const int p = dtile * 32 + c;
        int64_t v;
        if (NSPLIT == 1) {
            v = hist[idx];
        } else {
            v = ((int64_t)hist[hw + idx] << 16) + (int64_t)(uint32_t)hist[idx];
            hist[hw + idx] = 0;
        }
        hist[idx] = 0;
        if (p < d && v != 0) atomicAdd(out + (int64_t)p * T + q, (unsigned long long)v);
    }
    __syncthreads();
}

constexpr int kGatherGS = 8;

// Gather for one 32-direction tile straight from the global bin table: CTAs take chunks of
// P.chunk simplices (at most the flush bound), warps take groups of kGatherGS simplices.
// GH: no shared histogram; every signed weight is added to the int64 difference table in global
// memory (T beyond shared memory).
template <int NSPLIT, int M, bool GH>
__global__ void __launch_bounds__(kSimplexThreads, 1) simplex_fwd_kernel(const SimplexFwdArgs P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int GS = kGatherGS;
    const int T = P.T;
    int32_t *hist = reinterpret_cast<int32_t *>(smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t histLane = smem_addr(hist) + (uint32_t)lane * 4u;
    const uint32_t HOFF = (uint32_t)T * 128u;
    const int p = P.dtile * 32 + lane;
    unsigned long long *orow = (GH && p < P.d) ? P.out + (int64_t)p * T : nullptr;
    if (!GH) {
        for (int i = threadIdx.x; i < NSPLIT * T * 32; i += blockDim.x) hist[i] = 0;
        __syncthreads();
    }
    pdl_wait();             // a programmatic dependent: the bins and the table from here on
    pdl_trigger();
    const uint16_t *bins = P.bins + lane;
    const int64_t nchunks = (P.k + P.chunk - 1) / P.chunk;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t b0 = ch * P.chunk, b1 = min(P.k, b0 + P.chunk);
        for (int64_t bb = b0 + (int64_t)wid * GS; bb < b1; bb += (int64_t)nw * GS) {
            const int n = (int)(b1 - bb < (int64_t)GS ? b1 - bb : (int64_t)GS);
            const int32_t *ids = (M == 1) ? nullptr : P.simp + bb * M;
            if (n == GS)
                gather_group<NSPLIT, M, GS, true, GH>(ids, (int)bb, P.swp + bb, n, bins, histLane, HOFF,
                                                                      orow);
            else
                gather_group<NSPLIT, M, GS, false, GH>(ids, (int)bb, P.swp + bb, n, bins, histLane, HOFF,
                                                                       orow);
        }
        if (!GH) simplex_flush<NSPLIT>(hist, T, P.dtile, P.d, P.out);
    }
}

// Packed signed weights of a list for the gather: v = (-1)^dim w; one plane: {v, 0}; two planes:
// {low 16 bits of v, v >> 16}.
__global__ void pack_weights_kernel(const int64_t *__restrict__ sw, int64_t k, int sign, int nsplit,
                                    int2 *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = sign > 0 ? sw[i] : -sw[i];
        out[i] = nsplit == 1 ? make_int2((int)v, 0) : make_int2((int)(v & 0xFFFF), (int)(v >> 16));
    }
}

// The vertices' own scatter fused with their bins, for one 32-direction tile: each warp takes
// VG consecutive vertices per step (lane = direction column), loads all their coordinates and
// packed weights first, then computes each bin with the float32 filter (exact float64 path when
// undecided), stores it for the simplices' gathers and adds the vertex weight into the CTA's
// histogram.
template <int N, int NSPLIT>
__global__ void __launch_bounds__(kSimplexThreads, 1) vertex_scatter_kernel(const SimplexFwdArgs P,
                                                                            const double *__restrict__ coords,
                                                                            const float *__restrict__ xf, int64_t nv,
                                                                            const double *__restrict__ dirs,
                                                                            const float *__restrict__ tab,
                                                                            const double *__restrict__ beta,
                                                                            uint16_t *__restrict__ bins)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int VG = 8;
    const int T = P.T, d = P.d;
    int32_t *hist = reinterpret_cast<int32_t *>(smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t histLane = smem_addr(hist) + (uint32_t)lane * 4u;
    const uint32_t HOFF = (uint32_t)T * 128u;
    for (int i = threadIdx.x; i < NSPLIT * T * 32; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    pdl_wait();             // the previous tile's gathers have read the bins this kernel rewrites
    pdl_trigger();
    const int p = P.dtile * 32 + lane;
    const bool act = p < d;
    const int pc = act ? p : d - 1;
    const float4 t0 = __ldg(reinterpret_cast<const float4 *>(tab + (int64_t)pc * 8));
    const float Cf = __ldg(tab + (int64_t)pc * 8 + 4), eta = __ldg(tab + (int64_t)pc * 8 + 5);
    const float Af[4] = {t0.x, t0.y, t0.z, t0.w};
    // CTA-uniform steps of nw * VG vertices (so that the periodic flush is a block-wide barrier),
    // at most P.flush_every steps between flushes
    const int64_t cstep = (int64_t)nw * VG;
    const int nvm1 = (int)(nv - 1);                  // vertex ids are int32
    const int64_t gstep = (int64_t)gridDim.x * cstep;
    // coordinates and weights of the warp's next group, loaded one step ahead
    float xn[VG][N];
    int2 wn[VG];
    static_assert(VG % 2 == 0 && (VG * N) % 4 == 0, "128-bit group loads");
    auto load_group = [&](int64_t base) {
        const int v0 = (int)(base + (int64_t)wid * VG);
        if (v0 <= nvm1 - (VG - 1)) {
            // a whole group: its coordinates and packed weights are contiguous and 16-byte
            // aligned (v0 is a multiple of VG), so 128-bit loads
            const float4 *xs = reinterpret_cast<const float4 *>(xf + (int64_t)v0 * N);
            float xv[VG * N];
#pragma unroll
            for (int q = 0; q < VG * N / 4; ++q) {
                const float4 t = __ldg(xs + q);
                xv[4 * q] = t.x;
                xv[4 * q + 1] = t.y;
                xv[4 * q + 2] = t.z;
                xv[4 * q + 3] = t.w;
            }
#pragma unroll
            for (int g = 0; g < VG; ++g)
#pragma unroll
                for (int a = 0; a < N; ++a) xn[g][a] = xv[g * N + a];
            const int4 *ws = reinterpret_cast<const int4 *>(P.swp + v0);
#pragma unroll
            for (int q = 0; q < VG / 2; ++q) {
                const int4 t = __ldg(ws + q);
                wn[2 * q] = make_int2(t.x, t.y);
                wn[2 * q + 1] = make_int2(t.z, t.w);
            }
            return;
        }
#pragma unroll
        for (int g = 0; g < VG; ++g) {
            const int v = min(v0 + g, nvm1);
#pragma unroll
            for (int a = 0; a < N; ++a) xn[g][a] = __ldg(xf + (int64_t)v * N + a);
            wn[g] = (v0 + g <= nvm1) ? __ldg(P.swp + v) : make_int2(0, 0);
        }
    };
    if ((int64_t)blockIdx.x * cstep < nv) load_group((int64_t)blockIdx.x * cstep);
    int since = 0;
    for (int64_t base = (int64_t)blockIdx.x * cstep; base < nv; base += gstep) {
        const int v0 = (int)(base + (int64_t)wid * VG);
        float x[VG][N];
        int2 w[VG];
#pragma unroll
        for (int g = 0; g < VG; ++g) {
#pragma unroll
            for (int a = 0; a < N; ++a) x[g][a] = xn[g][a];
            w[g] = wn[g];
        }
        if (base + gstep < nv) load_group(base + gstep);
        // branch-free pass: candidate bins, stores and scatters; undecided bins are only marked
        int bc[VG];
        uint32_t pend = 0;
        uint16_t *brow = bins + (int64_t)v0 * 32 + lane;       // this lane's column of the group's rows
#pragma unroll
        for (int g = 0; g < VG; ++g) {
            float u = Cf;
#pragma unroll
            for (int a = N - 1; a >= 0; --a) u = __fmaf_rn(x[g][a], Af[a], u);
            const int tlo = __float_as_int(__fadd_ru(__fsub_rd(u, eta), kMagic));
            const int thi = __float_as_int(__fadd_ru(__fadd_ru(u, eta), kMagic));
            const int b = clamp_bin(thi, 0, T);
            bc[g] = b;
            pend |= (tlo != thi ? 1u : 0u) << g;
            // every column gets a valid bin (a padding column carries direction d - 1's), so the
            // gathers never read an unwritten entry
            if (v0 + g <= nvm1) brow[g * 32] = (uint16_t)b;
            const uint32_t addr = histLane + (uint32_t)b * 128u;
            red_shared_add(addr, w[g].x);
            if (NSPLIT == 2) red_shared_add(addr + HOFF, w[g].y);
        }
        // undecided bins: the exact float64 bin, and the contribution moved if it differs (the
        // entry it leaves received it above, so the low plane stays non-negative)
        if (__any_sync(0xffffffffu, pend != 0)) {
            while (pend) {
                const int g = __ffs(pend) - 1;
                pend &= pend - 1;
                const int v = min(v0 + g, nvm1);
                const double h = heightv<N>(coords + (int64_t)v * N, dirs + (int64_t)pc * N);
                int bg = 0, wx = 0, wy = 0;
#pragma unroll
                for (int k = 0; k < VG; ++k)
                    if (k == g) {
                        bg = bc[k];
                        wx = w[k].x;
                        wy = w[k].y;
                    }
                const int be = exact_bin_from(h, beta, T, bg);
                if (be != bg) {
                    if (v0 + g <= nvm1) bins[(int64_t)(v0 + g) * 32 + lane] = (uint16_t)be;
                    const uint32_t at = histLane + (uint32_t)bg * 128u, ae = histLane + (uint32_t)be * 128u;
                    red_shared_add(at, -wx);
                    red_shared_add(ae, wx);
                    if (NSPLIT == 2) {
                        red_shared_add(at + HOFF, -wy);
                        red_shared_add(ae + HOFF, wy);
                    }
                }
            }
        }
        if (++since >= P.flush_every) {
            simplex_flush<NSPLIT>(hist, T, P.dtile, d, P.out);
            since = 0;
        }
    }
    if (since > 0) simplex_flush<NSPLIT>(hist, T, P.dtile, d, P.out);
}

// ------------------------------------------------------------------ staged chunks

// Creation-time pass over a list of simplices with M >= 2 vertices, one CTA per chunk of
// chunk_simplices(M) simplices: sort the chunk's vertex ids, keep the distinct ones (thread 0, a
// serial pass over at most kChunkSlots sorted ids), and when there are at most kWinRows of them
// store them in cverts and rewrite the chunk's ids as the byte offsets of their rows in the
// staged window (rank * 64, below kWinRows * 64 = 34816: 16 bits).  cnu is the number
// of distinct vertices, or -1 for a chunk the gather reads straight from global memory.
template <int M>
__global__ void __launch_bounds__(512) chunk_local_kernel(const int32_t *__restrict__ simp, int64_t k,
                                                          uint16_t *__restrict__ local, int32_t *__restrict__ cverts,
                                                          int32_t *__restrict__ cnu)
{
    constexpr int C = chunk_simplices(M);
    constexpr int NK = 2048;              // power of two >= kChunkSlots
    __shared__ int keys[NK];
    __shared__ int U;
    const int64_t s0 = (int64_t)blockIdx.x * C;
    const int nslot = (int)(k - s0 < (int64_t)C ? k - s0 : (int64_t)C) * M;
    for (int j = threadIdx.x; j < NK; j += blockDim.x) keys[j] = (j < nslot) ? simp[s0 * M + j] : INT_MAX;
    __syncthreads();
    // bitonic sort, ascending
    for (int size = 2; size <= NK; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int j = threadIdx.x; j < NK / 2; j += blockDim.x) {
                const int lo = 2 * j - (j & (stride - 1)), hi = lo + stride;
                const int a = keys[lo], b = keys[hi];
                if ((a > b) == ((lo & size) == 0)) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        int u = 0;
        for (int j = 0; j < nslot; ++j)
            if (j == 0 || keys[j] != keys[j - 1]) keys[u++] = keys[j];
        U = u;
        cnu[blockIdx.x] = (u <= kWinRows) ? u : -1;
    }
    __syncthreads();
    const int u = U;
    if (u > kWinRows) return;
    for (int j = threadIdx.x; j < u; j += blockDim.x) cverts[(int64_t)blockIdx.x * kWinRows + j] = keys[j];
    for (int j = threadIdx.x; j < nslot; j += blockDim.x) {
        const int v = simp[s0 * M + j];
        int lo = 0, hi = u - 1;                 // keys[0..u) is sorted and holds v
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (keys[mid] < v) lo = mid + 1; else hi = mid;
        }
        local[s0 * M + j] = (uint16_t)(lo * 64);          // byte offset of the vertex's window row
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// 16-byte copy of which only the first n bytes come from src (the rest is zero-filled).
__device__ __forceinline__ void cp_async16_n(uint32_t dst, const void *src, int n)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Staged gather for lists of dim >= 1 (M >= 2 vertices per simplex), one 32-direction tile.  Each
// CTA walks a contiguous range of chunks.  For a staged chunk, cp.async copies its vertex-bin rows
// (64 bytes each, a window of at most kWinRows chunk vertices), its chunk-local ids and its packed
// weights into one of two shared-memory buffers while the previous chunk is reduced, so every
// load of the reduction is a shared-memory load.  Chunks with more than kWinRows distinct
// vertices read global memory as simplex_fwd_kernel does.  The histogram and flush are those of
// simplex_fwd_kernel.
template <int NSPLIT, int M>
__global__ void __launch_bounds__(kSimplexThreads, 1) simplex_fwd_staged_kernel(const SimplexFwdArgs P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int C = chunk_simplices(M);
    constexpr int GS = kGatherGS;
    constexpr int NWIN = 4 * kWinRows;                           // 16-byte pieces of a full window
    constexpr int NID = (C * M * 2 + 15) / 16;                    // ... of the chunk's ids
    constexpr int NWT = (C * 8 + 15) / 16;                        // ... of its weights
    constexpr int NCP = (NWIN + NID + NWT + kSimplexThreads - 1) / kSimplexThreads;
    const int T = P.T;
    int32_t *hist = reinterpret_cast<int32_t *>(smem);
    const size_t hbytes = ((size_t)NSPLIT * T * 128u + 15u) & ~(size_t)15u;
    const uint32_t histAddr = smem_addr(hist);
    const uint32_t bufAddr = histAddr + (uint32_t)hbytes;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const uint32_t histLane = histAddr + (uint32_t)lane * 4u;
    const uint32_t HOFF = (uint32_t)T * 128u;
    for (int i = tid; i < NSPLIT * T * 32; i += blockDim.x) hist[i] = 0;
    pdl_wait();             // a programmatic dependent: the tile's vertex bins from here on
    pdl_trigger();
    const int64_t cb = P.nchunks * blockIdx.x / gridDim.x, ce = P.nchunks * (blockIdx.x + 1) / gridDim.x;

    // window rows of this thread's copies of chunk c (vertex id, or -1) and the chunk's width u
    auto load_vids = [&](int64_t c, int *v, int &u) {
        u = (c < ce) ? __ldg(P.cnu + c) : -1;
#pragma unroll
        for (int i = 0; i < NCP; ++i) {
            const int q = tid + i * kSimplexThreads;
            v[i] = (q < 4 * u) ? __ldg(P.cverts + c * kWinRows + (q >> 2)) : -1;
        }
    };
    // cp.async of chunk c into buffer buf: 4u window pieces, then ids, then weights (the last
    // pieces of the lists are zero-filled beyond their ends)
    auto issue = [&](int buf, int64_t c, const int *v, int u) {
        if (u >= 0) {
            const int64_t s0 = c * C;
            const int ns = (int)(P.k - s0 < (int64_t)C ? P.k - s0 : (int64_t)C);
            const int idb = ns * M * 2, wtb = ns * 8;
            const int nid = (idb + 15) / 16, nwt = (wtb + 15) / 16;
            const uint32_t b0 = bufAddr + (uint32_t)buf * kStageBytes;
            const unsigned char *ids = reinterpret_cast<const unsigned char *>(P.local + s0 * M);
            const unsigned char *wts = reinterpret_cast<const unsigned char *>(P.swp + s0);
#pragma unroll
            for (int i = 0; i < NCP; ++i) {
                const int q = tid + i * kSimplexThreads;
                if (q < 4 * u) {
                    cp_async16(b0 + (uint32_t)q * 16u, P.bins + (int64_t)v[i] * 32 + (q & 3) * 8);
                } else if (q < 4 * u + nid) {
                    const int r = q - 4 * u;
                    cp_async16_n(b0 + kWinBytes + (uint32_t)r * 16u, ids + r * 16, min(16, idb - r * 16));
                } else if (q < 4 * u + nid + nwt) {
                    const int r = q - 4 * u - nid;
                    cp_async16_n(b0 + kWinBytes + kIdBytes + (uint32_t)r * 16u, wts + r * 16, min(16, wtb - r * 16));
                }
            }
        }
        cp_async_commit();
    };

    int vA[NCP], vB[NCP], uA, uB;
    load_vids(cb, vA, uA);
    issue(0, cb, vA, uA);
    load_vids(cb + 1, vB, uB);
    int since = 0, u = uA;
    for (int64_t c = cb; c < ce; ++c) {
        const int buf = (int)((c - cb) & 1);
        issue(buf ^ 1, c + 1, vB, uB);          // chunk c + 1 (nothing when past the range)
        const int unext = uB;
        load_vids(c + 2, vB, uB);               // consumed by the next iteration's issue
        cp_async_wait<1>();                     // this thread's copies of chunk c are done
        __syncthreads();                        // and everyone's (and the histogram is cleared)
        const int64_t s0 = c * C;
        const int ns = (int)(P.k - s0 < (int64_t)C ? P.k - s0 : (int64_t)C);
        if (u >= 0) {
            const uint32_t b0 = bufAddr + (uint32_t)buf * kStageBytes;
            const uint32_t winLane = b0 + 2u * (uint32_t)lane;
            for (int bb = wid * GS; bb < ns; bb += nw * GS)
                gather_group_staged<NSPLIT, M, GS>(b0 + kWinBytes + 2u * (uint32_t)(bb * M),
                                                   b0 + kWinBytes + kIdBytes + 8u * (uint32_t)bb, min(GS, ns - bb),
                                                   winLane, histLane, HOFF);
        } else {
            const uint16_t *gb = P.bins + lane;
            for (int bb = wid * GS; bb < ns; bb += nw * GS) {
                const int n = min(GS, ns - bb);
                const int32_t *ids = P.simp + (s0 + bb) * M;
                if (n == GS)
                    gather_group<NSPLIT, M, GS, true>(ids, 0, P.swp + s0 + bb, n, gb, histLane, HOFF);
                else
                    gather_group<NSPLIT, M, GS, false>(ids, 0, P.swp + s0 + bb, n, gb, histLane, HOFF);
            }
        }
        __syncthreads();                        // buffer buf is free for chunk c + 2
        if (++since >= P.flush_every) {
            simplex_flush<NSPLIT>(hist, T, P.dtile, P.d, P.out);
            since = 0;
        }
        u = unext;
    }
    cp_async_wait<0>();
    if (since > 0) simplex_flush<NSPLIT>(hist, T, P.dtile, P.d, P.out);
}

// ------------------------------------------------------------------ default range

constexpr int kMaxAbsDirs = 1024;

// The default range M = max over directions p and vertices v of |h_p(v)| (Section 3), exactly in
// float64, without evaluating every (p, v):
//   1. the vertex v* of largest norm (float32, argmax only);
//   2. L = max_p |h_p(v*)| in float64, a lower bound of M, and Smax >= max_p |s_p|;
//   3. the candidates: vertices with |x| Smax (rounded up, with margin for the float32 copy of x
//      and the float64 roundings of h) >= L; no other vertex can reach M (Cauchy-Schwarz);
//   4. for each candidate and direction, a float32 height with an error bound E, and the float64
//      height wherever |h| + E >= L.
// Typical point sets leave a handful of candidates; in the worst case (every vertex at the same
// norm) step 4 covers all vertices, as a plain screened pass would.
template <int N>
__global__ void __launch_bounds__(256) vertex_norm_argmax_kernel(const float *__restrict__ xf, int64_t nv,
                                                                 unsigned long long *key)
{
    unsigned long long best = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const float x = __ldg(xf + v * N + a);
            s = __fmaf_rn(x, x, s);
        }
        best = max(best, ((unsigned long long)__float_as_uint(s) << 32) | (unsigned long long)(uint32_t)v);
    }
    for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

// One block: L and Smax (step 2).  M starts at L; cand = {count, L rounded down, Smax, 0, list}.
template <int N>
__global__ void __launch_bounds__(256) range_lower_bound_kernel(const double *__restrict__ coords,
                                                                const double *__restrict__ dirs, int d,
                                                                const unsigned long long *key,
                                                                unsigned long long *Mbits, int *cand)
{
    __shared__ double sb[32];
    __shared__ float ss[32];
    const int v = (int)(uint32_t)(*key & 0xffffffffull);
    double xd[N];
#pragma unroll
    for (int a = 0; a < N; ++a) xd[a] = coords[(int64_t)v * N + a];
    double best = 0.0;
    float smax = 0.f;
    for (int p = threadIdx.x; p < d; p += blockDim.x) {
        best = fmax(best, fabs(heightv<N>(xd, dirs + (int64_t)p * N)));
        float s2 = 0.f;
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const float sa = __double2float_ru(fabs(dirs[(int64_t)p * N + a]));
            s2 = __fmaf_ru(sa, sa, s2);
        }
        smax = fmaxf(smax, __fsqrt_ru(s2));
    }
    for (int off = 16; off > 0; off >>= 1) {
        best = fmax(best, __shfl_down_sync(0xffffffffu, best, off));
        smax = fmaxf(smax, __shfl_down_sync(0xffffffffu, smax, off));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        sb[wid] = best;
        ss[wid] = smax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
            best = fmax(best, sb[w]);
            smax = fmaxf(smax, ss[w]);
        }
        atomicMax(Mbits, (unsigned long long)__double_as_longlong(best));
        cand[1] = __float_as_int(__double2float_rd(best));
        cand[2] = __float_as_int(smax);
    }
}

// Step 3: append every vertex whose norm bound reaches L to the list (warp-aggregated).
template <int N>
__global__ void __launch_bounds__(256) range_candidates_kernel(const float *__restrict__ xf, int64_t nv, int *cand)
{
    const float L = __int_as_float(cand[1]), Smax = __int_as_float(cand[2]);
    const int lane = threadIdx.x & 31;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < nv;
         v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + lane;
        bool c = false;
        if (v < nv) {
            float s = 0.f;
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const float x = fabsf(__ldg(xf + v * N + a));
                s = __fmaf_ru(x, x, s);
            }
            // |x| <= |x~| (1 + 2^-24) for the float32 copy x~; the float64 height rounds by far
            // less than the 2^-20 margin
            const float ub = __fadd_ru(__fmul_ru(__fmul_ru(__fsqrt_ru(s), Smax), 1.0f + 0x1p-20f), 0x1p-100f);
            c = ub >= L;
        }
        const unsigned m = __ballot_sync(0xffffffffu, c);
        if (m) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&cand[0], __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (c) cand[4 + base + __popc(m & ((1u << lane) - 1u))] = (int)v;
        }
    }
}

// Step 4: warps over candidates, lanes over a shared-memory chunk of directions.
template <int N>
__global__ void __launch_bounds__(256) max_abs_candidates_kernel(const double *__restrict__ coords,
                                                                 const float *__restrict__ xf,
                                                                 const double *__restrict__ dirs, int d,
                                                                 const int *__restrict__ cand,
                                                                 unsigned long long *Mbits)
{
    __shared__ float sd[kMaxAbsDirs][N];
    const int count = cand[0];
    const float L = __int_as_float(cand[1]);
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int p0 = 0; p0 < d; p0 += kMaxAbsDirs) {
        const int np = min(kMaxAbsDirs, d - p0);
        __syncthreads();
        for (int i = threadIdx.x; i < np * N; i += blockDim.x) sd[i / N][i % N] = __double2float_rn(dirs[(int64_t)p0 * N + i]);
        __syncthreads();
        for (int64_t ci = gw; ci < count; ci += nw) {
            const int v = cand[4 + ci];
            float x[N];
#pragma unroll
            for (int a = 0; a < N; ++a) x[a] = __ldg(xf + (int64_t)v * N + a);
            for (int j = lane; j < np; j += 32) {
                float h = 0.f, mag = 0.f;
#pragma unroll
                for (int a = N - 1; a >= 0; --a) {
                    h = __fmaf_rn(x[a], sd[j][a], h);
                    mag = __fmaf_ru(fabsf(x[a]), fabsf(sd[j][a]), mag);
                }
                const float E = __fmul_ru(mag, 0x1p-19f) + 0x1p-126f;
                if (__fadd_ru(fabsf(h), E) >= L) {
                    const double hd = fabs(heightv<N>(coords + (int64_t)v * N, dirs + (int64_t)(p0 + j) * N));
                    atomicMax(Mbits, (unsigned long long)__double_as_longlong(hd));
                }
            }
        }
    }
}

// ------------------------------------------------------------------ weights, adjoint, ECF

template <int M>
__global__ void simplex_weights_max_kernel(const int32_t *simp, int64_t k, const int64_t *vw, int64_t *sw)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = vw[simp[b * M]];
#pragma unroll
        for (int j = 1; j < M; ++j) m = max(m, vw[simp[b * M + j]]);
        sw[b] = m;
    }
}

// Adjoint of the simplex scatter for one dimension and one direction tile: per simplex
// g = sum_p S[p][max_j bin_p(v_j)], routed to the heaviest vertex (ties: lowest id) and summed
// exactly in 128 bits (lo word with carry into the hi word).
template <int M>
__global__ void simplex_bwd_kernel(const int32_t *simp, int64_t k, int sign, const int64_t *vw, const uint16_t *bins,
                                   int Dt, int dtile, int d, int T, const int64_t *S, unsigned long long *Iacc)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        int vid[M];
        for (int j = 0; j < M; ++j) vid[j] = (M == 1) ? (int)b : simp[b * M + j];
        int arg = vid[0];
        int64_t wm = vw[arg];
        for (int j = 1; j < M; ++j) {
            const int64_t w = vw[vid[j]];
            if (w > wm || (w == wm && vid[j] < arg)) {
                wm = w;
                arg = vid[j];
            }
        }
        long long g = 0;
        for (int c = 0; c < Dt; ++c) {
            const int p = dtile * Dt + c;
            if (p >= d) break;
            int bin = 0;
            for (int j = 0; j < M; ++j) bin = max(bin, (int)bins[(int64_t)vid[j] * Dt + c]);
            g += S[(int64_t)p * T + bin];
        }
        if (sign < 0) g = -g;
        const unsigned long long old = atomicAdd(Iacc + 2 * (int64_t)arg, (unsigned long long)g);
        const unsigned long long carry = (old + (unsigned long long)g < old) ? 1ull : 0ull;
        const unsigned long long hiadd = (unsigned long long)((g < 0 ? -1ll : 0ll) + (long long)carry);
        if (hiadd) atomicAdd(Iacc + 2 * (int64_t)arg + 1, hiadd);
    }
}

// grad[v] = I_v * scale, with the scale from device memory when scale_dev is not null.
__global__ void i128_to_grad_kernel(const unsigned long long *Iacc, int64_t nv, double scale, const double *scale_dev,
                                    float *grad)
{
    const double sc = scale_dev ? *scale_dev : scale;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x)
        grad[v] = (float)(i128_to_double((int64_t)Iacc[2 * v + 1], Iacc[2 * v]) * sc);
}

// WECF scatter of one list of M-vertex simplices for caller filters (Algorithm 1 with the vertex
// filter's bins): each simplex's bin is the max of its vertex bins (Eq. "msi"), its signed
// weight (or +-1) goes to a per-block histogram (int32, or int64 with H64) flushed once into
// the int64 output, or with GHIST straight to the output.  blockIdx.y selects the filter.
template <int M, bool H64, bool GHIST>
__global__ void __launch_bounds__(256) simplex_ecf_kernel(const int32_t *simp, const int64_t *sw, int64_t k, int sign,
                                                          int weighted, const uint16_t *bins, int T,
                                                          unsigned long long *out, int64_t nv)
{
    using H = typename std::conditional<H64, unsigned long long, int>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    H *h = reinterpret_cast<H *>(smem);
    bins += (int64_t)blockIdx.y * nv;       // filter blockIdx.y of [m][nv] bins, row of [m][T] out
    out += (int64_t)blockIdx.y * T;
    if (!GHIST) {
        for (int i = threadIdx.x; i < T; i += blockDim.x) h[i] = 0;
        __syncthreads();
    }
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        int bin = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) bin = max(bin, (int)bins[(M == 1) ? b : simp[b * M + j]]);
        const long long w = weighted ? (long long)sw[b] : 1ll;
        const long long v = sign > 0 ? w : -w;
        if (GHIST) atomicAdd(out + bin, (unsigned long long)v);
        else if (H64) atomicAdd(&h[bin], (unsigned long long)v);
        else atomicAdd(&h[bin], (int)v);
    }
    if (!GHIST) {
        __syncthreads();
        for (int i = threadIdx.x; i < T; i += blockDim.x)
            if (h[i]) atomicAdd(out + i, (unsigned long long)(long long)h[i]);
    }
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_dir_filters(int n, const double *dirs, int d, int T, const double *range, float *tab,
                               cudaStream_t st)
{
    const unsigned g = (unsigned)((d + 127) / 128);
    if (n == 1) dir_filter_kernel<1><<<g, 128, 0, st>>>(dirs, d, T, range, tab);
    else if (n == 2) dir_filter_kernel<2><<<g, 128, 0, st>>>(dirs, d, T, range, tab);
    else if (n == 3) dir_filter_kernel<3><<<g, 128, 0, st>>>(dirs, d, T, range, tab);
    else dir_filter_kernel<4><<<g, 128, 0, st>>>(dirs, d, T, range, tab);
    return cudaGetLastError();
}

cudaError_t launch_coords_to_f32(const double *x, int64_t n, float *xf, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    coords_to_f32_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(x, n, xf);
    return cudaGetLastError();
}

cudaError_t launch_vertex_bins(int n, const double *coords, const float *xf, int64_t nv, const double *dirs,
                               const float *tab, int d, int dtile, int Dt, int T, const double *beta, uint16_t *bins,
                               cudaStream_t st)
{
    const int threads = 256;
    const int vpb = threads / Dt;
    const unsigned g = (unsigned)std::min<int64_t>((nv + vpb - 1) / vpb, 152 * 16);
#define VB(NN) vertex_bins_kernel<NN><<<g, threads, 0, st>>>(coords, xf, nv, dirs, tab, d, dtile, Dt, T, beta, bins)
    if (n == 1) VB(1);
    else if (n == 2) VB(2);
    else if (n == 3) VB(3);
    else VB(4);
#undef VB
    return cudaGetLastError();
}

cudaError_t launch_vertex_scatter(int n, int nsplit, const SimplexFwdArgs &a, const double *coords, const float *xf,
                                  int64_t nv, const double *dirs, const float *tab, const double *beta, uint16_t *bins,
                                  int grid, cudaStream_t st)
{
    if (a.Dt != 32 || !a.swp) return cudaErrorInvalidValue;
    const size_t sm = (size_t)nsplit * a.T * 128u;
    cudaError_t e = cudaSuccess;
#define VS(NN, SS)                                                                                                   \
    do {                                                                                                             \
        e = cudaFuncSetAttribute(vertex_scatter_kernel<NN, SS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e == cudaSuccess)                                                                                        \
            e = launch_kernel(vertex_scatter_kernel<NN, SS>, dim3(grid), dim3(kSimplexThreads), sm, st, a.pdl != 0, a, \
                              coords, xf, nv, dirs, tab, beta, bins);                                                \
    } while (0)
    if (nsplit == 1) {
        if (n == 1) VS(1, 1); else if (n == 2) VS(2, 1); else if (n == 3) VS(3, 1); else VS(4, 1);
    } else {
        if (n == 1) VS(1, 2); else if (n == 2) VS(2, 2); else if (n == 3) VS(3, 2); else VS(4, 2);
    }
#undef VS
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

size_t simplex_fwd_smem(int nsplit, int T, int Dt) { return (size_t)nsplit * T * Dt * 4u; }

template <int NSPLIT, bool GH>
static cudaError_t launch_simplex_fwd_s(const SimplexFwdArgs &a, int grid, cudaStream_t st)
{
    const size_t sm = GH ? 0 : simplex_fwd_smem(NSPLIT, a.T, a.Dt);
    cudaError_t e = cudaSuccess;
#define SF(MM)                                                                                                      \
    do {                                                                                                            \
        e = cudaFuncSetAttribute(simplex_fwd_kernel<NSPLIT, MM, GH>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 (int)sm);                                                                          \
        if (e == cudaSuccess)                                                                                       \
            e = launch_kernel(simplex_fwd_kernel<NSPLIT, MM, GH>, dim3(grid), dim3(kSimplexThreads), sm, st,       \
                              a.pdl != 0, a);                                                                        \
    } while (0)
    switch (a.m) {
    case 1: SF(1); break;
    case 2: SF(2); break;
    case 3: SF(3); break;
    case 4: SF(4); break;
    default: SF(5); break;
    }
#undef SF
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_simplex_fwd(int nsplit, bool gh, const SimplexFwdArgs &a, int grid, cudaStream_t st)
{
    if (a.Dt != 32 || !a.swp) return cudaErrorInvalidValue;
    if (gh) return launch_simplex_fwd_s<1, true>(a, grid, st);
    return nsplit == 1 ? launch_simplex_fwd_s<1, false>(a, grid, st) : launch_simplex_fwd_s<2, false>(a, grid, st);
}

cudaError_t launch_pack_weights(const int64_t *sw, int64_t k, int sign, int nsplit, int2 *out, cudaStream_t st)
{
    if (k <= 0) return cudaSuccess;
    pack_weights_kernel<<<(unsigned)std::min<int64_t>((k + 255) / 256, 152 * 16), 256, 0, st>>>(sw, k, sign, nsplit, out);
    return cudaGetLastError();
}

cudaError_t launch_chunk_local(const int32_t *simp, int64_t k, int m, uint16_t *local, int32_t *cverts, int32_t *cnu,
                               cudaStream_t st)
{
    if (k <= 0 || m < 2) return cudaSuccess;
    const int64_t nch = (k + chunk_simplices(m) - 1) / chunk_simplices(m);
    switch (m) {
    case 2: chunk_local_kernel<2><<<(unsigned)nch, 512, 0, st>>>(simp, k, local, cverts, cnu); break;
    case 3: chunk_local_kernel<3><<<(unsigned)nch, 512, 0, st>>>(simp, k, local, cverts, cnu); break;
    case 4: chunk_local_kernel<4><<<(unsigned)nch, 512, 0, st>>>(simp, k, local, cverts, cnu); break;
    default: chunk_local_kernel<5><<<(unsigned)nch, 512, 0, st>>>(simp, k, local, cverts, cnu); break;
    }
    return cudaGetLastError();
}

size_t simplex_fwd_staged_smem(int nsplit, int T, int Dt)
{
    return (((size_t)nsplit * T * Dt * 4u + 15u) & ~(size_t)15u) + 2u * kStageBytes;
}

template <int NSPLIT>
static cudaError_t launch_simplex_fwd_staged_s(const SimplexFwdArgs &a, int grid, cudaStream_t st)
{
    const size_t sm = simplex_fwd_staged_smem(NSPLIT, a.T, a.Dt);
    cudaError_t e = cudaSuccess;
#define SS(MM)                                                                                                        \
    do {                                                                                                              \
        e = cudaFuncSetAttribute(simplex_fwd_staged_kernel<NSPLIT, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)sm);                                                                            \
        if (e == cudaSuccess)                                                                                         \
            e = launch_kernel(simplex_fwd_staged_kernel<NSPLIT, MM>, dim3(grid), dim3(kSimplexThreads), sm, st,      \
                              a.pdl != 0, a);                                                                          \
    } while (0)
    switch (a.m) {
    case 2: SS(2); break;
    case 3: SS(3); break;
    case 4: SS(4); break;
    default: SS(5); break;
    }
#undef SS
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_simplex_fwd_staged(int nsplit, const SimplexFwdArgs &a, int grid, cudaStream_t st)
{
    if (a.Dt != 32 || a.m < 2 || a.m > kMaxSimplexDim + 1 || !a.swp) return cudaErrorInvalidValue;
    return nsplit == 1 ? launch_simplex_fwd_staged_s<1>(a, grid, st) : launch_simplex_fwd_staged_s<2>(a, grid, st);
}

cudaError_t launch_simplicial_max_abs(int n, const double *coords, const float *xf, int64_t nv, const double *dirs,
                                      int d, unsigned long long *Mbits, unsigned long long *key, int *cand,
                                      cudaStream_t st)
{
    if (nv <= 0) return cudaSuccess;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nv + 255) / 256, 152 * 8));
    cudaError_t e = cudaMemsetAsync(cand, 0, 4 * sizeof(int), st);
    if (e != cudaSuccess) return e;
#define MA(NN)                                                                                          \
    do {                                                                                                \
        vertex_norm_argmax_kernel<NN><<<g, 256, 0, st>>>(xf, nv, key);                                 \
        range_lower_bound_kernel<NN><<<1, 256, 0, st>>>(coords, dirs, d, key, Mbits, cand);            \
        range_candidates_kernel<NN><<<g, 256, 0, st>>>(xf, nv, cand);                                  \
        max_abs_candidates_kernel<NN><<<g, 256, 0, st>>>(coords, xf, dirs, d, cand, Mbits);            \
    } while (0)
    if (n == 1) MA(1);
    else if (n == 2) MA(2);
    else if (n == 3) MA(3);
    else MA(4);
#undef MA
    return cudaGetLastError();
}

cudaError_t launch_simplex_weights_max(const int32_t *simp, int64_t k, int m, const int64_t *vw, int64_t *sw,
                                       cudaStream_t st)
{
    if (k <= 0) return cudaSuccess;
    const unsigned g = (unsigned)std::min<int64_t>((k + 255) / 256, 4096);
    switch (m) {
    case 2: simplex_weights_max_kernel<2><<<g, 256, 0, st>>>(simp, k, vw, sw); break;
    case 3: simplex_weights_max_kernel<3><<<g, 256, 0, st>>>(simp, k, vw, sw); break;
    case 4: simplex_weights_max_kernel<4><<<g, 256, 0, st>>>(simp, k, vw, sw); break;
    default: simplex_weights_max_kernel<5><<<g, 256, 0, st>>>(simp, k, vw, sw); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_simplicial_bwd(int n, const double *coords, const float *xf, int64_t nv, const int32_t *const *simp,
                                  const int64_t *counts, int max_dim, const int64_t *vw, const double *dirs, int d,
                                  int T, const float *tab, const double *beta, const int64_t *S,
                                  uint16_t *bins, unsigned long long *Iacc, float *grad, double scale,
                                  const double *scale_dev, cudaStream_t st)
{
    const int Dt = 32;
    cudaError_t e = cudaMemsetAsync(Iacc, 0, (size_t)nv * 16u, st);
    if (e != cudaSuccess) return e;
    for (int dt = 0; dt * Dt < d; ++dt) {
        if ((e = launch_vertex_bins(n, coords, xf, nv, dirs, tab, d, dt, Dt, T, beta, bins, st)) != cudaSuccess) return e;
        for (int i = 0; i <= max_dim; ++i) {
            const int64_t k = counts[i];
            if (k <= 0) continue;
            const unsigned g = (unsigned)std::min<int64_t>((k + 255) / 256, 4096);
            const int sign = (i & 1) ? -1 : 1;
            switch (i) {
            case 0: simplex_bwd_kernel<1><<<g, 256, 0, st>>>(nullptr, k, sign, vw, bins, Dt, dt, d, T, S, Iacc); break;
            case 1: simplex_bwd_kernel<2><<<g, 256, 0, st>>>(simp[1], k, sign, vw, bins, Dt, dt, d, T, S, Iacc); break;
            case 2: simplex_bwd_kernel<3><<<g, 256, 0, st>>>(simp[2], k, sign, vw, bins, Dt, dt, d, T, S, Iacc); break;
            case 3: simplex_bwd_kernel<4><<<g, 256, 0, st>>>(simp[3], k, sign, vw, bins, Dt, dt, d, T, S, Iacc); break;
            default: simplex_bwd_kernel<5><<<g, 256, 0, st>>>(simp[4], k, sign, vw, bins, Dt, dt, d, T, S, Iacc); break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    i128_to_grad_kernel<<<(unsigned)std::min<int64_t>((nv + 255) / 256, 4096), 256, 0, st>>>(Iacc, nv, scale, scale_dev,
                                                                                                 grad);
    return cudaGetLastError();
}

template <int M, bool H, bool G>
static cudaError_t launch_simplex_ecf_t(dim3 g, size_t sm, const int32_t *simp, const int64_t *sw, int64_t k, int sign,
                                        int weighted, const uint16_t *bins, int T, unsigned long long *out, int64_t nv,
                                        cudaStream_t st)
{
    if (sm > 48u * 1024u) {
        cudaError_t e = cudaFuncSetAttribute(simplex_ecf_kernel<M, H, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (e != cudaSuccess) return e;
    }
    simplex_ecf_kernel<M, H, G><<<g, 256, sm, st>>>(simp, sw, k, sign, weighted, bins, T, out, nv);
    return cudaGetLastError();
}

template <int M>
static cudaError_t launch_simplex_ecf_m(bool h64, bool ghist, dim3 g, size_t sm, const int32_t *simp,
                                        const int64_t *sw, int64_t k, int sign, int weighted, const uint16_t *bins,
                                        int T, unsigned long long *out, int64_t nv, cudaStream_t st)
{
    if (ghist) return launch_simplex_ecf_t<M, true, true>(g, sm, simp, sw, k, sign, weighted, bins, T, out, nv, st);
    if (h64) return launch_simplex_ecf_t<M, true, false>(g, sm, simp, sw, k, sign, weighted, bins, T, out, nv, st);
    return launch_simplex_ecf_t<M, false, false>(g, sm, simp, sw, k, sign, weighted, bins, T, out, nv, st);
}

// Signed scatter of one simplex list for m filters: int32 shared histograms when enough blocks
// keep each block's sum of |weight| (at most wbound per simplex) below 2^30, int64 otherwise,
// global atomics when the histogram does not fit in shared memory.
cudaError_t launch_simplex_ecf(const int32_t *simp, const int64_t *sw, int64_t k, int m, int sign, int weighted,
                               int64_t wbound, const uint16_t *bins, int T, unsigned long long *out, int64_t nv,
                               int nf, cudaStream_t st)
{
    if (k <= 0) return cudaSuccess;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int64_t maxblocks = (k + 255) / 256;
    const double wb = weighted ? (double)std::max<int64_t>(wbound, 1) : 1.0;
    const double need = std::ceil((double)k * wb / 1073741824.0) + 1.0;
    const bool h64 = need > (double)maxblocks;
    size_t sm = (size_t)T * (h64 ? 8u : 4u);
    const bool ghist = sm + 1024 > (size_t)optin;
    if (ghist) sm = 0;
    int64_t per = std::max<int64_t>(1, (int64_t)std::max(sms, 1) * 4 / std::max(nf, 1));
    if (!h64) per = std::max<int64_t>(per, (int64_t)need);
    const dim3 g((unsigned)std::min<int64_t>(maxblocks, per), (unsigned)nf);
    switch (m) {
    case 1: return launch_simplex_ecf_m<1>(h64, ghist, g, sm, simp, sw, k, sign, weighted, bins, T, out, nv, st);
    case 2: return launch_simplex_ecf_m<2>(h64, ghist, g, sm, simp, sw, k, sign, weighted, bins, T, out, nv, st);
    case 3: return launch_simplex_ecf_m<3>(h64, ghist, g, sm, simp, sw, k, sign, weighted, bins, T, out, nv, st);
    case 4: return launch_simplex_ecf_m<4>(h64, ghist, g, sm, simp, sw, k, sign, weighted, bins, T, out, nv, st);
    default: return launch_simplex_ecf_m<5>(h64, ghist, g, sm, simp, sw, k, sign, weighted, bins, T, out, nv, st);
    }
}

}  // namespace wect
