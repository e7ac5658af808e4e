// wect_cubical_bwd.cu -- the adjoint of the cubical (stencil) WECT with respect to the vertex
// weights (sm_103a).
//
// The forward scatters c_o(v) into diff_p[bin_p(v)] for the directions p of octant o (see
// wect_cubical.cu); c_o(v) sums the signed weights of the cells whose sign corner is v, and a
// cell's weight is the max of its vertex weights.  The chain rule therefore runs in two steps:
//   1. octant sums   Rv[o][v] = sum over p in octant o of S[p][bin_p(v)], with S the suffix
//      sums of the upstream gradient over the thresholds (the prefix sum of the forward, read
//      backwards);
//   2. routing       I_v = sum over cells s containing v whose heaviest vertex is v of
//      (-1)^dim(s) sum_o Rv[o][corner_o(s)]   (ties of the heaviest vertex go to the lowest
//      vertex index).
// Both are exact integer sums.  Bins are recomputed with the same float32 filter and float64
// fix-ups as the forward, not stored.
#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

// ------------------------------------------------------------------ backward

constexpr int kRsumG = 4;    // directions per group in the adjoint's octant sums

// Slots of the adjoint's direction table: octant-sorted directions, each octant padded to a
// multiple of kRsumG (an upper bound that does not depend on the octant counts).
__host__ __device__ inline int rsum_slots(int n, int d)
{
    return (d + (1 << n) * (kRsumG - 1) + kRsumG - 1) / kRsumG * kRsumG;
}

// Byte offsets of the adjoint kernel's shared memory.
struct RsumLayout {
    size_t ss, dfil, slotk, tab, flags, total;
};

__host__ __device__ inline RsumLayout rsum_layout(int n, int d, int T, int R)
{
    const int NS = rsum_slots(n, d);
    RsumLayout l;
    l.ss = 0;
    l.dfil = (size_t)(d + 1) * T * 8u;
    l.slotk = l.dfil + (size_t)d * sizeof(DirFilter);
    l.tab = (l.slotk + (size_t)NS * 4u + 15u) & ~(size_t)15u;
    l.flags = l.tab + (size_t)R * NS * 16u;
    l.total = l.flags + (size_t)R * (NS / kRsumG) + 16u;   // the flag loop reads one group ahead
    return l;
}


// Per-vertex octant sums of the suffix-scanned upstream gradient,
//     Rv[o][v] = sum over directions p of octant o of S[p][bin_p(v)]   (octant-major planes),
// for one item (complex, row range).  Each lane takes two vertices of a row, 32 apart, which
// share every table load; the direction loop is uniform across the warp and visits the
// directions octant by octant, kRsumG at a time, two per packed float32x2 filter step.
//
// Shared memory: the suffix table of the complex in octant order ([d + 1][T] int64, row d all
// zero), the direction filters, and per row tile a [R][slots] table of filter constants
// {S0, Glo, Ghi, W} with the constants of two neighbouring slots interleaved.  Slots are the
// octant-sorted directions with each octant padded to a multiple of kRsumG; a padding slot has
// S0 = Glo = Ghi = 0 and reads the zero row.  W is the shared address of the suffix row minus the
// magic bias, so the candidate bin's entry sits at (thi << 3) + W.  A group flag marks groups
// whose bins may leave [0, T-1] in that row; they take the clamped path.  Undecided bins are
// fixed with the exact float64 height.
// Shared-memory context of one item of the adjoint's octant sums.
struct RsumCtx {
    uint32_t ssAddr;              // suffix table [d + 1][T] (row d zero)
    const int *slotk;             // slot -> octant-sorted direction, -1 for padding
    const DirFilter *dfil;        // direction filters
    const int *L;                 // grid sides
    int T, d;
};

// Candidate suffix-table addresses of the kRsumG slots of group gi for the two vertices of a lane
// (k0 = KA, KB packed twice), from the row's filter table at address e.  With clampg the bins
// are clamped to [0, T-1] (the group may leave the range in this row).  Returns nonzero when a
// bin is undecided; with non-null t/h it also returns the filter ends.
template <int N>
__device__ __forceinline__ int rsum_group(uint32_t e, int gi, bool clampg, F2 KA, F2 KB, F2 M2, const RsumCtx &C,
                                          int i1, int i2, uint32_t *adA, uint32_t *adB, int *tAo, int *hAo,
                                          int *tBo, int *hBo)
{
    constexpr int G = kRsumG;
    int hA[G], hB[G];
    int bad = 0;
#pragma unroll
    for (int u = 0; u < G; u += 2) {
        unsigned long long s0, gl, gh, ww;
        lds_v2u64(e + u * 16u, s0, gl);
        lds_v2u64(e + u * 16u + 16u, gh, ww);
        int t0, t1, t2, t3;
        filter_ceil2(KA, F2{s0}, F2{gl}, F2{gh}, M2, t0, hA[u], t1, hA[u + 1]);
        filter_ceil2(KB, F2{s0}, F2{gl}, F2{gh}, M2, t2, hB[u], t3, hB[u + 1]);
        bad |= (t0 ^ hA[u]) | (t1 ^ hA[u + 1]) | (t2 ^ hB[u]) | (t3 ^ hB[u + 1]);
        if (tAo) {
            tAo[u] = t0;
            tAo[u + 1] = t1;
            tBo[u] = t2;
            tBo[u + 1] = t3;
        }
        const uint32_t w0 = (uint32_t)ww, w1 = (uint32_t)(ww >> 32);
        adA[u] = ((uint32_t)hA[u] << 3) + w0;
        adA[u + 1] = ((uint32_t)hA[u + 1] << 3) + w1;
        adB[u] = ((uint32_t)hB[u] << 3) + w0;
        adB[u + 1] = ((uint32_t)hB[u + 1] << 3) + w1;
    }
    if (clampg) {
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int k = C.slotk[gi * G + u];
            int nr = 0, kr = C.d;
            if (k >= 0) {
                nr = make_row_filter<N>(C.dfil[k], i1, i2, C.L).nr;
                kr = k;
            }
            const uint32_t rowAddr = C.ssAddr + 8u * (uint32_t)(kr * C.T);
            adA[u] = rowAddr + 8u * (uint32_t)(k >= 0 ? clamp_bin(hA[u], nr, C.T) : 0);
            adB[u] = rowAddr + 8u * (uint32_t)(k >= 0 ? clamp_bin(hB[u], nr, C.T) : 0);
        }
    }
    if (hAo) {
#pragma unroll
        for (int u = 0; u < G; ++u) {
            hAo[u] = hA[u];
            hBo[u] = hB[u];
        }
    }
    return bad;
}

// An octant sum as two int32 halves, value = hi * 2^32 + lo with lo the signed low word (so hi
// is the high word plus one when lo < 0).  The routing kernel then multiplies each half by its
// small coefficient with one 32 x 32 -> 64 multiply-add.  |value| < 2^63 / 3^n keeps hi in range.
__device__ __forceinline__ void store_split(int64_t *p, long long v, bool accumulate)
{
    if (accumulate) {            // a later direction chunk: add to the stored sum
        const int2 old = *reinterpret_cast<const int2 *>(p);
        v += (long long)(((unsigned long long)(long long)old.y << 32) + (unsigned long long)(long long)old.x);
    }
    const int lo = (int)(unsigned int)((unsigned long long)v & 0xffffffffull);
    const int hi = (int)((v - (long long)lo) >> 32);
    *reinterpret_cast<int2 *>(p) = make_int2(lo, hi);
}

template <int N>
__global__ void __launch_bounds__(1024, 1) cubical_bwd_rsum_kernel(const CubicalBwdArgs P)
{
    constexpr int NOCT = 1 << N;
    constexpr int G = kRsumG;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sb[NOCT + 1];
    const int T = P.T, d = P.d, RB = P.R;
    const int NS = rsum_slots(N, d), NG = NS / G;
    const RsumLayout lay = rsum_layout(N, d, T, RB);
    long long *Ss = reinterpret_cast<long long *>(smem + lay.ss);
    DirFilter *dfil = reinterpret_cast<DirFilter *>(smem + lay.dfil);
    int *slotk = reinterpret_cast<int *>(smem + lay.slotk);
    uint8_t *flags = smem + lay.flags;
    const uint32_t ssAddr = smem_addr(Ss), tabAddr = smem_addr(smem + lay.tab);
    const double lo = P.range[0], hi = P.range[1], step = P.range[2];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;

    if (tid == 0) {
        int s = 0;
        for (int o = 0; o < NOCT; ++o) {
            sb[o] = s;
            s += (P.octb[o + 1] - P.octb[o] + G - 1) / G * G;
        }
        sb[NOCT] = s;
    }
    __syncthreads();
    for (int j = tid; j < NS; j += blockDim.x) {
        int k = -1;
        for (int o = 0; o < NOCT; ++o)
            if (j >= sb[o] && j < sb[o + 1] && P.octb[o] + (j - sb[o]) < P.octb[o + 1]) k = P.octb[o] + (j - sb[o]);
        slotk[j] = k;
    }
    const uint32_t zeroW = ssAddr + 8u * (uint32_t)(d * T) - 8u * (uint32_t)kMagicBits;
    const int it0 = P.item_ranges ? P.item_ranges[blockIdx.x] : (int)blockIdx.x;
    const int it1 = P.item_ranges ? P.item_ranges[blockIdx.x + 1] : (int)blockIdx.x + 1;
    int staged = -1;                        // complex whose suffix rows and filters are staged
    for (int item = it0; item < it1; ++item) {
        const WorkItem W = P.items[item];
        const GridDesc g = P.grids[W.cx];
        const int L0 = g.L[0], L1 = g.L[1];
        if (W.cx != staged) {
            // the suffix rows of this complex (octant order; row d zero) and its direction filters
            __syncthreads();                    // the previous complex's readers are done
            const long long *S = reinterpret_cast<const long long *>(P.S) + ((int64_t)W.cx * P.d_all + P.p0) * T;
            for (int idx = tid; idx < (d + 1) * T; idx += blockDim.x) {
                const int k = idx / T, q = idx - k * T;
                Ss[idx] = (k < d) ? S[(int64_t)P.perm[k] * T + q] : 0ll;
            }
            for (int k = tid; k < d; k += blockDim.x) {
                const int p = P.perm[k];
                double sv[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int a = 0; a < N; ++a) sv[a] = P.dirs[(int64_t)p * N + a];
                dfil[k] = make_dir_filter<N>(sv, g.L, lo, hi, step, T);
            }
            staged = W.cx;
        }
        const int segs = (L0 + 63) >> 6;
        const RsumCtx C{ssAddr, slotk, dfil, g.L, T, d};
        for (int rt = W.r0; rt < W.r1; rt += RB) {
            const int nrt = min(RB, W.r1 - rt);
            __syncthreads();
            // filter table of the row tile: one warp per row, lanes over slots
            for (int rl = wid; rl < nrt; rl += nwarps) {
                const int r = rt + rl, i1 = r % L1, i2 = r / L1;
                for (int j0 = 0; j0 < NS; j0 += 32) {
                    const int j = j0 + lane;
                    const int k = (j < NS) ? slotk[j] : -1;
                    float S0 = 0.f, Glo = 0.f, Ghi = 0.f;
                    uint32_t Wj = zeroW;
                    unsigned cf = 0;
                    if (k >= 0) {
                        const DirFilter f = dfil[k];
                        const RowFilter rf = make_row_filter<N>(f, i1, i2, g.L);
                        // all bins of the row provably inside [0, T-1]?  (NaN/inf compare false)
                        const float A = __fmul_ru((float)(L0 - 1), fabsf(f.S0));
                        const float lowf = __fadd_rd(__fsub_rd(rf.Glo, A), (float)(rf.nr - 1));
                        const float highf = __fadd_ru(__fadd_ru(rf.Ghi, A), (float)(rf.nr + 1));
                        cf = (!(lowf >= 0.0f) || !(highf <= (float)(T - 1))) ? 1u : 0u;
                        S0 = f.S0;
                        Glo = rf.Glo;
                        Ghi = rf.Ghi;
                        Wj = ssAddr + 8u * (uint32_t)(k * T + rf.nr) - 8u * (uint32_t)kMagicBits;
                    }
                    cf |= __shfl_xor_sync(0xffffffffu, cf, 1);
                    cf |= __shfl_xor_sync(0xffffffffu, cf, 2);
                    if (j < NS) {
                        float *e = reinterpret_cast<float *>(smem + lay.tab + ((size_t)rl * NS + (j & ~1)) * 16u);
                        const int h = j & 1;
                        e[h] = S0;
                        e[2 + h] = Glo;
                        e[4 + h] = Ghi;
                        reinterpret_cast<uint32_t *>(e)[6 + h] = Wj;
                        if ((j & (G - 1)) == 0) flags[rl * NG + j / G] = (uint8_t)cf;
                    }
                }
            }
            __syncthreads();
            for (int job = wid; job < nrt * segs; job += nwarps) {
                const int rl = job / segs, seg = job - rl * segs;
                // two vertices per lane, 32 apart in the row
                const int ia = min(seg * 64 + lane, L0 - 1), ib = min(seg * 64 + 32 + lane, L0 - 1);
                const bool liveA = seg * 64 + lane < L0, liveB = seg * 64 + 32 + lane < L0;
                const int r = rt + rl, i1 = r % L1, i2 = r / L1;
                const float ka = (float)(2 * ia - (L0 - 1)), kb = (float)(2 * ib - (L0 - 1));
                const F2 KA = f2_pack(ka, ka), KB = f2_pack(kb, kb), M2 = f2_pack(kMagic, kMagic);
                const uint32_t rowTab = tabAddr + (uint32_t)(rl * NS) * 16u;
                const uint8_t *rowFlags = flags + rl * NG;
                const int64_t voutA = g.v_off + (int64_t)ia + (int64_t)L0 * r;
#pragma unroll 1
                for (int o = 0; o < NOCT; ++o) {
                    long long accA = 0, accB = 0;
                    const int g0 = sb[o] / G, g1 = sb[o + 1] / G;
                    int badOct = 0;
                    // fast pass: no vote and no flag load on the critical path (the next group's
                    // clamp flag is fetched one group ahead)
                    uint8_t fnext = rowFlags[g0];
#pragma unroll 1
                    for (int gi = g0; gi < g1; ++gi) {
                        const bool clampg = fnext != 0;
                        fnext = rowFlags[gi + 1];
                        uint32_t adA[G], adB[G];
                        badOct |= rsum_group<N>(rowTab + (uint32_t)gi * (G * 16u), gi, clampg, KA, KB, M2, C, i1, i2, adA,
                                                adB, nullptr, nullptr, nullptr, nullptr);
#pragma unroll
                        for (int u = 0; u < G; ++u) {
                            accA += lds_s64(adA[u]);
                            accB += lds_s64(adB[u]);
                        }
                    }
                    if (__any_sync(0xffffffffu, badOct != 0)) {
                        // undecided bins somewhere in this octant: replace their candidate entries
                        // by the entries of the exact float64 bins
#pragma unroll 1
                        for (int gi = g0; gi < g1; ++gi) {
                            uint32_t adA[G], adB[G];
                            int tA[G], hA[G], tB[G], hB[G];
                            if (!rsum_group<N>(rowTab + (uint32_t)gi * (G * 16u), gi, rowFlags[gi] != 0, KA, KB, M2, C, i1,
                                               i2, adA, adB, tA, hA, tB, hB))
                                continue;
#pragma unroll
                            for (int u = 0; u < G; ++u) {
                                const int k = slotk[gi * G + u];
                                if (k < 0) continue;
                                const double *sp = P.dirs + (int64_t)P.perm[k] * N;
                                if (tA[u] != hA[u]) {
                                    const int cand = (int)((adA[u] - ssAddr) >> 3) - k * T;
                                    const double h = height3<N>(gcoord(g, 0, ia), gcoord(g, 1, i1), gcoord(g, 2, i2), sp);
                                    accA += Ss[k * T + exact_bin_from(h, P.beta, T, cand)] - lds_s64(adA[u]);
                                }
                                if (tB[u] != hB[u]) {
                                    const int cand = (int)((adB[u] - ssAddr) >> 3) - k * T;
                                    const double h = height3<N>(gcoord(g, 0, ib), gcoord(g, 1, i1), gcoord(g, 2, i2), sp);
                                    accB += Ss[k * T + exact_bin_from(h, P.beta, T, cand)] - lds_s64(adB[u]);
                                }
                            }
                        }
                    }
                    if (liveA) store_split(P.Rv + (int64_t)o * P.total_nv + voutA, accA, P.accumulate != 0);
                    if (liveB) store_split(P.Rv + (int64_t)o * P.total_nv + voutA + 32, accB, P.accumulate != 0);
                }
            }
        }
    }   // items of this CTA
}

// Route each cell's gradient to its heaviest vertex:
//     I_v = sum over cells s containing v whose heaviest vertex is v (ties -> lowest index) of
//           (-1)^dim(s) sum_o Rv[o][corner_o(s)].
// Cells containing v are indexed like the 3^n neighbourhood: e in {-1,0,1}^n spans v and v + e.
// The neighbours that beat v (heavier, or as heavy with a lower index) form a bit mask; v is
// the heaviest vertex of a cell iff the mask misses every cell vertex, which gives the mask A
// of the cells v takes.  Under octant o (sg_a = +1 when bit a is set, else -1) the corner of a
// cell e is v + delta * sg with delta_a = [e_a == sg_a], so regrouping by (o, delta),
//     I_v = sum_o sum_delta K[o][delta] * Rv[o][v + delta * sg],
//     K[o][delta] = #(A & even cells of the class) - #(A & odd cells of the class),
// where the class of (o, delta) is the cells with e_a = sg_a on delta and e_a in {0, -sg_a}
// off it (computed below with one mask and one popcount each).  That is 2^n x 2^n coalesced
// loads per vertex and no divergence.  Every partial sum is
// a signed sum over at most 3^n cells of sums over disjoint direction sets, so with
// 3^n d max|S| < 2^63 (checked when the suffix table is built) int64 is exact.
__host__ __device__ constexpr int route_nb(int n) { return n == 1 ? 3 : (n == 2 ? 9 : 27); }

// Vertex mask (over the 3^n neighbourhood) of the cell with extent vector e = cell index t.
__host__ __device__ constexpr uint32_t route_cell_mask(int n, int t)
{
    uint32_t m = 0;
    for (int sub = 0; sub < (1 << n); ++sub) {
        int idx = 0, mul = 1;
        bool ok = true;
        for (int a = 0; a < n; ++a) {
            const int ea = (t / mul) % 3 - 1;
            int f = 0;
            if ((sub >> a) & 1) {
                if (ea == 0) ok = false;
                f = ea;
            }
            idx += (f + 1) * mul;
            mul *= 3;
        }
        if (ok) m |= 1u << idx;
    }
    return m;
}

// Cells of the class (o, delta) with even (par = 0) or odd (par = 1) dimension.
__host__ __device__ constexpr uint32_t route_class_mask(int n, int o, int delta, int par)
{
    uint32_t m = 0;
    for (int t = 0; t < route_nb(n); ++t) {
        int mul = 1, dim = 0;
        bool in = true;
        for (int a = 0; a < n; ++a) {
            const int ea = (t / mul) % 3 - 1;
            const int sg = ((o >> a) & 1) ? 1 : -1;
            dim += ea != 0;
            if ((delta >> a) & 1) in = in && ea == sg;
            else in = in && ea != sg;
            mul *= 3;
        }
        if (in && (dim & 1) == par) m |= 1u << t;
    }
    return m;
}

// Cells of odd dimension among the 3^n neighbourhood cells, and the population count of a mask
// (both for compile-time masks).
__host__ __device__ constexpr uint32_t route_odd_mask(int n)
{
    uint32_t m = 0;
    for (int t = 0; t < route_nb(n); ++t) {
        int mul = 1, dim = 0;
        for (int a = 0; a < n; ++a) {
            dim += (t / mul) % 3 != 1;
            mul *= 3;
        }
        if (dim & 1) m |= 1u << t;
    }
    return m;
}

__host__ __device__ constexpr int route_popcount(uint32_t m)
{
    int c = 0;
    for (; m; m &= m - 1) ++c;
    return c;
}

// Neighbourhood index of the corner v + delta * sg(o).
__host__ __device__ constexpr int route_corner(int n, int o, int delta)
{
    int idx = 0, mul = 1;
    for (int a = 0; a < n; ++a) {
        const int c = ((delta >> a) & 1) ? (((o >> a) & 1) ? 1 : -1) : 0;
        idx += (c + 1) * mul;
        mul *= 3;
    }
    return idx;
}

template <int N>
__global__ void __launch_bounds__(256) cubical_bwd_route_kernel(const CubicalBwdArgs P)
{
    constexpr int NOCT = 1 << N;
    constexpr int NB = route_nb(N);
    constexpr int CENTER = (NB - 1) / 2;
    const int64_t gid = P.v_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= P.v_end) return;
    int cx = 0;
    if (P.uniform_nv > 0) {
        cx = (int)(gid / P.uniform_nv);         // every grid of the batch has the same vertex count
    } else if (P.n_grids > 1) {
        int hi_c = P.n_grids - 1;
        while (cx < hi_c) {
            const int mid = (cx + hi_c + 1) >> 1;
            if (P.grids[mid].v_off <= gid) cx = mid; else hi_c = mid - 1;
        }
    }
    const GridDesc g = P.grids[cx];
    const int64_t v = gid - g.v_off;
    const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
    int i0, i1, i2;
    if (g.nv <= 0x7fffffff) {
        const uint32_t v32 = (uint32_t)v, q = v32 / (uint32_t)L0;
        i0 = (int)(v32 - q * (uint32_t)L0);
        i1 = (int)(q % (uint32_t)L1);
        i2 = (int)(q / (uint32_t)L1);
    } else {
        i0 = (int)(v % L0);
        i1 = (int)((v / L0) % L1);
        i2 = (int)(v / ((int64_t)L0 * L1));
    }
    const int32_t *wp = g.w + v;
    const int32_t wv = __ldg(wp);
    // neighbour offsets (flat, int32) and the "beats v" mask over the 3^n neighbourhood; a
    // position outside the grid counts as beating v, so that no cell holding it is v's
    const bool ox[3] = {i0 > 0, true, i0 < L0 - 1};
    const bool oy[3] = {i1 > 0, true, i1 < L1 - 1};
    const bool oz[3] = {i2 > 0, true, i2 < L2 - 1};
    int off[NB];
    uint32_t beat = 0;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const int dx = t % 3 - 1, dy = (N >= 2) ? (t / 3) % 3 - 1 : 0, dz = (N >= 3) ? t / 9 - 1 : 0;
        off[t] = dx + L0 * (dy + L1 * dz);
        const bool ok = ox[dx + 1] && oy[dy + 1] && oz[dz + 1];
        if (t != CENTER) {
            if (!ok) {
                beat |= 1u << t;
            } else {
                const int32_t wu = __ldg(wp + off[t]);
                // u's flat index is below v's iff its offset is lexicographically negative
                const bool below = (dz < 0) || (dz == 0 && (dy < 0 || (dy == 0 && dx < 0)));
                if (wu > wv || (wu == wv && below)) beat |= 1u << t;
            }
        }
    }
    // cells v takes: beaten nowhere (a cell leaving the grid holds a position that beats v)
    uint32_t A = 0;
#pragma unroll
    for (int t = 0; t < NB; ++t)
        if ((beat & route_cell_mask(N, t)) == 0) A |= 1u << t;
    // K = #(A & even & class) - #(A & odd & class) = #(X & class) - #(odd & class) with
    // X = A ^ odd: one mask and one popcount per coefficient, the second count a constant
    const uint32_t X = A ^ route_odd_mask(N);
    // the octant sums are stored as (lo, hi) int32 halves: sum K * lo and K * hi separately
    // (|K| <= 2^n, 4^n terms: both sums stay far inside int64), combined modulo 2^64 at the end
    long long acc_lo = 0, acc_hi = 0;
#pragma unroll
    for (int o = 0; o < NOCT; ++o) {
        const int2 *R = reinterpret_cast<const int2 *>(P.Rv) + (int64_t)o * P.total_nv + gid;
#pragma unroll
        for (int dl = 0; dl < NOCT; ++dl) {
            const uint32_t cls = route_class_mask(N, o, dl, 0) | route_class_mask(N, o, dl, 1);
            const int K = __popc(X & cls) - route_popcount(route_odd_mask(N) & cls);
            // K == 0 whenever the corner lies outside the grid (every cell of the class holds it)
            const int2 r = (K != 0) ? __ldg(R + off[route_corner(N, o, dl)]) : make_int2(0, 0);
            acc_lo += (long long)K * r.x;
            acc_hi += (long long)K * r.y;
        }
    }
    const long long acc = (long long)(((unsigned long long)acc_hi << 32) + (unsigned long long)acc_lo);
    const double scale = P.scale_dev ? *P.scale_dev : P.scale;
    P.grad[gid] = (float)((double)acc * scale);
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_cubical_bwd_rsum(int n, const CubicalBwdArgs &a, int n_items, size_t smem_rsum, cudaStream_t st)
{
    cudaError_t e;
    if (n_items <= 0) return cudaSuccess;
#define RS(NN)                                                                                                 \
    do {                                                                                                       \
        e = cudaFuncSetAttribute(cubical_bwd_rsum_kernel<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                 (int)smem_rsum);                                                              \
        if (e != cudaSuccess) return e;                                                                        \
        cubical_bwd_rsum_kernel<NN><<<n_items, 1024, smem_rsum, st>>>(a);                                      \
    } while (0)
    if (n == 1) RS(1);
    else if (n == 2) RS(2);
    else RS(3);
#undef RS
    return cudaGetLastError();
}

cudaError_t launch_cubical_bwd_route(int n, const CubicalBwdArgs &a, cudaStream_t st)
{
    const int blocks = (int)((a.v_end - a.v_begin + 255) / 256);
    if (blocks <= 0) return cudaSuccess;
    if (n == 1) cubical_bwd_route_kernel<1><<<blocks, 256, 0, st>>>(a);
    else if (n == 2) cubical_bwd_route_kernel<2><<<blocks, 256, 0, st>>>(a);
    else cubical_bwd_route_kernel<3><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

size_t cubical_bwd_rsum_smem(int n, int d, int T, int R)
{
    return rsum_layout(n, d, T, R).total;
}

}  // namespace wect
