// wect_ecf.cu -- the ECF and WECF of grids (Eq. "ecf", Algorithm 1 with caller-supplied
// vertex filters) and the exact bins of caller filters, shared with simplex lists (sm_103a).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

// ------------------------------------------------------------------ kernels

// Order-preserving int64 key of a float64: x < y <=> key(x) < key(y) for non-NaN x and y, with
// -0 and +0 equal.  Compares of keys are integer instructions, where float64 compares would run
// on the float64 pipe.
__device__ __forceinline__ long long f64_key(double x)
{
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b < 0 ? (b ^ 0x7fffffffffffffffll) : b;
}

// A float32 within a relative 2^-20 of x (its sign, exponent and top 20 mantissa bits; 0 below
// the float32 normal range, +-2^127 above it), from integer operations alone.  Only a guide: the
// bin is decided by key compares.
__device__ __forceinline__ float f32_guide(double x)
{
    const unsigned hi = (unsigned)((unsigned long long)__double_as_longlong(x) >> 32);
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;
    const unsigned sg = hi & 0x80000000u;
    const unsigned r = e <= 0 ? sg : (e >= 255 ? (sg | 0x7F000000u) : (sg | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3)));
    return __uint_as_float(r);
}

// Bins of caller-supplied vertex filters, bin(x) = #{q <= T-2 : beta[q] < x} exactly: a float32
// guess of (x - lo) / step, then integer compares of order-preserving keys against the threshold
// table (staged in shared memory when it fits, SMEM), stepping to the exact count.  Non-finite
// values set flag in *status (they still get a bin).  Grid-stride over the [m][nv] values.
template <bool SMEM>
__global__ void __launch_bounds__(512) filter_bins_kernel(const double *__restrict__ f, int64_t n,
                                                          const double *__restrict__ range,
                                                          const double *__restrict__ beta, int T,
                                                          uint16_t *__restrict__ bins, int *status, int flag)
{
    extern __shared__ long long kb[];
    if (SMEM) {
        for (int q = threadIdx.x; q < T - 1; q += blockDim.x) kb[q] = f64_key(beta[q]);
        __syncthreads();
    }
    const double lo = range[0], step = range[2];
    const bool deg = !(step > 0.0);                   // lo == hi: every beta equals lo
    const float inv = deg ? 0.f : 1.0f / (float)step;
    const float off = -(float)lo * inv;
    const long long klo = f64_key(lo);
    bool bad = false;
    constexpr int K = 4;                                // values in flight per thread
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += K * stride) {
        double xs[K];
#pragma unroll
        for (int k = 0; k < K; ++k) xs[k] = (base + k * stride < n) ? __ldg(f + base + k * stride) : 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t v = base + k * stride;
            if (v >= n) break;
            const double x = xs[k];
            const long long kx = f64_key(x);
            bad |= ((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF;
            int b;
            if (deg) {
                b = kx <= klo ? 0 : T - 1;
            } else {
                const float u = fminf(fmaxf(fmaf(f32_guide(x), inv, off), -1.0f), (float)T);
                b = min(max(__float_as_int(__fadd_ru(u, kMagic)) - kMagicBits, 0), T - 1);
            }
            while (b > 0 && kx <= (SMEM ? kb[b - 1] : f64_key(__ldg(beta + b - 1)))) --b;
            while (b < T - 1 && kx > (SMEM ? kb[b] : f64_key(__ldg(beta + b)))) ++b;
            bins[v] = (uint16_t)b;
        }
    }
    if (bad) atomicOr(status, flag);
}

// Cells of a grid by lower corner: each vertex v owns the 2^n cells (extent masks e) that have v
// as the lower corner.  A cell's bin is the max of its vertex bins (Eq. "msi"), here the max over
// the corners s of e of v's 2^n box, by a subset-max pass over the box; with WEIGHTED its weight
// is the max of its vertex weights the same way, else 1.  Every warp walks a contiguous span of
// 32-vertex row segments (one division per warp, then the row coordinates advance by
// increments).  The signed sums go to a per-block histogram in shared memory, int32 when the
// launch keeps each block's sum of |weights| below 2^31 and int64 (H64) otherwise, or with
// GHIST straight to the int64 output when the histogram does not fit.  blockIdx.y selects the
// filter of [m][nv] bins and the row of the [m][T] output.
template <int N, bool WEIGHTED, bool H64, bool GHIST>
__global__ void __launch_bounds__(1024) cubical_ecf_kernel(const GridDesc *grids, const uint16_t *__restrict__ bins,
                                                          int T, unsigned long long *__restrict__ out)
{
    using H = typename std::conditional<H64, unsigned long long, int>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    H *h = reinterpret_cast<H *>(smem);
    if (!GHIST) {
        for (int i = threadIdx.x; i < T; i += blockDim.x) h[i] = 0;
        __syncthreads();
    }
    const GridDesc g = grids[0];
    bins += (int64_t)blockIdx.y * g.nv;
    out += (int64_t)blockIdx.y * T;
    const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
    const int segs = (L0 + 31) >> 5;
    const int64_t units = (int64_t)L1 * L2 * segs;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t span = (units + nwarps - 1) / nwarps;
    int64_t unit = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * span;
    const int64_t uend = min(units, unit + span);
    int64_t row = unit / segs;
    int seg = (int)(unit - row * segs);
    int i1 = (int)(row % L1), i2 = (int)(row / L1);
    for (; unit < uend; ++unit) {
        const int i0 = seg * 32 + (threadIdx.x & 31);
        const int64_t v = (int64_t)i0 + (int64_t)L0 * row;
        const bool live = i0 < L0;
        const bool ok0 = i0 + 1 < L0, ok1 = N >= 2 && i1 + 1 < L1, ok2 = N >= 3 && i2 + 1 < L2;
        if (++seg == segs) {          // next segment's coordinates
            seg = 0;
            ++row;
            if (++i1 == L1) {
                i1 = 0;
                ++i2;
            }
        }
        if (!live) continue;
        int c[1 << N];
        int32_t w[1 << N];
#pragma unroll
        for (int s = 0; s < (1 << N); ++s) {
            const bool in = (!(s & 1) || ok0) && (!(s & 2) || ok1) && (!(s & 4) || ok2);
            const int64_t u = v + (s & 1) + (int64_t)L0 * (((s >> 1) & 1) + (int64_t)L1 * ((s >> 2) & 1));
            c[s] = in ? (int)bins[u] : 0;
            w[s] = (WEIGHTED && in) ? __ldg(g.w + u) : INT32_MIN;
        }
        // subset max: c[e] = max over the corners s of e (s a sub-mask of e) of the corner bins
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int s = 0; s < (1 << N); ++s)
                if ((s >> a) & 1) {
                    c[s] = max(c[s], c[s ^ (1 << a)]);
                    if (WEIGHTED) w[s] = max(w[s], w[s ^ (1 << a)]);
                }
#pragma unroll
        for (int e = 0; e < (1 << N); ++e) {
            const bool in = (!(e & 1) || ok0) && (!(e & 2) || ok1) && (!(e & 4) || ok2);
            if (!in) continue;
            const bool odd = __popc(e) & 1;
            if (GHIST) {
                const long long val = WEIGHTED ? (long long)w[e] : 1ll;
                atomicAdd(out + c[e], (unsigned long long)(odd ? -val : val));
            } else if (H64) {
                const long long val = WEIGHTED ? (long long)w[e] : 1ll;
                atomicAdd(&h[c[e]], (unsigned long long)(odd ? -val : val));
            } else {
                const int val = WEIGHTED ? w[e] : 1;
                atomicAdd(&h[c[e]], odd ? -val : val);
            }
        }
    }
    if (!GHIST) {
        __syncthreads();
        for (int i = threadIdx.x; i < T; i += blockDim.x)
            if (h[i]) atomicAdd(out + i, (unsigned long long)(long long)h[i]);
    }
}

// ------------------------------------------------------------------ launchers

static int device_attr(cudaDeviceAttr attr)
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, attr, dev);
    return v;
}

template <int N, bool W, bool H, bool G>
static cudaError_t launch_ecf_t(dim3 blocks, int threads, size_t sm, const GridDesc *grids, const uint16_t *bins,
                                int T, unsigned long long *out, cudaStream_t st)
{
    if (sm > 48u * 1024u) {
        cudaError_t e = cudaFuncSetAttribute(cubical_ecf_kernel<N, W, H, G>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    cubical_ecf_kernel<N, W, H, G><<<blocks, threads, sm, st>>>(grids, bins, T, out);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_ecf_n(bool weighted, bool h64, bool ghist, dim3 blocks, int threads, size_t sm,
                                const GridDesc *grids, const uint16_t *bins, int T, unsigned long long *out,
                                cudaStream_t st)
{
    if (ghist)
        return weighted ? launch_ecf_t<N, true, true, true>(blocks, threads, sm, grids, bins, T, out, st)
                        : launch_ecf_t<N, false, true, true>(blocks, threads, sm, grids, bins, T, out, st);
    if (weighted)
        return h64 ? launch_ecf_t<N, true, true, false>(blocks, threads, sm, grids, bins, T, out, st)
                   : launch_ecf_t<N, true, false, false>(blocks, threads, sm, grids, bins, T, out, st);
    return launch_ecf_t<N, false, false, false>(blocks, threads, sm, grids, bins, T, out, st);
}

cudaError_t launch_cubical_ecf(int n, const GridDesc *grids, const uint16_t *bins, int T, int weighted,
                               int64_t wbound, unsigned long long *out, int64_t nv, int nf, cudaStream_t st)
{
    static const int sms = std::max(1, device_attr(cudaDevAttrMultiProcessorCount));
    static const size_t optin = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin);
    const int threads = T > 2048 ? 1024 : 512;
    const int64_t maxblocks = std::max<int64_t>(1, (nv + threads - 1) / threads);
    // blocks per filter that keep a block's sum of |weight| (2^n cells per vertex, each at most
    // wbound) below 2^30 in an int32 histogram
    const double wb = weighted ? (double)std::max<int64_t>(wbound, 1) : 1.0;
    const double need = std::ceil((double)nv * (double)(1 << n) * wb / 1073741824.0) + 1.0;
    const bool h64 = need > (double)maxblocks;
    size_t sm = (size_t)T * (h64 ? 8u : 4u);
    const bool ghist = sm + 1024 > optin;
    if (ghist) sm = 0;
    // over all filters: four blocks of 512 per SM (full occupancy) for small T, one of 1024 when
    // the flush of each block's T-entry histogram (global atomics) would cost more
    int64_t per = std::max<int64_t>(1, (int64_t)sms * (T > 2048 ? 1 : 4) / std::max(nf, 1));
    if (!h64) per = std::max<int64_t>(per, (int64_t)need);
    const dim3 blocks((unsigned)std::min<int64_t>(maxblocks, per), (unsigned)nf);
    if (n == 1) return launch_ecf_n<1>(weighted != 0, h64, ghist, blocks, threads, sm, grids, bins, T, out, st);
    if (n == 2) return launch_ecf_n<2>(weighted != 0, h64, ghist, blocks, threads, sm, grids, bins, T, out, st);
    return launch_ecf_n<3>(weighted != 0, h64, ghist, blocks, threads, sm, grids, bins, T, out, st);
}

cudaError_t launch_filter_bins(const double *f, int64_t nv, const double *range, const double *beta, int T,
                               uint16_t *bins, int *status, int flag, cudaStream_t st)
{
    static const int sms = std::max(1, device_attr(cudaDevAttrMultiProcessorCount));
    static const size_t optin = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin);
    static const size_t persm = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerMultiprocessor);
    if (nv <= 0) return cudaSuccess;
    const size_t sm = (size_t)std::max(T - 1, 1) * 8u;
    const bool use_smem = sm + 1024 <= optin;
    const int per_sm = use_smem ? (int)std::max<size_t>(1, std::min<size_t>(4, persm / (sm + 1024))) : 4;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nv + 511) / 512, (int64_t)sms * per_sm));
    if (use_smem) {
        if (sm > 48u * 1024u) {
            cudaError_t e = cudaFuncSetAttribute(filter_bins_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
            if (e != cudaSuccess) return e;
        }
        filter_bins_kernel<true><<<grid, 512, sm, st>>>(f, nv, range, beta, T, bins, status, flag);
    } else {
        filter_bins_kernel<false><<<grid, 512, 0, st>>>(f, nv, range, beta, T, bins, status, flag);
    }
    return cudaGetLastError();
}

}  // namespace wect
