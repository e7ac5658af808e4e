// wect_simplicial.cu -- gather kernels for the WECT of simplicial complexes given as index lists
// (Section 3 "inputs": per dimension a [k_i][i+1] table of vertex ids and a weight per simplex).
//
// Per direction tile the vertex bins are computed once (float32 filter, exact float64 fallback)
// into a [nv][Dt] uint16 table; the simplex kernel then takes, for every simplex and direction,
// the max of its vertex bins (equal to the bin of the max height, Eq. "msi") and adds the
// signed simplex weight into a shared-memory histogram [T][Dt] (one column per lane, so a
// red.shared of a warp hits 32 distinct banks), flushed into the int64 output.
#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

constexpr int kSimplexThreads = 512;

// ------------------------------------------------------------------ vertex bins

// Per direction p, the float32 form u = sum_a x~_a A_a + C of the threshold coordinate
// (h - lo) / step, with x~_a = rn32(x_a), A_a = rn32(s_a / step), C = rn32(-lo / step), and a bound
// eta on |u - (h - lo) / step| (Sec. 3.2, the bin of a vertex height).  tab[p] = {A_0, A_1, A_2, C,
// eta, 0, 0, 0}.  A zero step (lo == hi) gives eta = inf, so every bin goes to the float64 path.
template <int N>
__global__ void dir_filter_kernel(const double *__restrict__ dirs, int d, int T, const double *__restrict__ range,
                                  float *__restrict__ tab)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d) return;
    const double lo = range[0], step = range[2];
    float Af[3] = {0.f, 0.f, 0.f}, Cf = 0.f, eta = __int_as_float(0x7f800000);
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
        Af[0] = Af[1] = Af[2] = Cf = 0.f;
        eta = __int_as_float(0x7f800000);
    }
    float4 *t = reinterpret_cast<float4 *>(tab + (int64_t)p * 8);
    t[0] = make_float4(Af[0], Af[1], Af[2], Cf);
    t[1] = make_float4(eta, 0.f, 0.f, 0.f);
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
    const float eta = __ldg(tab + (int64_t)pc * 8 + 4);
    const float Af[3] = {t0.x, t0.y, t0.z};
    for (int64_t v = (int64_t)blockIdx.x * vpb + threadIdx.x / Dt; v < nv; v += (int64_t)gridDim.x * vpb) {
        float u = t0.w;
#pragma unroll
        for (int a = N - 1; a >= 0; --a) u = __fmaf_rn(__ldg(xf + v * N + a), Af[a], u);
        const int tlo = __float_as_int(__fadd_ru(__fsub_rd(u, eta), kMagic));
        const int thi = __float_as_int(__fadd_ru(__fadd_ru(u, eta), kMagic));
        int b = clamp_bin(thi, 0, T);
        if (tlo != thi) {
            double xd[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < N; ++a) xd[a] = coords[v * N + a];
            const double h = height3<N>(xd[0], xd[1], xd[2], dirs + (int64_t)pc * N);
            b = exact_bin_from(h, beta, T, b);
        }
        if (act) bins[v * Dt + col] = (uint16_t)b;
    }
}

// ------------------------------------------------------------------ simplex scatter

template <int NSPLIT, int M>
__global__ void __launch_bounds__(kSimplexThreads, 1) simplex_fwd_kernel(const SimplexFwdArgs P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = P.T, Dt = P.Dt;
    const int hw = T * Dt;
    int32_t *hist = reinterpret_cast<int32_t *>(smem);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t histAddr = smem_addr(hist);
    const uint32_t HOFF = (uint32_t)hw * 4u;
    for (int i = threadIdx.x; i < NSPLIT * hw; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int64_t nchunks = (P.k + P.chunk - 1) / P.chunk;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t b0 = ch * P.chunk, b1 = min(P.k, b0 + P.chunk);
        // each warp takes GS simplices per step: their vertex ids, weights and vertex bins are all
        // loaded before any is reduced, so GS dependent load chains are in flight per warp
        constexpr int GS = 8;
        for (int64_t bb = b0 + (int64_t)wid * GS; bb < b1; bb += (int64_t)nw * GS) {
            int vid[GS][M];
            int64_t w[GS];
#pragma unroll
            for (int g = 0; g < GS; ++g) {
                const int64_t b = min(bb + g, b1 - 1);
#pragma unroll
                for (int j = 0; j < M; ++j) vid[g][j] = (M == 1) ? (int)b : __ldg(P.simp + b * M + j);
                w[g] = (bb + g < b1) ? __ldg(reinterpret_cast<const long long *>(P.sw) + b) : 0;
            }
            for (int c = lane; c < Dt; c += 32) {
                int bin[GS];
#pragma unroll
                for (int g = 0; g < GS; ++g) {
                    bin[g] = 0;
#pragma unroll
                    for (int j = 0; j < M; ++j) bin[g] = max(bin[g], (int)__ldg(P.bins + (int64_t)vid[g][j] * Dt + c));
                }
#pragma unroll
                for (int g = 0; g < GS; ++g) {
                    const int64_t sw = P.sign > 0 ? w[g] : -w[g];
                    const uint32_t addr = histAddr + ((uint32_t)bin[g] * (uint32_t)Dt + (uint32_t)c) * 4u;
                    if (NSPLIT == 1) {
                        red_shared_add(addr, (int32_t)sw);
                    } else {
                        red_shared_add_u32(addr, (uint32_t)(sw & 0xFFFF));
                        red_shared_add(addr + HOFF, (int32_t)(sw >> 16));
                    }
                }
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < hw; idx += blockDim.x) {
            const int q = idx / Dt, c = idx - q * Dt;
            const int p = P.dtile * Dt + c;
            int64_t v;
            if (NSPLIT == 1) {
                v = hist[idx];
            } else {
                v = ((int64_t)hist[hw + idx] << 16) + (int64_t)(uint32_t)hist[idx];
                hist[hw + idx] = 0;
            }
            hist[idx] = 0;
            if (p < P.d && v != 0) atomicAdd(P.out + (int64_t)p * T + q, (unsigned long long)v);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ default range

// Pass 1: a float32 lower bound L on max |h| (|h~| - E); pass 2: exact float64 |h| of every
// (vertex, direction) whose float32 upper bound reaches L.  Each thread keeps one vertex and
// walks the directions, staged in shared memory kMaxAbsDirs at a time.
constexpr int kMaxAbsDirs = 1024;

template <int N, int PASS>
__global__ void __launch_bounds__(256) simplicial_max_abs_kernel(const double *__restrict__ coords,
                                                                 const float *__restrict__ xf, int64_t nv,
                                                                 const double *__restrict__ dirs, int d,
                                                                 unsigned long long *Mbits, unsigned int *Lbits)
{
    __shared__ float sd[kMaxAbsDirs][N];
    const float L = (PASS == 2) ? __uint_as_float(*Lbits) : 0.f;
    unsigned int best = 0;
    for (int p0 = 0; p0 < d; p0 += kMaxAbsDirs) {
        const int np = min(kMaxAbsDirs, d - p0);
        __syncthreads();
        for (int i = threadIdx.x; i < np * N; i += blockDim.x) sd[i / N][i % N] = __double2float_rn(dirs[(int64_t)p0 * N + i]);
        __syncthreads();
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
            float x[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < N; ++a) x[a] = __ldg(xf + v * N + a);
            for (int j = 0; j < np; ++j) {
                float h = 0.f, mag = 0.f;
#pragma unroll
                for (int a = N - 1; a >= 0; --a) {
                    h = __fmaf_rn(x[a], sd[j][a], h);
                    mag = __fmaf_ru(fabsf(x[a]), fabsf(sd[j][a]), mag);
                }
                const float E = __fmul_ru(mag, 0x1p-19f) + 0x1p-126f;
                if (PASS == 1) {
                    const float lb = __fsub_rd(fabsf(h), E);
                    if (lb > 0.f) best = max(best, __float_as_uint(lb));
                } else if (__fadd_ru(fabsf(h), E) >= L) {
                    double xd[3] = {0.0, 0.0, 0.0};
                    for (int a = 0; a < N; ++a) xd[a] = coords[v * N + a];
                    const double hd = fabs(height3<N>(xd[0], xd[1], xd[2], dirs + (int64_t)(p0 + j) * N));
                    atomicMax(Mbits, (unsigned long long)__double_as_longlong(hd));
                }
            }
        }
    }
    if (PASS == 1) {
        for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, off));
        if ((threadIdx.x & 31) == 0) atomicMax(Lbits, best);
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

__global__ void i128_to_grad_kernel(const unsigned long long *Iacc, int64_t nv, double scale, float *grad)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x)
        grad[v] = (float)(i128_to_double((int64_t)Iacc[2 * v + 1], Iacc[2 * v]) * scale);
}

template <int M>
__global__ void simplex_ecf_kernel(const int32_t *simp, const int64_t *sw, int64_t k, int sign, int weighted,
                                   const uint16_t *bins, int T, unsigned long long *out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *h = reinterpret_cast<long long *>(smem);
    for (int i = threadIdx.x; i < T; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        int bin = 0;
        for (int j = 0; j < M; ++j) bin = max(bin, (int)bins[(M == 1) ? b : simp[b * M + j]]);
        const long long w = weighted ? (long long)sw[b] : 1ll;
        atomicAdd(reinterpret_cast<unsigned long long *>(&h[bin]), (unsigned long long)(sign > 0 ? w : -w));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T; i += blockDim.x)
        if (h[i]) atomicAdd(out + i, (unsigned long long)h[i]);
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_dir_filters(int n, const double *dirs, int d, int T, const double *range, float *tab,
                               cudaStream_t st)
{
    const unsigned g = (unsigned)((d + 127) / 128);
    if (n == 1) dir_filter_kernel<1><<<g, 128, 0, st>>>(dirs, d, T, range, tab);
    else if (n == 2) dir_filter_kernel<2><<<g, 128, 0, st>>>(dirs, d, T, range, tab);
    else dir_filter_kernel<3><<<g, 128, 0, st>>>(dirs, d, T, range, tab);
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
    else VB(3);
#undef VB
    return cudaGetLastError();
}

size_t simplex_fwd_smem(int nsplit, int T, int Dt) { return (size_t)nsplit * T * Dt * 4u; }

template <int NSPLIT>
static cudaError_t launch_simplex_fwd_s(const SimplexFwdArgs &a, int grid, cudaStream_t st)
{
    const size_t sm = simplex_fwd_smem(NSPLIT, a.T, a.Dt);
    cudaError_t e = cudaSuccess;
#define SF(MM)                                                                                                  \
    do {                                                                                                        \
        e = cudaFuncSetAttribute(simplex_fwd_kernel<NSPLIT, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 (int)sm);                                                                      \
        if (e == cudaSuccess) simplex_fwd_kernel<NSPLIT, MM><<<grid, kSimplexThreads, sm, st>>>(a);            \
    } while (0)
    switch (a.m) {
    case 1: SF(1); break;
    case 2: SF(2); break;
    case 3: SF(3); break;
    default: SF(4); break;
    }
#undef SF
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_simplex_fwd(int nsplit, const SimplexFwdArgs &a, int grid, cudaStream_t st)
{
    return nsplit == 1 ? launch_simplex_fwd_s<1>(a, grid, st) : launch_simplex_fwd_s<2>(a, grid, st);
}

cudaError_t launch_simplicial_max_abs(int n, const double *coords, const float *xf, int64_t nv, const double *dirs,
                                      int d, unsigned long long *Mbits, float *Lscratch, cudaStream_t st)
{
    unsigned int *Lbits = reinterpret_cast<unsigned int *>(Lscratch);
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nv + 255) / 256, 152 * 8));
    cudaError_t e = cudaMemsetAsync(Lbits, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
#define MA(NN)                                                                                      \
    do {                                                                                            \
        simplicial_max_abs_kernel<NN, 1><<<g, 256, 0, st>>>(coords, xf, nv, dirs, d, Mbits, Lbits); \
        simplicial_max_abs_kernel<NN, 2><<<g, 256, 0, st>>>(coords, xf, nv, dirs, d, Mbits, Lbits); \
    } while (0)
    if (n == 1) MA(1);
    else if (n == 2) MA(2);
    else MA(3);
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
    default: simplex_weights_max_kernel<4><<<g, 256, 0, st>>>(simp, k, vw, sw); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_simplicial_bwd(int n, const double *coords, const float *xf, int64_t nv, const int32_t *const *simp,
                                  const int64_t *counts, int max_dim, const int64_t *vw, const double *dirs, int d,
                                  int T, const float *tab, const double *beta, const int64_t *S,
                                  uint16_t *bins, unsigned long long *Iacc, float *grad, double scale,
                                  cudaStream_t st)
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
            default: simplex_bwd_kernel<4><<<g, 256, 0, st>>>(simp[3], k, sign, vw, bins, Dt, dt, d, T, S, Iacc); break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    i128_to_grad_kernel<<<(unsigned)std::min<int64_t>((nv + 255) / 256, 4096), 256, 0, st>>>(Iacc, nv, scale, grad);
    return cudaGetLastError();
}

cudaError_t launch_simplex_ecf(const int32_t *simp, const int64_t *sw, int64_t k, int m, int sign, int weighted,
                               const uint16_t *bins, int T, unsigned long long *out, cudaStream_t st)
{
    if (k <= 0) return cudaSuccess;
    const unsigned g = (unsigned)std::min<int64_t>((k + 255) / 256, 1024);
    const size_t sm = (size_t)T * 8u;
    cudaError_t e = cudaSuccess;
#define SE(MM)                                                                                              \
    do {                                                                                                    \
        e = cudaFuncSetAttribute(simplex_ecf_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        if (e == cudaSuccess) simplex_ecf_kernel<MM><<<g, 256, sm, st>>>(simp, sw, k, sign, weighted, bins, T, out); \
    } while (0)
    switch (m) {
    case 1: SE(1); break;
    case 2: SE(2); break;
    case 3: SE(3); break;
    default: SE(4); break;
    }
#undef SE
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace wect
