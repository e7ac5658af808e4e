// wect_common.cu -- small kernels shared by every path: threshold table, prefix scans over
// thresholds, direction grouping by octant, weight conversion and input validation.
#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

// Resolve the threshold range and fill beta (Section 3: beta(q) = q 2M/(T-1) - M, here for a
// range [lo, hi]; the default range is [-M, M] with M the largest |height|).
//   range[0] = lo, range[1] = hi, range[2] = step = (hi - lo)/(T - 1); beta[q] = lo + q*step.
// Thread t of nt (over one or more blocks) fills its share.
__device__ __forceinline__ void range_beta(double lo, double hi, int use_default, const unsigned long long *Mbits, int T,
                                           double *range, double *beta, int t, int nt)
{
    if (use_default) {
        const double M = __longlong_as_double((long long)*Mbits);
        lo = -M;
        hi = M;
    }
    const double step = __ddiv_rn(__dsub_rn(hi, lo), (double)(T - 1));
    if (t == 0) {
        range[0] = lo;
        range[1] = hi;
        range[2] = step;
    }
    for (int q = t; q < T; q += nt) beta[q] = __dadd_rn(lo, __dmul_rn((double)q, step));
}

__global__ void setup_range_beta_kernel(double lo, double hi, int use_default, const unsigned long long *Mbits, int T,
                                        double *range, double *beta)
{
    range_beta(lo, hi, use_default, Mbits, T, range, beta, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x);
}

// Grouping of the directions by octant (bit a set when s_a > 0): perm lists the directions
// octant by octant, octb[o] is where octant o starts.  One block; the order inside an octant
// is arbitrary (every consumer sums integers, so results do not depend on it).
// One block (any size); cnt/start/fill are shared arrays of the caller.
__device__ __forceinline__ void octant_sort_block(int n, const double *dirs, int d, int *perm, int *octb, int *cnt,
                                                  int *start, int *fill)
{
    if (threadIdx.x < 8) {
        cnt[threadIdx.x] = 0;
        fill[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < d; p += blockDim.x) {
        int o = 0;
        for (int a = 0; a < n; ++a)
            if (dirs[(int64_t)p * n + a] > 0.0) o |= 1 << a;
        atomicAdd(&cnt[o], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        start[0] = 0;
        for (int o = 0; o < 8; ++o) start[o + 1] = start[o] + cnt[o];
    }
    __syncthreads();
    if (threadIdx.x <= (1 << n)) octb[threadIdx.x] = start[threadIdx.x];
    for (int p = threadIdx.x; p < d; p += blockDim.x) {
        int o = 0;
        for (int a = 0; a < n; ++a)
            if (dirs[(int64_t)p * n + a] > 0.0) o |= 1 << a;
        perm[start[o] + atomicAdd(&fill[o], 1)] = p;
    }
}

__global__ void octant_sort_kernel(int n, const double *dirs, int d, int *perm, int *octb)
{
    __shared__ int cnt[8], start[9], fill[8];
    octant_sort_block(n, dirs, d, perm, octb, cnt, start, fill);
}

// Everything the cubical forward needs before its launch, in one kernel: block 0 checks the
// directions for non-finite values (status flag), resolves the range and fills beta, groups the
// directions by octant and clears the work-queue head; every block clears the output table
// (when given) with 16-byte stores.
// Key of a direction in the run order: |s_0| (a non-finite component sorts last; the direction is
// flagged as invalid anyway).
__device__ __forceinline__ double run_key(const double *dirs, int n, int p)
{
    const double x = dirs[(int64_t)p * n];
    return isfinite(x) ? fabs(x) : __longlong_as_double(0x7ff0000000000000ll);
}

__global__ void fwd_prep_kernel(int n, const double *dirs, int d, int T, double lo, double hi, int use_default,
                                const unsigned long long *Mbits, double *range, double *beta, int *perm, int *octb,
                                int *counter, int *status, unsigned long long *out, int64_t out_elems, int run_order,
                                int early)
{
    // A programmatic dependent: the forward kernel may launch at once.  When the kernel before is
    // known to be the library's weight conversion (early), this grid runs beside it, since it
    // reads none of its output, and waits for it only before exiting, so that the forward
    // kernel's griddepcontrol.wait covers both.  Otherwise the kernel before may be the caller's,
    // which may have written the directions or still read the table: wait first.
    pdl_trigger();
    if (!early) pdl_wait();
    if (blockIdx.x == 0) {
        __shared__ int cnt[8], start[9], fill[8];
        if (status)
            for (int i = threadIdx.x; i < d * n; i += blockDim.x)
                if (!isfinite(dirs[i])) atomicOr(status, kStatusBadIndex);
        if (use_default) pdl_wait();      // Mbits comes from the kernel before
        range_beta(lo, hi, use_default, Mbits, T, range, beta, threadIdx.x, blockDim.x);
        if (!run_order) octant_sort_block(n, dirs, d, perm, octb, cnt, start, fill);
        if (threadIdx.x == 0) *counter = 0;
    }
    if (run_order) {
        // directions in increasing |s_0| (ties by index: a total order, so perm is a permutation):
        // the run kernel's lanes then walk similar numbers of bin boundaries per row
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < d; p += gridDim.x * blockDim.x) {
            const double kp = run_key(dirs, n, p);
            int r = 0;
            for (int q = 0; q < d; ++q) {
                const double kq = run_key(dirs, n, q);
                r += (kq < kp || (kq == kp && q < p)) ? 1 : 0;
            }
            perm[r] = p;
        }
    }
    if (out && out_elems > 0) {
        // an 8-byte aligned table: one scalar head element when it is not 16-byte aligned
        const int head = (reinterpret_cast<uintptr_t>(out) & 15u) ? 1 : 0;
        ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(out + head);
        const int64_t n2 = (out_elems - head) >> 1;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
            o2[i] = make_ulonglong2(0ull, 0ull);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (head) out[0] = 0ull;
            if ((out_elems - head) & 1) out[out_elems - 1] = 0ull;
        }
    }
    pdl_wait();
}

// Inclusive prefix sum of each row of an int64 [rows][T] table (Algorithm 1's final cumulative
// sum) from src into dst (the same table, or another one, e.g. mapped host memory): one warp per
// row, 32-wide shuffle scans with a running carry.
__global__ void scan_rows_kernel(const unsigned long long *src, unsigned long long *dst, int64_t rows, int T)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const long long *r = reinterpret_cast<const long long *>(src) + row * T;
    long long *o = reinterpret_cast<long long *>(dst) + row * T;
    long long carry = 0;
    for (int base = 0; base < T; base += 32) {
        const int q = base + lane;
        long long v = (q < T) ? r[q] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        v += carry;
        if (q < T) o[q] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

// Long rows (T in the thousands): one block per row.  Each thread sums a contiguous piece of
// the row, the block scans the piece sums (warp shuffles, then the warp totals), and each thread
// rewrites its piece as running sums from its exclusive prefix.  A warp per row would walk T / 32
// dependent steps.
__global__ void __launch_bounds__(1024) scan_rows_block_kernel(const unsigned long long *src, unsigned long long *dst,
                                                               int T)
{
    __shared__ long long wsum[32];
    pdl_wait();
    const long long *r = reinterpret_cast<const long long *>(src) + (int64_t)blockIdx.x * T;
    long long *o = reinterpret_cast<long long *>(dst) + (int64_t)blockIdx.x * T;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (T + blockDim.x - 1) / blockDim.x;
    const int q0 = min(T, (int)threadIdx.x * per), q1 = min(T, q0 + per);
    long long s = 0;
    for (int q = q0; q < q1; ++q) s += r[q];
    long long v = s;                                  // inclusive scan of the piece sums
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += u;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += u;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    long long run = v - s + (wid > 0 ? wsum[wid - 1] : 0);   // exclusive prefix of the piece
    for (int q = q0; q < q1; ++q) {
        run += r[q];
        o[q] = run;
    }
}

// Suffix sums S[q] = sum_{q' >= q} G[q'] of each row (the adjoint of the prefix scan).  The
// adjoint later sums S over up to d directions in int64: entries with |S| > smax flag overflow.
__global__ void suffix_rows_kernel(const int64_t *in, int64_t *out, int64_t rows, int T, long long smax, int *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const long long *a = reinterpret_cast<const long long *>(in) + row * T;
    long long *o = reinterpret_cast<long long *>(out) + row * T;
    long long carry = 0;
    for (int top = T - 1; top >= 0; top -= 32) {
        const int q = top - lane;
        long long v = (q >= 0) ? a[q] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        v += carry;
        if (q >= 0) {
            o[q] = v;
            if (status && (v > smax || v < -smax)) atomicOr(status, kStatusOverflow);
        }
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
}

// Vertex weights to int64 fixed point, with max |w| and a flag for non-finite input.
template <int WT>
__global__ void weights_to_fixed_kernel(const void *w, int64_t nv, int frac_bits, int64_t *out,
                                        unsigned long long *maxabs, int *bad)
{
    unsigned long long m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        if (WT == WT_F32) {
            const float x = ((const float *)w)[v];
            if (!isfinite(x) || fabsf(x) >= 0x1p62f / ldexpf(1.0f, frac_bits)) {
                atomicOr(bad, 1);
                continue;
            }
        }
        const int64_t f = load_weight_fixed<WT>(w, v, frac_bits);
        if (out) out[v] = f;
        const unsigned long long a = (unsigned long long)(f < 0 ? -f : f);
        m = a > m ? a : m;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, m, off);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && maxabs) atomicMax(maxabs, m);
}

// Vertex weights to the int32 fixed-point copy the stencil kernels read; |w| above limit
// (or non-finite input) sets the overflow bit of the status word.
template <int WT>
__global__ void weights_to_w32_kernel(const void *w, int64_t nv, int frac_bits, int64_t limit, int32_t *out, int *status)
{
    pdl_trigger();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        if (WT == WT_F32) {
            const float x = ((const float *)w)[v];
            if (!isfinite(x) || fabsf(x) >= 0x1p62f / ldexpf(1.0f, frac_bits)) {
                atomicOr(status, kStatusOverflow);
                out[v] = 0;
                continue;
            }
        }
        const int64_t f = load_weight_fixed<WT>(w, v, frac_bits);
        if (f > limit || f < -limit) atomicOr(status, kStatusOverflow);
        out[v] = (int32_t)f;
    }
}

// u8 weights (which never exceed the limit, at least 255): 16 per thread step, one 16-byte load
// and four 16-byte stores, then the tail.  w is 16-byte aligned.
__global__ void weights_u8_to_w32_kernel(const uint8_t *__restrict__ w, int64_t nv, int32_t *__restrict__ out)
{
    pdl_trigger();          // the forward's preparation reads none of this
    const int64_t n16 = nv >> 4, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(w) + i);
        int4 *o = reinterpret_cast<int4 *>(out) + 4 * i;
        const unsigned q[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            o[k] = make_int4((int)(q[k] & 255u), (int)((q[k] >> 8) & 255u), (int)((q[k] >> 16) & 255u), (int)(q[k] >> 24));
    }
    for (int64_t v = (n16 << 4) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) out[v] = w[v];
}

template <int WT>
__global__ void weights_check_kernel(const void *w, int64_t nv, int frac_bits, int64_t limit, int *status)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        if (WT == WT_F32) {
            const float x = ((const float *)w)[v];
            if (!isfinite(x) || fabsf(x) >= 0x1p62f / ldexpf(1.0f, frac_bits)) {
                atomicOr(status, kStatusOverflow);
                continue;
            }
        }
        const int64_t f = load_weight_fixed<WT>(w, v, frac_bits);
        if (f > limit || f < -limit) atomicOr(status, kStatusOverflow);
    }
}

__global__ void max_abs_f64_kernel(const double *x, int64_t n, int stride, int offset, unsigned long long *Mbits)
{
    __shared__ unsigned long long wmax[32];
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = fabs(x[i * stride + offset]);
        const unsigned long long b = (unsigned long long)__double_as_longlong(a);
        m = b > m ? b : m;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, m, off);
        m = o > m ? o : m;
    }
    // one atomic per block (a per-warp atomic on a single address serialises in L2)
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wmax[w] > m ? wmax[w] : m;
        if (m) atomicMax(Mbits, m);
    }
}

// Upstream float64 gradient -> int64 table with the largest power-of-two scale 2^k that keeps
// hr * max|G| * 2^k < 2^62 (hr = headroom, d * T rounded up to a power of two), so the adjoint's
// int64 sums over thresholds and directions cannot overflow.  out = rint(G * 2^k) (ties to
// even), *scale = 2^-k.  Non-finite G flags the status word.
__global__ void grad_quantize_kernel(const double *G, int64_t n, const unsigned long long *maxbits, int log2_headroom,
                                     long long *out, double *scale, int *status)
{
    const double m = __longlong_as_double((long long)*maxbits);
    int k = 0;
    if (m > 0.0 && isfinite(m)) {
        int e;
        frexp(m, &e);                                      // m < 2^e
        k = 62 - log2_headroom - e;
        k = max(min(k, 1000), -1000);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *scale = ldexp(1.0, -k);
    // x * 2^k with 2^k an exact double (|k| <= 1000): the same value as ldexp(x, k), one multiply
    const double p2k = ldexp(1.0, k);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = G[i];
        if (!isfinite(x)) {
            atomicOr(status, kStatusBadIndex);
            out[i] = 0;
            continue;
        }
        out[i] = (m > 0.0) ? __double2ll_rn(__dmul_rn(x, p2k)) : 0ll;
    }
}

__global__ void finite_check_kernel(const double *x, int64_t n, int *bad, int flag)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) atomicOr(bad, flag);
}

__global__ void index_check_kernel(const int32_t *idx, int64_t n, int64_t nv, int *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = idx[i];
        if (v < 0 || (int64_t)v >= nv) atomicOr(bad, 1);
    }
}

// ------------------------------------------------------------------ launchers

static unsigned grid_for(int64_t n, int threads, unsigned cap = 4096)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (unsigned)(g > cap ? cap : g);
}

cudaError_t launch_setup_range_beta(double lo, double hi, int use_default, const unsigned long long *Mbits, int T,
                                    double *range, double *beta, cudaStream_t st)
{
    setup_range_beta_kernel<<<grid_for(T, 256, 64), 256, 0, st>>>(lo, hi, use_default, Mbits, T, range, beta);
    return cudaGetLastError();
}

cudaError_t launch_fwd_prep(int n, const double *dirs, int d, int T, double lo, double hi, int use_default,
                            const unsigned long long *Mbits, double *range, double *beta, int *perm, int *octb,
                            int *counter, int *status, unsigned long long *out, int64_t out_elems, cudaStream_t st,
                            int run_order, bool pdl, bool early)
{
    if (out && (reinterpret_cast<uintptr_t>(out) & 7u)) return cudaErrorMisalignedAddress;   // int64 alignment
    int64_t work = out ? (out_elems / 2 + 255) / 256 : 1;
    if (run_order) work = std::max<int64_t>(work, (d + 255) / 256);
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(work, 152 * 4));
    return launch_kernel(fwd_prep_kernel, dim3(g), dim3(256), 0, st, pdl, n, dirs, d, T, lo, hi, use_default, Mbits, range,
                         beta, perm, octb, counter, status, out, out_elems, run_order, early ? 1 : 0);
}

cudaError_t launch_octant_sort(int n, const double *dirs, int d, int *perm, int *octb, cudaStream_t st)
{
    octant_sort_kernel<<<1, 1024, 0, st>>>(n, dirs, d, perm, octb);
    return cudaGetLastError();
}

cudaError_t launch_scan_rows_to(const unsigned long long *src, unsigned long long *dst, int64_t rows, int T,
                                cudaStream_t st, bool pdl)
{
    if (rows <= 0) return cudaSuccess;
    if (T >= 1024 && rows <= 65535) {
        // a block of up to 1024 threads per row, about 8 entries per thread
        const int threads = std::min(1024, ((T + 7) / 8 + 31) / 32 * 32);
        return launch_kernel(scan_rows_block_kernel, dim3((unsigned)rows), dim3(threads), 0, st, pdl, src, dst, T);
    }
    const int wpb = 8;
    return launch_kernel(scan_rows_kernel, dim3((unsigned)((rows + wpb - 1) / wpb)), dim3(wpb * 32), 0, st, pdl, src, dst,
                         rows, T);
}

cudaError_t launch_scan_rows(unsigned long long *data, int64_t rows, int T, cudaStream_t st)
{
    return launch_scan_rows_to(data, data, rows, T, st);
}

// Copy of n doubles (src: device memory or mapped pinned host memory).
__global__ void copy_f64_kernel(const double *__restrict__ src, double *__restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

cudaError_t launch_copy_f64(const double *src, double *dst, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    copy_f64_kernel<<<grid_for(n, 256), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_suffix_rows(const int64_t *in, int64_t *out, int64_t rows, int T, long long smax, int *status,
                               cudaStream_t st)
{
    const int wpb = 8;
    suffix_rows_kernel<<<(unsigned)((rows + wpb - 1) / wpb), wpb * 32, 0, st>>>(in, out, rows, T, smax, status);
    return cudaGetLastError();
}

cudaError_t launch_weights_to_fixed(int wt, const void *w, int64_t nv, int frac_bits, int64_t *out,
                                    unsigned long long *maxabs, int *bad, cudaStream_t st)
{
    const unsigned g = grid_for(nv, 256);
    switch (wt) {
    case WT_U8: weights_to_fixed_kernel<WT_U8><<<g, 256, 0, st>>>(w, nv, frac_bits, out, maxabs, bad); break;
    case WT_I64: weights_to_fixed_kernel<WT_I64><<<g, 256, 0, st>>>(w, nv, frac_bits, out, maxabs, bad); break;
    case WT_F32: weights_to_fixed_kernel<WT_F32><<<g, 256, 0, st>>>(w, nv, frac_bits, out, maxabs, bad); break;
    default: weights_to_fixed_kernel<WT_ONE><<<g, 256, 0, st>>>(w, nv, frac_bits, out, maxabs, bad); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_weights_check(int wt, const void *w, int64_t nv, int frac_bits, int64_t limit, int *status,
                                 cudaStream_t st)
{
    const unsigned g = grid_for(nv, 256);
    switch (wt) {
    case WT_U8: weights_check_kernel<WT_U8><<<g, 256, 0, st>>>(w, nv, frac_bits, limit, status); break;
    case WT_I64: weights_check_kernel<WT_I64><<<g, 256, 0, st>>>(w, nv, frac_bits, limit, status); break;
    case WT_F32: weights_check_kernel<WT_F32><<<g, 256, 0, st>>>(w, nv, frac_bits, limit, status); break;
    default: return cudaSuccess;
    }
    return cudaGetLastError();
}

cudaError_t launch_max_abs_f64(const double *x, int64_t n, int stride, int offset, unsigned long long *Mbits,
                               cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    max_abs_f64_kernel<<<grid_for(n, 256), 256, 0, st>>>(x, n, stride, offset, Mbits);
    return cudaGetLastError();
}

cudaError_t launch_weights_to_w32(int wt, const void *w, int64_t nv, int frac_bits, int64_t limit, int32_t *out,
                                  int *status, cudaStream_t st)
{
    const unsigned g = grid_for(nv, 256);
    if (wt == WT_U8 && limit >= 255 && (reinterpret_cast<uintptr_t>(w) & 15u) == 0) {
        weights_u8_to_w32_kernel<<<grid_for(std::max<int64_t>(nv >> 4, 1), 256), 256, 0, st>>>(
            static_cast<const uint8_t *>(w), nv, out);
        return cudaGetLastError();
    }
    switch (wt) {
    case WT_U8: weights_to_w32_kernel<WT_U8><<<g, 256, 0, st>>>(w, nv, frac_bits, limit, out, status); break;
    case WT_I64: weights_to_w32_kernel<WT_I64><<<g, 256, 0, st>>>(w, nv, frac_bits, limit, out, status); break;
    case WT_F32: weights_to_w32_kernel<WT_F32><<<g, 256, 0, st>>>(w, nv, frac_bits, limit, out, status); break;
    default: weights_to_w32_kernel<WT_ONE><<<g, 256, 0, st>>>(w, nv, frac_bits, limit, out, status); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_quantize(const double *G, int64_t n, int log2_headroom, unsigned long long *maxbits,
                                 long long *out, double *scale, int *status, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        max_abs_f64_kernel<<<grid_for(n, 256), 256, 0, st>>>(G, n, 1, 0, maxbits);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    grad_quantize_kernel<<<grid_for(std::max<int64_t>(n, 1), 256), 256, 0, st>>>(G, n, maxbits, log2_headroom, out, scale,
                                                                               status);
    return cudaGetLastError();
}

cudaError_t launch_finite_check(const double *x, int64_t n, int *bad, int flag, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    finite_check_kernel<<<grid_for(n, 256), 256, 0, st>>>(x, n, bad, flag);
    return cudaGetLastError();
}

cudaError_t launch_index_check(const int32_t *idx, int64_t n, int64_t nv, int *bad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    index_check_kernel<<<grid_for(n, 256), 256, 0, st>>>(idx, n, nv, bad);
    return cudaGetLastError();
}

}  // namespace wect
