// wect_device.cuh -- device-side building blocks shared by the WECT kernels (sm_103a).
//
// Binning.  The transform needs, for every vertex v and direction p, the exact bin
//     bin(h) = #{q in [0, T-2] : beta[q] < h},   h = fma chain of x(v) . s_p in float64,
// i.e. the index alpha of Eq. "left-adjoint" taken as an exact count (Eq. "galois").  GB300's
// float64 rate is about 1/64 of its float32 rate, so the kernels decide each bin with a
// float32 filter and fall back to the exact float64 evaluation only when the filter cannot
// decide: with u = (h - lo)/step the thresholds sit (within e_q, |e_q| < 2^-40 T) at the
// integers, and if a rigorous enclosure [u_lo, u_hi] of u contains no integer then
// bin = clamp(ceil(u_hi), 0, T-1).  ceil is read off the low mantissa bits of
// u + 1.5 * 2^23 rounded upward.  The enclosure comes from directed-rounding fma on a
// per-row offset computed in double-single arithmetic (two float32 words).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wect {

constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
constexpr int32_t kMagicBits = 0x4B400000;     // bit pattern of kMagic
constexpr int kMaxN = 3;              // grid dimension (cubical complexes)
constexpr int kMaxSimplexN = 4;       // ambient dimension of simplicial complexes
constexpr int kMaxSimplexDim = 4;     // top simplex dimension of simplicial complexes

// device status word bits
constexpr int kStatusOverflow = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusBadIndex = 4;

// weight storage types (mirror wect_wtype)
constexpr int WT_U8 = 0;
constexpr int WT_I64 = 1;
constexpr int WT_F32 = 2;
constexpr int WT_ONE = 3;

// One cubical grid as seen by the kernels.
struct GridDesc {
    const int32_t *w;    // vertex weights as int32 fixed point (all ones when unweighted)
    int L[3];            // axis lengths, 1 for unused axes
    int rows;            // L[1] * L[2]
    int64_t nv;          // vertex count
    int64_t v_off;       // vertex offset of this complex in concatenated per-vertex arrays
    int *status;         // device status word of the complex
    const double *xg;    // grid coordinates [L0 + L1 + L2] (axis 0, then 1, then 2), or null
    const void *tmap;    // TMA tensor map of w as a 3-D [L2][L1][L0] int32 tensor, or null
    // the forward stencil kernel walks axis-0 rows in segments of seg vertices (nseg per row)
    // when the rows are longer than its shared row buffers; seg = 0: whole rows
    int seg = 0;
    int nseg = 1;
};

// A unit of work of the cubical kernels: one complex, one direction tile, a row range (units of
// rows or row segments), and for the forward stencil kernel a threshold tile (0 when untiled).
struct WorkItem {
    int cx;
    int dtile;
    int r0, r1;
    int tt = 0;
};

// ------------------------------------------------------------------ float64 exact path

__device__ __forceinline__ double grid_coord(int i, int L)
{
    if (L <= 1) return 0.0;
    return __ddiv_rn((double)(2 * i - (L - 1)), (double)(L - 1));
}

// Grid coordinate of index i on axis a, from the complex's table when it has one (the same
// correctly rounded quotient as grid_coord, computed once when the complex is created).
__device__ __forceinline__ double gcoord(const GridDesc &g, int a, int i)
{
    if (g.xg) return __ldg(g.xg + (a >= 1 ? g.L[0] : 0) + (a >= 2 ? g.L[1] : 0) + i);
    return grid_coord(i, g.L[a]);
}

// h = x[n-1]*s[n-1], then fma from n-2 down to 0 (every op rounded on its own).
template <int N>
__device__ __forceinline__ double height3(double x0, double x1, double x2, const double *s)
{
    if (N == 1) return __dmul_rn(x0, s[0]);
    if (N == 2) return __fma_rn(x0, s[0], __dmul_rn(x1, s[1]));
    return __fma_rn(x0, s[0], __fma_rn(x1, s[1], __dmul_rn(x2, s[2])));
}

// The same rule for N coordinates in an array (simplicial complexes, N <= 4).
template <int N>
__device__ __forceinline__ double heightv(const double *x, const double *s)
{
    double h = __dmul_rn(x[N - 1], s[N - 1]);
#pragma unroll
    for (int c = N - 2; c >= 0; --c) h = __fma_rn(x[c], s[c], h);
    return h;
}

// Exact bin of h against the float64 threshold table, starting from a nearby candidate.
// Both loops are bounded by T.
__device__ __forceinline__ int exact_bin_from(double h, const double *__restrict__ beta, int T, int cand)
{
    int b = cand < 0 ? 0 : (cand > T - 1 ? T - 1 : cand);
    while (b > 0 && h <= beta[b - 1]) --b;
    while (b < T - 1 && h > beta[b]) ++b;
    return b;
}

// ------------------------------------------------------------------ double-single helpers

struct DS {
    float hi, lo;
};

__device__ __forceinline__ DS ds_from_double(double v)
{
    DS r;
    r.hi = __double2float_rn(v);
    r.lo = __double2float_rn(__dsub_rn(v, (double)r.hi));
    return r;
}

// k * B for an exactly representable float k (|k| < 2^24).
__device__ __forceinline__ DS ds_mul_small(float k, DS b)
{
    DS r;
    r.hi = __fmul_rn(k, b.hi);
    r.lo = __fmaf_rn(k, b.hi, -r.hi);            // exact residual of k * b.hi
    r.lo = __fmaf_rn(k, b.lo, r.lo);
    return r;
}

__device__ __forceinline__ DS ds_add(DS a, DS b)
{
    float s = __fadd_rn(a.hi, b.hi);
    float z = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
    DS r;
    r.hi = s;
    r.lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return r;
}

// ------------------------------------------------------------------ per-direction filter setup

// Float32 filter constants of one direction for a grid with axis lengths L:
//   S0 = s0 / ((L0-1) step), B1, B2 = s_a / ((L_a-1) step) (double-single), C = -lo/step (double-single),
// eta = rigorous bound on |u_filter - u_exact| excluding the per-row offset rounding handled below.
struct DirFilter {
    float S0;
    DS B1, B2, C;
    float eta;
    int oct;     // bit a set when s_a > 0 (the cell maximum sits at the upper corner on axis a)
};

template <int N>
__device__ __forceinline__ DirFilter make_dir_filter(const double *s, const int *L, double lo, double hi, double step, int T)
{
    DirFilter f;
    f.oct = 0;
    for (int a = 0; a < N; ++a)
        if (s[a] > 0.0) f.oct |= 1 << a;
    double sumabs = 0.0;
    for (int a = 0; a < N; ++a) sumabs += fabs(s[a]);
    // |u| <= big for every vertex: the float32 filter is sound while big stays well inside the
    // magic-constant range (|u| < 2^22); beyond 2^21 every bin takes the exact path
    const double big = (step > 0.0) ? (double)T + (fabs(lo) + fabs(hi) + sumabs) / step + 1.0 : 0.0;
    if (!(step > 0.0) || !(big <= 0x1p21)) {
        // degenerate or very narrow range: force the exact path everywhere
        f.S0 = 0.f;
        f.B1 = f.B2 = f.C = DS{0.f, 0.f};
        f.eta = __int_as_float(0x7f800000);
        return f;
    }
    double b0 = (L[0] > 1) ? __ddiv_rn(s[0], __dmul_rn((double)(L[0] - 1), step)) : 0.0;
    double b1 = (N >= 2 && L[1] > 1) ? __ddiv_rn(s[1], __dmul_rn((double)(L[1] - 1), step)) : 0.0;
    double b2 = (N >= 3 && L[2] > 1) ? __ddiv_rn(s[2], __dmul_rn((double)(L[2] - 1), step)) : 0.0;
    f.S0 = __double2float_rn(b0);
    f.B1 = ds_from_double(b1);
    f.B2 = ds_from_double(b2);
    f.C = ds_from_double(__ddiv_rn(-lo, step));
    double A0 = fabs((double)f.S0) * (double)(L[0] > 1 ? L[0] - 1 : 0);
    double eta = (1.0 + 0x1p-10) * (0x1p-25 + A0 * 0x1p-24) + 0x1p-40 * big;
    f.eta = __double2float_ru(eta);
    return f;
}

// Per-row filter state of one direction: u(i0) = k0 * S0 + Goff, k0 = 2 i0 - (L0-1), shifted
// by the integer nr so that |Goff| <= 1/2.  Glo/Ghi enclose the exact offset within eta.
struct RowFilter {
    float Glo, Ghi;
    int nr;
};

template <int N>
__device__ __forceinline__ RowFilter make_row_filter(const DirFilter &f, int i1, int i2, const int *L)
{
    DS g = f.C;
    if (N >= 2) g = ds_add(g, ds_mul_small((float)(2 * i1 - (L[1] - 1)), f.B1));
    if (N >= 3) g = ds_add(g, ds_mul_small((float)(2 * i2 - (L[2] - 1)), f.B2));
    float nrf = rintf(g.hi);
    float off = __fadd_rn(__fsub_rn(g.hi, nrf), g.lo);
    RowFilter r;
    r.nr = (int)nrf;
    r.Glo = __fsub_rd(off, f.eta);
    r.Ghi = __fadd_ru(off, f.eta);
    return r;
}

// ceil() of the enclosure ends; equal results mean the bin is decided.
__device__ __forceinline__ void filter_ceil(float k0, float S0, float Glo, float Ghi, int &tlo, int &thi)
{
    float ul = __fmaf_rd(k0, S0, Glo);
    float uh = __fmaf_ru(k0, S0, Ghi);
    tlo = __float_as_int(__fadd_ru(ul, kMagic));
    thi = __float_as_int(__fadd_ru(uh, kMagic));
}

// Candidate bin from the upper end of the filter, clamped to [0, T-1].  A negative thi is a
// negative float32 sum, i.e. u far below the range (bin 0).
__device__ __forceinline__ int clamp_bin(int thi, int nr, int T)
{
    return thi < 0 ? 0 : min(max(thi - kMagicBits + nr, 0), T - 1);
}

// Two directions at once with the packed float32 pipe (sm_100+ f32x2): element-wise the same
// IEEE operations, with the same directed roundings, as filter_ceil.
struct F2 {
    unsigned long long v;
};

__device__ __forceinline__ F2 f2_pack(float a, float b)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ F2 f2_add_rn(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ void filter_ceil2(F2 k0, F2 S0, F2 Glo, F2 Ghi, F2 M, int &tlo_a, int &thi_a, int &tlo_b,
                                             int &thi_b)
{
    unsigned long long ul, uh, tl, th;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(ul) : "l"(k0.v), "l"(S0.v), "l"(Glo.v));
    asm("fma.rp.f32x2 %0, %1, %2, %3;" : "=l"(uh) : "l"(k0.v), "l"(S0.v), "l"(Ghi.v));
    asm("add.rp.f32x2 %0, %1, %2;" : "=l"(tl) : "l"(ul), "l"(M.v));
    asm("add.rp.f32x2 %0, %1, %2;" : "=l"(th) : "l"(uh), "l"(M.v));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(tlo_a), "=r"(tlo_b) : "l"(tl));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(thi_a), "=r"(thi_b) : "l"(th));
}

// ------------------------------------------------------------------ weights

template <int WT>
__device__ __forceinline__ int64_t load_weight_fixed(const void *w, int64_t v, int frac_bits)
{
    if (WT == WT_U8) return (int64_t)__ldg((const uint8_t *)w + v);
    if (WT == WT_I64) return __ldg((const long long *)w + v);
    if (WT == WT_F32) return __float2ll_rn(ldexpf(__ldg((const float *)w + v), frac_bits));
    return 1;
}

// ------------------------------------------------------------------ misc

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Programmatic dependent launch: let the next kernel of the stream (launched with the
// programmatic-serialization attribute) start, and wait until the kernels this grid depends on
// have completed with their memory visible.  Both are no-ops without such a launch.
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Bytes of dynamic shared memory the CTA was launched with.
__device__ __forceinline__ uint32_t dynamic_smem_bytes()
{
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// Orders this thread's generic-proxy shared-memory accesses before later async-proxy (TMA)
// accesses of the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void red_shared_add(uint32_t addr, int32_t v)
{
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v));
}

__device__ __forceinline__ void red_shared_add_u32(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

__device__ __forceinline__ void lds_v2u64(uint32_t addr, unsigned long long &a, unsigned long long &b)
{
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}

__device__ __forceinline__ int lds_s32(uint32_t addr)
{
    int v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ long long lds_s64(uint32_t addr)
{
    long long v;
    asm volatile("ld.shared.s64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ int4 lds128(uint32_t addr)
{
    int4 r;
    asm volatile("ld.shared.v4.s32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(addr));
    return r;
}

// ------------------------------------------------------------------ TMA and mbarriers

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// Makes mbarrier initialisations visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, at most about 2^20 polls with a short
// sleep between them (a few tens of milliseconds); false when the wait ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity)
{
    for (int k = 0; k < (1 << 20); ++k) {
        if (mbar_test_wait(mbar, parity)) return true;
        __nanosleep(32);
    }
    return false;
}

// TMA tile load of a 3-D box at coordinates (x, y, z) of the tensor described by tmap (a tensor
// map in global memory) into shared memory at dst, completing on the mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void *tmap, int x, int y, int z, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

// Round a signed 128-bit integer (hi:lo) to the nearest double, ties to even.
__device__ __forceinline__ double i128_to_double(int64_t hi, uint64_t lo)
{
    bool neg = hi < 0;
    uint64_t h = (uint64_t)hi, l = lo;
    if (neg) {                                    // two's complement negate
        l = ~l + 1ull;
        h = ~h + (l == 0ull ? 1ull : 0ull);
    }
    if (h == 0ull) {
        // |v| < 2^64: round the 64-bit magnitude
        if (l == 0ull) return 0.0;
        int lz = __clzll((long long)l);
        int top = 63 - lz;                        // index of the leading one
        double r;
        if (top <= 52) {
            r = (double)l;                        // exact
        } else {
            int sh = top - 52;
            uint64_t m = l >> sh;
            uint64_t rem = l & ((1ull << sh) - 1ull);
            uint64_t half = 1ull << (sh - 1);
            if (rem > half || (rem == half && (m & 1ull))) ++m;
            r = ldexp((double)m, sh);             // m <= 2^53, exact scaling
        }
        return neg ? -r : r;
    }
    int lz = __clzll((long long)h);
    int top = 127 - lz;                           // leading one of the 128-bit magnitude
    int sh = top - 52;                            // >= 12
    // m = magnitude >> sh (53 bits), guard = next bit, sticky = any bit below it
    uint64_t m, guard, sticky;
    if (sh >= 64) {
        int s2 = sh - 64;
        m = h >> s2;
        uint64_t remh = s2 ? (h & ((1ull << s2) - 1ull)) : 0ull;
        guard = s2 ? ((h >> (s2 - 1)) & 1ull) : (l >> 63);
        uint64_t below = s2 ? (remh & ((1ull << (s2 - 1)) - 1ull)) : 0ull;
        uint64_t lbelow = s2 ? l : (l & ~(1ull << 63));
        sticky = (below | lbelow) ? 1ull : 0ull;
    } else {
        m = (h << (64 - sh)) | (l >> sh);
        guard = (l >> (sh - 1)) & 1ull;
        sticky = (l & ((1ull << (sh - 1)) - 1ull)) ? 1ull : 0ull;
    }
    if (guard && (sticky || (m & 1ull))) ++m;
    double r = ldexp((double)m, sh);
    return neg ? -r : r;
}

}  // namespace wect
