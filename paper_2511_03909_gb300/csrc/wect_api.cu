// wect_api.cu -- the C ABI declared in include/wect.h: handles, validation, workspace,
// dispatch to the kernels, batches (persistent launch + CUDA graph) and the tile autotuner.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/wect.h"
#include "wect_device.cuh"
#include "wect_launch.h"

using namespace wect;

// ------------------------------------------------------------------ errors and accounting

static thread_local std::string g_last_error;
static std::atomic<int> g_last_stencil{0};      // 0 none, 1 per-vertex, 2 run-based, 3 global histogram
static std::atomic<int64_t> g_launches{0};

static wect_status fail(wect_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

// Allocation-failure injection for tests: the number of device allocations that still succeed
// before one fails (-1: disarmed).  The failing allocation disarms the hook.
static std::atomic<int64_t> g_alloc_fail_in{-1};

namespace wect {
void note_error(const char *msg) { g_last_error = msg; }
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t dev_malloc(void **p, size_t bytes)
{
    int64_t k = g_alloc_fail_in.load();
    while (k >= 0 && !g_alloc_fail_in.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
}  // namespace wect

static wect_status cuda_fail(cudaError_t e, const char *where)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(WECT_ERR_OUT_OF_MEMORY, "%s: %s", where, cudaGetErrorString(e));
    return fail(WECT_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

// a launch of one of our kernels (counted for launch accounting)
#define KL(call, where)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
        g_launches.fetch_add(1, std::memory_order_relaxed); \
    } while (0)

// ------------------------------------------------------------------ profiling hook

static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_events;

struct ProfScope {
    cudaStream_t st;
    cudaEvent_t e1 = nullptr;
    explicit ProfScope(cudaStream_t s) : st(s)
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_prof_on) return;
        cudaEvent_t e0;
        if (cudaEventCreate(&e0) != cudaSuccess) return;
        if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); e1 = nullptr; return; }
        cudaEventRecord(e0, st);
        g_prof_events.push_back({e0, e1});
    }
    ~ProfScope()
    {
        if (e1) cudaEventRecord(e1, st);
    }
};

static bool range_is_default(double lo, double hi) { return std::isnan(lo) && std::isnan(hi); }

static wect_status check_range(double lo, double hi, int T)
{
    if (T < 2) return fail(WECT_ERR_INVALID_ARG, "T must be >= 2 (got %d)", T);
    if (T > 65535) return fail(WECT_ERR_UNSUPPORTED, "T must be <= 65535 (got %d)", T);
    if (range_is_default(lo, hi)) return WECT_OK;
    if (!std::isfinite(lo) || !std::isfinite(hi)) return fail(WECT_ERR_INVALID_ARG, "lo/hi must be finite or both NaN");
    if (lo > hi) return fail(WECT_ERR_INVALID_ARG, "lo > hi");
    return WECT_OK;
}

static int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

static size_t smem_optin()
{
    static int v = 0;
    if (v == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (v <= 0) v = 48 * 1024;
    }
    return (size_t)v;
}

static size_t smem_per_sm()
{
    static int v = 0;
    if (v == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (v <= 0) v = 100 * 1024;
    }
    return (size_t)v;
}

// CTAs per SM that a grid is sized for: the shared-memory and thread-slot limits.  Registers may
// allow fewer to be resident; the kernels are persistent (work queue), so CTAs that start later
// find the remaining items or none.
static int ctas_per_sm_for(size_t smem, int threads)
{
    int k = (int)(smem_per_sm() / (smem + 2048));
    k = std::min(k, 2048 / threads);
    return std::max(1, k);
}

// ------------------------------------------------------------------ device buffers

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t cap = 0;   // elements
    cudaError_t ensure(size_t n)
    {
        if (n <= cap && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = dev_malloc((void **)&p, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) cap = std::max<size_t>(n, 1);
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// Per-call workspace shared by the compute entry points of one complex or batch.
struct Workspace {
    DBuf<double> range;           // [6]: lo, hi, step, max|x_0..2|
    DBuf<double> beta;            // [T]
    DBuf<unsigned long long> M;   // [2]: max-abs bits, scratch (argmax key of the default range)
    DBuf<int> cand;               // default range of a simplicial complex: {count, L, Smax, 0, candidates}
    DBuf<int> counter;            // work-queue head
    DBuf<int> perm, octb;         // octant grouping of the directions
    DBuf<uint16_t> bins;          // vertex bins
    DBuf<float> dtab;             // [d][8] float32 bin filter per direction (simplicial)
    DBuf<int64_t> S;              // suffix sums of the upstream gradient
    DBuf<int64_t> Rv;             // per-vertex octant sums (adjoint)
    DBuf<unsigned long long> Iacc;
    DBuf<long long> Gq;           // quantised upstream gradient
    DBuf<double> gscale;          // its power-of-two scale
    DBuf<WorkItem> items;
    DBuf<WorkItem> items_bwd;
    DBuf<int> ranges_bwd;         // per CTA of the octant sums: its first item (and the end)
    DBuf<double> hdirs;           // wect_compute_host: device copy of the directions
    DBuf<int64_t> hout;           // wect_compute_host: the difference table before its scan
    DBuf<unsigned char> hw;       // wect_compute_host: staged pageable weights
    // cache key of the uploaded item list
    std::tuple<int, int, int, int, int> items_key{-1, -1, -1, -1, -1};
    std::tuple<int, int> items_bwd_key{-1, -1};
    int n_items = 0, n_items_bwd = 0, n_ctas_bwd = 0;
    void release()
    {
        range.release(); beta.release(); M.release(); cand.release(); counter.release(); perm.release(); octb.release();
        bins.release(); dtab.release(); S.release(); Rv.release(); Iacc.release(); Gq.release(); gscale.release(); items.release();
        items_bwd.release(); ranges_bwd.release(); hdirs.release(); hout.release(); hw.release();
    }
};

// ------------------------------------------------------------------ handles

struct wect_complex_s {
    int kind = 0;                  // 0 = cubical, 1 = simplicial
    int n = 0;
    int64_t nv = 0;
    int L[3] = {1, 1, 1};
    int wtype = WECT_W_ONE;
    int frac_bits = 0;
    size_t wbytes = 0;             // bytes per raw vertex weight
    int32_t *d_w32 = nullptr;      // cubical: int32 fixed-point vertex weights read by the kernels
    double *d_xg = nullptr;        // cubical: grid coordinates [L0 + L1 + L2]
    void *d_tmap = nullptr;        // cubical: TMA tensor map of d_w32 (null when the grid does not qualify)
    int nsplit = 1;
    int64_t climit = 0;            // cubical: max |c_o(v)|; simplicial: max |w(s)|
    int kflush = 1 << 16;
    int64_t cells[kMaxSimplexDim + 1] = {};
    // simplicial
    double *d_coords = nullptr;
    float *d_xf = nullptr;         // float32 copies of the coordinates (round to nearest)
    int max_dim = 0;
    int64_t counts[kMaxSimplexDim + 1] = {};
    int32_t *d_simp[kMaxSimplexDim + 1] = {};
    int64_t *d_sw[kMaxSimplexDim + 1] = {};            // d_sw[0] = vertex weights (fixed)
    // staged gather: per list of dim >= 1, chunk-local ids and per-chunk vertex lists
    int2 *d_swp[kMaxSimplexDim + 1] = {};              // packed signed weights of the gather
    uint16_t *d_local[kMaxSimplexDim + 1] = {};
    int32_t *d_cverts[kMaxSimplexDim + 1] = {};
    int32_t *d_cnu[kMaxSimplexDim + 1] = {};
    int64_t nchunks[kMaxSimplexDim + 1] = {};
    int sw_mode = WECT_SW_MAX_OF_VERTICES;
    // device state
    int *d_status = nullptr;
    GridDesc *d_grid = nullptr;
    Workspace ws;
    std::mutex mu;
};

// What a captured forward graph reads from the batch's workspace besides the arguments in its
// key: the buffers' addresses and the uploaded item list (named by its key).  A later call with
// other sizes may grow a buffer (new address) or upload other items; the graph is then stale.
using GraphDeps = std::tuple<const void *, const void *, const void *, const void *, const void *, const void *,
                             const void *, std::tuple<int, int, int, int, int>, int>;

static GraphDeps graph_deps(const Workspace &ws)
{
    return GraphDeps(ws.M.p, ws.range.p, ws.beta.p, ws.perm.p, ws.octb.p, ws.counter.p, ws.items.p, ws.items_key,
                     ws.n_items);
}

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;
    GraphDeps deps{};
};

struct BatchConfig {
    int dpl = 0, Dt = 0;
    bool run = false;             // the run-based kernel (dpl 1)
    int threads = 512;            // CTA size of the per-vertex kernel
};

struct wect_batch_s {
    int count = 0;
    int n = 0;
    int wtype = WECT_W_ONE;
    int frac_bits = 0;
    int nsplit = 1;
    int64_t climit = 0;
    int kflush = 1 << 16;
    int64_t total_nv = 0;
    int maxL0 = 1;                 // longest unit of the forward stencil kernel (a row or a segment)
    double meanL0 = 1.0;           // mean unit length over all units of the batch
    bool segmented = false;        // some grid's rows are walked in segments
    std::vector<GridDesc> h_grids;
    std::vector<int64_t> v_off;
    GridDesc *d_grids = nullptr;
    int *d_status = nullptr;
    int32_t *d_w32 = nullptr;      // owned concatenated int32 weights (create_cubical), else nullptr
    double *d_xg = nullptr;        // owned grid-coordinate tables (create_cubical), else nullptr
    void *d_tmaps = nullptr;       // owned TMA tensor maps of the grids (create_cubical), else nullptr
    bool has_tmap = false;         // some grid has a tensor map
    bool owns_w = false;
    Workspace ws;
    std::map<std::pair<int, int>, BatchConfig> tuned;    // (d, T) -> tile shape
    std::vector<int> loop_starts;                        // per-complex item ranges of the loop path
    std::map<std::tuple<const void *, int, int, double, double, void *, void *, int, int>, GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr;
    std::mutex mu;
};

static size_t wtype_bytes(int wt)
{
    switch (wt) {
    case WECT_W_U8: return 1;
    case WECT_W_I64_FIXED: return 8;
    case WECT_W_F32: return 4;
    default: return 0;
    }
}

static wect_status check_wtype(int wt, int frac_bits)
{
    if (wt < WECT_W_U8 || wt > WECT_W_ONE) return fail(WECT_ERR_INVALID_ARG, "unknown weight type %d", wt);
    if (wt == WECT_W_F32 && (frac_bits < 0 || frac_bits > 40))
        return fail(WECT_ERR_INVALID_ARG, "frac_bits must be in [0, 40] (got %d)", frac_bits);
    return WECT_OK;
}

// Accumulator mode of a cubical complex from the largest fixed-point vertex weight.  The
// per-vertex contribution c_o(v) is a signed sum of 2^n cell weights, |c| <= 2^n max|w|.
static wect_status choose_cubical_mode(int n, int wt, uint64_t wmax, int &nsplit, int64_t &climit, int &kflush)
{
    const int64_t two_n = 1ll << n;
    if (wt == WECT_W_U8 || wt == WECT_W_ONE) {
        climit = two_n * 255;
        nsplit = 1;
        kflush = (int)std::min<int64_t>((((int64_t)1 << 31) - 1) / climit, 1 << 30);
        return WECT_OK;
    }
    const double cmax = (double)two_n * (double)wmax;
    if (cmax <= (double)(1 << 14)) {              // narrow: one plane, 2x headroom for later weights
        nsplit = 1;
        climit = 1 << 15;
        kflush = 1 << 16;
        return WECT_OK;
    }
    if (cmax < 2147483647.0) {                   // two planes: low 16 bits + signed high part
        nsplit = 2;
        climit = 2147483647ll;
        kflush = 1 << 16;
        return WECT_OK;
    }
    return fail(WECT_ERR_OVERFLOW, "cell contributions 2^n*max|w| = %.3g exceed 2^31", cmax);
}

// ------------------------------------------------------------------ tile shapes (cubical)

struct CubShape {
    int dpl, Dt, ctas_per_sm, grid;
    size_t smem;
    bool gh = false;              // global-histogram variant (T x Dt does not fit shared memory)
    bool run = false;             // run-based kernel (walks bin boundaries along the rows)
    int threads = 512;            // CTA size
    int L0s = 0;                  // > 0: TMA staging of the neighbouring rows (per-vertex kernel)
    int Tt = 0;                   // > 0: threshold tiles of Tt bins, one pass over the grid each
};


// Stencil variant selection: 0 = by cost estimate, 1 = per-vertex kernel only, 2 = the run-based
// kernel wherever it applies, 3 = per-vertex kernel without TMA row staging (test hook
// wect_debug_stencil_variant).
static std::atomic<int> g_stencil_variant{0};

// Should a grid with rows of L0 vertices (mean) take the run-based kernel for T thresholds over a
// range of width span (NaN: the default range)?  A row of a spread-out direction set crosses
// about 2 E|s_0| / step ~ 1.2 / step bin boundaries.  Measured on the 128^3 u8 volume with 256
// Fibonacci directions (CUDA events, the library's kernel hook): the run kernel costs ~140 us of
// row set-up (octant contributions, prefix sums, end bins; latency-bound) plus ~4 us per million
// boundaries, the per-vertex kernel 200-270 us whatever T.  So the runs win only with a few
// boundaries per long row: T = 8 took 178 us against 267 us, T = 32 286 us against 216 us.
static bool run_profitable(int n, double meanL0, int T, double span)
{
    if (!(span > 0.0)) span = 2.0 * std::sqrt((double)n);
    const double step = span / (double)(T - 1);
    const double runs = 1.0 + 1.2 / step;
    return runs <= 4.0 && meanL0 >= 96.0;
}

// Run-based kernel shape: one direction per lane, the widest tile up to 256 that fits.
static bool run_shape(int n, int d, int T, int maxL0, CubShape &out, int Dt_req = 0)
{
    const size_t limit = smem_optin() - 1024;
    int Dmax = 32;
    while (Dmax < d && Dmax < 256) Dmax *= 2;
    for (int Dt = (Dt_req > 0 ? Dt_req : Dmax); Dt >= 32; Dt /= 2) {
        const size_t sm = cubical_run_smem(n, T, Dt, maxL0);
        if (sm > limit) {
            if (Dt_req > 0) return false;
            continue;
        }
        out.dpl = 1;
        out.Dt = Dt;
        out.smem = sm;
        out.ctas_per_sm = ctas_per_sm_for(sm, cubical_run_threads());
        out.grid = sm_count() * out.ctas_per_sm;
        out.gh = false;
        out.run = true;
        out.threads = cubical_run_threads();
        return true;
    }
    return false;
}

// Tile shape of the stencil kernel: the widest direction tile (fewest passes over the grid)
// that fits shared memory, then the most directions per lane.  dpl_req / Dt_req pin a shape.
// With run_ok (one histogram plane) the run-based kernel is taken when it is estimated cheaper
// (meanL0 rows, a threshold range of width span), or always under the test hook.
static bool cub_shape(int n, int nsplit, int d, int T, int maxL0, CubShape &out, int dpl_req = 0, int Dt_req = 0,
                      double meanL0 = 0.0, double span = 0.0, int threads_req = 0, bool tma_ok = false,
                      bool segmented = false)
{
    const int threads = threads_req > 0 ? threads_req : cubical_fwd_threads();
    const int warps = threads / 32;
    out.threads = threads;
    out.L0s = 0;
    out.Tt = 0;
    // TMA staging of the neighbouring rows when some grid has a tensor map and it fits next to
    // the histogram (else plain loads)
    const int L0s = (tma_ok && g_stencil_variant.load() != 3) ? cubical_fwd_stage_len(n, maxL0) : 0;
    const size_t limit = smem_optin() - 1024;
    out.run = false;
    // (the run-based kernel walks whole rows: not for grids walked in segments)
    if (!segmented && nsplit == 1 && dpl_req == 0 && Dt_req == 0 && g_stencil_variant.load() != 1 &&
        g_stencil_variant.load() != 3) {
        const bool want = g_stencil_variant.load() == 2 ||
                          run_profitable(n, meanL0 > 0.0 ? meanL0 : (double)maxL0, T, span);
        if (want && run_shape(n, d, T, maxL0, out)) return true;
    }
    int Dmax = 32;
    while (Dmax < d && Dmax < 32 * 4 * warps) Dmax *= 2;
    for (int Dt = (Dt_req > 0 ? Dt_req : Dmax); Dt >= 32; Dt /= 2) {
        // two directions per lane first (measured fastest on the 128^3 workload), then four, then one
        for (int dpl : {2, 4, 1}) {
            if (dpl_req > 0 && dpl != dpl_req) continue;
            if (Dt % (32 * dpl)) continue;
            const int WC = Dt / (32 * dpl);
            if (WC > warps || warps % WC) continue;
            if (dpl > 1 && Dt / dpl < 32) continue;
            size_t sm = cubical_fwd_smem(n, nsplit, dpl, T, Dt, maxL0, false, threads);
            if (sm > limit) continue;
            if (L0s > 0) {
                const size_t smt = cubical_fwd_smem(n, nsplit, dpl, T, Dt, maxL0, false, threads, L0s);
                if (smt <= limit) {
                    sm = smt;
                    out.L0s = L0s;
                }
            }
            out.dpl = dpl;
            out.Dt = Dt;
            out.smem = sm;
            const int k = ctas_per_sm_for(sm, threads);
            out.ctas_per_sm = k;
            out.grid = sm_count() * k;
            out.gh = false;
            return true;
        }
        if (Dt_req > 0) break;
    }
    // no shared histogram of all T rows fits (for a pinned tile shape: that one): threshold tiles of Tt bins (plus a discard row on
    // each side), one pass over the grid per (direction tile, threshold tile).  A pass costs a
    // per-vertex part (octant contributions, row set-up) and a per-update part; measured on the
    // 128^3 volume (T = 128, 512, 1024 at tile widths 256, 64, 32) they weigh about 45 : 1 per
    // direction, so the cost is passes x (45 + Dt).  The cheapest shape wins (ties: the first,
    // widest), and it beats the global histogram.
    {
        int64_t bestCost = INT64_MAX;
        CubShape best;
        for (int Dt = (Dt_req > 0 ? Dt_req : Dmax); Dt >= 32; Dt /= 2)
            for (int dpl : {2, 4, 1}) {
                if ((Dt_req > 0 && Dt != Dt_req) || (dpl_req > 0 && dpl != dpl_req)) continue;
                if (Dt % (32 * dpl)) continue;
                const int WC = Dt / (32 * dpl);
                if (WC > warps || warps % WC) continue;
                if (dpl > 1 && Dt / dpl < 32) continue;
                const size_t fixed = cubical_fwd_smem(n, nsplit, dpl, 0, Dt, maxL0, false, threads);
                if (fixed >= limit) continue;
                int Tt = (int)((limit - fixed) / ((size_t)nsplit * Dt * 4u)) - 2;
                if (Tt < 16) continue;
                Tt = std::min(Tt, T);
                const int64_t cost = (int64_t)((d + Dt - 1) / Dt) * ((T + Tt - 1) / Tt) * (45 + Dt);
                if (cost >= bestCost) continue;
                bestCost = cost;
                best = CubShape{};
                best.threads = threads;
                best.dpl = dpl;
                best.Dt = Dt;
                best.Tt = Tt;
                best.smem = cubical_fwd_smem(n, nsplit, dpl, Tt + 2, Dt, maxL0, false, threads);
                if (L0s > 0) {
                    const size_t smt = cubical_fwd_smem(n, nsplit, dpl, Tt + 2, Dt, maxL0, false, threads, L0s);
                    if (smt <= limit) {
                        best.smem = smt;
                        best.L0s = L0s;
                    }
                }
            }
        if (bestCost < INT64_MAX) {
            out = best;
            const int k = ctas_per_sm_for(out.smem, threads);
            out.ctas_per_sm = k;
            out.grid = sm_count() * k;
            out.gh = false;
            out.run = false;
            return true;
        }
    }
    if (dpl_req > 0 || Dt_req > 0) return false;
    // not even threshold tiles fit: scatter into the global int64 difference table instead
    const int Dt = std::min(Dmax, 256);
    out.dpl = Dt >= 64 ? 2 : 1;
    out.Dt = Dt;
    out.smem = cubical_fwd_smem(n, 1, out.dpl, T, Dt, maxL0, true, threads);
    if (out.smem > limit) return false;
    if (L0s > 0) {
        const size_t smt = cubical_fwd_smem(n, 1, out.dpl, T, Dt, maxL0, true, threads, L0s);
        if (smt <= limit) {
            out.smem = smt;
            out.L0s = L0s;
        }
    }
    const int k = ctas_per_sm_for(out.smem, threads);
    out.ctas_per_sm = k;
    out.grid = sm_count() * k;
    out.gh = true;
    return true;
}

// Items for a set of grids: per complex, direction tiles x row chunks, largest first.  An item
// never holds more than kflush vertices (the int32 histogram bound); whole=true keeps one chunk
// per complex (the caller has checked that every complex fits).
// Axis-0 rows longer than seg_len(n, nsplit) vertices are walked by the forward stencil kernel in
// segments of that length (each a unit of work with its own shared row of octant contributions);
// shorter rows are whole units.  The length keeps the row buffers of the worst-case shape (16 row
// groups of one warp, NSPLIT planes of 2^n octant rows) within 128 KB for n = 3 and 64 KB for
// n = 1, 2, so every grid has a shape, and a one-warp direction tile keeps its shared histogram
// up to T ~ 1000 beside them (beyond, the global histogram).
static int seg_len(int n, int nsplit)
{
    const int base = (n >= 2) ? 256 : 512;
    return nsplit >= 2 ? base / 2 : base;
}

static void set_segments(GridDesc &g, int n, int nsplit)
{
    const int S = seg_len(n, nsplit);
    g.seg = (g.L[0] > S) ? S : 0;
    g.nseg = (g.L[0] > S) ? (g.L[0] + S - 1) / S : 1;
}

// Vertices of one unit (a row, or a segment of one) of the forward stencil kernel.
static int unit_len(const GridDesc &g) { return g.seg > 0 ? g.seg : g.L[0]; }

static std::vector<WorkItem> make_items(const std::vector<GridDesc> &grids, int d, int Dt, int T, int kflush,
                                        int target_items, bool whole, int Tt = 0)
{
    // direction tiles x threshold tiles (Tt > 0: each item covers Tt bins of one tile)
    const int nttiles = (Tt > 0) ? (T + Tt - 1) / Tt : 1;
    const int ntiles = (d + Dt - 1) / Dt * nttiles;
    const int HR = (Tt > 0) ? std::min(T, Tt + 2) : T;
    std::vector<std::pair<int64_t, WorkItem>> v;
    // items are ranges of units: rows, or row segments of long rows (unit u = row u / nseg,
    // segment u % nseg)
    int64_t total_units = 0;
    for (auto &g : grids) total_units += (int64_t)g.rows * g.nseg;
    for (int c = 0; c < (int)grids.size(); ++c) {
        const GridDesc &g = grids[c];
        const int units = g.rows * g.nseg, ul = unit_len(g);
        const int max_units = std::max(1, kflush / std::max(1, ul));
        int chunks = 1;
        if (!whole) {
            const double share = (double)units / (double)std::max<int64_t>(total_units, 1);
            chunks = (int)std::ceil(share * target_items / ntiles);
            // no item smaller than 8x its histogram flush (HR x Dt entries): units * length >= 8 HR
            const int min_units = (int)std::min<int64_t>(units, (8ll * HR + ul - 1) / std::max(1, ul));
            chunks = std::min(chunks, std::max(1, units / std::max(1, min_units)));
            chunks = std::max(chunks, (units + max_units - 1) / max_units);
            chunks = std::max(1, std::min(chunks, units));
            if (grids.size() == 1) {
                // one complex: the chunk count whose items fill the CTAs' rounds best (makespan
                // ceil(items / target) / chunks), fewest chunks on ties
                const int lo_c = std::max(1, (units + max_units - 1) / max_units);
                const int hi_c = std::max(lo_c, std::min(units, units / std::max(1, min_units)));
                double best = 1e30;
                for (int c2 = lo_c; c2 <= std::min(hi_c, lo_c + 4 * std::max(1, target_items)); ++c2) {
                    const int64_t items_n = (int64_t)ntiles * c2;
                    const double span = (double)((items_n + target_items - 1) / std::max(1, target_items)) / c2;
                    if (span < best - 1e-12) {
                        best = span;
                        chunks = c2;
                    }
                }
            }
        }
        const int per = (units + chunks - 1) / chunks;
        for (int t = 0; t < ntiles; ++t)
            for (int r0 = 0; r0 < units; r0 += per) {
                WorkItem w{c, t % ((d + Dt - 1) / Dt), r0, std::min(units, r0 + per), t / ((d + Dt - 1) / Dt)};
                v.push_back({(int64_t)(w.r1 - w.r0) * ul, w});
            }
    }
    std::stable_sort(v.begin(), v.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<WorkItem> out;
    out.reserve(v.size());
    for (auto &x : v) out.push_back(x.second);
    return out;
}

// ------------------------------------------------------------------ cubical launch sequence

struct CubLaunch {
    int n, nsplit, wt, frac_bits, kflush, maxL0;   // maxL0: longest unit (row or row segment)
    int64_t climit;
    const GridDesc *d_grids;
    Workspace *ws;
    int *status;                  // device status word (non-finite directions are flagged here)
    bool segmented = false;       // some grid walks its rows in segments
};

// Enqueue the forward transform of a set of grids: [range], beta, work queue, stencil kernel,
// [scan].  items must be uploaded in ws->items already.
static wect_status enqueue_cubical_fwd(const CubLaunch &L, const CubShape &sh, int n_items, bool direct,
                                       const double *dirs, int d, int T, double lo, double hi, bool dflt,
                                       int64_t out_rows, int64_t *out, cudaStream_t st, int64_t *final_out = nullptr,
                                       bool prep_early = false)
{
    Workspace &ws = *L.ws;
    if (dflt) {
        CK(cudaMemsetAsync(ws.M.p, 0, sizeof(unsigned long long), st), "memset");
        KL(launch_grid_max_abs(L.n, L.d_grids, dirs, d, ws.M.p, st), "grid_max_abs");
    }
    // outside a stream capture the preparation, the forward kernel and the scan are programmatic
    // dependent launches (each starts while the kernel before it finishes)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs), "capture status");
    const bool pdl = cs == cudaStreamCaptureStatusNone;
    KL(launch_fwd_prep(L.n, dirs, d, T, lo, hi, dflt ? 1 : 0, ws.M.p, ws.range.p, ws.beta.p, ws.perm.p, ws.octb.p,
                       ws.counter.p, L.status, direct ? nullptr : reinterpret_cast<unsigned long long *>(out),
                       out_rows * T, st, sh.run ? 1 : 0, pdl, pdl && prep_early && !dflt),
       "fwd_prep");
    CubicalFwdArgs a{};
    a.grids = L.d_grids;
    a.items = ws.items.p;
    a.n_items = n_items;
    a.counter = ws.counter.p;
    a.dirs = dirs;
    a.d = d;
    a.T = T;
    a.range = ws.range.p;
    a.beta = ws.beta.p;
    a.Dt = sh.Dt;
    a.CP = sh.run ? cubical_run_pitch(L.maxL0) : cubical_fwd_pitch(L.maxL0);
    a.perm = ws.perm.p;
    a.kflush = L.kflush;
    a.climit = L.climit;
    a.direct = direct ? 1 : 0;
    a.out = reinterpret_cast<unsigned long long *>(out);
    a.threads = sh.threads;
    a.L0s = sh.L0s;
    a.segmented = L.segmented ? 1 : 0;
    a.Tt = sh.Tt;
    {
        // with the profiling hook on, the kernel is launched in plain stream order, so that the
        // hook's events bracket all of it (an early start would fall before the first event)
        std::lock_guard<std::mutex> lk(g_prof_mu);
        a.pdl = (pdl && !g_prof_on) ? 1 : 0;
    }
    const int grid = std::max(1, std::min(sh.grid, n_items));
    {
        g_last_stencil.store(sh.run ? 2 : (sh.gh ? 3 : 1));
        auto launch = [&]() {
            return sh.run ? launch_cubical_run(L.n, a, grid, sh.smem, st)
                          : launch_cubical_fwd(L.n, L.nsplit, sh.dpl, sh.gh, a, grid, sh.smem, st);
        };
        if (cs == cudaStreamCaptureStatusNone) {
            ProfScope prof(st);
            KL(launch(), "cubical_fwd");
        } else {
            KL(launch(), "cubical_fwd");
        }
    }
    if (!direct)
        KL(launch_scan_rows_to(reinterpret_cast<unsigned long long *>(out),
                               reinterpret_cast<unsigned long long *>(final_out ? final_out : out), out_rows, T, st,
                               pdl && !sh.run),
           "scan_rows");
    return WECT_OK;
}

static int ceil_log2(int64_t x)
{
    int k = 0;
    while (((int64_t)1 << k) < x) ++k;
    return k;
}

static wect_status ensure_common_ws(Workspace &ws, int T, int d = 1)
{
    CK(ws.perm.ensure((size_t)d), "alloc");
    CK(ws.octb.ensure(9), "alloc");
    CK(ws.range.ensure(8), "alloc");      // lo, hi, step, max |x_a| for a < n <= 4, spare
    CK(ws.beta.ensure((size_t)T), "alloc");
    CK(ws.M.ensure(2), "alloc");
    CK(ws.counter.ensure(1), "alloc");
    return WECT_OK;
}

static wect_status upload_items(Workspace &ws, const std::vector<WorkItem> &items, cudaStream_t st)
{
    ws.items_key = std::make_tuple(-1, -1, -1, -1, -1);     // the callers set it once the upload is done
    ws.n_items = 0;
    CK(ws.items.ensure(items.size()), "alloc");
    CK(cudaMemcpyAsync(ws.items.p, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, st),
       "upload items");
    CK(cudaStreamSynchronize(st), "sync");     // the host vector goes out of scope
    ws.n_items = (int)items.size();
    return WECT_OK;
}

// ------------------------------------------------------------------ create / destroy

static wect_status pack_simplicial_weights(wect_complex c, cudaStream_t st);

// Grid coordinates x_a(i) = (2i - (L_a-1)) / (L_a-1) (0 when L_a = 1) of every axis of a grid,
// axis 0 first: one correctly rounded float64 division each, as grid_coord on the device.
static void append_grid_coords(const int *L, std::vector<double> &out)
{
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < L[a]; ++i)
            out.push_back(L[a] <= 1 ? 0.0 : (double)(2 * i - (L[a] - 1)) / (double)(L[a] - 1));
}

static cudaError_t upload_doubles(const std::vector<double> &h, double **d, cudaStream_t st)
{
    cudaError_t e = dev_malloc((void **)d, std::max<size_t>(h.size(), 1) * sizeof(double));
    if (e == cudaSuccess && !h.empty()) e = cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

static wect_status new_status_word(int **p)
{
    CK(dev_malloc((void **)p, sizeof(int)), "alloc");
    CK(cudaMemset(*p, 0, sizeof(int)), "memset");
    return WECT_OK;
}

extern "C" wect_status wect_complex_create_cubical(int n, const int64_t *dims, const void *vertex_weights,
                                                   wect_wtype wtype, int frac_bits, wect_stream stream,
                                                   wect_complex *out)
{
    if (!out) return fail(WECT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 3) return fail(WECT_ERR_INVALID_ARG, "n must be 1..3 (got %d)", n);
    if (!dims) return fail(WECT_ERR_INVALID_ARG, "dims is NULL");
    wect_status s = check_wtype(wtype, frac_bits);
    if (s) return s;
    int64_t nv = 1;
    for (int a = 0; a < n; ++a) {
        if (dims[a] < 1 || dims[a] > (1 << 24)) return fail(WECT_ERR_INVALID_ARG, "dims[%d] = %lld out of range", a, (long long)dims[a]);
        nv *= dims[a];
        if (nv >= (1ll << 31)) return fail(WECT_ERR_INVALID_ARG, "grid has >= 2^31 vertices");
    }
    if (wtype != WECT_W_ONE && !vertex_weights) return fail(WECT_ERR_INVALID_ARG, "vertex_weights is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    auto *c = new wect_complex_s();
    c->kind = 0;
    c->n = n;
    c->nv = nv;
    for (int a = 0; a < n; ++a) c->L[a] = (int)dims[a];
    c->wtype = wtype;
    c->frac_bits = (wtype == WECT_W_F32) ? frac_bits : 0;
    c->wbytes = wtype_bytes(wtype);
    // cells per dimension: number of (corner, mask) boxes with |mask| = k
    for (int e = 0; e < (1 << n); ++e) {
        int64_t cnt = 1;
        for (int a = 0; a < n; ++a) cnt *= ((e >> a) & 1) ? (c->L[a] - 1) : c->L[a];
        c->cells[__builtin_popcount(e)] += cnt;
    }
    auto cleanup = [&](wect_status st_) { wect_complex_destroy(c); return st_; };
    if ((s = new_status_word(&c->d_status))) return cleanup(s);
    if ((s = ensure_common_ws(c->ws, 2))) return cleanup(s);
    cudaError_t e;
    uint64_t wmax = 255;
    if (wtype == WECT_W_F32 || wtype == WECT_W_I64_FIXED) {
        int *d_bad = c->d_status;   // reuse the status word as a flag before it is published
        unsigned long long m = 0;
        int bad = 0;
        e = cudaMemsetAsync(c->ws.M.p, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = launch_weights_to_fixed(wtype, vertex_weights, nv, c->frac_bits, nullptr, c->ws.M.p, d_bad, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&m, c->ws.M.p, sizeof m, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "create weights"));
        g_launches++;
        if (bad) return cleanup(fail(WECT_ERR_INVALID_ARG, "vertex weights are not finite or too large for int64 fixed point"));
        wmax = m;
    }
    if ((s = choose_cubical_mode(n, wtype, wmax, c->nsplit, c->climit, c->kflush))) return cleanup(s);
    if ((e = cudaMemsetAsync(c->d_status, 0, sizeof(int), st))) return cleanup(cuda_fail(e, "memset"));
    if ((e = dev_malloc((void **)&c->d_w32, (size_t)nv * sizeof(int32_t)))) return cleanup(cuda_fail(e, "alloc weights"));
    if ((e = launch_weights_to_w32(wtype, vertex_weights, nv, c->frac_bits, c->climit >> n, c->d_w32, c->d_status, st)))
        return cleanup(cuda_fail(e, "weights_to_w32"));
    g_launches++;
    {
        std::vector<double> xg;
        append_grid_coords(c->L, xg);
        if ((e = upload_doubles(xg, &c->d_xg, st))) return cleanup(cuda_fail(e, "grid coordinates"));
    }
    {
        // TMA tensor map of the int32 weights, for grids that qualify (rows of a multiple of 4
        // vertices, at most 256)
        alignas(64) unsigned char map[128];
        if (encode_grid_tmap(n, c->L, c->d_w32, map)) {
            if ((e = dev_malloc(&c->d_tmap, sizeof map))) return cleanup(cuda_fail(e, "alloc tensor map"));
            if ((e = cudaMemcpy(c->d_tmap, map, sizeof map, cudaMemcpyHostToDevice))) return cleanup(cuda_fail(e, "tensor map"));
        }
    }
    GridDesc g{};
    g.w = c->d_w32;
    for (int a = 0; a < 3; ++a) g.L[a] = c->L[a];
    g.rows = c->L[1] * c->L[2];
    set_segments(g, n, c->nsplit);
    g.nv = nv;
    g.v_off = 0;
    g.status = c->d_status;
    g.xg = c->d_xg;
    g.tmap = c->d_tmap;
    e = dev_malloc((void **)&c->d_grid, sizeof(GridDesc));
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_grid, &g, sizeof g, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "upload grid"));
    *out = c;
    return WECT_OK;
}

extern "C" wect_status wect_complex_create_simplicial(int n, int64_t n_vertices, const double *coords, int max_dim,
                                                      const int64_t *counts, const int32_t *const *simplices,
                                                      const void *vertex_weights, wect_wtype wtype, int frac_bits,
                                                      wect_simplex_weight_mode sw_mode,
                                                      const int64_t *const *simplex_weights, wect_stream stream,
                                                      wect_complex *out)
{
    if (!out) return fail(WECT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxSimplexN) return fail(WECT_ERR_INVALID_ARG, "n must be 1..%d (got %d)", kMaxSimplexN, n);
    if (n_vertices < 1 || n_vertices >= (1ll << 31)) return fail(WECT_ERR_INVALID_ARG, "n_vertices out of range");
    if (max_dim < 0 || max_dim > kMaxSimplexDim) return fail(WECT_ERR_INVALID_ARG, "max_dim must be 0..%d", kMaxSimplexDim);
    if (!coords || !counts) return fail(WECT_ERR_INVALID_ARG, "coords/counts is NULL");
    if (counts[0] != n_vertices) return fail(WECT_ERR_INVALID_ARG, "counts[0] must equal n_vertices");
    if (sw_mode != WECT_SW_MAX_OF_VERTICES && sw_mode != WECT_SW_EXPLICIT)
        return fail(WECT_ERR_INVALID_ARG, "unknown simplex weight mode");
    wect_status s = check_wtype(wtype, frac_bits);
    if (s) return s;
    for (int i = 1; i <= max_dim; ++i) {
        if (counts[i] < 0 || counts[i] >= (1ll << 31)) return fail(WECT_ERR_INVALID_ARG, "counts[%d] out of range", i);
        if (counts[i] > 0 && (!simplices || !simplices[i])) return fail(WECT_ERR_INVALID_ARG, "simplices[%d] is NULL", i);
        if (sw_mode == WECT_SW_EXPLICIT && counts[i] > 0 && (!simplex_weights || !simplex_weights[i]))
            return fail(WECT_ERR_INVALID_ARG, "simplex_weights[%d] is NULL", i);
    }
    const bool vw_explicit = sw_mode == WECT_SW_EXPLICIT && simplex_weights && simplex_weights[0];
    if (!vw_explicit && wtype != WECT_W_ONE && !vertex_weights) return fail(WECT_ERR_INVALID_ARG, "vertex_weights is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    auto *c = new wect_complex_s();
    c->kind = 1;
    c->n = n;
    c->nv = n_vertices;
    c->max_dim = max_dim;
    c->wtype = wtype;
    c->frac_bits = (wtype == WECT_W_F32) ? frac_bits : 0;
    c->wbytes = wtype_bytes(wtype);
    c->sw_mode = sw_mode;
    for (int i = 0; i <= max_dim; ++i) c->counts[i] = counts[i];
    for (int i = 0; i <= max_dim; ++i) c->cells[i] = counts[i];
    auto cleanup = [&](wect_status st_) { wect_complex_destroy(c); return st_; };
    cudaError_t e;
    if ((s = new_status_word(&c->d_status))) return cleanup(s);
    if ((s = ensure_common_ws(c->ws, 2))) return cleanup(s);
    int *d_bad = nullptr;
    if ((e = dev_malloc((void **)&d_bad, 4 * sizeof(int))) != cudaSuccess) return cleanup(cuda_fail(e, "alloc"));
    struct FreeBad { int *p; ~FreeBad() { if (p) cudaFree(p); } } fb{d_bad};
    if ((e = cudaMemsetAsync(d_bad, 0, 4 * sizeof(int), st)) != cudaSuccess) return cleanup(cuda_fail(e, "memset"));
    // coordinates
    if ((e = dev_malloc((void **)&c->d_coords, (size_t)n_vertices * n * sizeof(double))) != cudaSuccess)
        return cleanup(cuda_fail(e, "alloc coords"));
    if ((e = cudaMemcpyAsync(c->d_coords, coords, (size_t)n_vertices * n * sizeof(double), cudaMemcpyDeviceToDevice, st)))
        return cleanup(cuda_fail(e, "copy coords"));
    if ((e = launch_finite_check(c->d_coords, n_vertices * n, d_bad + 0, 1, st))) return cleanup(cuda_fail(e, "finite_check"));
    g_launches++;
    if ((e = dev_malloc((void **)&c->d_xf, (size_t)n_vertices * n * sizeof(float))) != cudaSuccess)
        return cleanup(cuda_fail(e, "alloc coords"));
    if ((e = launch_coords_to_f32(c->d_coords, n_vertices * n, c->d_xf, st))) return cleanup(cuda_fail(e, "coords_to_f32"));
    g_launches++;
    // per-axis max |x| into range[3..5]
    std::vector<unsigned long long> zeros(3, 0ull);
    unsigned long long *d_xm = reinterpret_cast<unsigned long long *>(c->ws.range.p + 3);
    if ((e = cudaMemsetAsync(c->ws.range.p, 0, 8 * sizeof(double), st))) return cleanup(cuda_fail(e, "memset"));
    for (int a = 0; a < n; ++a) {
        if ((e = launch_max_abs_f64(c->d_coords, n_vertices, n, a, d_xm + a, st))) return cleanup(cuda_fail(e, "max_abs"));
        g_launches++;
    }
    // simplex lists
    for (int i = 1; i <= max_dim; ++i) {
        const size_t cnt = (size_t)counts[i] * (i + 1);
        if ((e = dev_malloc((void **)&c->d_simp[i], std::max<size_t>(cnt, 1) * sizeof(int32_t)))) return cleanup(cuda_fail(e, "alloc"));
        if (cnt) {
            if ((e = cudaMemcpyAsync(c->d_simp[i], simplices[i], cnt * sizeof(int32_t), cudaMemcpyDeviceToDevice, st)))
                return cleanup(cuda_fail(e, "copy simplices"));
            if ((e = launch_index_check(c->d_simp[i], (int64_t)cnt, n_vertices, d_bad + 1, st))) return cleanup(cuda_fail(e, "index_check"));
            g_launches++;
        }
    }
    // weights
    for (int i = 0; i <= max_dim; ++i)
        if ((e = dev_malloc((void **)&c->d_sw[i], std::max<int64_t>(counts[i], 1) * sizeof(int64_t))))
            return cleanup(cuda_fail(e, "alloc weights"));
    if ((e = cudaMemsetAsync(c->ws.M.p, 0, 2 * sizeof(unsigned long long), st))) return cleanup(cuda_fail(e, "memset"));
    if (vw_explicit) {
        if ((e = cudaMemcpyAsync(c->d_sw[0], simplex_weights[0], n_vertices * sizeof(int64_t), cudaMemcpyDeviceToDevice, st)))
            return cleanup(cuda_fail(e, "copy"));
        if ((e = launch_weights_to_fixed(WT_I64, c->d_sw[0], n_vertices, 0, nullptr, c->ws.M.p, d_bad + 2, st)))
            return cleanup(cuda_fail(e, "weights"));
        g_launches++;
    } else {
        if ((e = launch_weights_to_fixed(wtype, vertex_weights, n_vertices, c->frac_bits, c->d_sw[0], c->ws.M.p, d_bad + 2, st)))
            return cleanup(cuda_fail(e, "weights"));
        g_launches++;
    }
    for (int i = 1; i <= max_dim; ++i) {
        if (counts[i] == 0) continue;
        if (sw_mode == WECT_SW_EXPLICIT) {
            if ((e = cudaMemcpyAsync(c->d_sw[i], simplex_weights[i], counts[i] * sizeof(int64_t), cudaMemcpyDeviceToDevice, st)))
                return cleanup(cuda_fail(e, "copy"));
            if ((e = launch_weights_to_fixed(WT_I64, c->d_sw[i], counts[i], 0, nullptr, c->ws.M.p, d_bad + 2, st)))
                return cleanup(cuda_fail(e, "weights"));
        } else {
            if ((e = launch_simplex_weights_max(c->d_simp[i], counts[i], i + 1, c->d_sw[0], c->d_sw[i], st)))
                return cleanup(cuda_fail(e, "simplex weights"));
        }
        g_launches++;
    }
    int bad[4] = {0, 0, 0, 0};
    unsigned long long wmax = 0;
    double xm[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(&wmax, c->ws.M.p, sizeof wmax, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(xm, c->ws.range.p + 3, sizeof xm, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cleanup(cuda_fail(e, "create sync"));
    if (bad[0]) return cleanup(fail(WECT_ERR_INVALID_ARG, "coordinates are not finite"));
    if (bad[1]) return cleanup(fail(WECT_ERR_INVALID_ARG, "a simplex vertex index is outside [0, n_vertices)"));
    if (bad[2]) return cleanup(fail(WECT_ERR_INVALID_ARG, "vertex weights are not finite or too large"));
    if (wtype == WECT_W_U8 || wtype == WECT_W_ONE) wmax = std::max<unsigned long long>(wmax, 255);
    if (wmax >= (1ull << 40)) return cleanup(fail(WECT_ERR_OVERFLOW, "a weight magnitude reaches 2^40"));
    // accumulator: one int32 plane when 65536 updates of max|w| fit, else low 16 bits + high part
    if (wmax <= (1ull << 14)) {
        c->nsplit = 1;
        c->climit = 1 << 15;
        c->kflush = 1 << 16;
    } else {
        c->nsplit = 2;
        const int64_t lim = (int64_t)std::max<unsigned long long>(wmax, 1ull << 31) * 2;    // headroom for later weights
        c->climit = std::min<int64_t>(lim, (1ll << 40) - 1);
        const int64_t hb = (c->climit >> 16) + 1;
        c->kflush = (int)std::max<int64_t>(1, std::min<int64_t>(1 << 16, (((int64_t)1 << 31) - 1) / hb));
    }
    // lists sorted by a spatial key (results do not depend on the order; the gather's chunks then
    // cover compact patches and reference few distinct vertices)
    bool any_list = false;
    for (int i = 1; i <= max_dim; ++i) any_list |= counts[i] > 1;
    if (any_list) {
        unsigned long long *vkey = nullptr;
        if ((e = dev_malloc((void **)&vkey, (size_t)n_vertices * sizeof(unsigned long long))))
            return cleanup(cuda_fail(e, "alloc sort keys"));
        e = vertex_morton_keys(c->d_coords, n_vertices, n, xm, vkey, st);
        g_launches++;
        for (int i = 1; i <= max_dim && e == cudaSuccess; ++i)
            if (counts[i] > 1) e = sort_simplices_spatial(c->d_simp[i], counts[i], i + 1, c->d_sw[i], vkey, st);
        cudaStreamSynchronize(st);
        cudaFree(vkey);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "sort lists"));
    }
    for (int i = 0; i <= max_dim; ++i)
        if ((e = dev_malloc((void **)&c->d_swp[i], std::max<int64_t>(counts[i], 1) * sizeof(int2))))
            return cleanup(cuda_fail(e, "alloc packed weights"));
    if ((s = pack_simplicial_weights(c, st))) return cleanup(s);
    // chunk-local ids of the lists of dim >= 1, for the staged gather (indices are valid here)
    for (int i = 1; i <= max_dim; ++i) {
        if (counts[i] == 0) continue;
        const int m = i + 1;
        const int64_t nch = (counts[i] + chunk_simplices(m) - 1) / chunk_simplices(m);
        if ((e = dev_malloc((void **)&c->d_local[i], (size_t)counts[i] * m * sizeof(uint16_t))) ||
            (e = dev_malloc((void **)&c->d_cverts[i], (size_t)nch * kWinRows * sizeof(int32_t))) ||
            (e = dev_malloc((void **)&c->d_cnu[i], (size_t)nch * sizeof(int32_t))))
            return cleanup(cuda_fail(e, "alloc chunks"));
        if ((e = launch_chunk_local(c->d_simp[i], counts[i], m, c->d_local[i], c->d_cverts[i], c->d_cnu[i], st)))
            return cleanup(cuda_fail(e, "chunk_local"));
        g_launches++;
        c->nchunks[i] = nch;
    }
    *out = c;
    return WECT_OK;
}

extern "C" void wect_complex_destroy(wect_complex c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    if (c->d_w32) cudaFree(c->d_w32);
    if (c->d_xg) cudaFree(c->d_xg);
    if (c->d_tmap) cudaFree(c->d_tmap);
    if (c->d_coords) cudaFree(c->d_coords);
    if (c->d_xf) cudaFree(c->d_xf);
    for (int i = 0; i <= kMaxSimplexDim; ++i) {
        if (c->d_simp[i]) cudaFree(c->d_simp[i]);
        if (c->d_sw[i]) cudaFree(c->d_sw[i]);
        if (c->d_swp[i]) cudaFree(c->d_swp[i]);
        if (c->d_local[i]) cudaFree(c->d_local[i]);
        if (c->d_cverts[i]) cudaFree(c->d_cverts[i]);
        if (c->d_cnu[i]) cudaFree(c->d_cnu[i]);
    }
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_grid) cudaFree(c->d_grid);
    c->ws.release();
    delete c;
}

extern "C" int64_t wect_complex_num_vertices(wect_complex c) { return c ? c->nv : 0; }

extern "C" wect_status wect_complex_cell_counts(wect_complex c, int64_t *counts5)
{
    if (!c || !counts5) return fail(WECT_ERR_INVALID_ARG, "NULL argument");
    for (int i = 0; i <= kMaxSimplexDim; ++i) counts5[i] = c->cells[i];
    return WECT_OK;
}

static wect_status status_from_bits(int bits)
{
    if (bits & kStatusOverflow) return fail(WECT_ERR_OVERFLOW, "weights exceeded the accumulator chosen at create time");
    if (bits & kStatusTimeout) return fail(WECT_ERR_TIMEOUT, "a bounded device wait ran out");
    if (bits & kStatusBadIndex) return fail(WECT_ERR_INVALID_ARG, "device-side validation failed (non-finite input)");
    return WECT_OK;
}

extern "C" wect_status wect_complex_device_status(wect_complex c, wect_stream stream)
{
    if (!c) return fail(WECT_ERR_INVALID_ARG, "NULL complex");
    cudaStream_t st = (cudaStream_t)stream;
    int bits = 0;
    CK(cudaStreamSynchronize(st), "sync");
    CK(cudaMemcpy(&bits, c->d_status, sizeof bits, cudaMemcpyDeviceToHost), "read status");
    CK(cudaMemset(c->d_status, 0, sizeof(int)), "clear status");
    return status_from_bits(bits);
}

static wect_status set_weights_locked(wect_complex c, const void *w, cudaStream_t st);

extern "C" wect_status wect_complex_set_weights(wect_complex c, const void *w, wect_stream stream)
{
    if (!c) return fail(WECT_ERR_INVALID_ARG, "NULL complex");
    cudaStream_t st = (cudaStream_t)stream;
    if (c->wtype == WECT_W_ONE) return WECT_OK;
    if (!w) return fail(WECT_ERR_INVALID_ARG, "weights is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    return set_weights_locked(c, w, st);
}

// w: device-accessible weights of the complex's type (device memory or mapped pinned host memory)
static wect_status set_weights_locked(wect_complex c, const void *w, cudaStream_t st)
{
    if (c->kind == 0) {
        KL(launch_weights_to_w32(c->wtype, w, c->nv, c->frac_bits, c->climit >> c->n, c->d_w32, c->d_status, st),
           "weights_to_w32");
        return WECT_OK;
    }
    if (c->sw_mode == WECT_SW_EXPLICIT) return fail(WECT_ERR_UNSUPPORTED, "set_weights on a complex with explicit simplex weights");
    KL(launch_weights_to_fixed(c->wtype, w, c->nv, c->frac_bits, c->d_sw[0], nullptr, c->d_status, st), "weights_to_fixed");
    KL(launch_weights_check(WT_I64, c->d_sw[0], c->nv, 0, c->climit, c->d_status, st), "weights_check");
    for (int i = 1; i <= c->max_dim; ++i)
        if (c->counts[i] > 0) KL(launch_simplex_weights_max(c->d_simp[i], c->counts[i], i + 1, c->d_sw[0], c->d_sw[i], st), "sw");
    return pack_simplicial_weights(c, st);
}

// Packed signed weights of every list (after the weights or the accumulator mode change).
static wect_status pack_simplicial_weights(wect_complex c, cudaStream_t st)
{
    for (int i = 0; i <= c->max_dim; ++i) {
        if (c->counts[i] == 0) continue;
        KL(launch_pack_weights(c->d_sw[i], c->counts[i], (i & 1) ? -1 : 1, c->nsplit, c->d_swp[i], st), "pack_weights");
    }
    return WECT_OK;
}

// ------------------------------------------------------------------ forward

static wect_status dirs_check(wect_complex c, const double *dirs, int d, cudaStream_t st)
{
    KL(launch_finite_check(dirs, (int64_t)d * c->n, c->d_status, kStatusBadIndex, st), "finite_check");
    return WECT_OK;
}

// out: the int64 [d][T] table the forward accumulates into; final_out (null: out) receives its
// scan (simplicial_compute likewise).
// prep_early: the kernel enqueued just before is this call's own weight conversion.
static wect_status cubical_compute(wect_complex c, const double *dirs, int d, int T, double lo, double hi, int64_t *out,
                                   cudaStream_t st, int64_t *final_out = nullptr, bool prep_early = false)
{
    CubShape sh;
    GridDesc gd{};
    gd.L[0] = c->L[0]; gd.L[1] = c->L[1]; gd.L[2] = c->L[2];
    gd.rows = c->L[1] * c->L[2];
    gd.nv = c->nv;
    set_segments(gd, c->n, c->nsplit);
    const int ul = unit_len(gd);
    if (!cub_shape(c->n, c->nsplit, d, T, ul, sh, 0, 0, (double)ul, hi - lo, 0, c->d_tmap != nullptr && gd.nseg == 1,
                   gd.nseg > 1))
        return fail(WECT_ERR_UNSUPPORTED, "grid rows of %d vertices do not fit the kernel's shared row buffers", ul);
    if (ul > c->kflush && !sh.gh) return fail(WECT_ERR_UNSUPPORTED, "grid rows longer than %d vertices", c->kflush);
    wect_status s = ensure_common_ws(c->ws, T, d);
    if (s) return s;
    const bool direct = false;
    auto key = std::make_tuple(d, T, sh.Dt, sh.run ? 100 : sh.dpl * (sh.gh ? -1 : 1) + sh.Tt * 100000, sh.grid);
    if (c->ws.items_key != key) {   // (items do not depend on the TMA staging)
        std::vector<GridDesc> gv(1, gd);
        std::vector<WorkItem> items = make_items(gv, d, sh.Dt, T, c->kflush, sh.grid, false, sh.Tt);
        if ((s = upload_items(c->ws, items, st))) return s;
        c->ws.items_key = key;
    }
    CubLaunch L{c->n, c->nsplit, c->wtype, c->frac_bits, c->kflush, ul, c->climit, c->d_grid, &c->ws, c->d_status,
                gd.nseg > 1};
    return enqueue_cubical_fwd(L, sh, c->ws.n_items, direct, dirs, d, T, lo, hi, range_is_default(lo, hi), d, out, st,
                               final_out, prep_early);
}

static wect_status simplicial_range(wect_complex c, const double *dirs, int d, int T, double lo, double hi, cudaStream_t st)
{
    const bool dflt = range_is_default(lo, hi);
    if (dflt) {
        CK(c->ws.cand.ensure((size_t)c->nv + 4), "alloc range candidates");
        CK(cudaMemsetAsync(c->ws.M.p, 0, 2 * sizeof(unsigned long long), st), "memset");
        KL(launch_simplicial_max_abs(c->n, c->d_coords, c->d_xf, c->nv, dirs, d, c->ws.M.p, c->ws.M.p + 1,
                                     c->ws.cand.p, st), "max_abs");
        g_launches += 3;    // four kernels
    }
    KL(launch_setup_range_beta(lo, hi, dflt ? 1 : 0, c->ws.M.p, T, c->ws.range.p, c->ws.beta.p, st), "setup_range_beta");
    CK(c->ws.dtab.ensure((size_t)d * 8), "alloc filter table");
    KL(launch_dir_filters(c->n, dirs, d, T, c->ws.range.p, c->ws.dtab.p, st), "dir_filters");
    return WECT_OK;
}

static wect_status simplicial_compute(wect_complex c, const double *dirs, int d, int T, double lo, double hi,
                                      int64_t *out, cudaStream_t st, int64_t *final_out = nullptr)
{
    const int Dt = 32;
    const size_t sm = simplex_fwd_smem(c->nsplit, T, Dt);
    // T x 32 int32 entries beyond shared memory: every signed weight goes to the int64 table in
    // global memory instead (same bins and sums)
    const bool gh = sm > std::min<size_t>(smem_optin(), 200 * 1024);
    wect_status s = ensure_common_ws(c->ws, T);
    if (s) return s;
    CK(c->ws.bins.ensure((size_t)c->nv * Dt), "alloc bins");
    if ((s = simplicial_range(c, dirs, d, T, lo, hi, st))) return s;
    CK(cudaMemsetAsync(out, 0, (size_t)d * T * sizeof(int64_t), st), "memset");
    const int grid = sm_count();
    const bool staged_ok = simplex_fwd_staged_smem(c->nsplit, T, Dt) <= smem_optin() - 1024;
    // outside a stream capture the gathers after the first are programmatic dependent launches
    // (each clears its histogram while the one before finishes)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs), "capture status");
    bool pdl = false;
    ProfScope prof(st);
    for (int dt = 0; dt * Dt < d; ++dt) {
        for (int i = 0; i <= c->max_dim; ++i) {
            if (i > 0 && c->counts[i] == 0) continue;
            SimplexFwdArgs a{};
            a.pdl = pdl ? 1 : 0;
            pdl = cs == cudaStreamCaptureStatusNone;
            a.simp = (i == 0) ? nullptr : c->d_simp[i];
            a.sw = c->d_sw[i];
            a.swp = c->d_swp[i];
            a.k = c->counts[i];
            a.m = i + 1;
            a.sign = (i & 1) ? -1 : 1;
            a.bins = c->ws.bins.p;
            a.Dt = Dt;
            a.dtile = dt;
            a.d = d;
            a.T = T;
            // a multiple of 8 simplices, so that groups start on 16-byte boundaries
            a.chunk = std::max<int64_t>(8, std::min<int64_t>(c->kflush, std::max<int64_t>(4096, (a.k + grid - 1) / grid)) & ~7ll);
            a.out = reinterpret_cast<unsigned long long *>(out);
            if (gh) {
                // vertex bins of the tile first, then every list (vertices included) from the table
                if (i == 0)
                    KL(launch_vertex_bins(c->n, c->d_coords, c->d_xf, c->nv, dirs, c->ws.dtab.p, d, dt, Dt, T,
                                          c->ws.beta.p, c->ws.bins.p, st),
                       "vertex_bins");
                const int g = (int)std::min<int64_t>(grid, (a.k + a.chunk - 1) / a.chunk);
                KL(launch_simplex_fwd(c->nsplit, true, a, std::max(g, 1), st), "simplex_fwd");
                continue;
            }
            if (i == 0) {
                // vertex bins of the tile, fused with the vertices' own scatter (16 warps x 8
                // vertices per CTA step)
                a.flush_every = std::max(1, c->kflush / (16 * 8));
                KL(launch_vertex_scatter(c->n, c->nsplit, a, c->d_coords, c->d_xf, c->nv, dirs, c->ws.dtab.p, c->ws.beta.p,
                                         c->ws.bins.p, grid, st),
                   "vertex_scatter");
                continue;
            }
            const int cs = chunk_simplices(a.m);
            if (i >= 1 && staged_ok && c->d_local[i] && c->kflush >= cs) {
                a.local = c->d_local[i];
                a.cverts = c->d_cverts[i];
                a.cnu = c->d_cnu[i];
                a.nchunks = c->nchunks[i];
                a.flush_every = c->kflush / cs;           // at most kflush simplices between flushes
                const int g = (int)std::min<int64_t>(grid, a.nchunks);
                KL(launch_simplex_fwd_staged(c->nsplit, a, std::max(g, 1), st), "simplex_fwd_staged");
                continue;
            }
            const int g = (int)std::min<int64_t>(grid, (a.k + a.chunk - 1) / a.chunk);
            KL(launch_simplex_fwd(c->nsplit, false, a, std::max(g, 1), st), "simplex_fwd");
        }
    }
    KL(launch_scan_rows_to(reinterpret_cast<unsigned long long *>(out),
                           reinterpret_cast<unsigned long long *>(final_out ? final_out : out), d, T, st, pdl),
       "scan_rows");
    return WECT_OK;
}

extern "C" wect_status wect_compute(wect_complex c, const double *dirs, int d, int T, double lo, double hi,
                                    int64_t *out, wect_stream stream)
{
    if (!c) return fail(WECT_ERR_INVALID_ARG, "NULL complex");
    if (!dirs || !out) return fail(WECT_ERR_INVALID_ARG, "dirs/out is NULL");
    if (d < 1) return fail(WECT_ERR_INVALID_ARG, "d must be >= 1");
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->kind == 0) return cubical_compute(c, dirs, d, T, lo, hi, out, st);   // directions checked in fwd_prep
    if ((s = dirs_check(c, dirs, d, st))) return s;
    return simplicial_compute(c, dirs, d, T, lo, hi, out, st);
}

// The device address of a caller buffer: device memory of the current device and managed memory
// as they are, page-locked host memory through its mapping into the device's address space
// (kernels read and write it over the host link); null for pageable host memory (and memory of
// another device), which is copied instead (cudaMemcpyDefault: the unified address space tells
// the direction).
static void *device_alias(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (a.type == cudaMemoryTypeDevice && a.device != dev) return nullptr;
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeHost)
        return a.devicePointer;
    return nullptr;
}

extern "C" wect_status wect_compute_host(wect_complex c, const void *weights, const double *dirs, int d, int T,
                                         double lo, double hi, int64_t *out, wect_stream stream)
{
    if (!c) return fail(WECT_ERR_INVALID_ARG, "NULL complex");
    if (!dirs || !out) return fail(WECT_ERR_INVALID_ARG, "dirs/out is NULL");
    if (d < 1) return fail(WECT_ERR_INVALID_ARG, "d must be >= 1");
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(c->mu);
    // the directions: a device copy (every CTA of the forward reads them), made before the
    // weight conversion, which the forward's preparation overlaps
    const int64_t nd = (int64_t)d * c->n;
    CK(c->ws.hdirs.ensure((size_t)nd), "alloc direction copy");
    const double *dd = static_cast<const double *>(device_alias(dirs));
    if (dd)
        KL(launch_copy_f64(dd, c->ws.hdirs.p, nd, st), "copy_f64");
    else
        CK(cudaMemcpyAsync(c->ws.hdirs.p, dirs, (size_t)nd * sizeof(double), cudaMemcpyDefault, st), "copy dirs");
    // the weights: read in place by the conversion kernel, or staged when pageable
    if (weights && c->wtype != WECT_W_ONE) {
        const void *wd = device_alias(weights);
        if (!wd) {
            const size_t bytes = (size_t)c->nv * c->wbytes;
            CK(c->ws.hw.ensure(bytes), "alloc weight staging");
            CK(cudaMemcpyAsync(c->ws.hw.p, weights, bytes, cudaMemcpyDefault, st), "copy weights");
            wd = c->ws.hw.p;
        }
        if ((s = set_weights_locked(c, wd, st))) return s;
    }
    // the difference table on the device; its scan writes out directly when out is mapped
    CK(c->ws.hout.ensure((size_t)d * T), "alloc table");
    int64_t *od = static_cast<int64_t *>(device_alias(out));
    if (c->kind == 0) {
        // (the kernel just before is this call's weight conversion or direction copy)
        s = cubical_compute(c, c->ws.hdirs.p, d, T, lo, hi, c->ws.hout.p, st, od, true);
    } else {
        if ((s = dirs_check(c, c->ws.hdirs.p, d, st))) return s;
        s = simplicial_compute(c, c->ws.hdirs.p, d, T, lo, hi, c->ws.hout.p, st, od);
    }
    if (s) return s;
    if (!od)
        CK(cudaMemcpyAsync(out, c->ws.hout.p, (size_t)d * T * sizeof(int64_t), cudaMemcpyDefault, st), "copy table");
    return WECT_OK;
}

// Algorithm 1 for m caller-supplied vertex filters [m][nv]: exact float64 bins of every filter,
// then the per-cell max of the bins and the signed scatter, one histogram row per filter.
static wect_status wecf_impl(wect_complex c, const double *filters, int m, int T, double lo, double hi, int weighted,
                             int64_t *out, cudaStream_t st)
{
    if (!c) return fail(WECT_ERR_INVALID_ARG, "NULL complex");
    if (!filters || !out) return fail(WECT_ERR_INVALID_ARG, "filters/out is NULL");
    if (m < 1 || m > 65535) return fail(WECT_ERR_INVALID_ARG, "m must be in [1, 65535] (got %d)", m);
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    std::lock_guard<std::mutex> lk(c->mu);
    if ((s = ensure_common_ws(c->ws, T))) return s;
    const int64_t total = (int64_t)m * c->nv;
    CK(c->ws.bins.ensure((size_t)total), "alloc bins");
    const bool dflt = range_is_default(lo, hi);
    if (dflt) {
        // the paper's M is the largest |f| over all m filters
        CK(cudaMemsetAsync(c->ws.M.p, 0, sizeof(unsigned long long), st), "memset");
        KL(launch_max_abs_f64(filters, total, 1, 0, c->ws.M.p, st), "max_abs");
    }
    KL(launch_setup_range_beta(lo, hi, dflt ? 1 : 0, c->ws.M.p, T, c->ws.range.p, c->ws.beta.p, st), "setup_range_beta");
    // exact bins of every filter value, and the finite check of the filters
    KL(launch_filter_bins(filters, total, c->ws.range.p, c->ws.beta.p, T, c->ws.bins.p, c->d_status, kStatusBadIndex,
                          st),
       "filter_bins");
    CK(cudaMemsetAsync(out, 0, (size_t)m * T * sizeof(int64_t), st), "memset");
    if (c->kind == 0) {
        KL(launch_cubical_ecf(c->n, c->d_grid, c->ws.bins.p, T, weighted ? 1 : 0, c->climit >> c->n,
                              reinterpret_cast<unsigned long long *>(out), c->nv, m, st),
           "cubical_ecf");
    } else {
        for (int i = 0; i <= c->max_dim; ++i) {
            if (c->counts[i] == 0) continue;
            KL(launch_simplex_ecf(i == 0 ? nullptr : c->d_simp[i], c->d_sw[i], c->counts[i], i + 1, (i & 1) ? -1 : 1,
                                  weighted ? 1 : 0, c->climit, c->ws.bins.p, T,
                                  reinterpret_cast<unsigned long long *>(out), c->nv, m, st),
               "simplex_ecf");
        }
    }
    KL(launch_scan_rows(reinterpret_cast<unsigned long long *>(out), m, T, st), "scan_rows");
    return WECT_OK;
}

extern "C" wect_status ecf_compute(wect_complex c, const double *filter, int T, double lo, double hi, int weighted,
                                   int64_t *out, wect_stream stream)
{
    return wecf_impl(c, filter, 1, T, lo, hi, weighted, out, (cudaStream_t)stream);
}

extern "C" wect_status wecf_compute(wect_complex c, const double *filters, int m, int T, double lo, double hi,
                                    int weighted, int64_t *out, wect_stream stream)
{
    return wecf_impl(c, filters, m, T, lo, hi, weighted, out, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ adjoint

static wect_status cubical_backward(const GridDesc *d_grids, int n_grids, const std::vector<GridDesc> &h_grids, int n,
                                    int wt, int frac_bits, int64_t total_nv, Workspace &ws, const double *dirs, int d,
                                    int T, double lo, double hi, const int64_t *dW, double scale, float *grad,
                                    int *status, cudaStream_t st, const double *scale_dev = nullptr)
{
    if (range_is_default(lo, hi) && n_grids != 1) return fail(WECT_ERR_UNSUPPORTED, "default range in a batch");
    wect_status s = ensure_common_ws(ws, T, d);
    if (s) return s;
    const int noct = 1 << n;
    CK(ws.S.ensure((size_t)n_grids * d * T), "alloc S");
    CK(ws.Rv.ensure((size_t)total_nv * noct), "alloc Rv");
    CK(ws.perm.ensure((size_t)d), "alloc perm");
    CK(ws.octb.ensure(9), "alloc octb");
    // directions per chunk of the octant sums: the chunk's suffix rows ([dc + 1][T] int64) must fit
    // shared memory next to one row tile of filter constants; then rows per filter tile: as many
    // as fit (up to 32)
    const size_t lim = smem_optin() - 1024;
    int dc = d;
    while (dc > 1 && cubical_bwd_rsum_smem(n, dc, T, 1) > lim) dc = (dc + 1) / 2;
    if (cubical_bwd_rsum_smem(n, dc, T, 1) > lim)
        return fail(WECT_ERR_UNSUPPORTED, "T = %d: one direction's suffix row does not fit the adjoint's shared table", T);
    int R = 32;
    while (R > 1 && cubical_bwd_rsum_smem(n, dc, T, R) > lim) R /= 2;
    const size_t sm = cubical_bwd_rsum_smem(n, dc, T, R);
    auto key = std::make_tuple(d, R);
    if (ws.items_bwd_key != key) {
        // one CTA per SM (the suffix table fills shared memory), each taking a contiguous share of
        // all rows with about the same number of vertices, cut at complex boundaries into items;
        // a CTA stages a complex's suffix rows once for all its rows of that complex
        int64_t total = 0;
        for (int c = 0; c < n_grids; ++c) total += (int64_t)h_grids[c].rows * h_grids[c].L[0];
        const int nctas = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count(), total / 64));
        std::vector<WorkItem> items;
        std::vector<int> ranges(1, 0);
        int64_t done = 0;                   // vertices assigned so far
        int c = 0, r = 0;
        for (int b = 0; b < nctas; ++b) {
            const int64_t goal = (b == nctas - 1) ? total : total * (b + 1) / nctas;
            while (c < n_grids && done < goal) {
                const int L0 = std::max(1, h_grids[c].L[0]);
                const int rows = h_grids[c].rows;
                const int take = (int)std::min<int64_t>(rows - r, std::max<int64_t>(1, (goal - done + L0 - 1) / L0));
                items.push_back(WorkItem{c, 0, r, r + take});
                done += (int64_t)take * L0;
                r += take;
                if (r >= rows) {
                    ++c;
                    r = 0;
                }
            }
            ranges.push_back((int)items.size());
        }
        ws.items_bwd_key = std::make_tuple(-1, -1);         // set again once the upload is done
        ws.n_items_bwd = 0;
        CK(ws.items_bwd.ensure(items.size()), "alloc");
        CK(ws.ranges_bwd.ensure(ranges.size()), "alloc");
        CK(cudaMemcpyAsync(ws.items_bwd.p, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, st), "upload");
        CK(cudaMemcpyAsync(ws.ranges_bwd.p, ranges.data(), ranges.size() * sizeof(int), cudaMemcpyHostToDevice, st),
           "upload");
        CK(cudaStreamSynchronize(st), "sync");
        ws.n_items_bwd = (int)items.size();
        ws.n_ctas_bwd = nctas;
        ws.items_bwd_key = key;
    }
    const bool dflt = range_is_default(lo, hi);
    if (dflt) {
        CK(cudaMemsetAsync(ws.M.p, 0, sizeof(unsigned long long), st), "memset");
        KL(launch_grid_max_abs(n, d_grids, dirs, d, ws.M.p, st), "grid_max_abs");
    }
    KL(launch_setup_range_beta(lo, hi, dflt ? 1 : 0, ws.M.p, T, ws.range.p, ws.beta.p, st), "setup_range_beta");
    // the routing kernel sums in int64: 3^n d max|S| must stay below 2^63
    const int64_t pow3 = n == 1 ? 3 : (n == 2 ? 9 : 27);
    KL(launch_suffix_rows(dW, ws.S.p, (int64_t)n_grids * d, T, INT64_MAX / ((int64_t)d * pow3), status, st), "suffix_rows");
    CubicalBwdArgs a{};
    a.grids = d_grids;
    a.n_grids = n_grids;
    a.items = ws.items_bwd.p;
    a.d_all = d;
    a.T = T;
    a.range = ws.range.p;
    a.beta = ws.beta.p;
    a.perm = ws.perm.p;
    a.octb = ws.octb.p;
    a.R = R;
    a.S = ws.S.p;
    a.Rv = ws.Rv.p;
    a.grad = grad;
    a.v_begin = 0;
    a.v_end = total_nv;
    a.scale = scale;
    a.scale_dev = scale_dev;
    a.frac_bits = frac_bits;
    a.total_nv = total_nv;
    a.uniform_nv = h_grids.empty() ? 0 : h_grids[0].nv;
    for (const auto &hg : h_grids)
        if (hg.nv != a.uniform_nv) a.uniform_nv = 0;
    {
        ProfScope prof(st);
        for (int p0 = 0; p0 < d; p0 += dc) {
            const int dn = std::min(dc, d - p0);
            KL(launch_octant_sort(n, dirs + (int64_t)p0 * n, dn, ws.perm.p, ws.octb.p, st), "octant_sort");
            a.dirs = dirs + (int64_t)p0 * n;
            a.d = dn;
            a.p0 = p0;
            a.accumulate = p0 > 0 ? 1 : 0;
            a.item_ranges = ws.ranges_bwd.p;
            KL(launch_cubical_bwd_rsum(n, a, ws.n_ctas_bwd, sm, st), "cubical_bwd_rsum");
        }
        KL(launch_cubical_bwd_route(n, a, st), "cubical_bwd_route");
    }
    return WECT_OK;
}

// The adjoint of one complex (the caller holds its lock).  grad_w = I_v * scale, or I_v times
// the device-side scale *scale_dev when that is not null (the quantised float64 upstream).
static wect_status complex_backward(wect_complex c, const double *dirs, int d, int T, double lo, double hi,
                                    const int64_t *dW, double scale, const double *scale_dev, float *grad_w,
                                    cudaStream_t st)
{
    wect_status s;
    if (c->kind == 0) {
        std::vector<GridDesc> hg(1);
        hg[0].L[0] = c->L[0]; hg[0].L[1] = c->L[1]; hg[0].L[2] = c->L[2];
        hg[0].rows = c->L[1] * c->L[2];
        hg[0].nv = c->nv;
        return cubical_backward(c->d_grid, 1, hg, c->n, c->wtype, c->frac_bits, c->nv, c->ws, dirs, d, T, lo, hi, dW, scale,
                                grad_w, c->d_status, st, scale_dev);
    }
    if ((s = ensure_common_ws(c->ws, T))) return s;
    CK(c->ws.S.ensure((size_t)d * T), "alloc S");
    CK(c->ws.bins.ensure((size_t)c->nv * 32), "alloc bins");
    CK(c->ws.Iacc.ensure((size_t)c->nv * 2), "alloc Iacc");
    if ((s = simplicial_range(c, dirs, d, T, lo, hi, st))) return s;
    KL(launch_suffix_rows(dW, c->ws.S.p, d, T, INT64_MAX / d, c->d_status, st), "suffix_rows");
    const int32_t *simp[kMaxSimplexDim + 1] = {nullptr, c->d_simp[1], c->d_simp[2], c->d_simp[3], c->d_simp[4]};
    CK(launch_simplicial_bwd(c->n, c->d_coords, c->d_xf, c->nv, simp, c->counts, c->max_dim, c->d_sw[0], dirs, d, T, c->ws.dtab.p,
                             c->ws.beta.p, c->ws.S.p, c->ws.bins.p, c->ws.Iacc.p, grad_w, scale, scale_dev, st),
       "simplicial_bwd");
    g_launches += 1 + ((d + 31) / 32) * (1 + c->max_dim + 1);
    return WECT_OK;
}

static wect_status backward_checks(wect_complex c, const double *dirs, int d, int T, double lo, double hi,
                                   const void *up, float *grad_w)
{
    if (!c) return fail(WECT_ERR_INVALID_ARG, "NULL complex");
    if (!dirs || !up || !grad_w) return fail(WECT_ERR_INVALID_ARG, "NULL pointer argument");
    if (d < 1) return fail(WECT_ERR_INVALID_ARG, "d must be >= 1");
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    if (c->kind != 0 && c->sw_mode != WECT_SW_MAX_OF_VERTICES)
        return fail(WECT_ERR_UNSUPPORTED, "the adjoint needs simplex weights that are the max of the vertex weights");
    return WECT_OK;
}

extern "C" wect_status wect_backward(wect_complex c, const double *dirs, int d, int T, double lo, double hi,
                                     const int64_t *dW, double scale, float *grad_w, wect_stream stream)
{
    wect_status s = backward_checks(c, dirs, d, T, lo, hi, dW, grad_w);
    if (s) return s;
    if (!std::isfinite(scale)) return fail(WECT_ERR_INVALID_ARG, "scale must be finite");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(c->mu);
    if ((s = dirs_check(c, dirs, d, st))) return s;
    return complex_backward(c, dirs, d, T, lo, hi, dW, scale, nullptr, grad_w, st);
}

extern "C" wect_status wect_backward_f64(wect_complex c, const double *dirs, int d, int T, double lo, double hi,
                                         const double *G, float *grad_w, wect_stream stream)
{
    wect_status s = backward_checks(c, dirs, d, T, lo, hi, G, grad_w);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(c->mu);
    if ((s = dirs_check(c, dirs, d, st))) return s;
    if ((s = ensure_common_ws(c->ws, T, d))) return s;
    const int64_t n = (int64_t)d * T;
    CK(c->ws.Gq.ensure((size_t)n), "alloc");
    CK(c->ws.gscale.ensure(1), "alloc");
    // headroom: suffix sums over T and sums over d directions, and on a grid the signed sums over
    // the 3^n cells of a vertex
    const int head = ceil_log2(T) + ceil_log2(d) +
                     (c->kind == 0 ? ceil_log2(c->n == 1 ? 3 : (c->n == 2 ? 9 : 27)) : 0);
    KL(launch_grad_quantize(G, n, head, c->ws.M.p, c->ws.Gq.p, c->ws.gscale.p, c->d_status, st), "grad_quantize");
    g_launches++;
    return complex_backward(c, dirs, d, T, lo, hi, reinterpret_cast<const int64_t *>(c->ws.Gq.p), 1.0, c->ws.gscale.p,
                            grad_w, st);
}

// ------------------------------------------------------------------ batches

static wect_status batch_finish(wect_batch b, cudaStream_t st)
{
    b->v_off.resize(b->count);
    int64_t off = 0;
    b->maxL0 = 1;
    for (int i = 0; i < b->count; ++i) {
        set_segments(b->h_grids[i], b->n, b->nsplit);       // with the batch's accumulator mode
        b->h_grids[i].v_off = off;
        b->v_off[i] = off;
        off += b->h_grids[i].nv;
        b->maxL0 = std::max(b->maxL0, unit_len(b->h_grids[i]));
        b->segmented = b->segmented || b->h_grids[i].nseg > 1;
    }
    b->total_nv = off;
    int64_t units = 0;
    for (auto &g : b->h_grids) units += (int64_t)g.rows * g.nseg;
    b->meanL0 = (double)off / (double)std::max<int64_t>(units, 1);
    CK(dev_malloc((void **)&b->d_grids, b->h_grids.size() * sizeof(GridDesc)), "alloc grids");
    CK(cudaMemcpy(b->d_grids, b->h_grids.data(), b->h_grids.size() * sizeof(GridDesc), cudaMemcpyHostToDevice), "upload grids");
    CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream");
    (void)st;
    return ensure_common_ws(b->ws, 2);
}

extern "C" wect_status wect_batch_create(int count, const wect_complex *cxs, wect_batch *out)
{
    if (!out) return fail(WECT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !cxs) return fail(WECT_ERR_INVALID_ARG, "empty batch");
    const wect_complex c0 = cxs[0];
    if (!c0) return fail(WECT_ERR_INVALID_ARG, "NULL complex");
    for (int i = 0; i < count; ++i) {
        const wect_complex c = cxs[i];
        if (!c || c->kind != 0) return fail(WECT_ERR_UNSUPPORTED, "batches hold cubical complexes only");
        if (c->n != c0->n || c->wtype != c0->wtype || c->frac_bits != c0->frac_bits)
            return fail(WECT_ERR_INVALID_ARG, "batch complexes must share n, weight type and frac_bits");
    }
    auto *b = new wect_batch_s();
    b->count = count;
    b->n = c0->n;
    b->wtype = c0->wtype;
    b->frac_bits = c0->frac_bits;
    b->nsplit = 1;
    b->climit = INT64_MAX;
    b->kflush = 1 << 30;
    for (int i = 0; i < count; ++i) {
        b->nsplit = std::max(b->nsplit, cxs[i]->nsplit);
        b->kflush = std::min(b->kflush, cxs[i]->kflush);
    }
    for (int i = 0; i < count; ++i)
        if (cxs[i]->nsplit == b->nsplit) b->climit = std::min(b->climit, cxs[i]->climit);
    b->h_grids.resize(count);
    for (int i = 0; i < count; ++i) {
        GridDesc g{};
        g.w = cxs[i]->d_w32;
        for (int a = 0; a < 3; ++a) g.L[a] = cxs[i]->L[a];
        g.rows = g.L[1] * g.L[2];
        g.nv = cxs[i]->nv;
        g.status = cxs[i]->d_status;
        g.xg = cxs[i]->d_xg;
        g.tmap = cxs[i]->d_tmap;
        b->has_tmap = b->has_tmap || g.tmap != nullptr;
        b->h_grids[i] = g;
    }
    cudaError_t e = dev_malloc((void **)&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
    if (e != cudaSuccess) { wect_batch_destroy(b); return cuda_fail(e, "alloc"); }
    wect_status s = batch_finish(b, nullptr);
    if (s) { wect_batch_destroy(b); return s; }
    *out = b;
    return WECT_OK;
}

extern "C" wect_status wect_batch_create_cubical(int count, int n, const int64_t *dims, const void *vertex_weights,
                                                 wect_wtype wtype, int frac_bits, wect_stream stream, wect_batch *out)
{
    if (!out) return fail(WECT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !dims) return fail(WECT_ERR_INVALID_ARG, "empty batch");
    if (n < 1 || n > 3) return fail(WECT_ERR_INVALID_ARG, "n must be 1..3");
    wect_status s = check_wtype(wtype, frac_bits);
    if (s) return s;
    if (wtype != WECT_W_ONE && !vertex_weights) return fail(WECT_ERR_INVALID_ARG, "vertex_weights is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    auto *b = new wect_batch_s();
    b->count = count;
    b->n = n;
    b->wtype = wtype;
    b->frac_bits = (wtype == WECT_W_F32) ? frac_bits : 0;
    b->h_grids.resize(count);
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        int64_t nv = 1;
        GridDesc g{};
        g.L[0] = g.L[1] = g.L[2] = 1;
        for (int a = 0; a < n; ++a) {
            const int64_t L = dims[(int64_t)i * n + a];
            if (L < 1 || L > (1 << 24)) { delete b; return fail(WECT_ERR_INVALID_ARG, "dims out of range"); }
            g.L[a] = (int)L;
            nv *= L;
        }
        if (nv >= (1ll << 31)) { delete b; return fail(WECT_ERR_INVALID_ARG, "grid too large"); }
        g.rows = g.L[1] * g.L[2];
        g.nv = nv;
        b->h_grids[i] = g;
        total += nv;
    }
    cudaError_t e = dev_malloc((void **)&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = dev_malloc((void **)&b->d_w32, (size_t)total * sizeof(int32_t));
    if (e != cudaSuccess) { wect_batch_destroy(b); return cuda_fail(e, "alloc batch"); }
    b->owns_w = true;
    {
        std::vector<double> xg;
        std::vector<size_t> xoff(count);
        for (int i = 0; i < count; ++i) {
            xoff[i] = xg.size();
            append_grid_coords(b->h_grids[i].L, xg);
        }
        if ((e = upload_doubles(xg, &b->d_xg, st))) { wect_batch_destroy(b); return cuda_fail(e, "grid coordinates"); }
        for (int i = 0; i < count; ++i) b->h_grids[i].xg = b->d_xg + xoff[i];
    }
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        b->h_grids[i].w = b->d_w32 + off;
        b->h_grids[i].status = b->d_status;
        off += b->h_grids[i].nv;
    }
    {
        // TMA tensor maps of the grids that qualify (16-byte aligned start, rows of a multiple of
        // 4 vertices, at most 256), 128 bytes each in one device array
        std::vector<unsigned char> maps;
        std::vector<int> which(count, -1);
        for (int i = 0; i < count; ++i) {
            alignas(64) unsigned char map[128];
            if (encode_grid_tmap(n, b->h_grids[i].L, b->h_grids[i].w, map)) {
                which[i] = (int)(maps.size() / 128);
                maps.insert(maps.end(), map, map + 128);
            }
        }
        if (!maps.empty()) {
            if ((e = dev_malloc(&b->d_tmaps, maps.size()))) { wect_batch_destroy(b); return cuda_fail(e, "alloc tensor maps"); }
            if ((e = cudaMemcpy(b->d_tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice))) {
                wect_batch_destroy(b);
                return cuda_fail(e, "tensor maps");
            }
            for (int i = 0; i < count; ++i)
                if (which[i] >= 0) b->h_grids[i].tmap = static_cast<unsigned char *>(b->d_tmaps) + 128 * which[i];
            b->has_tmap = true;
        }
    }
    if ((s = batch_finish(b, st))) { wect_batch_destroy(b); return s; }
    uint64_t wmax = 255;
    if (wtype == WECT_W_F32 || wtype == WECT_W_I64_FIXED) {
        int *d_bad = nullptr;
        e = dev_malloc((void **)&d_bad, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->ws.M.p, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = launch_weights_to_fixed(wtype, vertex_weights, total, b->frac_bits, nullptr, b->ws.M.p, d_bad, st);
        unsigned long long m = 0;
        int bad = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&m, b->ws.M.p, sizeof m, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (d_bad) cudaFree(d_bad);
        if (e != cudaSuccess) { wect_batch_destroy(b); return cuda_fail(e, "batch weights"); }
        g_launches++;
        if (bad) { wect_batch_destroy(b); return fail(WECT_ERR_INVALID_ARG, "vertex weights are not finite or too large"); }
        wmax = m;
    }
    if ((s = choose_cubical_mode(n, wtype, wmax, b->nsplit, b->climit, b->kflush))) { wect_batch_destroy(b); return s; }
    e = launch_weights_to_w32(wtype, vertex_weights, total, b->frac_bits, b->climit >> n, b->d_w32, b->d_status, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { wect_batch_destroy(b); return cuda_fail(e, "weights_to_w32"); }
    g_launches++;
    *out = b;
    return WECT_OK;
}

extern "C" wect_status wect_batch_set_weights(wect_batch b, const void *w, wect_stream stream)
{
    if (!b) return fail(WECT_ERR_INVALID_ARG, "NULL batch");
    if (!b->owns_w) return fail(WECT_ERR_UNSUPPORTED, "batch does not own its weights");
    if (b->wtype == WECT_W_ONE) return WECT_OK;
    if (!w) return fail(WECT_ERR_INVALID_ARG, "weights is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(b->mu);
    KL(launch_weights_to_w32(b->wtype, w, b->total_nv, b->frac_bits, b->climit >> b->n, b->d_w32, b->d_status, st),
       "weights_to_w32");
    return WECT_OK;
}

extern "C" int wect_batch_count(wect_batch b) { return b ? b->count : 0; }
extern "C" int64_t wect_batch_total_vertices(wect_batch b) { return b ? b->total_nv : 0; }

static bool batch_shape(wect_batch b, int d, int T, double span, CubShape &sh)
{
    auto it = b->tuned.find({d, T});
    if (it != b->tuned.end()) {
        if (it->second.run) return !b->segmented && b->nsplit == 1 && run_shape(b->n, d, T, b->maxL0, sh, it->second.Dt);
        return cub_shape(b->n, b->nsplit, d, T, b->maxL0, sh, it->second.dpl, it->second.Dt, 0.0, 0.0,
                         it->second.threads, b->has_tmap, b->segmented);
    }
    return cub_shape(b->n, b->nsplit, d, T, b->maxL0, sh, 0, 0, b->meanL0, span, 0, b->has_tmap, b->segmented);
}

// Tile-shape code for cache keys: dpl, negative for the global-histogram variant, 100 for runs.
static int shape_code(const CubShape &sh)
{
    return sh.run ? 100
                  : (sh.dpl * (sh.gh ? -1 : 1) + (sh.threads == 256 ? 1000 : 0) + (sh.L0s > 0 ? 10000 : 0) +
                     sh.Tt * 100000);
}

// Work items of a batch for a tile shape.  Whole-complex items (scanned in the CTA, stored
// directly) when every complex fits one flush; otherwise row chunks balanced over the grid.
static wect_status batch_items(wect_batch b, int d, int T, const CubShape &sh, bool &direct, cudaStream_t st)
{
    int64_t maxnv = 0;
    for (auto &g : b->h_grids) maxnv = std::max<int64_t>(maxnv, g.nv);
    const int ntiles = (d + sh.Dt - 1) / sh.Dt;
    direct = !sh.gh && sh.Tt == 0 && maxnv <= b->kflush && (int64_t)b->count * ntiles >= 2 * (int64_t)sh.grid;
    auto key = std::make_tuple(d, T, sh.Dt, shape_code(sh), direct ? 1 : 0);
    if (b->ws.items_key == key) return WECT_OK;
    std::vector<WorkItem> items = make_items(b->h_grids, d, sh.Dt, T, b->kflush, 4 * sh.grid, direct, sh.Tt);
    wect_status s = upload_items(b->ws, items, st);
    if (s) return s;
    b->ws.items_key = key;
    return WECT_OK;
}

static wect_status batch_enqueue(wect_batch b, const CubShape &sh, bool direct, const double *dirs, int d, int T,
                                 double lo, double hi, int64_t *out, cudaStream_t st)
{
    CubLaunch L{b->n, b->nsplit, b->wtype, b->frac_bits, b->kflush, b->maxL0, b->climit, b->d_grids, &b->ws, b->d_status,
                b->segmented};
    return enqueue_cubical_fwd(L, sh, b->ws.n_items, direct, dirs, d, T, lo, hi, false, (int64_t)b->count * d, out, st);
}

extern "C" wect_status wect_batch_compute(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                          int64_t *out, wect_stream stream)
{
    if (!b) return fail(WECT_ERR_INVALID_ARG, "NULL batch");
    if (!dirs || !out) return fail(WECT_ERR_INVALID_ARG, "dirs/out is NULL");
    if (d < 1) return fail(WECT_ERR_INVALID_ARG, "d must be >= 1");
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    if (range_is_default(lo, hi)) return fail(WECT_ERR_UNSUPPORTED, "batches need an explicit threshold range");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(b->mu);
    CubShape sh;
    if (!batch_shape(b, d, T, hi - lo, sh))
        return fail(WECT_ERR_UNSUPPORTED, "no tile shape of the stencil kernel fits (T = %d)", T);
    if (b->maxL0 > b->kflush && !sh.gh) return fail(WECT_ERR_UNSUPPORTED, "grid rows too long");
    if ((s = ensure_common_ws(b->ws, T, d))) return s;
    bool direct = false;
    if ((s = batch_items(b, d, T, sh, direct, st))) return s;
    auto key = std::make_tuple((const void *)dirs, d, T, lo, hi, (void *)out, (void *)st, sh.Dt, shape_code(sh));
    auto it = b->graphs.find(key);
    if (it != b->graphs.end() && it->second.deps != graph_deps(b->ws)) {
        CK(cudaStreamSynchronize(st), "sync");          // a replay of it may still be running
        cudaGraphExecDestroy(it->second.exec);
        cudaGraphDestroy(it->second.graph);
        b->graphs.erase(it);
        it = b->graphs.end();
    }
    if (it == b->graphs.end()) {
        // capture the launch sequence once on a private stream, replay it on the caller's stream
        CK(sh.run ? prepare_cubical_run(b->n, sh.smem) : prepare_cubical_fwd(b->n, b->nsplit, sh.dpl, sh.gh, sh.smem),
           "prepare");
        CK(cudaStreamSynchronize(st), "sync");
        GraphEntry ge;
        const int64_t before = g_launches.load();
        CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        wect_status s2 = batch_enqueue(b, sh, direct, dirs, d, T, lo, hi, out, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &ge.graph);
        if (s2) return s2;
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        ge.nodes = (int)(g_launches.load() - before);
        ge.deps = graph_deps(b->ws);
        g_launches -= ge.nodes;          // counted at each replay instead
        if ((e = cudaGraphInstantiate(&ge.exec, ge.graph, 0)) != cudaSuccess) {
            cudaGraphDestroy(ge.graph);
            return cuda_fail(e, "instantiate");
        }
        it = b->graphs.emplace(key, ge).first;
    }
    {
        ProfScope prof(st);
        CK(cudaGraphLaunch(it->second.exec, st), "graph launch");
    }
    g_launches += it->second.nodes;
    return WECT_OK;
}

extern "C" wect_status wect_batch_compute_loop(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                               int64_t *out, wect_stream stream)
{
    if (!b) return fail(WECT_ERR_INVALID_ARG, "NULL batch");
    if (!dirs || !out) return fail(WECT_ERR_INVALID_ARG, "dirs/out is NULL");
    if (d < 1) return fail(WECT_ERR_INVALID_ARG, "d must be >= 1");
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    if (range_is_default(lo, hi)) return fail(WECT_ERR_UNSUPPORTED, "batches need an explicit threshold range");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(b->mu);
    CubShape sh;
    if (!batch_shape(b, d, T, hi - lo, sh)) return fail(WECT_ERR_UNSUPPORTED, "no tile shape fits");
    if (b->maxL0 > b->kflush && !sh.gh) return fail(WECT_ERR_UNSUPPORTED, "grid rows too long");
    if ((s = ensure_common_ws(b->ws, T, d))) return s;
    // one item list per complex, concatenated; each complex launched on its own
    std::vector<int> &starts = b->loop_starts;
    auto key = std::make_tuple(d, T, sh.Dt, shape_code(sh), 7);
    if (b->ws.items_key != key) {
        std::vector<WorkItem> all;
        starts.assign(b->count + 1, 0);
        for (int i = 0; i < b->count; ++i) {
            std::vector<GridDesc> one(1, b->h_grids[i]);
            std::vector<WorkItem> it = make_items(one, d, sh.Dt, T, b->kflush, sh.grid, false, sh.Tt);
            for (auto &w : it) w.cx = i;
            starts[i] = (int)all.size();
            all.insert(all.end(), it.begin(), it.end());
        }
        starts[b->count] = (int)all.size();
        if ((s = upload_items(b->ws, all, st))) return s;
        b->ws.items_key = key;
    }
    // range, beta and the direction order of the shape (octant groups, or |s_0| for the runs)
    KL(launch_fwd_prep(b->n, dirs, d, T, lo, hi, 0, b->ws.M.p, b->ws.range.p, b->ws.beta.p, b->ws.perm.p,
                       b->ws.octb.p, b->ws.counter.p, b->d_status, nullptr, 0, st, sh.run ? 1 : 0),
       "fwd_prep");
    CK(cudaMemsetAsync(out, 0, (size_t)b->count * d * T * sizeof(int64_t), st), "memset");
    for (int i = 0; i < b->count; ++i) {
        CK(cudaMemsetAsync(b->ws.counter.p, 0, sizeof(int), st), "memset");
        CubicalFwdArgs a{};
        a.grids = b->d_grids;
        a.items = b->ws.items.p + starts[i];
        a.n_items = starts[i + 1] - starts[i];
        a.counter = b->ws.counter.p;
        a.dirs = dirs;
        a.d = d;
        a.T = T;
        a.range = b->ws.range.p;
        a.beta = b->ws.beta.p;
        a.Dt = sh.Dt;
        a.CP = sh.run ? cubical_run_pitch(b->maxL0) : cubical_fwd_pitch(b->maxL0);
        a.perm = b->ws.perm.p;
        a.kflush = b->kflush;
        a.climit = b->climit;
        a.direct = 0;
        a.out = reinterpret_cast<unsigned long long *>(out);
        a.threads = sh.threads;
        a.L0s = sh.L0s;
        a.segmented = b->h_grids[i].nseg > 1 ? 1 : 0;
        a.Tt = sh.Tt;
        const int grid = std::max(1, std::min(sh.grid, a.n_items));
        KL(sh.run ? launch_cubical_run(b->n, a, grid, sh.smem, st)
                  : launch_cubical_fwd(b->n, b->nsplit, sh.dpl, sh.gh, a, grid, sh.smem, st),
           "fwd");
        KL(launch_scan_rows(reinterpret_cast<unsigned long long *>(out) + (int64_t)i * d * T, d, T, st), "scan");
    }
    return WECT_OK;
}

extern "C" wect_status wect_batch_backward(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                           const int64_t *dW, double scale, float *grad_w, wect_stream stream)
{
    if (!b) return fail(WECT_ERR_INVALID_ARG, "NULL batch");
    if (!dirs || !dW || !grad_w) return fail(WECT_ERR_INVALID_ARG, "NULL pointer argument");
    if (d < 1) return fail(WECT_ERR_INVALID_ARG, "d must be >= 1");
    if (!std::isfinite(scale)) return fail(WECT_ERR_INVALID_ARG, "scale must be finite");
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    if (range_is_default(lo, hi)) return fail(WECT_ERR_UNSUPPORTED, "batches need an explicit threshold range");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(b->mu);
    return cubical_backward(b->d_grids, b->count, b->h_grids, b->n, b->wtype, b->frac_bits, b->total_nv, b->ws, dirs, d, T,
                            lo, hi, dW, scale, grad_w, b->d_status, st);
}

extern "C" wect_status wect_batch_backward_f64(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                               const double *G, float *grad_w, wect_stream stream)
{
    if (!b) return fail(WECT_ERR_INVALID_ARG, "NULL batch");
    if (!dirs || !G || !grad_w) return fail(WECT_ERR_INVALID_ARG, "NULL pointer argument");
    if (d < 1) return fail(WECT_ERR_INVALID_ARG, "d must be >= 1");
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    if (range_is_default(lo, hi)) return fail(WECT_ERR_UNSUPPORTED, "batches need an explicit threshold range");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(b->mu);
    if ((s = ensure_common_ws(b->ws, T, d))) return s;
    const int64_t n = (int64_t)b->count * d * T;
    CK(b->ws.Gq.ensure((size_t)n), "alloc");
    CK(b->ws.gscale.ensure(1), "alloc");
    // headroom: suffix sums over T, sums over d directions, signed sums over the 3^n cells of a vertex
    const int head = ceil_log2(T) + ceil_log2(d) + ceil_log2(b->n == 1 ? 3 : (b->n == 2 ? 9 : 27));
    KL(launch_grad_quantize(G, n, head, b->ws.M.p, b->ws.Gq.p, b->ws.gscale.p, b->d_status, st), "grad_quantize");
    g_launches++;
    return cubical_backward(b->d_grids, b->count, b->h_grids, b->n, b->wtype, b->frac_bits, b->total_nv, b->ws, dirs, d, T,
                            lo, hi, reinterpret_cast<const int64_t *>(b->ws.Gq.p), 1.0, grad_w, b->d_status, st,
                            b->ws.gscale.p);
}

extern "C" wect_status wect_batch_autotune(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                           int64_t *scratch_out, wect_stream stream)
{
    if (!b || !dirs || !scratch_out) return fail(WECT_ERR_INVALID_ARG, "NULL argument");
    wect_status s = check_range(lo, hi, T);
    if (s) return s;
    if (range_is_default(lo, hi)) return fail(WECT_ERR_UNSUPPORTED, "batches need an explicit threshold range");
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(b->mu);
    if ((s = ensure_common_ws(b->ws, T, d))) return s;
    const int warps = cubical_fwd_threads() / 32;
    // candidates: (directions per lane, tile width, run-based kernel, CTA size)
    std::vector<std::tuple<int, int, bool, int>> cands;
    for (int threads : {512, 256})
        for (int dpl : {1, 2, 4})
            for (int Dt = 32 * dpl; Dt <= 32 * dpl * (threads / 32); Dt *= 2) cands.push_back({dpl, Dt, false, threads});
    if (b->nsplit == 1 && !b->segmented)
        for (int Dt = 32; Dt <= 256; Dt *= 2) cands.push_back({1, Dt, true, cubical_run_threads()});
    (void)warps;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    float best = 1e30f;
    BatchConfig bc{0, 0, false, 512};
    for (auto [dpl, Dt, run, threads] : cands) {
        if (Dt > 2 * std::max(d, 32 * dpl)) continue;
        CubShape sh;
        if (run) {
            if (!run_shape(b->n, d, T, b->maxL0, sh, Dt)) continue;
        } else if (!cub_shape(b->n, b->nsplit, d, T, b->maxL0, sh, dpl, Dt, 0.0, 0.0, threads, b->has_tmap) ||
                   sh.Dt != Dt || sh.dpl != dpl) {
            continue;
        }
        bool direct = false;
        if ((s = batch_items(b, d, T, sh, direct, st))) break;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaEventRecord(e0, st), "event");
            if ((s = batch_enqueue(b, sh, direct, dirs, d, T, lo, hi, scratch_out, st))) break;
            CK(cudaEventRecord(e1, st), "event");
            CK(cudaEventSynchronize(e1), "event sync");
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
            ms_best = std::min(ms_best, ms);
        }
        if (s) break;
        if (ms_best < best) {
            best = ms_best;
            bc = BatchConfig{dpl, Dt, run, threads};
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    if (bc.Dt == 0) {
        // no shared-histogram shape fits this T: compute keeps the global-histogram shape
        CubShape sh;
        if (!cub_shape(b->n, b->nsplit, d, T, b->maxL0, sh, 0, 0, 0.0, 0.0, 0, b->has_tmap))
            return fail(WECT_ERR_UNSUPPORTED, "no tile shape fits");
        return WECT_OK;
    }
    b->tuned[{d, T}] = bc;
    for (auto &kv : b->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
    }
    b->graphs.clear();
    b->ws.items_key = std::make_tuple(-1, -1, -1, -1, -1);
    return WECT_OK;
}

extern "C" wect_status wect_batch_tuned_shape(wect_batch b, int d, int T, int *shape4)
{
    if (!b || !shape4) return fail(WECT_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->tuned.find({d, T});
    if (it == b->tuned.end()) {
        shape4[0] = shape4[1] = shape4[2] = shape4[3] = 0;
        return WECT_OK;
    }
    shape4[0] = it->second.dpl;
    shape4[1] = it->second.Dt;
    shape4[2] = it->second.run ? 1 : 0;
    shape4[3] = it->second.threads;
    return WECT_OK;
}

extern "C" wect_status wect_debug_stencil_variant(int variant)
{
    if (variant < 0 || variant > 3) return fail(WECT_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
    g_stencil_variant.store(variant);
    return WECT_OK;
}

extern "C" void wect_batch_destroy(wect_batch b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    for (auto &kv : b->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->d_grids) cudaFree(b->d_grids);
    if (b->d_status) cudaFree(b->d_status);
    if (b->owns_w && b->d_w32) cudaFree(b->d_w32);
    if (b->d_tmaps) cudaFree(b->d_tmaps);
    if (b->d_xg) cudaFree(b->d_xg);
    b->ws.release();
    delete b;
}

// ------------------------------------------------------------------ misc

extern "C" const char *wect_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *wect_version(void) { return "wect-gb300 0.2 (sm_103a)"; }

extern "C" const char *wect_last_stencil_kernel(void)
{
    switch (g_last_stencil.load()) {
    case 1: return "cubical_fwd_kernel";
    case 2: return "cubical_run_kernel";
    case 3: return "cubical_fwd_kernel (global histogram)";
    default: return "";
    }
}
extern "C" int64_t wect_kernel_launch_count(void) { return g_launches.load(); }

extern "C" wect_status wect_debug_fail_alloc(int64_t k)
{
    g_alloc_fail_in.store(k < 0 ? -1 : k);
    return WECT_OK;
}

extern "C" wect_status wect_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return WECT_OK;
}

extern "C" wect_status wect_profile_read(double *kernel_ms, int64_t *launches)
{
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        ev.swap(g_prof_events);
    }
    double tot = 0.0;
    wect_status st = WECT_OK;
    for (auto &p : ev) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(p.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.first, p.second);
        if (e != cudaSuccess && st == WECT_OK) st = cuda_fail(e, "profile events");
        tot += ms;
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    if (kernel_ms) *kernel_ms = tot;
    if (launches) *launches = (int64_t)ev.size();
    return st;
}
