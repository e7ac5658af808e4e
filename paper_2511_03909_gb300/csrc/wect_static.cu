// wect_static.cu -- an allocation-free variant of the cubical forward transform.
//
// Some callers cannot call cudaMalloc at all: frameworks and inference servers whose caching
// allocator owns every device byte (an allocation from outside its pool fails or fragments
// it), real-time and embedded services that fix their memory plan at start-up and must not
// allocate afterwards, and plugin hosts that give a plugin no way to allocate.
// wect_cubical_compute_static serves them.  It runs the same kernels as wect_compute on a
// cubical grid, but its scratch memory (threshold table, direction grouping, work-queue head,
// work items, int32 copy of the weights, status word) lives in one file-scope device array of
// fixed size.  Each device reserves the array when this module is loaded on it (with lazy
// module loading, at the latest when the first call looks up its address) and holds it until
// the process exits.
//
// Host code never uses the array's name as a device address.  Every call asks the runtime for
// the array's address on the current device (cudaGetSymbolAddress, with that device current)
// and passes it to the kernels; the first call on a device is the one that does this set-up,
// so it should come before any stream capture.  A call whose stream is capturing does not
// repeat the lookup and uses the address found by the last call on that device.  Calls share
// the array: two calls whose work overlaps on the GPU (different streams, or different host
// threads without ordering) race on it.  Everything that must start at zero is cleared on the
// stream at the start of each call, and wect_cubical_static_status reads (and clears) the
// status word that the last call's device-side checks left.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/wect.h"
#include "wect_device.cuh"
#include "wect_launch.h"

using namespace wect;

namespace {

// Limits of the static scratch (about 8.1 MB in total).
constexpr int64_t kStaticMaxVertices = int64_t(1) << 21;   // 2,097,152 vertices (a 128^3 grid)
constexpr int kStaticMaxDirs = 4096;
constexpr int kStaticMaxT = 4096;
constexpr int kStaticMaxItems = 4096;
constexpr int kStaticMaxDevices = 64;

// Byte offsets inside the array, each on a 256-byte boundary.
constexpr size_t kOffRange = 0;                                   // 6 doubles: lo, hi, step, ...
constexpr size_t kOffM = 256;                                     // 2 x u64: max |h| bits, scratch
constexpr size_t kOffCounter = 512;                               // work-queue head
constexpr size_t kOffStatus = 768;                                // status word
constexpr size_t kOffOctb = 1024;                                 // 9 ints
constexpr size_t kOffGrid = 1280;                                 // one GridDesc
constexpr size_t kOffPerm = 1536;                                 // kStaticMaxDirs ints
constexpr size_t kOffBeta = kOffPerm + sizeof(int) * kStaticMaxDirs;
constexpr size_t kOffItems = kOffBeta + sizeof(double) * kStaticMaxT;
constexpr size_t kOffW32 = kOffItems + sizeof(WorkItem) * kStaticMaxItems;
constexpr size_t kStaticBytes = kOffW32 + sizeof(int32_t) * kStaticMaxVertices;

static_assert(sizeof(GridDesc) <= 256, "grid descriptor slot");
static_assert(kOffBeta % 256 == 0 && kOffItems % 256 == 0 && kOffW32 % 256 == 0, "alignment");

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Writes the grid descriptor and the work items (direction tile x row chunk) into the scratch.
__global__ void static_setup_kernel(unsigned char *scratch, GridDesc g, int ntiles, int chunks, int per)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<GridDesc *>(scratch + kOffGrid) = g;
    WorkItem *items = reinterpret_cast<WorkItem *>(scratch + kOffItems);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntiles * chunks; i += gridDim.x * blockDim.x) {
        const int t = i / chunks, c = i - t * chunks;
        WorkItem w;
        w.cx = 0;
        w.dtile = t;
        w.r0 = c * per;
        w.r1 = min(g.rows, w.r0 + per);
        items[i] = w;
    }
}

static std::mutex g_static_mu;
static void *g_static_ptr[kStaticMaxDevices];

// Device address of the scratch array on the current device.  It is looked up again on every
// call whose stream is not capturing (a module reloaded after cudaDeviceReset may sit at another
// address); a capturing call reuses the last address found on the device.
static cudaError_t static_scratch(cudaStream_t st, unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cs == cudaStreamCaptureStatusNone || !g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_static_ptr[dev]);
    return cudaSuccess;
}

static wect_status sfail(wect_status st, const char *msg)
{
    note_error(msg);
    return st;
}

extern "C" wect_status wect_cubical_compute_static(int n, const int64_t *dims, const void *vertex_weights,
                                                   wect_wtype wtype, const double *dirs, int d, int T, double lo,
                                                   double hi, int64_t *out, wect_stream stream)
{
    if (n < 1 || n > 3 || !dims) return sfail(WECT_ERR_INVALID_ARG, "n must be 1..3 and dims non-NULL");
    if (wtype != WECT_W_U8 && wtype != WECT_W_ONE)
        return sfail(WECT_ERR_UNSUPPORTED, "only uint8 or unweighted grids (accumulator fixed without reading data)");
    if (wtype == WECT_W_U8 && !vertex_weights) return sfail(WECT_ERR_INVALID_ARG, "vertex_weights is NULL");
    if (!dirs || !out) return sfail(WECT_ERR_INVALID_ARG, "dirs/out is NULL");
    if (d < 1 || d > kStaticMaxDirs) return sfail(WECT_ERR_INVALID_ARG, "d must be in [1, 4096]");
    if (T < 2 || T > kStaticMaxT) return sfail(WECT_ERR_INVALID_ARG, "T must be in [2, 4096]");
    const bool dflt = std::isnan(lo) && std::isnan(hi);
    if (!dflt && (!std::isfinite(lo) || !std::isfinite(hi) || lo > hi))
        return sfail(WECT_ERR_INVALID_ARG, "lo <= hi finite, or both NaN");
    int L[3] = {1, 1, 1};
    int64_t nv = 1;
    for (int a = 0; a < n; ++a) {
        if (dims[a] < 1 || dims[a] > (1 << 24)) return sfail(WECT_ERR_INVALID_ARG, "dims out of range");
        L[a] = (int)dims[a];
        nv *= dims[a];
        if (nv > kStaticMaxVertices) return sfail(WECT_ERR_INVALID_ARG, "grid larger than 2^21 vertices");
    }
    // accumulator: u8 weights bound every per-vertex contribution by 2^n * 255
    const int nsplit = 1;
    const int64_t climit = (int64_t(1) << n) * 255;
    const int kflush = (int)((((int64_t)1 << 31) - 1) / climit);
    if (L[0] > kflush) return sfail(WECT_ERR_UNSUPPORTED, "grid rows too long");     // (2^31 - 1) / (2^n 255)

    // tile shape: widest direction tile, then most directions per lane, that fits shared memory
    int dev = 0, sms = 1, optin = 48 * 1024, per_sm = 100 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int threads = cubical_fwd_threads(), warps = threads / 32;
    int dpl = 0, Dt = 0;
    size_t smem = 0;
    int Dmax = 32;
    while (Dmax < d && Dmax < 32 * 4 * warps) Dmax *= 2;
    for (int t = Dmax; t >= 32 && !dpl; t /= 2)
        for (int p : {2, 4, 1}) {
            if (t % (32 * p) || warps % (t / (32 * p)) || (p > 1 && t / p < 32)) continue;
            const size_t sm = cubical_fwd_smem(n, nsplit, p, T, t, L[0]);
            if (sm > (size_t)optin - 1024) continue;
            dpl = p;
            Dt = t;
            smem = sm;
            break;
        }
    bool gh = false;
    if (!dpl) {
        // no shared histogram fits this T: scatter into the int64 table in global memory
        gh = true;
        Dt = std::min(Dmax, 256);
        dpl = Dt >= 64 ? 2 : 1;
        smem = cubical_fwd_smem(n, nsplit, dpl, T, Dt, L[0], true);
        if (smem > (size_t)optin - 1024) return sfail(WECT_ERR_UNSUPPORTED, "grid rows too long for the row buffers");
    }
    const int ctas = sms * std::max(1, std::min((int)(per_sm / (smem + 2048)), 2048 / threads));
    const int rows = L[1] * L[2];
    const int ntiles = (d + Dt - 1) / Dt;
    int chunks = std::max(1, std::min(rows, (ctas + ntiles - 1) / ntiles));
    chunks = std::max(chunks, (rows + std::max(1, kflush / L[0]) - 1) / std::max(1, kflush / L[0]));
    const int per = (rows + chunks - 1) / chunks;
    chunks = (rows + per - 1) / per;
    if ((int64_t)ntiles * chunks > kStaticMaxItems) return sfail(WECT_ERR_UNSUPPORTED, "too many work items");

    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *S = nullptr;
    cudaError_t e = static_scratch(st, &S);
    if (e != cudaSuccess) return sfail(WECT_ERR_CUDA, cudaGetErrorString(e));
    double *range = reinterpret_cast<double *>(S + kOffRange);
    unsigned long long *M = reinterpret_cast<unsigned long long *>(S + kOffM);
    int *counter = reinterpret_cast<int *>(S + kOffCounter);
    int *status = reinterpret_cast<int *>(S + kOffStatus);
    int *octb = reinterpret_cast<int *>(S + kOffOctb);
    GridDesc *grid = reinterpret_cast<GridDesc *>(S + kOffGrid);
    int *perm = reinterpret_cast<int *>(S + kOffPerm);
    double *beta = reinterpret_cast<double *>(S + kOffBeta);
    WorkItem *items = reinterpret_cast<WorkItem *>(S + kOffItems);
    int32_t *w32 = reinterpret_cast<int32_t *>(S + kOffW32);

    GridDesc g{};
    g.w = w32;
    g.L[0] = L[0];
    g.L[1] = L[1];
    g.L[2] = L[2];
    g.rows = rows;
    g.nv = nv;
    g.v_off = 0;
    g.status = status;

#define SCK(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return sfail(WECT_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)
    SCK(cudaMemsetAsync(S + kOffM, 0, 1024 - kOffM, st));     // max-|h| bits, queue head, status word
    static_setup_kernel<<<(ntiles * chunks + 255) / 256, 256, 0, st>>>(S, g, ntiles, chunks, per);
    SCK(cudaGetLastError());
    note_launches(dflt ? 6 : 5);
    SCK(launch_weights_to_w32(wtype, vertex_weights, nv, 0, climit >> n, w32, status, st));
    if (dflt) SCK(launch_grid_max_abs(n, grid, dirs, d, M, st));
    // direction check, range and beta, octant grouping, queue head and a cleared output table
    SCK(launch_fwd_prep(n, dirs, d, T, lo, hi, dflt ? 1 : 0, M, range, beta, perm, octb, counter, status,
                        reinterpret_cast<unsigned long long *>(out), (int64_t)d * T, st));
    CubicalFwdArgs a{};
    a.grids = grid;
    a.items = items;
    a.n_items = ntiles * chunks;
    a.counter = counter;
    a.dirs = dirs;
    a.d = d;
    a.T = T;
    a.range = range;
    a.beta = beta;
    a.Dt = Dt;
    a.CP = cubical_fwd_pitch(L[0]);
    a.perm = perm;
    a.kflush = kflush;
    a.climit = climit;
    a.direct = 0;
    a.out = reinterpret_cast<unsigned long long *>(out);
    SCK(launch_cubical_fwd(n, nsplit, dpl, gh, a, std::min(ctas, a.n_items), smem, st));
    SCK(launch_scan_rows(reinterpret_cast<unsigned long long *>(out), d, T, st));
#undef SCK
    return WECT_OK;
}

extern "C" wect_status wect_cubical_static_status(wect_stream stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *S = nullptr;
    cudaError_t e = static_scratch(st, &S);
    if (e != cudaSuccess) return sfail(WECT_ERR_CUDA, cudaGetErrorString(e));
    int bits = 0;
    e = cudaMemcpyAsync(&bits, S + kOffStatus, sizeof bits, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S + kOffStatus, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return sfail(WECT_ERR_CUDA, cudaGetErrorString(e));
    if (bits & kStatusOverflow) return sfail(WECT_ERR_OVERFLOW, "a per-vertex contribution exceeded the accumulator");
    if (bits & kStatusBadIndex) return sfail(WECT_ERR_INVALID_ARG, "device-side validation failed (non-finite direction)");
    if (bits) return sfail(WECT_ERR_CUDA, "unexpected device status bits");
    return WECT_OK;
}
