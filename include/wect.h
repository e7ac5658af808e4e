/*
 * wect.h -- C ABI of the GB300 (sm_103a) weighted Euler characteristic transform library.
 *
 * The library computes, for a weighted geometric simplicial or cubical complex (K, w), a
 * set of d directions s_p and T thresholds beta[0..T-1],
 *
 *     W[p][q] = sum over cells s of K with bin(max_{v in s} h_p(v)) <= q of (-1)^dim(s) w(s),
 *
 * the discretised weighted Euler characteristic transform (Definition "wect"; Algorithm 1
 * with the height filters of Example "ex:wect"); ecf_compute does the same for one caller
 * supplied vertex filter (Eq. "ecf", Remark "which-ecf").
 *
 * Numerical contract (identical on every call, independent of launch shape):
 *   heights      h = x[n-1]*s[n-1], then h = fma(x[c], s[c], h) for c = n-2..0, float64;
 *   thresholds   step = (hi-lo)/(T-1), beta[q] = lo + q*step (float64, each op rounded);
 *   bins         bin(t) = #{q in [0, T-2] : beta[q] < t}  (exact; values above hi fall in
 *                T-1, so the last column is the weighted Euler characteristic of K);
 *   weights      int64 fixed point: u8 as is, f32 as rint(w * 2^frac_bits); the weight of a
 *                cell of dimension >= 1 is the max of its vertex weights (Figure 1) unless
 *                explicit simplex weights are given;
 *   output       int64 in the same fixed-point units, exact (order-independent sums).
 * Grid coordinates of a cubical complex are x_a(i) = (2i - (L_a-1)) / (L_a-1) (0 when
 * L_a = 1); axis 0 is the fastest-varying axis of every grid array.
 *
 * Conventions.
 *   - Pointers marked (dev) are CUDA device pointers; (host) are host pointers.  The
 *     caller owns every pointer it passes; create calls copy what they keep, so inputs may
 *     be freed after they return.  Outputs must not alias inputs.
 *   - Every compute call is asynchronous and ordered on the given stream (a cudaStream_t;
 *     NULL is the legacy default stream).  Create calls synchronise the stream once.
 *     Outside a stream capture some kernels of a call are programmatic dependent launches of
 *     the call's own kernels; the first kernel of a call waits for everything before it, and
 *     the last one signals completion only when it ends.  The weight conversion of
 *     wect_complex_set_weights signals dependents at its start: a caller's kernel launched
 *     right after it as a programmatic dependent must wait (cudaGridDependencySynchronize)
 *     before touching the weights it was given.
 *   - Every call returns a wect_status; no C++ exception crosses the ABI.  On an argument
 *     error nothing is launched and outputs are untouched.  wect_last_error() returns a
 *     thread-local description of the last failure.
 *   - Device-side conditions that cannot be checked before launch (weights that outgrow the
 *     accumulator chosen at create time, a bounded wait that ran out) set a per-complex
 *     status word, read and cleared by wect_complex_device_status().
 */
#ifndef WECT_H
#define WECT_H

#include <stdint.h>

#if defined(__GNUC__)
#define WECT_API __attribute__((visibility("default")))
#else
#define WECT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wect_complex_s *wect_complex;   /* opaque, owned by the library */
typedef struct wect_batch_s *wect_batch;       /* opaque, owned by the library */
typedef void *wect_stream;                     /* a cudaStream_t */

typedef enum {
    WECT_OK = 0,
    WECT_ERR_INVALID_ARG = 1,   /* bad sizes, T < 2, lo > hi, NaN/Inf input, index out of range */
    WECT_ERR_OUT_OF_MEMORY = 2, /* a device allocation failed */
    WECT_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in wect_last_error) */
    WECT_ERR_OVERFLOW = 4,      /* weights too large for exact int64 accumulation */
    WECT_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
    WECT_ERR_UNSUPPORTED = 6    /* a valid request this build does not implement */
} wect_status;

typedef enum {
    WECT_W_U8 = 0,        /* uint8 vertex weights, used as integers */
    WECT_W_I64_FIXED = 1, /* int64 vertex weights already in fixed point */
    WECT_W_F32 = 2,       /* float32 vertex weights, converted to rint(w * 2^frac_bits) */
    WECT_W_ONE = 3        /* unweighted: every cell has weight 1 (weights pointer ignored) */
} wect_wtype;

typedef enum {
    WECT_SW_MAX_OF_VERTICES = 0, /* w(s) = max of the vertex weights of s (Figure 1) */
    WECT_SW_EXPLICIT = 1         /* per-simplex int64 fixed-point weights supplied */
} wect_simplex_weight_mode;

/* ---------------------------------------------------------------- complexes */

/*
 * Cubical complex of a full n-dimensional grid (n = 1, 2, 3): every vertex, edge, square and
 * cube of the grid (Section 2: the method applies to cubical complexes; cells are boxes of the
 * grid with one corner per sub-mask of their extent).
 *   n               ambient dimension, 1..3
 *   dims (host)     [n] axis lengths, dims[0] = fastest axis, each >= 1, product < 2^31
 *   vertex_weights  (dev) [prod dims] of the type given by wtype (ignored for WECT_W_ONE)
 *   frac_bits       fractional bits for WECT_W_F32 (0..40), else ignored
 * Errors: INVALID_ARG for bad sizes or non-finite f32 weights; OVERFLOW when a cell's signed
 * contribution 2^n * max|w| does not fit 31 bits.
 */
WECT_API wect_status wect_complex_create_cubical(int n, const int64_t *dims, const void *vertex_weights,
                                        wect_wtype wtype, int frac_bits, wect_stream stream,
                                        wect_complex *out);

/*
 * The Freudenthal (Kuhn) triangulation of a full grid, built on the device: the paper's
 * triangulated image (Section 2), an alternative to the cubical complex of the same pixels.
 * Vertices are the grid points at the grid coordinates above; the k-simplices are the chains
 * 0 = c_0 < c_1 < ... < c_k of nested axis masks in {0,1}^n anchored at a grid point v, i.e.
 * {v + c_0, ..., v + c_k}, whenever v + c_k lies in the grid (n! top simplices per unit cube,
 * closed under faces).  The result is a simplicial complex (every simplicial call applies) whose
 * simplex weights are the max of their vertex weights.  Arguments as wect_complex_create_cubical.
 * Errors: as wect_complex_create_simplicial; OUT_OF_MEMORY/CUDA for device failures.
 */
WECT_API wect_status wect_complex_create_freudenthal(int n, const int64_t *dims, const void *vertex_weights,
                                            wect_wtype wtype, int frac_bits, wect_stream stream,
                                            wect_complex *out);

/*
 * Geometric simplicial complex in R^n (Section 3 "inputs": per dimension a list of vertex
 * index rows and a weight per simplex; Section 2: the method holds in any R^n).
 *   n                ambient dimension, 1..4
 *   n_vertices       k_0 >= 1
 *   coords (dev)     [k_0][n] float64 vertex positions l(v), finite
 *   max_dim          highest simplex dimension present, 0..4
 *   counts (host)    [max_dim+1], counts[0] = k_0, counts[i] = k_i >= 0
 *   simplices (host) [max_dim+1] device pointers; simplices[i] (i >= 1) is int32 [k_i][i+1],
 *                    each index in [0, k_0); simplices[0] is ignored.  Closure under faces
 *                    is not checked: the transform sums over exactly the simplices given.
 *   vertex_weights   (dev) [k_0] of type wtype
 *   sw_mode          WECT_SW_MAX_OF_VERTICES or WECT_SW_EXPLICIT
 *   simplex_weights  (host) [max_dim+1] device pointers to int64 [k_i] fixed-point weights
 *                    (EXPLICIT only; entry 0 overrides the vertex weights), else NULL.
 * Errors: INVALID_ARG for bad sizes, indices or non-finite data; OVERFLOW when a weight
 * magnitude reaches 2^40.
 */
WECT_API wect_status wect_complex_create_simplicial(int n, int64_t n_vertices, const double *coords, int max_dim,
                                           const int64_t *counts, const int32_t *const *simplices,
                                           const void *vertex_weights, wect_wtype wtype, int frac_bits,
                                           wect_simplex_weight_mode sw_mode,
                                           const int64_t *const *simplex_weights, wect_stream stream,
                                           wect_complex *out);

/*
 * Replace the vertex weights of an existing complex (same count, same wtype, same frac_bits
 * as at create time); asynchronous, allocates nothing.  For a simplicial complex in
 * MAX_OF_VERTICES mode the simplex weights are recomputed on the device.  Weights larger than
 * the accumulator chosen at create time set WECT_ERR_OVERFLOW in the device status word.
 */
WECT_API wect_status wect_complex_set_weights(wect_complex cx, const void *vertex_weights, wect_stream stream);

/* Number of vertices k_0 (0 for a NULL handle). */
WECT_API int64_t wect_complex_num_vertices(wect_complex cx);

/* Number of cells of each dimension 0..4 (host array of 5, zero beyond the top dimension). */
WECT_API wect_status wect_complex_cell_counts(wect_complex cx, int64_t *counts5);

/* Synchronise the stream, return and clear the device status word of the complex. */
WECT_API wect_status wect_complex_device_status(wect_complex cx, wect_stream stream);

WECT_API void wect_complex_destroy(wect_complex cx);

/* ---------------------------------------------------------------- forward transform */

/*
 * WECT of cx over d directions (Definition "wect", Example "ex:wect", Algorithm 1).
 *   dirs (dev)  [d][n] float64 direction vectors (finite; not required to be unit length)
 *   d >= 1, T >= 2
 *   lo, hi      threshold range; both NaN selects the paper's default [-M, M] with
 *               M = max over directions and vertices of |h_p(v)| (computed exactly on the
 *               device); otherwise lo <= hi, finite.
 *   out (dev)   [d][T] int64, row p = WECF of direction p at thresholds beta[0..T-1]
 * Errors: INVALID_ARG for NULL pointers, d < 1, T < 2 or a bad range; UNSUPPORTED for
 * T > 65535.  Every T up to 65535 is supported.  On a cubical grid, when the int32 histogram of
 * all T thresholds of a direction tile does not fit shared memory, the stencil kernel makes one
 * pass per threshold tile (a band of bins with a discard row on each side); a simplicial
 * complex's gather adds each update to the int64 table in global memory instead.  Any axis-0
 * row length is supported: on a cubical grid, rows longer than 256 vertices (512 for n = 1,
 * half that for two-plane weights) are walked in segments.
 */
WECT_API wect_status wect_compute(wect_complex cx, const double *dirs, int d, int T, double lo, double hi,
                         int64_t *out, wect_stream stream);

/*
 * wect_compute for inputs and output in host memory: optionally new vertex weights, then the
 * WECT of cx (the same table, bit for bit, as wect_complex_set_weights + wect_compute).
 *   weights (host)  nv weights of the complex's weight type (as wect_complex_set_weights), or
 *                   NULL to keep the current weights (ignored for WECT_W_ONE)
 *   dirs (host)     [d][n] float64
 *   out (host)      [d][T] int64
 * Page-locked host buffers (cudaHostAlloc, cudaHostRegister, torch pin_memory) are read and
 * written by the kernels themselves through their device mapping: the weight conversion reads
 * the weights, a copy kernel reads the directions, and the final scan writes out.  Pageable
 * buffers go through cudaMemcpyAsync and device staging kept with the complex (for a pageable
 * out the call returns after the table has arrived).  Device or managed pointers are also
 * accepted and used in place.  Asynchronous otherwise: out is complete once the stream reaches
 * this point, so synchronise the stream before reading it.  Calls on one complex share its
 * staging: order them on one stream.
 * Errors: as wect_compute and wect_complex_set_weights.
 */
WECT_API wect_status wect_compute_host(wect_complex cx, const void *weights, const double *dirs, int d, int T,
                                       double lo, double hi, int64_t *out, wect_stream stream);

/*
 * ECF / WECF of cx for one vertex filter f (Eq. "ecf"; Remark "which-ecf": the ECF of an
 * image when f is the pixel intensity and weighted = 0).
 *   filter (dev) [k_0] float64, finite
 *   weighted     0 => every cell has weight 1; otherwise the complex's weights
 *   out (dev)    [T] int64
 */
WECT_API wect_status ecf_compute(wect_complex cx, const double *filter, int T, double lo, double hi, int weighted,
                        int64_t *out, wect_stream stream);

/*
 * The WECF table of m caller-supplied vertex filters (Algorithm 1 with m filters, Section 3):
 *   out[p][q] = sum over cells s with bin(max_{v in s} f_p(v)) <= q of (-1)^dim(s) w(s),
 * with the same thresholds and bins as wect_compute.  Both lo and hi NaN select [-M, M] with M
 * the largest |f_p(v)| over all m filters, as in the paper.  ecf_compute is the case m = 1.
 *   filters (dev) [m][k_0] float64, finite (a non-finite value sets the status word)
 *   m             number of filters, 1..65535
 *   weighted      0 => every cell has weight 1; otherwise the complex's weights
 *   out (dev)     [m][T] int64
 * Errors: INVALID_ARG for NULL pointers, m out of range or a bad range; UNSUPPORTED for
 * T > 65535.  Workspace: m * k_0 uint16 bins, grown on demand and kept with the complex.
 */
WECT_API wect_status wecf_compute(wect_complex cx, const double *filters, int m, int T, double lo, double hi,
                         int weighted, int64_t *out, wect_stream stream);

/* ---------------------------------------------------------------- adjoint */

/*
 * Adjoint of wect_compute with respect to the vertex weights (the paper names differentiable
 * transforms as future work, Section 6; this is the exact chain rule of Algorithm 1):
 *   S[p][q]  = sum_{q' >= q} dW[p][q']                       (suffix sum of the upstream)
 *   g(s)     = sum_p S[p][bin_p(s)]                           (per cell)
 *   I_v      = sum over cells s whose heaviest vertex is v of (-1)^dim(s) g(s)
 *              (ties of the heaviest vertex go to the lowest vertex index)
 *   grad_w[v] = (float)((double)I_v * scale)
 * All sums are exact integers.  On a simplicial complex I_v is accumulated in 128 bits and the
 * upstream must satisfy d * max_q |S[p][q]| < 2^63.  On a cubical grid every partial sum of I_v
 * is int64, and the bound is 3^n * d * max_q |S[p][q]| < 2^63, because a vertex lies in 3^n
 * cells.  When the bound fails, WECT_ERR_OVERFLOW is set in the device status word and grad_w
 * is unspecified.  Only complexes whose cell weights are the max of their vertex weights
 * (cubical, or simplicial in MAX_OF_VERTICES mode) are supported.
 *   dW (dev)      [d][T] int64 upstream gradient in fixed-point units
 *   grad_w (dev)  [k_0] float32
 * Errors: as wect_compute; on a cubical grid the octant sums stage the suffix rows of a chunk of
 * directions in shared memory (chunks shrink as d x T grows), and T beyond one direction's
 * row in shared memory (about T > 14,000) returns UNSUPPORTED.
 */
WECT_API wect_status wect_backward(wect_complex cx, const double *dirs, int d, int T, double lo, double hi,
                          const int64_t *dW, double scale, float *grad_w, wect_stream stream);

/*
 * Adjoint of wect_compute for a float64 upstream gradient G = dL/dW (dev [d][T]) with W in real
 * units (the fixed-point table times 2^-frac_bits), so grad_w[v] = dL/dw_v for the real-valued
 * vertex weights (the vertex-weight gradient of Section 3's differentiable transform; the
 * autograd function of the Python binding calls this).  G is quantised on the device to int64
 * with the largest power-of-two scale 2^k that keeps H * max|G| * 2^k below 2^62, H = d * T on
 * a simplicial complex and 3^n * d * T on a grid (each rounded up to a power of two): exact
 * when G's values are multiples of 2^-k.  The rest is wect_backward with scale 2^-k.
 * Asynchronous: no host synchronisation.  A non-finite entry of G counts as zero and flags
 * the device status word, which wect_complex_device_status then reports as
 * WECT_ERR_INVALID_ARG.  Errors: as wect_backward.
 */
WECT_API wect_status wect_backward_f64(wect_complex cx, const double *dirs, int d, int T, double lo, double hi,
                                       const double *G, float *grad_w, wect_stream stream);

/* ---------------------------------------------------------------- batches */

/*
 * A batch of cubical complexes computed by one persistent launch over a work queue of
 * (complex, direction tile, row range) items ordered largest first.  The batch refers to the
 * complexes' device data: they must outlive it.  All complexes must be cubical with the same n.
 */
WECT_API wect_status wect_batch_create(int count, const wect_complex *cxs, wect_batch *out);

/*
 * A batch that owns its complexes: count cubical grids of dimension n with per-complex axis
 * lengths dims (host [count][n]) and one concatenated weight array (dev, complexes in order).
 */
WECT_API wect_status wect_batch_create_cubical(int count, int n, const int64_t *dims, const void *vertex_weights,
                                      wect_wtype wtype, int frac_bits, wect_stream stream, wect_batch *out);

/* Replace all weights of a batch made by wect_batch_create_cubical (one device copy). */
WECT_API wect_status wect_batch_set_weights(wect_batch b, const void *vertex_weights, wect_stream stream);

WECT_API int wect_batch_count(wect_batch b);
WECT_API int64_t wect_batch_total_vertices(wect_batch b);

/*
 * WECT of every complex of the batch; out (dev) [count][d][T] int64.  The launch sequence is
 * captured into a CUDA graph on first use for a given (dirs, d, T, range, out, stream) and
 * replayed afterwards.  Tile shapes come from the batch's autotuner (wect_batch_autotune) or a
 * size-based default.
 */
WECT_API wect_status wect_batch_compute(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                               int64_t *out, wect_stream stream);

/* Same result as wect_batch_compute, launched as one ordinary kernel sequence per complex
 * (the per-complex loop the batched path is measured against). */
WECT_API wect_status wect_batch_compute_loop(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                    int64_t *out, wect_stream stream);

/* Adjoint for every complex of the batch: dW (dev) [count][d][T], grad_w (dev) concatenated
 * [sum of k_0] float32 in complex order. */
WECT_API wect_status wect_batch_backward(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                const int64_t *dW, double scale, float *grad_w, wect_stream stream);

/*
 * Adjoint of wect_batch_compute for a float64 upstream gradient G = dL/dW (dev [count][d][T])
 * with W in real units (the fixed-point table times 2^-frac_bits), so grad_w[v] = dL/dw_v for
 * the real-valued vertex weights.  G is quantised on the device to int64 with the largest
 * power-of-two scale 2^k that keeps 3^n * d * T * max|G| * 2^k below 2^62, the headroom of the
 * int64 adjoint (exact when G's values are multiples of 2^-k, as for the gradient of a squared
 * error between fixed-point transforms);
 * the rest is wect_batch_backward.  Asynchronous: no host synchronisation.
 */
WECT_API wect_status wect_batch_backward_f64(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                             const double *G, float *grad_w, wect_stream stream);

/*
 * Time the candidate tile shapes for (d, T) on this batch (synchronises) and keep the fastest:
 * for the per-vertex stencil kernel every tile width Dt (32 .. 32 x directions per lane x warps),
 * 1, 2 or 4 directions per lane, and CTAs of 512 or 256 threads; for the run-based kernel (one
 * histogram plane) Dt = 32 .. 256.  A per-vertex candidate whose histogram cannot hold all T
 * thresholds runs in threshold tiles (the largest band of bins that fits beside its row
 * buffers), so the tuner also chooses the threshold tile.  wect_batch_tuned_shape reports the
 * choice (the threshold tile follows from the direction tile).
 */
WECT_API wect_status wect_batch_autotune(wect_batch b, const double *dirs, int d, int T, double lo, double hi,
                                int64_t *scratch_out, wect_stream stream);

/*
 * The tile shape wect_batch_autotune chose for (d, T) (host int[4]): directions per lane, tile
 * width, 1 for the run-based stencil kernel (else 0), CTA size; all zero when (d, T) is not tuned.
 */
WECT_API wect_status wect_batch_tuned_shape(wect_batch b, int d, int T, int *shape4);

WECT_API void wect_batch_destroy(wect_batch b);

/* ---------------------------------------------------------------- allocation-free variant */

/*
 * The paper has no counterpart to this entry point.  It serves callers that cannot allocate
 * device memory: frameworks and inference servers whose caching allocator owns every device
 * byte (an allocation from outside its pool fails or fragments it), real-time and embedded
 * services that fix their memory at start-up and must not allocate afterwards, and plugin
 * hosts that give a plugin no way to allocate.  It computes exactly what wect_compute computes
 * for the full cubical complex of a grid, with the same kernels, but allocates nothing: its
 * scratch (threshold table, direction grouping, work queue, int32 copy of the weights, status
 * word) lives in one static device array of about 8.1 MB that every GPU loading this library
 * holds until the process exits.
 *   n, dims (host)   grid rank 1..3 and axis lengths (axis 0 fastest); at most 2^21 vertices
 *   vertex_weights   (dev) uint8 [prod dims] for WECT_W_U8; ignored for WECT_W_ONE (other types:
 *                    WECT_ERR_UNSUPPORTED)
 *   dirs (dev)       [d][n] float64, 1 <= d <= 4096;  2 <= T <= 4096;  lo, hi as wect_compute
 *   out (dev)        [d][T] int64, caller-allocated
 * d, T, dims or the vertex count beyond these limits return WECT_ERR_INVALID_ARG; rows (axis 0)
 * longer than the kernel's shared row buffers hold (about 800 vertices for n = 3, 1,600 for
 * n = 2, 3,200 for n = 1) or a grid that needs more than 4096 work items return
 * WECT_ERR_UNSUPPORTED.  Nothing is launched then
 * and the message is in wect_last_error.  Every call looks up the array's device address on the
 * current device (cudaGetSymbolAddress); the first call on a device is the one that sets the
 * array up, so make it before any stream capture.  Every call shares the one array and clears
 * on its stream what must start at zero, so calls whose work overlaps on the GPU (other streams,
 * or unordered host threads) race; order them.  Directions are checked on the device:
 * wect_cubical_static_status reports what the last call's checks found.
 */
WECT_API wect_status wect_cubical_compute_static(int n, const int64_t *dims, const void *vertex_weights,
                                                 wect_wtype wtype, const double *dirs, int d, int T, double lo,
                                                 double hi, int64_t *out, wect_stream stream);

/*
 * Status of the device-side checks of the last wect_cubical_compute_static call on the current
 * device (the paper has no counterpart): synchronises the stream, reads the status word in the
 * static scratch and clears it.  WECT_ERR_INVALID_ARG when a direction was not finite (the
 * table written by that call is then meaningless), else WECT_OK.  Allocates nothing.
 */
WECT_API wect_status wect_cubical_static_status(wect_stream stream);

/* ---------------------------------------------------------------- misc */

/* Thread-local message for the last non-OK status on this thread ("" if none). */
WECT_API const char *wect_last_error(void);

/* Library version string. */
WECT_API const char *wect_version(void);

/*
 * Name of the stencil kernel that the last cubical forward enqueued by this process used
 * ("cubical_fwd_kernel", "cubical_run_kernel", ...; "" before the first), for benchmark reports.
 */
WECT_API const char *wect_last_stencil_kernel(void);

/*
 * Number of kernels this library launched (or replayed inside its graphs) on the calling
 * process since load, for launch accounting.
 */
WECT_API int64_t wect_kernel_launch_count(void);

/*
 * Kernel timing hook for benchmarks.  While enabled, every compute call records a pair of CUDA
 * events on its stream around its dominant kernel (the stencil or gather scatter kernel, or
 * the replayed batch graph, or the adjoint's kernels).  wect_profile_read synchronises on the
 * recorded events, returns the summed kernel milliseconds and the number of timed launches
 * since the last read, and releases the events.  Outside a stream capture the cubical forward
 * launches its preparation, stencil kernel and scan as programmatic dependent launches (each
 * may start while the kernel before it finishes); while the hook is on, the stencil kernel is
 * launched in plain stream order instead, so that its events bracket all of it.
 */
WECT_API wect_status wect_profile_enable(int on);
WECT_API wect_status wect_profile_read(double *kernel_ms, int64_t *launches);

/*
 * Allocation-failure injection, a test hook for the error paths.  With k >= 0 the next k
 * device allocations the library makes (in any call, on any thread) succeed and the one after
 * fails as if the device were out of memory: the call that made it returns
 * WECT_ERR_OUT_OF_MEMORY, frees what it had allocated, and leaves its handles and outputs as
 * they were.  The failing allocation disarms the hook; k < 0 disarms it at once.  No CUDA
 * call fails for real, so the context stays usable.  Always returns WECT_OK.
 */
WECT_API wect_status wect_debug_fail_alloc(int64_t k);

/*
 * Stencil-kernel selection for full cubical grids, a test and tuning hook.  The transform of a
 * grid has two exact kernels that give identical integers: one adds each vertex's octant
 * contribution to its bin, the other (one histogram plane only: u8, unweighted or narrow
 * weights) walks the bin boundaries of each grid row and adds prefix-sum differences.
 *   variant 0   choose by a cost estimate (default): the run kernel for long rows and few
 *               thresholds per row
 *   variant 1   the per-vertex kernel only
 *   variant 2   the run kernel wherever it applies
 *   variant 3   the per-vertex kernel, reading the neighbouring rows from global memory
 *               instead of staging them in shared memory by TMA
 * Process-wide; affects compute calls made afterwards (a batch's tuned shape takes precedence,
 * and graphs already captured keep their kernel).  INVALID_ARG for another value.
 */
WECT_API wect_status wect_debug_stencil_variant(int variant);

#ifdef __cplusplus
}
#endif

#endif /* WECT_H */
