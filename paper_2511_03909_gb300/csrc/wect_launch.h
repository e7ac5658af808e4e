// wect_launch.h -- argument blocks and launchers shared between the kernels and the host API.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "wect_device.cuh"

namespace wect {

struct CubicalFwdArgs {
    const GridDesc *grids;
    const WorkItem *items;
    int n_items;
    int *counter;                 // work-queue head, zero before the launch
    const double *dirs;           // [d][n]
    int d, T;
    const double *range;          // [3] = lo, hi, step (resolved on the device)
    const double *beta;           // [T]
    int Dt;                       // direction-tile width (columns of the shared histogram)
    int CP;                       // pitch (words) of the octant-contribution planes of a row
    const int *perm;              // column -> direction (directions grouped by octant)
    int kflush;                   // max vertices of one item (int32 histogram bound)
    int64_t climit;               // largest |c_o(v)| the accumulator mode supports
    int direct;                   // items cover whole complexes: scan in the CTA and store W
    unsigned long long *out;      // int64 difference tables (or W when direct) [count][d][T]
    int threads;                  // CTA size of the per-vertex stencil kernel (256 or 512; 0 = 512)
    int L0s;                      // > 0: rows are staged by TMA from grids with a tensor map, into
                                  // per-row-group buffers of 2 x 3^(n-1) rows of L0s int32
    int segmented;                // some grid walks its rows in segments (GridDesc::seg, nseg)
    int Tt;                       // > 0: threshold tiles of Tt bins (WorkItem::tt); the shared
                                  // histogram then holds Tt + 2 rows (a discard row on each side)
    int pdl;                      // launch as a programmatic dependent of the preceding kernel
};

// Launch k<<<g, b, smem, st>>>(args...), as a programmatic dependent launch when pdl is set: the
// grid may start once every CTA of the preceding kernel in the stream has signalled
// (griddepcontrol.launch_dependents) or exited, and it reads that kernel's results only after
// its own griddepcontrol.wait.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t st, bool pdl,
                                 Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

struct CubicalBwdArgs {
    const GridDesc *grids;
    int n_grids;
    const WorkItem *items;
    const double *dirs;
    int d, T;
    const double *range;
    const double *beta;
    const int *perm;              // directions ordered by octant
    const int *octb;              // [2^n + 1] octant bounds in perm
    int R;
    const int64_t *S;             // suffix sums [count][d][T]
    int64_t *Rv;                  // [2^n][total_nv] octant sums (octant-major planes), as int32 halves
    float *grad;                  // [total_nv]
    int64_t v_begin, v_end;       // vertex range the routing kernel covers
    double scale;
    const double *scale_dev;      // when set, the scale is read from the device (quantised upstream)
    int frac_bits;
    int64_t total_nv;
    int64_t uniform_nv;           // vertex count shared by every grid (0 when they differ)
    // direction chunks of the octant sums (d x T larger than the shared suffix table): dirs, d,
    // perm and octb describe the chunk, whose rows start at direction p0 of the d_all rows of S;
    // accumulate adds the chunk's sums to Rv instead of storing them
    int d_all, p0, accumulate;
    // CTA b of the octant sums takes items [item_ranges[b], item_ranges[b + 1]) in order (a
    // balanced contiguous share of all rows), or item b alone when null
    const int *item_ranges;
};

struct SimplexFwdArgs {
    const int32_t *simp;          // [k][m] vertex ids (m = dim + 1)
    const int64_t *sw;            // [k] fixed-point simplex weights
    const int2 *swp;              // [k] packed signed weights (launch_pack_weights)
    int64_t k;
    int m;                        // vertices per simplex (1 = vertices themselves)
    int sign;                     // (-1)^dim
    const uint16_t *bins;         // [nv][Dt] vertex bins of the current direction tile
    int Dt, dtile, d, T;
    int64_t chunk;                // simplices per CTA work unit (<= flush bound)
    unsigned long long *out;      // [d][T] int64
    // staged chunks (lists of dim >= 1, prepared at creation by launch_chunk_local)
    const uint16_t *local;        // [k][m] chunk-local vertex ids
    const int32_t *cverts;        // [nchunks][kWinRows] vertex ids of each chunk
    const int32_t *cnu;           // [nchunks] distinct vertices of each chunk, -1 above kWinRows
    int64_t nchunks;
    int flush_every;              // chunks between histogram flushes
    int pdl;                      // launch as a programmatic dependent of the preceding kernel
};

// Staged simplex chunks: kChunkSlots vertex slots per chunk (kChunkSlots / m simplices), and a
// chunk is staged when it references at most kWinRows distinct vertices.
constexpr int kChunkSlots = 1536;
constexpr int kWinRows = 544;
// Simplices per chunk: a multiple of 8 so that chunks and 8-simplex groups start on 16-byte
// boundaries of the id and weight arrays.
__host__ __device__ constexpr int chunk_simplices(int m) { return (kChunkSlots / m) & ~7; }
// One shared-memory stage of the staged gather: the vertex-bin window (32 u16 per row), the
// chunk-local ids and the packed weights of the chunk.
constexpr int kWinBytes = kWinRows * 64;
constexpr int kIdBytes = kChunkSlots * 2;
constexpr int kWtBytes = chunk_simplices(2) * 8;
constexpr int kStageBytes = kWinBytes + kIdBytes + kWtBytes;
static_assert(kWinBytes % 16 == 0 && kIdBytes % 16 == 0 && kWtBytes % 16 == 0, "16-byte stage pieces");

// cubical
// gh selects the global-histogram variant (large T): every update goes to the int64 difference
// table in global memory; it needs items that are not scanned in the CTA (direct = 0).
cudaError_t launch_cubical_fwd(int n, int nsplit, int dpl, bool gh, const CubicalFwdArgs &a, int grid, size_t smem,
                               cudaStream_t st);
cudaError_t prepare_cubical_fwd(int n, int nsplit, int dpl, bool gh, size_t smem);   // dynamic smem attribute, outside capture
size_t cubical_fwd_smem(int n, int nsplit, int dpl, int T, int Dt, int maxL0, bool gh = false, int threads = 0,
                        int L0s = 0);
// Row length of the TMA staging buffers for grids whose rows are at most maxL0 long (0: no TMA).
int cubical_fwd_stage_len(int n, int maxL0);
// TMA tensor map of an int32 grid [dims[2]][dims[1]][dims[0]] at w (16-byte aligned, dims[0] a
// multiple of 4 and at most 256, n >= 2), box {dims[0], 3, 3 or 1}, into host memory map (128
// bytes, 64-byte aligned).  False when the grid does not qualify or encoding fails.
bool encode_grid_tmap(int n, const int *dims, const int32_t *w, void *map);
int cubical_fwd_pitch(int maxL0);
int cubical_fwd_threads();           // the largest CTA size of the per-vertex stencil kernel
// The adjoint's octant sums for one direction chunk, then (once every chunk is summed) the routing.
// The run-based stencil kernel (one int32 histogram plane; directions in the run order of
// launch_fwd_prep; CP = cubical_run_pitch): same arguments and items as launch_cubical_fwd.
cudaError_t launch_cubical_run(int n, const CubicalFwdArgs &a, int grid, size_t smem, cudaStream_t st);
cudaError_t prepare_cubical_run(int n, size_t smem);
int cubical_run_pitch(int maxL0);
size_t cubical_run_smem(int n, int T, int Dt, int maxL0);
int cubical_run_threads();
cudaError_t launch_cubical_bwd_rsum(int n, const CubicalBwdArgs &a, int n_items, size_t smem_rsum, cudaStream_t st);
cudaError_t launch_cubical_bwd_route(int n, const CubicalBwdArgs &a, cudaStream_t st);
size_t cubical_bwd_rsum_smem(int n, int d, int T, int R);
// ECF kernels for nf filters: bins [nf][nv], out [nf][T] (blockIdx.y = filter).
cudaError_t launch_cubical_ecf(int n, const GridDesc *grids, const uint16_t *bins, int T, int weighted,
                               int64_t wbound, unsigned long long *out, int64_t nv, int nf, cudaStream_t st);
cudaError_t launch_filter_bins(const double *f, int64_t nv, const double *range, const double *beta, int T,
                               uint16_t *bins, int *status, int flag, cudaStream_t st);
cudaError_t launch_grid_max_abs(int n, const GridDesc *grids, const double *dirs, int d, unsigned long long *Mbits,
                                cudaStream_t st);

// simplicial
cudaError_t launch_dir_filters(int n, const double *dirs, int d, int T, const double *range, float *tab,
                               cudaStream_t st);
cudaError_t launch_coords_to_f32(const double *x, int64_t n, float *xf, cudaStream_t st);
cudaError_t launch_vertex_bins(int n, const double *coords, const float *xf, int64_t nv, const double *dirs,
                               const float *tab, int d, int dtile, int Dt, int T, const double *beta, uint16_t *bins,
                               cudaStream_t st);
// gh: every signed weight goes to the int64 difference table in global memory (no shared
// histogram; any T).
cudaError_t launch_simplex_fwd(int nsplit, bool gh, const SimplexFwdArgs &a, int grid, cudaStream_t st);
// Vertex bins of a 32-direction tile fused with the vertices' own scatter (a: the list of dim 0).
cudaError_t launch_vertex_scatter(int n, int nsplit, const SimplexFwdArgs &a, const double *coords, const float *xf,
                                  int64_t nv, const double *dirs, const float *tab, const double *beta, uint16_t *bins,
                                  int grid, cudaStream_t st);
// Packed signed weights for the gather: v = sign * sw; nsplit 1: {v, 0}, 2: {v & 0xFFFF, v >> 16}.
cudaError_t launch_pack_weights(const int64_t *sw, int64_t k, int sign, int nsplit, int2 *out, cudaStream_t st);
// Morton code of every vertex (coordinates [nv][n], quantised on the box [-xm_a, xm_a]), and the
// stable sort of a list of k simplices (m vertices each, in place) by the smallest code among each
// simplex's vertices; sw (may be null) is permuted alike.  The sort is creation-time only: it
// allocates and synchronises the stream.
cudaError_t vertex_morton_keys(const double *coords, int64_t nv, int n, const double *xm, unsigned long long *vkey,
                               cudaStream_t st);
cudaError_t sort_simplices_spatial(int32_t *simp, int64_t k, int m, int64_t *sw, const unsigned long long *vkey,
                                   cudaStream_t st);
// Chunk-local ids of a list of k simplices with m vertices (m >= 2): per chunk its distinct vertices
// (cverts, cnu) and the list rewritten as the 16-bit byte offsets of their rows in the staged
// window (local).
cudaError_t launch_chunk_local(const int32_t *simp, int64_t k, int m, uint16_t *local, int32_t *cverts, int32_t *cnu,
                               cudaStream_t st);
// The staged gather (two shared-memory windows of kWinRows vertex rows next to the histogram);
// returns cudaErrorInvalidValue when they do not fit.
cudaError_t launch_simplex_fwd_staged(int nsplit, const SimplexFwdArgs &a, int grid, cudaStream_t st);
size_t simplex_fwd_staged_smem(int nsplit, int T, int Dt);
size_t simplex_fwd_smem(int nsplit, int T, int Dt);
cudaError_t launch_simplicial_max_abs(int n, const double *coords, const float *xf, int64_t nv, const double *dirs,
                                      int d, unsigned long long *Mbits, unsigned long long *key, int *cand,
                                      cudaStream_t st);
cudaError_t launch_simplex_weights_max(const int32_t *simp, int64_t k, int m, const int64_t *vw, int64_t *sw,
                                       cudaStream_t st);
cudaError_t launch_simplicial_bwd(int n, const double *coords, const float *xf, int64_t nv, const int32_t *const *simp,
                                  const int64_t *counts, int max_dim, const int64_t *vw, const double *dirs, int d,
                                  int T, const float *tab, const double *beta, const int64_t *S,
                                  uint16_t *bins, unsigned long long *Iacc, float *grad, double scale,
                                  const double *scale_dev, cudaStream_t st);
cudaError_t launch_simplex_ecf(const int32_t *simp, const int64_t *sw, int64_t k, int m, int sign, int weighted,
                               int64_t wbound, const uint16_t *bins, int T, unsigned long long *out, int64_t nv,
                               int nf, cudaStream_t st);

// common
cudaError_t launch_setup_range_beta(double lo, double hi, int use_default, const unsigned long long *Mbits, int T,
                                    double *range, double *beta, cudaStream_t st);
cudaError_t launch_octant_sort(int n, const double *dirs, int d, int *perm, int *octb, cudaStream_t st);
// Fused preparation of the cubical forward: direction check (status may be null), range and beta,
// octant grouping, work-queue head, and (out non-null) a cleared output table of out_elems int64.
// run_order: perm lists the directions by increasing |s_0| (the run kernel's order) instead of
// grouped by octant (octb is then not written).
// pdl: a programmatic dependent launch; early (with pdl): the kernel before is the library's weight
// conversion, which the preparation may overlap (it reads its own inputs before waiting).
cudaError_t launch_fwd_prep(int n, const double *dirs, int d, int T, double lo, double hi, int use_default,
                            const unsigned long long *Mbits, double *range, double *beta, int *perm, int *octb,
                            int *counter, int *status, unsigned long long *out, int64_t out_elems, cudaStream_t st,
                            int run_order = 0, bool pdl = false, bool early = false);
cudaError_t launch_scan_rows(unsigned long long *data, int64_t rows, int T, cudaStream_t st);
// The same scan from src into dst (dst may be mapped pinned host memory; src == dst is in place).
cudaError_t launch_scan_rows_to(const unsigned long long *src, unsigned long long *dst, int64_t rows, int T,
                                cudaStream_t st, bool pdl = false);
cudaError_t launch_copy_f64(const double *src, double *dst, int64_t n, cudaStream_t st);
cudaError_t launch_suffix_rows(const int64_t *in, int64_t *out, int64_t rows, int T, long long smax, int *status,
                               cudaStream_t st);
cudaError_t launch_weights_to_fixed(int wt, const void *w, int64_t nv, int frac_bits, int64_t *out,
                                    unsigned long long *maxabs, int *bad, cudaStream_t st);
cudaError_t launch_weights_to_w32(int wt, const void *w, int64_t nv, int frac_bits, int64_t limit, int32_t *out,
                                  int *status, cudaStream_t st);
cudaError_t launch_weights_check(int wt, const void *w, int64_t nv, int frac_bits, int64_t limit, int *status,
                                 cudaStream_t st);
cudaError_t launch_max_abs_f64(const double *x, int64_t n, int stride, int offset, unsigned long long *Mbits,
                               cudaStream_t st);
cudaError_t launch_grad_quantize(const double *G, int64_t n, int log2_headroom, unsigned long long *maxbits,
                                 long long *out, double *scale, int *status, cudaStream_t st);
cudaError_t launch_finite_check(const double *x, int64_t n, int *bad, int flag, cudaStream_t st);
cudaError_t launch_index_check(const int32_t *idx, int64_t n, int64_t nv, int *bad, cudaStream_t st);

// host-side bookkeeping shared with the C entry points (last error message, launch counter)
void note_error(const char *msg);
void note_launches(int64_t n);
// cudaMalloc behind the library's allocation-failure test hook (wect_debug_fail_alloc).
cudaError_t dev_malloc(void **p, size_t bytes);

}  // namespace wect
