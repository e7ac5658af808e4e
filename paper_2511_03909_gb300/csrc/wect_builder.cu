// wect_builder.cu -- the Freudenthal (Kuhn) triangulation of a full grid, built on the device.
//
// The paper offers a triangulated image as an alternative to the cubical complex of its pixels
// (Section 2).  Here the vertices are the grid points, placed by the grid coordinate rule
// x_a(i) = (2i - (L_a-1)) / (L_a-1) (0 when L_a = 1), and the simplices of dimension k are the
// chains 0 = c_0 < c_1 < ... < c_k of nested axis masks in {0,1}^n: the simplex anchored at v is
// {v + c_0, ..., v + c_k} (offsets read as vectors), present when v + c_k is in the grid.  Every
// unit cube is cut into n! top simplices along these chains; the lists of every dimension are
// closed under faces.  The complex is then created as a simplicial complex whose simplex
// weights are the max of their vertex weights.
#include <vector>

#include "../../include/wect.h"
#include "wect_device.cuh"
#include "wect_launch.h"

namespace wect {

__global__ void grid_coords_kernel(int n, int L0, int L1, int L2, int64_t nv, double *__restrict__ coords)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        const int i0 = (int)(v % L0), i1 = (int)((v / L0) % L1), i2 = (int)(v / ((int64_t)L0 * L1));
        coords[v * n] = grid_coord(i0, L0);
        if (n >= 2) coords[v * n + 1] = grid_coord(i1, L1);
        if (n >= 3) coords[v * n + 2] = grid_coord(i2, L2);
    }
}

struct ChainType {
    int m;                        // vertices per simplex (k + 1)
    int off[4];                   // flat vertex offsets of c_0..c_k
    int A[3];                     // anchor box: L_a - (bit a of c_k)
};

// The simplices of one chain type, anchors in row-major order of the anchor box.
__global__ void chain_cells_kernel(ChainType t, int L0, int L1, int64_t count, int32_t *__restrict__ out)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x) {
        const int a0 = (int)(j % t.A[0]), a1 = (int)((j / t.A[0]) % t.A[1]), a2 = (int)(j / ((int64_t)t.A[0] * t.A[1]));
        const int v = a0 + L0 * (a1 + L1 * a2);
        for (int s = 0; s < t.m; ++s) out[j * t.m + s] = v + t.off[s];
    }
}

}  // namespace wect

using namespace wect;

// Chains 0 = c_0 < c_1 < ... < c_k of masks in {0,1}^n (strict inclusion), by dimension k.
static void chains(int n, int last, std::vector<int> &cur, std::vector<std::vector<int>> *by_dim)
{
    const int k = (int)cur.size() - 1;
    if (k >= 1) by_dim[k].push_back(cur);
    for (int nxt = 1; nxt < (1 << n); ++nxt)
        if ((nxt & last) == last && nxt != last) {
            cur.push_back(nxt);
            chains(n, nxt, cur, by_dim);
            cur.pop_back();
        }
}

extern "C" wect_status wect_complex_create_freudenthal(int n, const int64_t *dims, const void *vertex_weights,
                                                       wect_wtype wtype, int frac_bits, wect_stream stream,
                                                       wect_complex *out)
{
    if (!out) return WECT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || n > 3 || !dims) {
        note_error("n must be 1..3 and dims non-NULL");
        return WECT_ERR_INVALID_ARG;
    }
    int L[3] = {1, 1, 1};
    int64_t nv = 1;
    for (int a = 0; a < n; ++a) {
        if (dims[a] < 1 || dims[a] > (1 << 24)) {
            note_error("dims out of range");
            return WECT_ERR_INVALID_ARG;
        }
        L[a] = (int)dims[a];
        nv *= dims[a];
        if (nv >= (1ll << 31)) {
            note_error("grid has >= 2^31 vertices");
            return WECT_ERR_INVALID_ARG;
        }
    }
    std::vector<std::vector<int>> by_dim[4];
    std::vector<int> cur{0};
    chains(n, 0, cur, by_dim);
    const int stride[3] = {1, L[0], L[0] * L[1]};
    cudaStream_t st = (cudaStream_t)stream;
    double *coords = nullptr;
    int32_t *lists[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t counts[4] = {nv, 0, 0, 0};
    wect_status status = WECT_OK;
    cudaError_t e = dev_malloc((void **)&coords, (size_t)nv * n * sizeof(double));
    if (e == cudaSuccess) {
        grid_coords_kernel<<<(unsigned)std::min<int64_t>((nv + 255) / 256, 152 * 16), 256, 0, st>>>(n, L[0], L[1], L[2],
                                                                                                    nv, coords);
        e = cudaGetLastError();
        note_launches(1);
    }
    for (int k = 1; k <= n && e == cudaSuccess; ++k) {
        std::vector<ChainType> types;
        std::vector<int64_t> tcount;
        for (const auto &ch : by_dim[k]) {
            ChainType t{};
            t.m = k + 1;
            for (int s = 0; s <= k; ++s) {
                int o = 0;
                for (int a = 0; a < n; ++a)
                    if ((ch[s] >> a) & 1) o += stride[a];
                t.off[s] = o;
            }
            int64_t cnt = 1;
            for (int a = 0; a < 3; ++a) {
                t.A[a] = (a < n) ? L[a] - ((ch[k] >> a) & 1) : 1;
                cnt *= std::max(t.A[a], 0);
            }
            types.push_back(t);
            tcount.push_back(cnt);
            counts[k] += cnt;
        }
        if (counts[k] == 0) continue;
        if ((e = dev_malloc((void **)&lists[k], (size_t)counts[k] * (k + 1) * sizeof(int32_t)))) break;
        int64_t base = 0;
        for (size_t t = 0; t < types.size(); ++t) {
            if (tcount[t] > 0) {
                chain_cells_kernel<<<(unsigned)std::min<int64_t>((tcount[t] + 255) / 256, 152 * 16), 256, 0, st>>>(
                    types[t], L[0], L[1], tcount[t], lists[k] + base * (k + 1));
                note_launches(1);
            }
            base += tcount[t];
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        note_error(cudaGetErrorString(e));
        status = e == cudaErrorMemoryAllocation ? WECT_ERR_OUT_OF_MEMORY : WECT_ERR_CUDA;
    } else {
        int max_dim = 0;
        for (int k = 1; k <= n; ++k)
            if (counts[k] > 0) max_dim = k;
        status = wect_complex_create_simplicial(n, nv, coords, max_dim, counts, lists, vertex_weights, wtype, frac_bits,
                                                WECT_SW_MAX_OF_VERTICES, nullptr, stream, out);
    }
    cudaStreamSynchronize(st);      // the create copied what it keeps
    cudaFree(coords);
    for (int k = 1; k <= 3; ++k) cudaFree(lists[k]);
    return status;
}
