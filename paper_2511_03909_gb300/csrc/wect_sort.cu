// wect_sort.cu -- creation-time reordering of simplex lists for locality (sm_103a).
//
// The transform is a sum over simplices, so the order of a list does not change any result.  The
// gather reads the vertex bins of each simplex; it is fastest when consecutive simplices share
// vertices, because then a chunk of the list references few distinct vertices and its bins can be
// staged in shared memory.  Lists are therefore stably sorted once, when the complex is created
// (CUB's device radix sort, a one-time library sort), by a spatial key: the smallest Morton code
// among the simplex's vertices, the code interleaving the bits of each vertex's coordinates
// quantised on the box [-max|x_a|, max|x_a|].  A chunk then covers a compact patch of the complex
// (on a triangulated grid, a square of about 16 x 16 vertices instead of a strip two rows high),
// which roughly halves the distinct vertices per chunk.  Ties keep the caller's order, so the
// layout is deterministic.
#include <cub/device/device_radix_sort.cuh>

#include "wect_launch.h"

namespace wect {

// Morton code of every vertex: b = 64 / n bits per axis (63 for n = 1), coordinate a quantised
// as floor((x_a / xm_a + 1) / 2 * (2^b - 1)) (0 on an axis with xm_a = 0), bit i of axis a at
// bit i * n + a of the code.
__global__ void vertex_morton_kernel(const double *__restrict__ coords, int64_t nv, int n, double xm0, double xm1,
                                     double xm2, double xm3, unsigned long long *__restrict__ vkey)
{
    const int b = (n == 1) ? 63 : 64 / n;
    const double top = ldexp(1.0, b) - 1.0;
    const double xm[4] = {xm0, xm1, xm2, xm3};
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long key = 0;
        for (int a = 0; a < n; ++a) {
            double t = (xm[a] > 0.0) ? (coords[v * n + a] / xm[a] + 1.0) * 0.5 * top : 0.0;
            t = fmin(fmax(t, 0.0), top);
            const unsigned long long q = (unsigned long long)t;
            for (int i = 0; i < b; ++i) key |= ((q >> i) & 1ull) << (i * n + a);
        }
        vkey[v] = key;
    }
}

__global__ void min_key_kernel(const int32_t *__restrict__ simp, int64_t k, int m,
                               const unsigned long long *__restrict__ vkey, unsigned long long *__restrict__ key,
                               int32_t *__restrict__ idx)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long kk = vkey[simp[j * m]];
        for (int t = 1; t < m; ++t) kk = min(kk, vkey[simp[j * m + t]]);
        key[j] = kk;
        idx[j] = (int32_t)j;
    }
}

__global__ void gather_simplices_kernel(const int32_t *__restrict__ simp, const int64_t *__restrict__ sw, int64_t k,
                                        int m, const int32_t *__restrict__ perm, int32_t *__restrict__ simp_out,
                                        int64_t *__restrict__ sw_out)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = perm[j];
        for (int t = 0; t < m; ++t) simp_out[j * m + t] = simp[s * m + t];
        if (sw) sw_out[j] = sw[s];
    }
}

cudaError_t vertex_morton_keys(const double *coords, int64_t nv, int n, const double *xm, unsigned long long *vkey,
                               cudaStream_t st)
{
    if (nv <= 0) return cudaSuccess;
    const unsigned g = (unsigned)std::min<int64_t>((nv + 255) / 256, 152 * 16);
    vertex_morton_kernel<<<g, 256, 0, st>>>(coords, nv, n, xm[0], n > 1 ? xm[1] : 0.0, n > 2 ? xm[2] : 0.0,
                                            n > 3 ? xm[3] : 0.0, vkey);
    return cudaGetLastError();
}

cudaError_t sort_simplices_spatial(int32_t *simp, int64_t k, int m, int64_t *sw, const unsigned long long *vkey,
                                   cudaStream_t st)
{
    if (k <= 1) return cudaSuccess;
    if (k > INT32_MAX) return cudaErrorInvalidValue;
    unsigned long long *key = nullptr, *key2 = nullptr;
    int32_t *idx = nullptr, *idx2 = nullptr, *simp2 = nullptr;
    int64_t *sw2 = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t e = cudaSuccess;
    const unsigned g = (unsigned)std::min<int64_t>((k + 255) / 256, 152 * 16);
    do {
        if ((e = dev_malloc((void **)&key, k * sizeof(unsigned long long))) ||
            (e = dev_malloc((void **)&key2, k * sizeof(unsigned long long))) ||
            (e = dev_malloc((void **)&idx, k * sizeof(int32_t))) || (e = dev_malloc((void **)&idx2, k * sizeof(int32_t))) ||
            (e = dev_malloc((void **)&simp2, (size_t)k * m * sizeof(int32_t))))
            break;
        if (sw && (e = dev_malloc((void **)&sw2, k * sizeof(int64_t)))) break;
        min_key_kernel<<<g, 256, 0, st>>>(simp, k, m, vkey, key, idx);
        if ((e = cudaGetLastError())) break;
        if ((e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key, key2, idx, idx2, (int)k, 0, 64, st))) break;
        if ((e = dev_malloc(&tmp, tmp_bytes))) break;
        if ((e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key, key2, idx, idx2, (int)k, 0, 64, st))) break;
        gather_simplices_kernel<<<g, 256, 0, st>>>(simp, sw, k, m, idx2, simp2, sw2);
        if ((e = cudaGetLastError())) break;
        if ((e = cudaMemcpyAsync(simp, simp2, (size_t)k * m * sizeof(int32_t), cudaMemcpyDeviceToDevice, st))) break;
        if (sw && (e = cudaMemcpyAsync(sw, sw2, k * sizeof(int64_t), cudaMemcpyDeviceToDevice, st))) break;
        e = cudaStreamSynchronize(st);          // before the temporaries are freed
    } while (0);
    if (e != cudaSuccess) cudaStreamSynchronize(st);    // work queued before the failure uses them too
    cudaFree(key);
    cudaFree(key2);
    cudaFree(idx);
    cudaFree(idx2);
    cudaFree(simp2);
    cudaFree(sw2);
    cudaFree(tmp);
    return e;
}

}  // namespace wect
