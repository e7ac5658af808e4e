// wect_sort.cu -- creation-time reordering of simplex lists for locality (sm_103a).
//
// The transform is a sum over simplices, so the order of a list does not change any result.  The
// gather reads the vertex bins of each simplex; it is fastest when consecutive simplices share
// vertices, because then a chunk of the list references few distinct vertices and its bins can be
// staged in shared memory.  Lists are therefore stably sorted by their smallest vertex id once,
// when the complex is created (CUB's device radix sort, a one-time library sort).  Ties keep the
// caller's order, so the layout is deterministic.
#include <cub/device/device_radix_sort.cuh>

#include "wect_launch.h"

namespace wect {

__global__ void min_vertex_kernel(const int32_t *__restrict__ simp, int64_t k, int m, int32_t *__restrict__ key,
                                  int32_t *__restrict__ idx)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        int v = simp[j * m];
        for (int t = 1; t < m; ++t) v = min(v, simp[j * m + t]);
        key[j] = v;
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

cudaError_t sort_simplices_by_min_vertex(int32_t *simp, int64_t k, int m, int64_t *sw, int64_t nv, cudaStream_t st)
{
    if (k <= 1) return cudaSuccess;
    if (k > INT32_MAX) return cudaErrorInvalidValue;
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < nv) ++bits;
    int32_t *key = nullptr, *key2 = nullptr, *idx = nullptr, *idx2 = nullptr, *simp2 = nullptr;
    int64_t *sw2 = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t e = cudaSuccess;
    const unsigned g = (unsigned)std::min<int64_t>((k + 255) / 256, 152 * 16);
    do {
        if ((e = dev_malloc((void **)&key, k * sizeof(int32_t))) || (e = dev_malloc((void **)&key2, k * sizeof(int32_t))) ||
            (e = dev_malloc((void **)&idx, k * sizeof(int32_t))) || (e = dev_malloc((void **)&idx2, k * sizeof(int32_t))) ||
            (e = dev_malloc((void **)&simp2, (size_t)k * m * sizeof(int32_t))))
            break;
        if (sw && (e = dev_malloc((void **)&sw2, k * sizeof(int64_t)))) break;
        min_vertex_kernel<<<g, 256, 0, st>>>(simp, k, m, key, idx);
        if ((e = cudaGetLastError())) break;
        if ((e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key, key2, idx, idx2, (int)k, 0, bits, st))) break;
        if ((e = dev_malloc(&tmp, tmp_bytes))) break;
        if ((e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, key, key2, idx, idx2, (int)k, 0, bits, st))) break;
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
