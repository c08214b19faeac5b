// Sum of the per-site map contributions (Eq. map-sum, incoherent sum over
// sites), each optionally weighted by the site's occupancy.  The partials are zero outside each site's crop mask (the map
// clears them before the per-site evaluation writes the in-crop scans), so
// the sum runs over all sites.  It is done in FP64 with Neumaier
// compensation in a fixed order -- sites in chunks of kChunk in site order,
// then the chunks in order -- so the result does not depend on how the
// sites were batched or scheduled.
#include <algorithm>

#include "bip_internal.h"

namespace {

constexpr int kChunk = 64;
constexpr int kThreads = 256;

// Neumaier step: s + x with the rounding error of the addition kept in c
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

__global__ void __launch_bounds__(kThreads) reduce_chunk_kernel(const float* __restrict__ partial, int n_sites,
                                                                int P, const double* __restrict__ occ,
                                                                double2* __restrict__ chunk_sum) {
    const int p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= P) return;
    const int k0 = blockIdx.y * kChunk, k1 = min(k0 + kChunk, n_sites);
    double s = 0.0, c = 0.0;
    if (occ) {
        for (int k = k0; k < k1; ++k) neumaier(s, c, __ldg(&occ[k]) * (double)__ldg(&partial[(size_t)k * P + p]));
    } else {
#pragma unroll 8
        for (int k = k0; k < k1; ++k) neumaier(s, c, (double)__ldg(&partial[(size_t)k * P + p]));
    }
    chunk_sum[(size_t)blockIdx.y * P + p] = make_double2(s, c);
}

__global__ void __launch_bounds__(kThreads) reduce_final_kernel(const double2* __restrict__ chunk_sum, int n_chunks,
                                                                int P, double* __restrict__ out) {
    const int p = blockIdx.x * kThreads + threadIdx.x;
    if (p >= P) return;
    double s = 0.0, c = 0.0;
    for (int j = 0; j < n_chunks; ++j) {
        const double2 v = chunk_sum[(size_t)j * P + p];
        neumaier(s, c, v.x);
        neumaier(s, c, v.y);
    }
    out[p] = s + c;
}

}  // namespace

size_t bip_reduce_scratch_bytes(int n_sites, int P) {
    return (size_t)((n_sites + kChunk - 1) / kChunk) * P * sizeof(double2);
}

cudaError_t bip_reduce_sites(const float* partial, int n_sites, int P, void* scratch, double* out, cudaStream_t s,
                             const double* occ) {
    const int n_chunks = (n_sites + kChunk - 1) / kChunk;
    if (n_chunks == 0) return cudaMemsetAsync(out, 0, (size_t)P * sizeof(double), s);
    double2* cs = static_cast<double2*>(scratch);
    reduce_chunk_kernel<<<dim3((P + kThreads - 1) / kThreads, n_chunks), kThreads, 0, s>>>(partial, n_sites, P, occ,
                                                                                         cs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final_kernel<<<(P + kThreads - 1) / kThreads, kThreads, 0, s>>>(cs, n_chunks, P, out);
    return cudaGetLastError();
}

// Count of NaN or infinite values in an output (the optional finite check
// of the map, cube, qEELS and gradient calls): n values of 4 or 8 bytes,
// grid-stride, one atomic add per block of its non-zero count.
namespace {

template <class T>
__global__ void __launch_bounds__(kThreads) count_nonfinite_kernel(const T* __restrict__ v, int64_t n,
                                                                   unsigned long long* __restrict__ count) {
    __shared__ unsigned int warp_bad[kThreads / 32];
    unsigned int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
        bad += isfinite(v[i]) ? 0u : 1u;
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) warp_bad[threadIdx.x >> 5] = bad;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += warp_bad[w];
        if (t) atomicAdd(count, (unsigned long long)t);
    }
}

}  // namespace

cudaError_t bip_count_nonfinite(const void* v, int64_t n, int elem_bytes, unsigned long long* count,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
    if (elem_bytes == 8)
        count_nonfinite_kernel<double><<<(int)blocks, kThreads, 0, s>>>((const double*)v, n, count);
    else
        count_nonfinite_kernel<float><<<(int)blocks, kThreads, 0, s>>>((const float*)v, n, count);
    return cudaGetLastError();
}
