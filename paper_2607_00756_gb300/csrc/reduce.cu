// Sum of the per-site map contributions (Eq. map-sum, incoherent sum over
// sites): every scan adds the in-crop contributions of all sites in site
// order, in FP64 with Neumaier compensation, so the result does not depend
// on how the sites were batched.
#include "bip_device.cuh"
#include "bip_internal.h"

namespace {

__global__ void reduce_kernel(const float* __restrict__ partial, int n_sites, int P,
                              const double* __restrict__ scans, const SiteDev* __restrict__ sites, int ny,
                              int nx, int fy, int fx, double* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double ry = scans[2 * p], rx = scans[2 * p + 1];
    double s = 0.0, c = 0.0;
    for (int k = 0; k < n_sites; ++k) {
        const SiteDev st = sites[k];
        if (!in_crop(ry, rx, st.ty, st.tx, ny, nx, fy, fx)) continue;
        const double x = (double)partial[(size_t)k * P + p];
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    out[p] = s + c;
}

__global__ void zero_outside_kernel(float* __restrict__ partial, int n_sites, int P,
                                    const double* __restrict__ scans, const SiteDev* __restrict__ sites, int ny,
                                    int nx, int fy, int fx) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (p >= P) return;
    const SiteDev st = sites[k];
    if (!in_crop(scans[2 * p], scans[2 * p + 1], st.ty, st.tx, ny, nx, fy, fx)) partial[(size_t)k * P + p] = 0.f;
}

}  // namespace

cudaError_t bip_reduce_sites(const float* partial, int n_sites, int P, const double* scans, const SiteDev* sites,
                             int ny, int nx, int fy, int fx, double* out, cudaStream_t s) {
    reduce_kernel<<<(P + 255) / 256, 256, 0, s>>>(partial, n_sites, P, scans, sites, ny, nx, fy, fx, out);
    return cudaGetLastError();
}

cudaError_t bip_zero_outside(float* partial, int n_sites, int P, const double* scans, const SiteDev* sites,
                             int ny, int nx, int fy, int fx, cudaStream_t s) {
    if (n_sites == 0) return cudaSuccess;
    dim3 grid((P + 255) / 256, n_sites);
    zero_outside_kernel<<<grid, 256, 0, s>>>(partial, n_sites, P, scans, sites, ny, nx, fy, fx);
    return cudaGetLastError();
}
