// Sum of the per-site map contributions (Eq. map-sum, incoherent sum over
// sites): every scan adds the in-crop contributions of all sites in site
// order, in FP64 with Neumaier compensation, so the result does not depend
// on how the sites were batched.  Also builds the illumination table
// c_b(rho) (Eq. probe with the PRISM rescale).
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

// Ct[rho][b] = coef_b exp(-2 pi i (h_y rho_y / N_y + h_x rho_x / N_x)),
// the phase reduced to [0, 1) turns in FP64 before the sine/cosine.
__global__ void illum_kernel(const double* __restrict__ scans, int P, const int2* __restrict__ h,
                             const double2* __restrict__ coef, int B, int Bpad, int ny, int nx, float2* Ct,
                             uint16_t* Ctb, size_t plane) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (b >= Bpad) return;
    float2 v = make_float2(0.f, 0.f);
    if (b < B) {
        const double ph = (double)h[b].x * scans[2 * p] / ny + (double)h[b].y * scans[2 * p + 1] / nx;
        const double fr = ph - floor(ph);
        double sn, cs;
        sincospi(-2.0 * fr, &sn, &cs);
        const double2 cf = coef[b];
        v = make_float2((float)(cf.x * cs - cf.y * sn), (float)(cf.x * sn + cf.y * cs));
    }
    const size_t o = (size_t)p * Bpad + b;
    if (Ct) Ct[o] = v;
    if (Ctb) {
        auto rn = [](float x) {
            uint32_t u = __float_as_uint(x);
            u += 0x7fffu + ((u >> 16) & 1u);
            return (uint16_t)(u >> 16);
        };
        auto up = [](uint16_t x) { return __uint_as_float((uint32_t)x << 16); };
        const uint16_t rh = rn(v.x), ih = rn(v.y);
        Ctb[o] = rh;
        Ctb[plane + o] = rn(v.x - up(rh));
        Ctb[2 * plane + o] = ih;
        Ctb[3 * plane + o] = rn(v.y - up(ih));
    }
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

cudaError_t bip_illumination(const double* scans, int P, const int2* h_beam, const double2* coef, int B, int Bpad,
                             int ny, int nx, float2* Ct, uint16_t* Ctb, size_t plane, cudaStream_t s) {
    dim3 grid((Bpad + 127) / 128, P);
    illum_kernel<<<grid, 128, 0, s>>>(scans, P, h_beam, coef, B, Bpad, ny, nx, Ct, Ctb, plane);
    return cudaGetLastError();
}
