// The probe order of the scan contraction (Sec. 2.2.5, Eq. coupling and
// Eq. map-sum contracted in the other order): with the windowed probes
// Psi(rho, r) = sum_b c_b(rho) S1_b(r) of every scan,
//   a^(n)_d(rho) = sum_r S2_d(r) H_n(r) Psi(rho, r).
// This kernel forms the second operand, Y^(n)(rho, r) = H_n(r) Psi(rho, r),
// as BF16 planes (re, im) with the channel in the column index
// (Y[site][plane][rho][n K + r]); the contraction with S2 and the |.|^2
// detector and channel sums run on the cube kernel.
#include <cuda_bf16.h>

#include "bip_internal.h"

namespace {

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// thread = 8 consecutive pixels r of one (site, scan, channel): two 16-byte
// loads of H and four of Psi, one 16-byte store per plane
__global__ void probe_y_kernel(ProbeYArgs a) {
    const int k8 = a.K / 8;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_site = (int64_t)a.rows * a.nch * k8;
    if (i >= per_site * a.n_sites) return;
    const int bs = (int)(i / per_site);
    int64_t rem = i - (int64_t)bs * per_site;
    const int rho = (int)(rem / ((int64_t)a.nch * k8));
    rem -= (int64_t)rho * a.nch * k8;
    const int n = (int)(rem / k8);
    const int r0 = (int)(rem - (int64_t)n * k8) * 8;
    const SiteDev st = a.sites[a.site_ids[bs]];
    const float4* ps = reinterpret_cast<const float4*>(a.psi + ((int64_t)bs * a.psi_rows + rho) * a.K + r0);
    uint32_t re[4], im[4];
    if (n < st.nch) {
        const float4* hp = reinterpret_cast<const float4*>(a.H + (int64_t)st.h_off + (int64_t)n * a.K + r0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 p = __ldg(&ps[j]), h = __ldg(&hp[j]);
            // (p.x + i p.y) (h.x + i h.y), (p.z + i p.w) (h.z + i h.w)
            re[j] = pack2(p.x * h.x - p.y * h.y, p.z * h.z - p.w * h.w);
            im[j] = pack2(p.x * h.y + p.y * h.x, p.z * h.w + p.w * h.z);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) re[j] = im[j] = 0u;
    }
    uint16_t* y = a.Y + ((int64_t)bs * 2 * a.y_rows + rho) * ((int64_t)a.nch * a.K) + (int64_t)n * a.K + r0;
    *reinterpret_cast<uint4*>(y) = make_uint4(re[0], re[1], re[2], re[3]);
    *reinterpret_cast<uint4*>(y + a.y_rows * (int64_t)a.nch * a.K) = make_uint4(im[0], im[1], im[2], im[3]);
}

}  // namespace

cudaError_t bip_probe_y(const ProbeYArgs& a, cudaStream_t s) {
    if (a.n_sites < 1 || a.rows < 1) return cudaSuccess;
    if (a.K % 8 || a.nch < 1 || a.rows > a.psi_rows || a.rows > a.y_rows) return cudaErrorInvalidValue;
    if (((uintptr_t)a.psi | (uintptr_t)a.H | (uintptr_t)a.Y) & 15) return cudaErrorMisalignedAddress;
    const int64_t n = (int64_t)a.n_sites * a.rows * a.nch * (a.K / 8);
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    probe_y_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}
