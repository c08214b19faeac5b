// The energy-filtered 4D cube (Sec. 2.2.6): Eq. map-sum with the detector
// sum left open,
//   cube[rho][d] = sum_tau scale sum_n |sum_b M^(n)_{d,b} c_b(rho)|^2
// over the sites tau whose crop mask holds rho.
//
//   illum_kernel : c_b(rho) = coef_b exp(-2 pi i h_b.rho/N), [Bpad][P]
//                  complex64 (the angle reduced to [0, 1) turns in FP64)
//   cube_kernel  : block = 64 detector beams x 64 scans; for the sites of a
//                  batch in order, the contraction over b per channel in
//                  16-beam shared tiles, |.|^2 summed over the channels and
//                  added to the block's cube entries -- each entry has one
//                  writer per launch and the sites come in a fixed order, so
//                  the result does not depend on scheduling.
#include "bip_device.cuh"
#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int kTile = 64;        // detector beams and scans per block
constexpr int kKb = 16;          // aperture beams per shared tile
constexpr int kThreads = 256;    // 16 x 16 threads, 4 x 4 outputs each

__global__ void illum_kernel(IllumArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (p >= a.P) return;
    float2 v = make_float2(0.f, 0.f);
    if (b < a.B) {
        const int2 h = a.h[b];
        double t = -((double)h.x * a.scans[2 * p] / a.ny + (double)h.y * a.scans[2 * p + 1] / a.nx);
        t -= floor(t);
        float s, c;
        sincospif(2.0f * (float)t, &s, &c);
        const double2 cf = a.coef[b];
        v = make_float2((float)(cf.x * c - cf.y * s), (float)(cf.x * s + cf.y * c));
    }
    a.C[(size_t)b * a.P + p] = v;
}

// M^(n)_{d,b} is the complex64 coupling at element (b m_ld + n Dp + d)
__global__ void __launch_bounds__(kThreads) cube_kernel(CubeArgs a) {
    __shared__ float2 ms[kKb][kTile];     // [b][d]
    __shared__ float2 cs[kKb][kTile];     // [b][rho]
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int d0 = blockIdx.x * kTile, p0 = blockIdx.y * kTile;
    for (int bs = 0; bs < a.n_sites; ++bs) {
        const SiteDev st = a.sites[a.site_ids[bs]];
        bool in[4];
        bool any = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = p0 + ty * 4 + j;
            in[j] = p < a.P && in_crop(a.scans[2 * p], a.scans[2 * p + 1], st.ty, st.tx, a.ny, a.nx, a.fy, a.fx);
            any |= in[j];
        }
        if (!__syncthreads_or(any)) continue;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int n = 0; n < a.nch; ++n) {
            float ar[4][4], ai[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0.f;
            for (int b0 = 0; b0 < a.Bpad; b0 += kKb) {
                for (int k = threadIdx.x; k < kKb * kTile; k += kThreads) {
                    const int bb = k / kTile, x = k % kTile;
                    const int d = d0 + x, p = p0 + x;
                    ms[bb][x] = d < a.n_det ? a.m32[(size_t)bs * a.m_site + (int64_t)(b0 + bb) * a.m_ld +
                                                    (int64_t)n * a.Dp + d]
                                            : make_float2(0.f, 0.f);
                    cs[bb][x] = p < a.P ? a.C[(size_t)(b0 + bb) * a.P + p] : make_float2(0.f, 0.f);
                }
                __syncthreads();
#pragma unroll
                for (int bb = 0; bb < kKb; ++bb) {
                    float2 mv[4], cv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) mv[i] = ms[bb][tx * 4 + i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) cv[j] = cs[bb][ty * 4 + j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            ar[i][j] = fmaf(mv[i].x, cv[j].x, fmaf(-mv[i].y, cv[j].y, ar[i][j]));
                            ai[i][j] = fmaf(mv[i].x, cv[j].y, fmaf(mv[i].y, cv[j].x, ai[i][j]));
                        }
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i][j], ar[i][j], fmaf(ai[i][j], ai[i][j], acc[i][j]));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!in[j]) continue;
            float* row = a.cube + (size_t)(p0 + ty * 4 + j) * a.cube_ld;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int d = d0 + tx * 4 + i;
                if (d < a.n_det) row[d] += a.scale * acc[i][j];
            }
        }
    }
}

// qEELS: row rho of the cube binned by each beam's bin (beams in order,
// one thread per scan row, so the sums are deterministic)
__global__ void qeels_kernel(const float* __restrict__ cube, int P, int n_det, const int32_t* __restrict__ bin_of,
                             int n_bins, float* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float* o = out + (size_t)p * n_bins;
    for (int i = 0; i < n_bins; ++i) o[i] = 0.f;
    const float* c = cube + (size_t)p * n_det;
    for (int d = 0; d < n_det; ++d) o[__ldg(&bin_of[d])] += c[d];
}

}  // namespace

cudaError_t bip_illum(const IllumArgs& a, cudaStream_t s) {
    if (a.P < 1 || a.Bpad < a.B) return cudaErrorInvalidValue;
    illum_kernel<<<dim3((a.P + 255) / 256, a.Bpad), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t bip_cube_accumulate(const CubeArgs& a, cudaStream_t s) {
    if (a.n_sites < 1) return cudaSuccess;
    if (a.Bpad % kKb || a.cube_ld < a.n_det) return cudaErrorInvalidValue;
    const dim3 grid((a.n_det + kTile - 1) / kTile, (a.P + kTile - 1) / kTile);
    cube_kernel<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t bip_qeels_bin(const float* cube, int P, int n_det, const int32_t* bin_of, int n_bins, float* out,
                          cudaStream_t s) {
    if (P < 1 || n_det < 1 || n_bins < 1) return cudaErrorInvalidValue;
    qeels_kernel<<<(P + 127) / 128, 128, 0, s>>>(cube, P, n_det, bin_of, n_bins, out);
    return cudaGetLastError();
}
