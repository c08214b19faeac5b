// Per-window scales of the FP8 (E4M3) coupling operands.
//
// Each operand row is one beam's 64x64 window (and, on the S1 side, one
// channel's), the contracted index of Eq. coupling; its scale is fixed
// before the row is written, from an a-priori bound of the row's elements:
// a reconstructed window is a convex combination of the site's parent
// windows (Eq. window-recon, Eq. magpreserve: non-negative weights summing
// to one), so |S^t(r)| <= sum_p w_tp max_r |dt_p(r)|, and H_n S1^b is
// bounded by max_r |H_n| times that.  With kappa = 1 + 2^-6 of headroom for
// the rounding on the way, the row is stored as e4m3(v 448 / bound) and the
// product of two rows' scales is applied to the FP32 accumulator.
//
//   f8_hmax_kernel  : once per map call, block per site: max_r |H_n(r)| of
//                     each channel, and H_n divided by it
//   f8_scale_kernel : per batch, warp per target row: the bound from the
//                     row's 64 weights (hi + lo BF16, one coalesced 128-byte
//                     line per plane) and the parents' window maxima
#include <cuda_fp16.h>

#include "bip_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr float kKappa = 1.0f + 1.0f / 64.0f;
constexpr float kE4m3Max = 448.0f;

__global__ void __launch_bounds__(kThreads) f8_hmax_kernel(F8HmaxArgs a) {
    __shared__ float red[kThreads / 32];
    const int site = blockIdx.x;
    const SiteDev st = a.sites[site];
    const int K = st.w * st.w;                 // the site's window
    for (int n = 0; n < 9; ++n) {
        float m = 0.f;
        if (n < st.nch) {
            const float2* h = a.H + (size_t)st.h_off + (size_t)n * K;
            for (int i = threadIdx.x; i < K; i += kThreads) {
                const float2 v = __ldg(&h[i]);
                m = fmaxf(m, fmaf(v.x, v.x, v.y * v.y));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        float r = red[0];
        for (int w = 1; w < kThreads / 32; ++w) r = fmaxf(r, red[w]);
        const float hm = sqrtf(r);
        if (threadIdx.x == 0) a.hmax[(size_t)site * 9 + n] = hm;
        // H_n / max|H_n| for the E4M3 rows (the reconstruction multiplies by it)
        if (n < st.nch) {
            const float inv = hm > 0.f ? 1.f / hm : 0.f;
            const float2* h = a.H + (size_t)st.h_off + (size_t)n * K;
            float2* o = a.Hs + (size_t)st.h_off + (size_t)n * K;
            for (int i = threadIdx.x; i < K; i += kThreads) {
                const float2 v = __ldg(&h[i]);
                o[i] = make_float2(v.x * inv, v.y * inv);
            }
        }
        __syncthreads();
    }
}

// the two FP16 weights of a 32-bit word (the reconstruction's W planes)
__device__ __forceinline__ float f16_word_lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
__device__ __forceinline__ float f16_word_hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }

// grid: (row groups of 8, site in batch, side); warp = one target row
__global__ void __launch_bounds__(kThreads) f8_scale_kernel(F8ScaleArgs a) {
    const int side = blockIdx.z, bs = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * (kThreads / 32) + warp;
    if (t >= a.rows_pad[side]) return;
    float bound = 0.f;
    if (t < a.n_targets[side]) {
        // lane: parents 2 lane and 2 lane + 1
        const uint32_t* whi = reinterpret_cast<const uint32_t*>(a.W + (size_t)(a.w_row0[side] + t) * 64);
        const uint32_t* wlo = whi + (size_t)a.w_pad[side] * 32;
        const uint32_t h = __ldg(&whi[lane]), l = __ldg(&wlo[lane]);
        const unsigned* pm = a.pmax + ((size_t)side * a.n_sites + bs) * 64;
        const float m0 = __uint_as_float(__ldg(&pm[2 * lane])), m1 = __uint_as_float(__ldg(&pm[2 * lane + 1]));
        float s = fmaf(f16_word_lo(h) + f16_word_lo(l), m0, (f16_word_hi(h) + f16_word_hi(l)) * m1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        bound = kKappa * s;
    }
    if (lane == 0) a.inv_row[side][(size_t)bs * a.rows_pad[side] + t] = bound > 0.f ? kE4m3Max / bound : 0.f;
    if (side == 0) {
        if (lane == 0) a.scaleB[(size_t)bs * a.rows_pad[0] + t] = bound / kE4m3Max;
    } else if (lane < a.nch) {
        const int site = a.site_ids[bs];
        const int nuse = min(a.sites[site].nch, a.nch);
        a.scaleA[(size_t)bs * a.nch * a.rows_pad[1] + (size_t)lane * a.rows_pad[1] + t] =
            lane < nuse ? __ldg(&a.hmax[(size_t)site * 9 + lane]) * bound / kE4m3Max : 0.f;
    }
}

}  // namespace

cudaError_t bip_f8_hmax(const F8HmaxArgs& a, cudaStream_t s) {
    if (a.n_sites < 1) return cudaErrorInvalidValue;
    f8_hmax_kernel<<<a.n_sites, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t bip_f8_scales(const F8ScaleArgs& a, cudaStream_t s) {
    if (a.n_sites < 1 || a.nch < 0 || a.nch > 9) return cudaErrorInvalidValue;
    for (int i = 0; i < 2; ++i)
        if (a.n_targets[i] > a.rows_pad[i] || a.n_targets[i] > a.w_pad[i]) return cudaErrorInvalidValue;
    const int rows = a.rows_pad[0] > a.rows_pad[1] ? a.rows_pad[0] : a.rows_pad[1];
    const int per = kThreads / 32;
    f8_scale_kernel<<<dim3((rows + per - 1) / per, a.n_sites, 2), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
