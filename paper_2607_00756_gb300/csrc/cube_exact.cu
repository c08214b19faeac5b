// The 4D cube's exit side (Sec. 2.2.6): the cube keeps every output beam,
// so S2 is not partitioned -- each beam of the complete basis is its own
// column, propagated back from the exit surface (Eq. s2) by the multislice
// sweep in the de-tilted frame, its windows stashed per site.  This kernel
// turns such a stash into the coupling's detector-side operand: the value
// of beam d at window pixel r is the stashed value times the carrier
// exp(-2 pi i h_d.r/N) (the frame removed exp(-2 pi i h_d.r/N) -- the
// conjugate detector plane wave -- when the sweep started from a
// constant), written as complex64, or as BF16 planes (re, im) or split
// BF16 (re_hi, re_lo, im_hi, im_lo).
//
// Grid: (pixel-pair chunks of 256 threads, beams, sites of the batch); a
// thread re-tilts two adjacent pixels of one beam (16-byte load).  HBM
// bound: 8 B read and 4-8 B written per pixel and beam.
#include "bip_device.cuh"
#include "bip_internal.h"
#include "fft_smem.cuh"
#include "tc_common.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) retilt_kernel(RetiltArgs a) {
    const int pair = blockIdx.x * kThreads + threadIdx.x;
    const int d = blockIdx.y, bs = blockIdx.z;
    const int K2 = a.K / 2;
    if (pair >= K2) return;
    const int site = a.site_ids[bs];
    const SiteDev st = a.sites[site];
    const int px = 2 * pair;
    const int u = px / a.win, v = px - u * a.win;              // v even: v, v + 1 on one row
    // the batch's window: the central win x win block (offset wo) of the
    // stashed stash_win x stash_win one
    const size_t sk = (size_t)a.stash_win * a.stash_win;
    const float4 w = __ldg(reinterpret_cast<const float4*>(a.stash + ((size_t)site * a.nd + d) * sk +
                                                           (size_t)(u + a.wo) * a.stash_win + v + a.wo));
    const int2 h = __ldg(&a.h[d]);
    const int oy = st.oy + a.wo, ox = st.ox + a.wo;
    // exp(+2 pi i (h_y y + h_x x) / N) from the per-axis tables, the
    // products reduced modulo N (also when negative)
    const float2 ty = __ldg(&a.ey[wrap_n(h.x * (oy + u), a.ny)]);
    const float2 tx0 = __ldg(&a.ex[wrap_n(h.y * (ox + v), a.nx)]);
    const float2 tx1 = __ldg(&a.ex[wrap_n(h.y * (ox + v + 1), a.nx)]);
    float2 p0 = c_mul(ty, tx0), p1 = c_mul(ty, tx1);
    p0.y = -p0.y;                                               // the conjugate: exp(-2 pi i h.r/N)
    p1.y = -p1.y;
    const float2 o0 = c_mul(make_float2(w.x, w.y), p0), o1 = c_mul(make_float2(w.z, w.w), p1);
    const size_t off = (size_t)bs * a.site_stride + (size_t)d * a.K + px;
    if (a.out_c64) {
        *reinterpret_cast<float4*>(a.out_c64 + off) = make_float4(o0.x, o0.y, o1.x, o1.y);
    } else if (a.out_planes == 4) {
        const size_t plane = (size_t)a.rows_pad * a.K;
        uint16_t* o = a.out_bf16 + off;
        const uint32_t rh = pack_bf16x2(o0.x, o1.x), ih = pack_bf16x2(o0.y, o1.y);
        *reinterpret_cast<uint32_t*>(o) = rh;
        *reinterpret_cast<uint32_t*>(o + plane) = pack_bf16x2(o0.x - bf16_lo(rh), o1.x - bf16_hi(rh));
        *reinterpret_cast<uint32_t*>(o + 2 * plane) = ih;
        *reinterpret_cast<uint32_t*>(o + 3 * plane) = pack_bf16x2(o0.y - bf16_lo(ih), o1.y - bf16_hi(ih));
    } else {
        const size_t plane = (size_t)a.rows_pad * a.K;
        uint16_t* o = a.out_bf16 + off;
        *reinterpret_cast<uint32_t*>(o) = pack_bf16x2(o0.x, o1.x);
        *reinterpret_cast<uint32_t*>(o + plane) = pack_bf16x2(o0.y, o1.y);
    }
}

}  // namespace

cudaError_t bip_retilt(const RetiltArgs& a, cudaStream_t s) {
    if (a.n_sites < 1 || a.nd < 1) return cudaSuccess;
    if (a.K % 2 || a.win % 2 || a.nd > a.rows_pad || a.nd > 65535 || a.n_sites > 65535 || a.ny < 1 || a.nx < 1)
        return cudaErrorInvalidValue;
    if (a.K != a.win * a.win || a.wo < 0 || a.wo % 2 || a.win + 2 * a.wo != a.stash_win) return cudaErrorInvalidValue;
    if (!a.out_c64 && (!a.out_bf16 || (a.out_planes != 2 && a.out_planes != 4))) return cudaErrorInvalidValue;
    const int pairs = a.K / 2;
    retilt_kernel<<<dim3((pairs + kThreads - 1) / kThreads, a.nd, a.n_sites), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
