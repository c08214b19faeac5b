// Window reconstruction of S1 / S2 from the stashed parent windows
// (Eq. window-recon with Eq. magpreserve), written straight into the
// operand layout of the coupling contraction.
//
// For target beam t (an aperture beam for S1, a detector beam for S2) and
// window pixel r:
//   U = sum_p w_{t,p} S^dt_p(r),   A = sum_p w_{t,p} |S^dt_p(r)|
//   S = A U / |U|  (magnitude mode; A where U = 0)  or  S = U  (complex)
//   S_t(r) = S * exp(sign 2 pi i h_t.r/N)   (re-tilt, sign +1 S1, -1 S2)
// The S1 side is multiplied by each channel's transition potential H_n(r)
// (the diag(H_n) of Eq. coupling), giving one operand row per (n, t).
//
// Block: 128 consecutive window pixels of one site; the parents' values
// and magnitudes for those pixels are staged in shared memory once, then
// the block's targets are reconstructed from there.  Consecutive threads
// own consecutive pixels, so every operand row is written coalesced.
#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int kPix = 128;        // pixels per block
constexpr int kThreads = 256;    // two target groups of 128 threads

__device__ __forceinline__ uint16_t bf16_rn(float x) {
    // round-to-nearest-even to bfloat16 (finite inputs)
    uint32_t u = __float_as_uint(x);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

__global__ void __launch_bounds__(kThreads) gather_kernel(GatherArgs a, int targets_per_block) {
    extern __shared__ unsigned char smraw[];
    const int Bp = a.Bp;
    float2* sv = reinterpret_cast<float2*>(smraw);            // [Bp][kPix]
    float* sm = reinterpret_cast<float*>(sv + (size_t)Bp * kPix);  // [Bp][kPix]

    const int bs = blockIdx.z;                 // site within the batch
    const int site = a.site_ids[bs];
    const SiteDev st = a.sites[site];
    const int r0 = blockIdx.x * kPix;
    const float2* src = a.stash + (size_t)site * Bp * a.K;
    for (int i = threadIdx.x; i < Bp * kPix; i += kThreads) {
        const int p = i / kPix, r = i % kPix;
        float2 v = src[(size_t)p * a.K + r0 + r];
        sv[i] = v;
        sm[i] = sqrtf(v.x * v.x + v.y * v.y);
    }
    __syncthreads();

    const int r = threadIdx.x % kPix;
    const int grp = threadIdx.x / kPix;
    const int rr = r0 + r;
    const int u = rr / a.win, v = rr % a.win;
    int iy = (st.oy + u) % a.ny; if (iy < 0) iy += a.ny;
    int ix = (st.ox + v) % a.nx; if (ix < 0) ix += a.nx;

    // transition potentials of this pixel (S1 side)
    float2 hv[9];
    const int nch = a.nch;
    for (int n = 0; n < nch; ++n)
        hv[n] = (n < st.nch) ? a.H[(size_t)(st.ch_off + n) * a.K + rr] : make_float2(0.f, 0.f);

    const int t0 = blockIdx.y * targets_per_block;
    const int t1 = min(t0 + targets_per_block, a.n_targets);
    for (int t = t0 + grp; t < t1; t += kThreads / kPix) {
        float ur = 0.f, ui = 0.f, am = 0.f;
        const int* idx = a.ell.idx + (size_t)t * a.ell.k;
        const float* wt = a.ell.w + (size_t)t * a.ell.k;
        for (int e = 0; e < a.ell.k; ++e) {
            const float w = __ldg(&wt[e]);
            const int p = __ldg(&idx[e]);
            const float2 s = sv[p * kPix + r];
            ur = fmaf(w, s.x, ur);
            ui = fmaf(w, s.y, ui);
            am = fmaf(w, sm[p * kPix + r], am);
        }
        float2 S;
        if (a.magnitude) {
            const float m2 = ur * ur + ui * ui;
            if (m2 > 0.f) {
                const float sc = am * rsqrtf(m2);
                S = make_float2(ur * sc, ui * sc);
            } else {
                S = make_float2(am, 0.f);
            }
        } else {
            S = make_float2(ur, ui);
        }
        // re-tilt exp(sign 2 pi i h_t.r/N) from the integer phase index
        const int2 h = __ldg(&a.h_t[t]);
        int my = (int)(((long long)h.x * iy) % a.ny); if (my < 0) my += a.ny;
        int mx = (int)(((long long)h.y * ix) % a.nx); if (mx < 0) mx += a.nx;
        float2 tilt = c_mul(__ldg(&a.ey[my]), __ldg(&a.ex[mx]));
        if (a.tilt_sign < 0) tilt.y = -tilt.y;
        S = c_mul(S, tilt);

        const int nrep = nch > 0 ? nch : 1;
        for (int n = 0; n < nrep; ++n) {
            const float2 o = nch > 0 ? c_mul(hv[n], S) : S;
            const size_t row = (size_t)n * a.rows_pad + t;
            if (a.out_c64) {
                a.out_c64[(size_t)bs * a.site_stride + row * a.K + rr] = o;
            } else {
                const size_t plane = (size_t)(nrep * a.rows_pad) * a.K;
                uint16_t* base = a.out_bf16 + (size_t)bs * a.site_stride + row * a.K + rr;
                const uint16_t rh = bf16_rn(o.x), ih = bf16_rn(o.y);
                base[0] = rh;
                base[plane] = bf16_rn(o.x - bf16_to_f(rh));
                base[2 * plane] = ih;
                base[3 * plane] = bf16_rn(o.y - bf16_to_f(ih));
            }
        }
    }
}

}  // namespace

cudaError_t bip_gather(const GatherArgs& a, cudaStream_t s) {
    if (a.K % kPix != 0 || a.nch > 9) return cudaErrorInvalidValue;
    const int tpb = 256;
    dim3 grid(a.K / kPix, (a.n_targets + tpb - 1) / tpb, a.n_sites);
    const size_t sm = (size_t)a.Bp * kPix * (sizeof(float2) + sizeof(float));
    static size_t attr = 0;
    if (sm > 48 * 1024 && sm > attr) {
        cudaFuncSetAttribute(gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = sm;
    }
    gather_kernel<<<grid, kThreads, sm, s>>>(a, tpb);
    return cudaGetLastError();
}
