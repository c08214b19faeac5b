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
// Block: 64 consecutive window pixels of one site.  The parents' values
// and magnitudes for those pixels are staged in shared memory once; then
// each half-warp takes one target at a time (its weight row and nonzero
// count are half-warp-uniform loads) and each lane four consecutive pixels
// of one window row, so the y part of the tilt is shared and the x part
// advances by one fixed factor; results leave as 8-byte (bf16 planes) or
// 16-byte (complex64) stores covering whole 128-byte segments.
#include <cuda_bf16.h>

#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int kPix = 64;         // pixels per block
constexpr int kThreads = 256;    // 8 warps = 16 half-warps
constexpr int kPer = 4;          // pixels per lane
constexpr int kLanes = kPix / kPer;          // lanes per target (16)
constexpr int kGroups = kThreads / kLanes;   // targets in flight per block

// Two floats to packed bfloat16 (round to nearest even, one cvt), and the
// residuals x - bf16(x) packed the same way: hi + lo splits of each value.
struct Split4 {   // four values as hi and lo bf16, packed for 8-byte stores
    uint2 hi, lo;
};
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // .x = a (low half)
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float lo_f(uint32_t packed) { return __uint_as_float(packed << 16); }
__device__ __forceinline__ float hi_f(uint32_t packed) { return __uint_as_float(packed & 0xffff0000u); }
__device__ __forceinline__ Split4 split4(float a, float b, float c, float d) {
    const uint32_t h01 = pack_bf16x2(a, b), h23 = pack_bf16x2(c, d);
    Split4 s;
    s.hi = make_uint2(h01, h23);
    s.lo = make_uint2(pack_bf16x2(a - lo_f(h01), b - hi_f(h01)), pack_bf16x2(c - lo_f(h23), d - hi_f(h23)));
    return s;
}

// per-target data, loaded one target ahead of its use
template <int KE>
struct Target {
    int nnz;
    uint32_t idx[KE / 2];    // parent indices, two uint16 per word
    float wt[KE];
    int2 h;
    __device__ int parent(int e) const { return (idx[e / 2] >> (16 * (e & 1))) & 0xffff; }
};
template <int KE>
__device__ __forceinline__ void load_target(const GatherArgs& a, int t, Target<KE>& d) {
    d.nnz = __ldg(&a.ell.nnz[t]);
#pragma unroll
    for (int e = 0; e < KE; e += 8) {
        const uint4 i8 = __ldg(reinterpret_cast<const uint4*>(a.ell.idx + (size_t)t * KE + e));
        d.idx[e / 2] = i8.x; d.idx[e / 2 + 1] = i8.y; d.idx[e / 2 + 2] = i8.z; d.idx[e / 2 + 3] = i8.w;
    }
#pragma unroll
    for (int e = 0; e < KE; e += 4) {
        const float4 w4 = __ldg(reinterpret_cast<const float4*>(a.ell.w + (size_t)t * KE + e));
        d.wt[e] = w4.x; d.wt[e + 1] = w4.y; d.wt[e + 2] = w4.z; d.wt[e + 3] = w4.w;
    }
    d.h = __ldg(&a.h_t[t]);
}

template <int KE, int MAXCH>
__global__ void __launch_bounds__(kThreads, 3) gather_kernel(GatherArgs a, int targets_per_block) {
    extern __shared__ unsigned char smraw[];
    const int Bp = a.Bp;
    float2* sv = reinterpret_cast<float2*>(smraw);                  // [Bp][kPix]
    float* sm = reinterpret_cast<float*>(sv + (size_t)Bp * kPix);   // [Bp][kPix]
    float2* hs = reinterpret_cast<float2*>(sm + (size_t)Bp * kPix); // [MAXCH][kPix]

    const int bs = blockIdx.z;                 // site within the batch
    const int site = a.site_ids[bs];
    const SiteDev st = a.sites[site];
    const int r0 = blockIdx.x * kPix;
    const float2* src = a.stash + (size_t)site * Bp * a.K;
    for (int i = threadIdx.x; i < Bp * kPix; i += kThreads) {
        const int p = i / kPix, r = i % kPix;
        const float2 v = src[(size_t)p * a.K + r0 + r];
        sv[i] = v;
        sm[i] = sqrtf(v.x * v.x + v.y * v.y);
    }
    __syncthreads();

    const int grp = threadIdx.x / kLanes, lane = threadIdx.x % kLanes;
    const int rl = lane * kPer;                // first local pixel of this lane
    const int rr = r0 + rl;                    // first window pixel
    const int u = rr / a.win, v0 = rr % a.win; // the lane's pixels share the row u
    int iy = (st.oy + u) % a.ny;
    if (iy < 0) iy += a.ny;
    int ix0 = (st.ox + v0) % a.nx;
    if (ix0 < 0) ix0 += a.nx;

    // transition potentials of the block's pixels (S1 side), in shared memory
    const int nch = a.nch;
    if (nch > 0) {
        for (int i = threadIdx.x; i < MAXCH * kPix; i += kThreads) {
            const int n = i / kPix, r = i % kPix;
            hs[i] = (n < nch && n < st.nch) ? a.H[(size_t)(st.ch_off + n) * a.K + r0 + r] : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();

    const int t0 = blockIdx.y * targets_per_block;
    const int t1 = min(t0 + targets_per_block, a.n_targets);
    const int nrep = nch > 0 ? nch : 1;
    const size_t plane = (size_t)(nrep * a.rows_pad) * a.K;
    if (t0 + grp >= t1) return;
    Target<KE> cur, nxt;
    load_target(a, t0 + grp, cur);
    float2 ty, tx, step;
    {
        ty = __ldg(&a.ey[(cur.h.x * iy) & (a.ny - 1)]);
        tx = __ldg(&a.ex[(cur.h.y * ix0) & (a.nx - 1)]);
        step = __ldg(&a.ex[cur.h.y & (a.nx - 1)]);
    }
    for (int t = t0 + grp; t < t1; t += kGroups) {
        const bool more = t + kGroups < t1;
        if (more) load_target(a, t + kGroups, nxt);       // in flight during this target
        float ur[kPer], ui[kPer], am[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) ur[j] = ui[j] = am[j] = 0.f;
#pragma unroll
        for (int e = 0; e < KE; ++e) {
            if (e >= cur.nnz) break;
            const float w = cur.wt[e];
            const int pe = cur.parent(e);
            const float4* pv = reinterpret_cast<const float4*>(sv + pe * kPix + rl);
            const float4 m4 = *reinterpret_cast<const float4*>(sm + pe * kPix + rl);
            const float4 p01 = pv[0], p23 = pv[1];
            ur[0] = fmaf(w, p01.x, ur[0]); ui[0] = fmaf(w, p01.y, ui[0]);
            ur[1] = fmaf(w, p01.z, ur[1]); ui[1] = fmaf(w, p01.w, ui[1]);
            ur[2] = fmaf(w, p23.x, ur[2]); ui[2] = fmaf(w, p23.y, ui[2]);
            ur[3] = fmaf(w, p23.z, ur[3]); ui[3] = fmaf(w, p23.w, ui[3]);
            am[0] = fmaf(w, m4.x, am[0]); am[1] = fmaf(w, m4.y, am[1]);
            am[2] = fmaf(w, m4.z, am[2]); am[3] = fmaf(w, m4.w, am[3]);
        }
        // tilt tables of the next target, in flight during this one's epilogue
        float2 ty_n = ty, tx_n = tx, step_n = step;
        if (more) {
            ty_n = __ldg(&a.ey[(nxt.h.x * iy) & (a.ny - 1)]);
            tx_n = __ldg(&a.ex[(nxt.h.y * ix0) & (a.nx - 1)]);
            step_n = __ldg(&a.ex[nxt.h.y & (a.nx - 1)]);
        }
        // re-tilt exp(sign 2 pi i h_t.r/N): y factor shared by the lane's
        // pixels, x factor stepped by exp(sign 2 pi i h_x/N_x)
        float2 sty = ty, stx = tx, sst = step;
        if (a.tilt_sign < 0) {
            sty.y = -sty.y;
            stx.y = -stx.y;
            sst.y = -sst.y;
        }
        float2 tilt = c_mul(sty, stx);
        float2 S[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            float2 sval;
            if (a.magnitude) {
                const float m2 = ur[j] * ur[j] + ui[j] * ui[j];
                if (m2 > 0.f) {
                    const float sc = am[j] * rsqrtf(m2);
                    sval = make_float2(ur[j] * sc, ui[j] * sc);
                } else {
                    sval = make_float2(am[j], 0.f);
                }
            } else {
                sval = make_float2(ur[j], ui[j]);
            }
            S[j] = c_mul(sval, tilt);
            tilt = c_mul(tilt, sst);
        }
#pragma unroll
        for (int n = 0; n < MAXCH; ++n) {
            if (n >= nrep) break;
            float2 o[kPer];
            if (nch > 0) {
                const float4* hp = reinterpret_cast<const float4*>(hs + n * kPix + rl);
                const float4 h01 = hp[0], h23 = hp[1];
                o[0] = c_mul(make_float2(h01.x, h01.y), S[0]);
                o[1] = c_mul(make_float2(h01.z, h01.w), S[1]);
                o[2] = c_mul(make_float2(h23.x, h23.y), S[2]);
                o[3] = c_mul(make_float2(h23.z, h23.w), S[3]);
            } else {
#pragma unroll
                for (int j = 0; j < kPer; ++j) o[j] = S[j];
            }
            const size_t row = (size_t)n * a.rows_pad + t;
            if (a.out_c64) {
                float4* dst = reinterpret_cast<float4*>(a.out_c64 + (size_t)bs * a.site_stride + row * a.K + rr);
                dst[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                dst[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
            } else if (a.out_planes == 4) {
                uint16_t* base = a.out_bf16 + (size_t)bs * a.site_stride + row * a.K + rr;
                const Split4 re = split4(o[0].x, o[1].x, o[2].x, o[3].x);
                const Split4 im = split4(o[0].y, o[1].y, o[2].y, o[3].y);
                *reinterpret_cast<uint2*>(base) = re.hi;
                *reinterpret_cast<uint2*>(base + plane) = re.lo;
                *reinterpret_cast<uint2*>(base + 2 * plane) = im.hi;
                *reinterpret_cast<uint2*>(base + 3 * plane) = im.lo;
            } else {
                uint16_t* base = a.out_bf16 + (size_t)bs * a.site_stride + row * a.K + rr;
                *reinterpret_cast<uint2*>(base) =
                    make_uint2(pack_bf16x2(o[0].x, o[1].x), pack_bf16x2(o[2].x, o[3].x));
                *reinterpret_cast<uint2*>(base + plane) =
                    make_uint2(pack_bf16x2(o[0].y, o[1].y), pack_bf16x2(o[2].y, o[3].y));
            }
        }
        cur = nxt;
        ty = ty_n;
        tx = tx_n;
        step = step_n;
    }
}

template <int KE, int MAXCH>
cudaError_t launch(const GatherArgs& a, cudaStream_t s) {
    const int tpb = 256;
    dim3 grid(a.K / kPix, (a.n_targets + tpb - 1) / tpb, a.n_sites);
    const size_t sm = (size_t)a.Bp * kPix * (sizeof(float2) + sizeof(float)) + (size_t)MAXCH * kPix * sizeof(float2);
    static size_t attr = 0;
    if (sm > 48 * 1024 && sm > attr) {
        cudaError_t e =
            cudaFuncSetAttribute(gather_kernel<KE, MAXCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = sm;
    }
    gather_kernel<KE, MAXCH><<<grid, kThreads, sm, s>>>(a, tpb);
    return cudaGetLastError();
}

}  // namespace

cudaError_t bip_gather(const GatherArgs& a, cudaStream_t s) {
    if (a.K % kPix != 0 || a.win % kPer != 0 || a.nch > 9) return cudaErrorInvalidValue;
    // channel count: 1 stands for the S2 side (no channel product)
    const int mc = a.nch <= 1 ? 1 : (a.nch <= 3 ? 3 : 9);
    switch (a.ell.k * 16 + mc) {
        case 8 * 16 + 1: return launch<8, 1>(a, s);
        case 8 * 16 + 3: return launch<8, 3>(a, s);
        case 8 * 16 + 9: return launch<8, 9>(a, s);
        case 16 * 16 + 1: return launch<16, 1>(a, s);
        case 16 * 16 + 3: return launch<16, 3>(a, s);
        case 16 * 16 + 9: return launch<16, 9>(a, s);
        default: return cudaErrorInvalidValue;
    }
}
