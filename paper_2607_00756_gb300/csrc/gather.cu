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
// and magnitudes for those pixels are staged in shared memory once.  Each
// warp then takes groups of kGatherGroup consecutive targets; a group's
// targets are close on the beam lattice and share most natural neighbours,
// so the warp walks the union of their parents once, loading each parent's
// values for its 64 pixels (two adjacent pixels per lane) and accumulating
// all the group's targets from them.  The re-tilt is the product of a
// per-target factor and two table entries indexed by the lane's window row
// and column; results leave as 4-byte (bf16 pairs) or 16-byte (complex64
// pairs) stores, a warp covering whole 128-byte segments.
#include <cuda_bf16.h>

#include "bip_device.cuh"
#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int kPix = 64;                     // pixels per block, two per lane
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kGroupsPerWarp = 8;            // target groups per warp and block
constexpr int kG = kGatherGroup;

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // .x = a (low half)
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float lo_f(uint32_t packed) { return __uint_as_float(packed << 16); }
__device__ __forceinline__ float hi_f(uint32_t packed) { return __uint_as_float(packed & 0xffff0000u); }

// Magnitude-preserving value A U / |U| (A where U = 0), or U itself.
__device__ __forceinline__ float2 recon_value(float ur, float ui, float am, int magnitude) {
    if (!magnitude) return make_float2(ur, ui);
    const float m2 = ur * ur + ui * ui;
    if (m2 > 0.f) {
        const float sc = am * rsqrtf(m2);
        return make_float2(ur * sc, ui * sc);
    }
    return make_float2(am, 0.f);
}

template <int MAXCH>
__global__ void __launch_bounds__(kThreads, 3) gather_kernel(GatherArgs a) {
    extern __shared__ float4 smraw[];
    const int Bp = a.Bp;
    float4* sv = smraw;                                        // [Bp][32] pixels 2l, 2l+1
    float2* sm = reinterpret_cast<float2*>(sv + Bp * 32);      // [Bp][32] their magnitudes
    float4* hs = reinterpret_cast<float4*>(sm + Bp * 32);      // [MAXCH][32] H_n (MAXCH > 3)
    constexpr int HR = MAXCH <= 3 ? MAXCH : 1;                 // H_n held in registers

    const int bs = blockIdx.z;                 // site within the batch
    const int site = a.site_ids[bs];
    const SiteDev st = a.sites[site];
    const int r0 = blockIdx.x * kPix;
    // the batch's window is the central win x win block of the stashed
    // stash_win x stash_win windows; a lane's two pixels are adjacent in both
    // (win, stash_win and wo even)
    const int SK = a.stash_win * a.stash_win;
    const float2* src = a.stash + (size_t)site * Bp * SK;
    for (int i = threadIdx.x; i < Bp * 32; i += kThreads) {
        const int p = i >> 5, l = i & 31;
        const int rl = r0 + 2 * l, ul = rl / a.win;
        const int idx = (ul + a.wo) * a.stash_win + (rl - ul * a.win) + a.wo;
        const float4 v = __ldg(reinterpret_cast<const float4*>(src + (size_t)p * SK + idx));
        sv[i] = v;
        sm[i] = make_float2(sqrtf(v.x * v.x + v.y * v.y), sqrtf(v.z * v.z + v.w * v.w));
    }
    const int nch = a.nch;
    const int nuse = min(nch, st.nch);         // channels this site has
    const float4* H4 = reinterpret_cast<const float4*>(a.H);
    float4 hr[HR];
    if (MAXCH > 3) {
        for (int i = threadIdx.x; i < MAXCH * 32; i += kThreads) {
            const int n = i >> 5, l = i & 31;
            hs[i] = n < nuse ? __ldg(H4 + ((size_t)st.h_off + (size_t)n * a.K + r0) / 2 + l) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (MAXCH <= 3) {
#pragma unroll
        for (int n = 0; n < HR; ++n)
            hr[n] = n < nuse ? __ldg(H4 + ((size_t)st.h_off + (size_t)n * a.K + r0) / 2 + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int rr = r0 + 2 * lane;              // the lane's first window pixel
    const int u = rr / a.win, v = rr - u * a.win;   // window row, column (v even)
    const int nrep = nch > 0 ? nch : 1;
    const size_t plane = (size_t)(nrep * a.rows_pad) * a.K;
    const int gb = blockIdx.y * (kWarps * kGroupsPerWarp);
    const int ge = min(gb + kWarps * kGroupsPerWarp, a.grp.n_groups);

    const int oy = st.oy + a.wo, ox = st.ox + a.wo;   // origin of the batch's window
    float2 stp0 = __ldg(&a.ex[wrap_n(a.fx * (ox + v), a.nx)]);
    float2 stp1 = __ldg(&a.ex[wrap_n(a.fx * (ox + v + 1), a.nx)]);
    if (a.tilt_sign < 0) {
        stp0.y = -stp0.y;
        stp1.y = -stp1.y;
    }
    for (int gi = gb + warp; gi < ge; gi += kWarps) {
        float ur[kG][2], ui[kG][2], am[kG][2];
#pragma unroll
        for (int t = 0; t < kG; ++t)
#pragma unroll
            for (int j = 0; j < 2; ++j) ur[t][j] = ui[t][j] = am[t][j] = 0.f;
        const int e1 = __ldg(&a.grp.off[gi + 1]);
        for (int e = __ldg(&a.grp.off[gi]); e < e1; ++e) {
            const int p = __ldg(&a.grp.par[e]);
            const float4 w4 = __ldg(&a.grp.w[e]);
            const float4 pv = sv[p * 32 + lane];
            const float2 pm = sm[p * 32 + lane];
            const float w[kG] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int t = 0; t < kG; ++t) {
                ur[t][0] = fmaf(w[t], pv.x, ur[t][0]);
                ui[t][0] = fmaf(w[t], pv.y, ui[t][0]);
                ur[t][1] = fmaf(w[t], pv.z, ur[t][1]);
                ui[t][1] = fmaf(w[t], pv.w, ui[t][1]);
                am[t][0] = fmaf(w[t], pm.x, am[t][0]);
                am[t][1] = fmaf(w[t], pm.y, am[t][1]);
            }
        }
        float2 t0 = make_float2(1.f, 0.f), t1 = t0;
        int2 hp = make_int2(a.ny, 0);          // no previous target
#pragma unroll
        for (int tt = 0; tt < kG; ++tt) {
            const int t = gi * kG + tt;
            if (t < a.n_targets) {
                const int2 h = __ldg(&a.h_t[t]);
                if (h.x == hp.x && h.y == hp.y + a.fx) {
                    t0 = c_mul(t0, stp0);
                    t1 = c_mul(t1, stp1);
                } else {
                    const float2 base = c_mul(__ldg(&a.ey[wrap_n(h.x * oy, a.ny)]),
                                              __ldg(&a.ex[wrap_n(h.y * ox, a.nx)]));
                    const float2 ty = __ldg(&a.ytab[(size_t)(wrap_n(h.x, a.ny)) * a.stash_win + u]);
                    const float4 tx = __ldg(
                        reinterpret_cast<const float4*>(a.xtab + (size_t)(wrap_n(h.y, a.nx)) * a.stash_win + v));
                    const float2 by = c_mul(base, ty);
                    t0 = c_mul(by, make_float2(tx.x, tx.y));
                    t1 = c_mul(by, make_float2(tx.z, tx.w));
                    if (a.tilt_sign < 0) {
                        t0.y = -t0.y;
                        t1.y = -t1.y;
                    }
                }
                hp = h;
                const float2 S0 = c_mul(recon_value(ur[tt][0], ui[tt][0], am[tt][0], a.magnitude), t0);
                const float2 S1 = c_mul(recon_value(ur[tt][1], ui[tt][1], am[tt][1], a.magnitude), t1);
#pragma unroll
                for (int n = 0; n < MAXCH; ++n) {
                    if (n >= nrep) break;
                    float2 o0 = S0, o1 = S1;
                    if (nch > 0) {
                        const float4 hv = MAXCH <= 3 ? hr[n < HR ? n : 0] : hs[n * 32 + lane];
                        o0 = c_mul(make_float2(hv.x, hv.y), S0);
                        o1 = c_mul(make_float2(hv.z, hv.w), S1);
                    }
                    const size_t off = (size_t)bs * a.site_stride + ((size_t)n * a.rows_pad + t) * a.K + rr;
                    if (a.out_c64) {
                        *reinterpret_cast<float4*>(a.out_c64 + off) = make_float4(o0.x, o0.y, o1.x, o1.y);
                    } else if (a.out_planes == 4) {
                        // hi + lo bf16 splits of re and im
                        uint16_t* o = a.out_bf16 + off;
                        const uint32_t rh = pack_bf16x2(o0.x, o1.x), ih = pack_bf16x2(o0.y, o1.y);
                        *reinterpret_cast<uint32_t*>(o) = rh;
                        *reinterpret_cast<uint32_t*>(o + plane) = pack_bf16x2(o0.x - lo_f(rh), o1.x - hi_f(rh));
                        *reinterpret_cast<uint32_t*>(o + 2 * plane) = ih;
                        *reinterpret_cast<uint32_t*>(o + 3 * plane) = pack_bf16x2(o0.y - lo_f(ih), o1.y - hi_f(ih));
                    } else {
                        uint16_t* o = a.out_bf16 + off;
                        *reinterpret_cast<uint32_t*>(o) = pack_bf16x2(o0.x, o1.x);
                        *reinterpret_cast<uint32_t*>(o + plane) = pack_bf16x2(o0.y, o1.y);
                    }
                }
            }
        }
    }
}

template <int MAXCH>
cudaError_t launch(const GatherArgs& a, cudaStream_t s) {
    const int gpb = kWarps * kGroupsPerWarp;
    dim3 grid(a.K / kPix, (a.grp.n_groups + gpb - 1) / gpb, a.n_sites);
    const size_t sm = (size_t)a.Bp * 32 * (sizeof(float4) + sizeof(float2)) +
                      (MAXCH > 3 ? (size_t)MAXCH * 32 * sizeof(float4) : 0);
    static std::atomic<size_t> attr{0};
    if (sm > 48 * 1024) {
        const cudaError_t e = bip_raise_once(attr, sm, [&] {
            return cudaFuncSetAttribute(gather_kernel<MAXCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        });
        if (e != cudaSuccess) return e;
    }
    gather_kernel<MAXCH><<<grid, kThreads, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t bip_gather(const GatherArgs& a, cudaStream_t s) {
    if (a.K % kPix != 0 || a.win % 2 != 0 || a.nch > 9 || a.n_targets > a.grp.n_groups * kG) return cudaErrorInvalidValue;
    if (a.K != a.win * a.win || a.stash_win % 2 || a.wo % 2 || a.wo < 0 || a.win + 2 * a.wo != a.stash_win)
        return cudaErrorInvalidValue;
    if (a.nch > 0 && (reinterpret_cast<uintptr_t>(a.H) & 15) != 0) return cudaErrorMisalignedAddress;
    if (a.n_sites == 0 || a.grp.n_groups == 0) return cudaSuccess;
    // channel count: 1 stands for the S2 side (no channel product)
    switch (a.nch <= 1 ? 1 : (a.nch <= 3 ? 3 : 9)) {
        case 1: return launch<1>(a, s);
        case 3: return launch<3>(a, s);
        default: return launch<9>(a, s);
    }
}
