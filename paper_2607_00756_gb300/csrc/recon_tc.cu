// Window reconstruction on the tensor cores (mixed path): Eq. window-recon
// with Eq. magpreserve, the re-tilt and diag(H_n), written as the BF16
// operands of the coupling contraction.
//
// For the targets t of one side (detector beams for S2, aperture beams for
// S1) and the window pixels r of one site, the three sums
//   U_re(t, r) = sum_p w_tp Re S_p(r),  U_im(t, r) = sum_p w_tp Im S_p(r),
//   A(t, r)    = sum_p w_tp |S_p(r)|
// are one product W X with W [targets x 64 parents] and X [64 parents x
// pixels] per plane (re, im, magnitude), K = the parents (zero-padded to 64).
// The products are FP16 (kind::f16 with FP16 operands): W exact to FP32 as
// hi + lo FP16 (two products per plane), X rounded once to FP16 (relative
// 2^-11; the parent windows are O(1) plane-wave sums, far inside its range).
//
//   xprep_kernel    stash [Bp][K] complex64 -> X [3 planes][K px][64] fp16
//                   (transposed so the parents are contiguous: K-major B)
//   recon_tc_kernel persistent, one CTA per SM, 576 threads:
//     warp 0     TMA producer: the unit's W tile (128 targets x 64 parents,
//                hi and lo) once, then X tiles (64 pixels x 64 parents, three
//                planes) through a 4-stage ring
//     warp 1     TMEM allocator and MMA issuer: per 64-pixel tile, 8 MMAs
//                (M=128, N=192: the three planes side by side, K=16) into
//                three accumulators, two TMEM buffers so the epilogue of one
//                tile overlaps the next
//     warps 2-17 epilogue: thread = target row (TMEM lane), 16 pixels per
//                warp and tile; magnitude preservation, re-tilt stepped
//                along the window row in four independent chains, H_n
//                (staged per tile in shared memory) products, 16 bf16
//                stored per thread as one 32-byte sector -- or, for the FP8
//                coupling, 16 E4M3 bytes, the row scale folded into the
//                magnitude factor (H_n comes pre-divided by its maximum);
//                a side may instead be written transposed (pixels x targets,
//                no H_n), the probe order's operand
// Work unit: (side, site in batch, 128-target tile, chunk of up to 1024
// pixels).  Every wait is bounded; on a timeout the kernel sets *err, stops,
// drains the copies and MMAs it issued and frees TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bip_device.cuh"
#include "fft_smem.cuh"
#include "tc_common.cuh"

namespace {

constexpr int kEpiWarps = 16;                    // 4 per TMEM lane quadrant
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kN = 64;                           // pixels per MMA tile
constexpr int kChunk = 1024;                     // pixels per work unit (at most)
constexpr int kStages = 4;
constexpr int kAPlane = 128 * 64;                // bytes: 128 rows x 32 bf16 (one K block)
constexpr int kABuf = 2 * 2 * kAPlane;           // hi, lo x two K blocks
constexpr int kBPlane = kN * 64;                 // bytes: 64 rows x 32 bf16
constexpr int kBStage = 3 * 2 * kBPlane;         // re, im, mag x two K blocks
constexpr int kAccCols = 3 * kN;                 // TMEM columns per accumulator set
constexpr int kHBuf = 9 * 16 * 8;                // H_n of one warp's 16 pixels, up to 9 channels
constexpr size_t kSmem = 1024 + 2 * (size_t)kABuf + (size_t)kStages * kBStage + (size_t)kEpiWarps * kHBuf + 256;

struct Unit {
    int side, bs, mt, pc;
};

__device__ __forceinline__ bool unit_of(const ReconArgs& a, int idx, Unit& u) {
    int per0 = a.n_sites * a.side[0].mt_tiles * a.chunks;
    int per1 = a.n_sites * a.side[1].mt_tiles * a.chunks;
    if (idx >= per0 + per1) return false;
    u.side = idx < per0 ? 0 : 1;
    if (u.side) idx -= per0;
    const int per_site = a.side[u.side].mt_tiles * a.chunks;
    u.bs = idx / per_site;
    const int r = idx % per_site;
    u.mt = r / a.chunks;
    u.pc = r % a.chunks;
    return true;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// four E4M3 bytes (satfinite, nearest-even), a in the lowest byte
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ void st_v4(void* p, const uint32_t (&v)[4]) {
    asm volatile("st.global.v4.b32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                 : "memory");
}

// the hardware reciprocal square root (relative error near 2^-23; the
// operands leave in BF16 or E4M3)
__device__ __forceinline__ float rsqrt_hw(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Magnitude step with no branch: U = 0 must give the real A (the phase of a
// vanishing sum is taken as 0).  Adding 2^-60 to Re U before |U| does that
// (then U = (2^-60, 0), whose phase is 0, and |U|^2 = 2^-120 is still a
// normal FP32 number) and moves the phase of any other U by at most
// 2^-60 / |U|, far below the rounding of the parents' FP16 values.
constexpr float kPhaseGuard = 8.67361737988403547e-19f;   // 2^-60
constexpr float kTinyNormal = 1.17549435e-38f;             // 2^-126

// F8: the operands are written as E4M3 bytes, row t scaled by
// inv_row[side][t] and channel n by inv_h[n] (per-window scales)
template <bool F8>
__global__ void __launch_bounds__(kThreads, 1)
    recon_tc_kernel(const __grid_constant__ CUtensorMap mapW, const __grid_constant__ CUtensorMap mapX,
                    const ReconArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* abuf = smem;                                   // [2][kABuf]
    uint8_t* bbuf = smem + 2 * kABuf;                       // [kStages][kBStage]
    float2* hsm = (float2*)(bbuf + kStages * kBStage);     // [kEpiWarps][9][16] H_n per warp
    uint64_t* full = (uint64_t*)((uint8_t*)hsm + kEpiWarps * kHBuf);
    uint64_t* empty = full + kStages;
    uint64_t* a_full = empty + kStages;
    uint64_t* a_empty = a_full + 2;
    uint64_t* acc_full = a_empty + 2;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], 1);
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kEpiWarps);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const int tiles = a.chunk_px / kN;                      // MMA tiles per unit

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.err, 1);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;                    // X stages issued
            int a_last[2] = {-1, -1};          // last unit whose W went to each buffer
            bool ok = true;
            Unit u;
            for (int i = 0; ok && unit_of(a, blockIdx.x + i * gridDim.x, u); ++i) {
                const ReconSide& sd = a.side[u.side];
                const int ab = i & 1;
                if (!mbar_wait(&a_empty[ab], ((i >> 1) & 1) ^ 1, abort_flag, wait_limit(a.wait_ns))) {
                    fail();
                    ok = false;
                    break;
                }
                uint8_t* at = abuf + ab * kABuf;
                mbar_expect_tx(&a_full[ab], kABuf);
#pragma unroll
                for (int pl = 0; pl < 2; ++pl)
#pragma unroll
                    for (int kb = 0; kb < 2; ++kb)
                        tma_2d(at + (pl * 2 + kb) * kAPlane, &mapW, kb * 32,
                               sd.w_row0 + pl * sd.w_pad + u.mt * 128, &a_full[ab]);
                a_last[ab] = i;
                const int xrow0 = (sd.x_site0 + u.bs * 3) * a.K + u.pc * a.chunk_px;
                for (int t = 0; t < tiles; ++t) {
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, wait_limit(a.wait_ns))) {
                        fail();
                        ok = false;
                        break;
                    }
                    uint8_t* st = bbuf + s * kBStage;
                    mbar_expect_tx(&full[s], kBStage);
                    // per K block, the three planes' 64-row tiles back to back:
                    // one 192-row B operand
#pragma unroll
                    for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                        for (int pl = 0; pl < 3; ++pl)
                            tma_2d(st + (kb * 3 + pl) * kBPlane, &mapX, kb * 32, xrow0 + pl * a.K + t * kN, &full[s]);
                    ++issued;
                    if (++s == kStages) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            if (!ok) {
                // let the copies in flight land before the CTA exits
                const uint64_t t0 = gtimer();
                for (int k = 0; k < kStages && k < issued; ++k) {
                    s = (s + kStages - 1) % kStages;
                    if (s == kStages - 1) ph ^= 1;
                    while (!mbar_try(&full[s], ph) && gtimer() - t0 < kTimeoutNs) {
                    }
                }
                for (int ab = 0; ab < 2; ++ab)
                    if (a_last[ab] >= 0)
                        while (!mbar_try(&a_full[ab], (a_last[ab] >> 1) & 1) && gtimer() - t0 < kTimeoutNs) {
                        }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            const uint32_t id = idesc_f16(128, 3 * kN, false);   // re, im, magnitude side by side
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool any = false, ok = true;
            Unit u;
            for (int i = 0; ok && unit_of(a, blockIdx.x + i * gridDim.x, u); ++i) {
                const int ab = i & 1;
                if (!mbar_wait(&a_full[ab], (i >> 1) & 1, abort_flag, wait_limit(a.wait_ns))) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t abase = smem_u32(abuf + ab * kABuf);
                for (int t = 0; t < tiles; ++t) {
                    if (!mbar_wait(&acc_empty[acc], aph ^ 1, abort_flag, wait_limit(a.wait_ns)) || !mbar_wait(&full[s], ph, abort_flag, wait_limit(a.wait_ns))) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t bbase = smem_u32(bbuf + s * kBStage);
                    const uint32_t d0 = tbase + (uint32_t)(acc * kAccCols);
#pragma unroll
                    for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t whi = sdesc(abase + (0 * 2 + kb) * kAPlane + kk * 32);
                            const uint64_t wlo = sdesc(abase + (1 * 2 + kb) * kAPlane + kk * 32);
                            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
                            const uint64_t xd = sdesc(bbase + kb * 3 * kBPlane + kk * 32);
                            mma(d0, whi, xd, id, first);
                            mma(d0, wlo, xd, id, 1);
                        }
                    any = true;
                    mma_commit(&empty[s]);
                    mma_commit(&acc_full[acc]);
                    if (++s == kStages) {
                        s = 0;
                        ph ^= 1;
                    }
                    if (++acc == 2) {
                        acc = 0;
                        aph ^= 1;
                    }
                }
                mma_commit(&a_empty[ab]);
            }
            if (any) {
                mma_commit(drain);
                const uint64_t t0 = gtimer();
                while (!mbar_try(drain, 0) && gtimer() - t0 < kTimeoutNs) {
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2 .. 2 + kEpiWarps - 1; TMEM lane
        // quadrant warp % 4, 16-pixel quarter (warp - 2) / 4 of each tile.
        // Warps run independently: each waits on the accumulator barrier
        // itself and stages its own H_n.
        const int q = warp & 3;
        const int quarter = (warp - 2) >> 2;
        const int c0 = quarter * 16;                          // first column of this warp
        float2* hw = hsm + (warp - 2) * 9 * 16;               // this warp's H_n [9][16]
        int acc = 0;
        uint32_t aph = 0;
        Unit u;
        bool ok = true;
        for (int i = 0; ok && unit_of(a, blockIdx.x + i * gridDim.x, u); ++i) {
            const ReconSide& sd = a.side[u.side];
            const int t = u.mt * 128 + q * 32 + lane;       // target of this thread
            const bool valid = t < sd.n_targets;
            const int site = a.site_ids[u.bs];
            const SiteDev st = a.sites[site];
            const int nrep = sd.nch > 0 ? sd.nch : 1;
            const int nuse = min(sd.nch, st.nch);
            // re-tilt exp(sign 2 pi i (h_y (oy + u)/ny + h_x (ox + v)/nx)) at the
            // first pixel of this warp's columns, carried from tile to tile:
            // +64 pixels is X^64 and, per window-row wrap, Z = Y X^-win, with
            // X = exp(sign 2 pi i h_x/nx), Y = exp(sign 2 pi i h_y/ny)
            float2 F = make_float2(1.f, 0.f), sx1 = F, sx4 = F, sx8 = F, X64 = F, Z = F;
            int wv = 0;
            if (valid) {
                const int2 h = __ldg(&sd.h_t[t]);
                const int px0 = u.pc * a.chunk_px + c0;
                const int wu = px0 / a.win;
                wv = px0 - wu * a.win;
                // origin of the batch's window: wo pixels into the stashed one
                const float2 base = c_mul(__ldg(&a.ey[wrap_n(h.x * (st.oy + a.wo), a.ny)]),
                                          __ldg(&a.ex[wrap_n(h.y * (st.ox + a.wo), a.nx)]));
                F = c_mul(base, c_mul(__ldg(&a.ytab[(size_t)(wrap_n(h.x, a.ny)) * a.stash_win + wu]),
                                      __ldg(&a.xtab[(size_t)(wrap_n(h.y, a.nx)) * a.stash_win + wv])));
                sx1 = __ldg(&a.ex[wrap_n(h.y, a.nx)]);
                sx4 = __ldg(&a.ex[wrap_n(4 * h.y, a.nx)]);
                sx8 = __ldg(&a.ex[wrap_n(8 * h.y, a.nx)]);
                X64 = __ldg(&a.ex[wrap_n(64 * h.y, a.nx)]);
                Z = c_mul(__ldg(&a.ey[wrap_n(h.x, a.ny)]), __ldg(&a.ex[wrap_n(-a.win * h.y, a.nx)]));
                if (sd.tilt_sign < 0) {
                    F.y = -F.y;
                    sx1.y = -sx1.y;
                    sx4.y = -sx4.y;
                    sx8.y = -sx8.y;
                    X64.y = -X64.y;
                    Z.y = -Z.y;
                }
            }
            // output element offset of this row (bf16 or E4M3 elements)
            const size_t out_off = (size_t)u.bs * sd.site_stride + (size_t)t * a.K;
            float ir = 1.f;                                    // F8: 448 / bound of this row
            if (F8 && valid) ir = __ldg(&a.inv_row[u.side][(size_t)u.bs * sd.rows_pad + t]);
            const size_t ch_stride = (size_t)sd.rows_pad * a.K;
            const float2* Hs = a.H + (size_t)st.h_off;
            const int nh = sd.nch * 16;                       // H_n values of a warp per tile
            for (int tt = 0; tt < tiles; ++tt) {
                const int px = u.pc * a.chunk_px + tt * kN + c0;     // this warp's 16 pixels
                // this tile's H_n, in flight during the waits below
                float2 hv[5];
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    const int k = lane + 32 * r;
                    hv[r] = make_float2(0.f, 0.f);
                    if (k < nh && k / 16 < nuse) hv[r] = __ldg(&Hs[(size_t)(k / 16) * a.K + px + (k % 16)]);
                }
                int okw = 1;
                if (lane == 0) {
                    okw = mbar_wait(&acc_full[acc], aph, abort_flag, wait_limit(a.wait_ns)) ? 1 : 0;
                    if (!okw) fail();
                }
                okw = __shfl_sync(0xffffffffu, okw, 0);
                if (!okw) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kAccCols);
                float vr[16], vi[16], vm[16];
                tmem_ld16(tr + c0, vr);
                tmem_ld16(tr + kN + c0, vi);
                tmem_ld16(tr + 2 * kN + c0, vm);
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    const int k = lane + 32 * r;
                    if (k < nh) hw[k] = hv[r];
                }
                tmem_ld_wait();
                // the accumulator buffer is free for the next MMA once read
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[acc]);
                if (++acc == 2) {
                    acc = 0;
                    aph ^= 1;
                }
                if (valid) {
                    // re-tilt in four independent chains (pixels j, j + 4, j + 8, j + 12)
                    float2 tc[4];
                    tc[0] = F;
                    tc[1] = c_mul(F, sx4);
                    tc[2] = c_mul(F, sx8);
                    tc[3] = c_mul(tc[1], sx8);
                    float2 S[16];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int k = 4 * c + j;
                            float2 v;
                            if (a.magnitude) {
                                const float ur = vr[k] + kPhaseGuard;
                                const float m2 = fmaf(ur, ur, vi[k] * vi[k]);
                                const float mk = F8 ? vm[k] * ir : vm[k];
                                const float sc = mk * rsqrt_hw(fmaxf(m2, kTinyNormal));
                                v = make_float2(ur * sc, vi[k] * sc);
                            } else {
                                v = F8 ? make_float2(vr[k] * ir, vi[k] * ir) : make_float2(vr[k], vi[k]);
                            }
                            S[k] = c_mul(v, tc[c]);
                            tc[c] = c_mul(tc[c], sx1);
                        }
                    }
                    if constexpr (F8) {
                        uint8_t* o = (uint8_t*)a.out[u.side] + out_off + px;
                        for (int n = 0; n < nrep; ++n) {
                            uint32_t re[4], im[4];
                            if (sd.nch > 0) {
                                const float4* hp = reinterpret_cast<const float4*>(hw + n * 16);
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const float4 h0 = hp[2 * j], h1 = hp[2 * j + 1];
                                    const float2 e0 = c_mul(make_float2(h0.x, h0.y), S[4 * j]);
                                    const float2 e1 = c_mul(make_float2(h0.z, h0.w), S[4 * j + 1]);
                                    const float2 e2 = c_mul(make_float2(h1.x, h1.y), S[4 * j + 2]);
                                    const float2 e3 = c_mul(make_float2(h1.z, h1.w), S[4 * j + 3]);
                                    re[j] = pack_e4m3x4(e0.x, e1.x, e2.x, e3.x);
                                    im[j] = pack_e4m3x4(e0.y, e1.y, e2.y, e3.y);
                                }
                            } else {
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    re[j] = pack_e4m3x4(S[4 * j].x, S[4 * j + 1].x, S[4 * j + 2].x, S[4 * j + 3].x);
                                    im[j] = pack_e4m3x4(S[4 * j].y, S[4 * j + 1].y, S[4 * j + 2].y, S[4 * j + 3].y);
                                }
                            }
                            st_v4(o, re);
                            st_v4(o + sd.plane_stride, im);
                            o += ch_stride;
                        }
                    } else if (sd.trans) {
                        // targets contiguous: element (t, px + j) at (px + j) ld + t,
                        // so each store of the warp's 32 targets is one 64-byte run
                        uint16_t* o = a.out[u.side] + (size_t)u.bs * sd.site_stride + (size_t)px * sd.ld + t;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const uint32_t v = pack2(S[j].x, S[j].y);
                            o[(size_t)j * sd.ld] = (uint16_t)(v & 0xffffu);
                            o[sd.plane_stride + (size_t)j * sd.ld] = (uint16_t)(v >> 16);
                        }
                    } else {
                        uint16_t* o = a.out[u.side] + out_off + px;
                        for (int n = 0; n < nrep; ++n) {
                            uint32_t re[8], im[8];
                            if (sd.nch > 0) {
                                const float4* hp = reinterpret_cast<const float4*>(hw + n * 16);
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const float4 hq = hp[j];
                                    const float2 o0 = c_mul(make_float2(hq.x, hq.y), S[2 * j]);
                                    const float2 o1 = c_mul(make_float2(hq.z, hq.w), S[2 * j + 1]);
                                    re[j] = pack2(o0.x, o1.x);
                                    im[j] = pack2(o0.y, o1.y);
                                }
                            } else {
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    re[j] = pack2(S[2 * j].x, S[2 * j + 1].x);
                                    im[j] = pack2(S[2 * j].y, S[2 * j + 1].y);
                                }
                            }
                            st_v8(o, re);
                            st_v8(o + sd.plane_stride, im);
                            o += ch_stride;
                        }
                    }
                    // tilt at this warp's first pixel of the next tile
                    F = c_mul(F, X64);
                    wv += kN;
                    while (wv >= a.win) {
                        wv -= a.win;
                        F = c_mul(F, Z);
                    }
                }
                __syncwarp();                                  // hw reads done before the next tile's writes
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols));
    }
}

// stash [Bp][stash_win^2] complex64 of one site -> X planes [3][K][64] fp16
// (re, im, magnitude; parents past Bp zero) of the batch's w x w window, the
// central block at offset wo of the stashed one.  Block: 64 pixels of one
// site and side.
constexpr int kPrepThreads = 256;
__global__ void __launch_bounds__(kPrepThreads) xprep_kernel(XprepArgs a) {
    __shared__ float2 s[64][65];
    const int side = blockIdx.z;
    const XprepSide& sd = a.side[side];
    const int bs = blockIdx.y;
    const int site = a.site_ids[bs];
    const int px0 = blockIdx.x * 64;
    const int SK = a.stash_win * a.stash_win;
    const float2* src = sd.stash + (size_t)site * sd.Bp * SK;
    // stash index of this thread's pixel px0 + (threadIdx.x & 63) (the same
    // for its 16 loads: i & 63 does not change with r)
    const int pix = px0 + (threadIdx.x & 63), pu = pix / a.w;
    const int sidx = (pu + a.wo) * a.stash_win + (pix - pu * a.w) + a.wo;
    // (FP8 path: the parents' window maxima are taken from the same tile)
    // 16 loads per thread in flight at once (parents p = i / 64, pixels i % 64)
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int i = threadIdx.x + r * kPrepThreads, p = i >> 6;
        v[r] = p < sd.Bp ? __ldg(&src[(size_t)p * SK + sidx]) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int i = threadIdx.x + r * kPrepThreads;
        s[i >> 6][i & 63] = v[r];
    }
    __syncthreads();
    if (a.pmax) {
        // four threads per parent, 16 pixels each
        const int p = threadIdx.x >> 2, x0 = (threadIdx.x & 3) * 16;
        float m = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float2 e = s[p][x0 + j];
            m = fmaxf(m, sqrtf(e.x * e.x + e.y * e.y));
        }
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
        // non-negative floats order like their bit patterns
        if ((threadIdx.x & 3) == 0 && p < sd.Bp && m > 0.f)
            atomicMax(&a.pmax[((size_t)side * a.n_sites + bs) * 64 + p], __float_as_uint(m));
    }
    // thread: one pixel (lane) and eight consecutive parents, for one plane
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;   // 8 warps
    uint16_t* dst = a.X + ((size_t)(sd.x_site0 + bs * 3) * a.K + px0) * 64;
    for (int job = w; job < 2 * 3 * 8; job += 8) {
        const int xh = job / 24, r = job % 24, pl = r / 8, p0 = (r % 8) * 8;
        const int x = xh * 32 + lane;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 e0 = s[p0 + 2 * k][x], e1 = s[p0 + 2 * k + 1][x];
            float f0, f1;
            if (pl == 0) {
                f0 = e0.x; f1 = e1.x;
            } else if (pl == 1) {
                f0 = e0.y; f1 = e1.y;
            } else {
                f0 = sqrtf(e0.x * e0.x + e0.y * e0.y);
                f1 = sqrtf(e1.x * e1.x + e1.y * e1.y);
            }
            const __half2 hv = __floats2half2_rn(f0, f1);
            v[k] = *reinterpret_cast<const uint32_t*>(&hv);
        }
        *reinterpret_cast<uint4*>(dst + ((size_t)pl * a.K + x) * 64 + p0) = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

}  // namespace

cudaError_t bip_xprep(const XprepArgs& a, cudaStream_t s) {
    if (a.K % 64 || a.n_sites < 1) return cudaErrorInvalidValue;
    if (a.side[0].Bp > 64 || a.side[1].Bp > 64) return cudaErrorInvalidValue;
    if (a.K != a.w * a.w || a.wo < 0 || a.w + 2 * a.wo != a.stash_win) return cudaErrorInvalidValue;
    xprep_kernel<<<dim3(a.K / 64, a.n_sites, 2), kPrepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t bip_recon_tc(const ReconArgs& a, cudaStream_t s) {
    if (a.K % kN || a.chunk_px % kN || a.K % a.chunk_px || a.chunk_px > kChunk || a.win % 16) return cudaErrorInvalidValue;
    if (a.K != a.win * a.win || a.wo < 0 || a.win + 2 * a.wo != a.stash_win) return cudaErrorInvalidValue;
    if (a.n_sites < 1 || a.chunks != a.K / a.chunk_px) return cudaErrorInvalidValue;
    for (int i = 0; i < 2; ++i) {
        const ReconSide& sd = a.side[i];
        if (sd.mt_tiles * 128 != sd.w_pad || sd.n_targets > sd.rows_pad || sd.n_targets > sd.w_pad || sd.nch > 9)
            return cudaErrorInvalidValue;
        if (sd.nch > 0 && ((uintptr_t)a.H & 15)) return cudaErrorMisalignedAddress;
        if (sd.trans && (sd.nch != 0 || a.f8 || sd.ld < sd.n_targets || sd.plane_stride < (int64_t)a.K * sd.ld ||
                         sd.site_stride < 2 * sd.plane_stride))
            return cudaErrorInvalidValue;
        if (sd.w_row0 + 2 * sd.w_pad > a.w_rows) return cudaErrorInvalidValue;
        if ((int64_t)(sd.x_site0 + 3 * a.n_sites) * a.K > a.x_rows) return cudaErrorInvalidValue;
    }
    CUtensorMap mw, mx;
    cudaError_t e = make_map_2d(&mw, a.W, a.w_rows, 64, 128);
    if (e != cudaSuccess) return e;
    e = make_map_2d(&mx, a.Xb, a.x_rows, 64, kN);
    if (e != cudaSuccess) return e;
    if (a.f8 && (!a.inv_row[0] || !a.inv_row[1])) return cudaErrorInvalidValue;
    static std::atomic<bool> attr[2];
    e = bip_set_once(attr[a.f8 ? 1 : 0], [&] {
        return a.f8 ? cudaFuncSetAttribute(recon_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kSmem)
                    : cudaFuncSetAttribute(recon_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kSmem);
    });
    if (e != cudaSuccess) return e;
    const int units = a.n_sites * (a.side[0].mt_tiles + a.side[1].mt_tiles) * a.chunks;
    const int grid = units < num_sms() ? units : num_sms();
    if (a.f8)
        recon_tc_kernel<true><<<grid, kThreads, kSmem, s>>>(mw, mx, a);
    else
        recon_tc_kernel<false><<<grid, kThreads, kSmem, s>>>(mw, mx, a);
    return cudaGetLastError();
}
