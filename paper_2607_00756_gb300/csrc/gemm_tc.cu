// Complex contractions on the 5th-generation tensor cores (tcgen05.mma,
// TMEM accumulators, TMA operand staging), in split BF16, BF16 or E4M3.
//
// Split BF16: every complex FP32 operand is stored as four BF16 planes,
// x = hi + lo with hi = bf16(x), lo = bf16(x - hi), for the real and the
// imaginary part.  A real product A B is taken as A_hi B_hi + A_hi B_lo +
// A_lo B_hi (the lo*lo term is below FP32 rounding), accumulated in FP32 in
// TMEM, and the complex product as
//   Re += Ar Br -/+ Ai Bi,   Im += Ar Bi +/- Ai Br     (-/+: op(A) = A / conj A)
// -- twelve MMAs per K step into two accumulators, the signs carried by the
// instruction descriptor's negate-A bit.  BF16: two planes (re, im), one
// product per real product, four MMAs per K step.  E4M3 (kind::f8f6f4):
// as BF16 with 64 values per 64-byte row, each operand row carrying one
// scale (its 64x64 window) that the epilogue applies to the FP32 sums.
//
// Kernel: persistent, one CTA per SM, 192 threads:
//   warp 0      TMA producer (one elected thread): 4 A planes + 4 B planes
//               per 32-wide K block into a 64B-swizzled shared stage;
//   warp 1      TMEM allocator and MMA issuer (one elected thread);
//   warps 2-5   epilogue: tcgen05.ld of the accumulators, then
//     MT   : coupling M written transposed as bf16 planes for the Gram step
//     C32  : complex64 row-major copy (the Gram matrix for the scan
//            contraction, or the coupling for validation).
// Every wait is bounded (a few seconds of %globaltimer); on a timeout the
// kernel sets *err, stops issuing work, drains what it issued and frees
// TMEM before returning.
#include "tc_common.cuh"

namespace {

constexpr int kThreads = 192;
constexpr int kATile = 128 * 64;                 // one plane: 128 rows x 32 bf16

// Work units: (site in batch, M tile, N tile).
struct Unit {
    int bs, mt, nt, w;
    bool skip;    // tile below the diagonal of a Hermitian Gram matrix
    int kb0;      // first K block
    int nc;       // columns of this tile: N, or fewer for the last one
};

template <int EPI>
struct UnitIter {
    const TcArgs& p;
    int total;
    __device__ int N_of() const { return p.N; }
    __device__ UnitIter(const TcArgs& a) : p(a) { total = a.n_sites * a.mt_per * a.nt_per; }
    // the i-th unit of this CTA (i = 0, 1, ...), false past the end
    __device__ bool get(int i, Unit& u) const {
        const int idx = blockIdx.x + i * gridDim.x;
        if (idx >= total) return false;
        const int per = p.mt_per * p.nt_per;
        u.bs = idx / per;
        const int r = idx % per;
        u.mt = r / p.nt_per;
        u.nt = r % p.nt_per;
        u.w = 0;
        u.skip = p.tri && (u.nt + 1) * N_of() <= u.mt * 128;
        u.kb0 = 0;
        const int left = p.n_cols - u.nt * N_of();
        u.nc = left < N_of() ? left : N_of();
        return true;
    }
};

template <int N, int NPL>
struct TcShape {
    static constexpr int B_TILE = N * 64;
    static constexpr int STAGE = NPL * kATile + NPL * B_TILE;
    static constexpr int STAGES = (196608 / STAGE) > 6 ? 6 : (196608 / STAGE);
    static constexpr int NACC = N == 256 ? 1 : 2;
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256;
};

template <int N, int EPI, int NPL, bool F8>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapBt, const TcArgs p) {
    using Sh = TcShape<N, NPL>;
    constexpr int STAGES = Sh::STAGES;
    constexpr int NACC = Sh::NACC;
    constexpr int B_TILE = Sh::B_TILE;
    constexpr int STAGE = Sh::STAGE;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;
    uint64_t* acc_empty = acc_full + NACC;
    uint64_t* drain = acc_empty + NACC;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* ep_ok = abort_flag + 1;                    // epilogue's shared wait result

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 4);
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
    const UnitIter<EPI> it(p);

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(p.err, 1);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            Unit u;
            bool ok = true;
            for (int i = 0; ok && it.get(i, u); ++i) {
                if (u.skip) continue;
                const int64_t a0 = (int64_t)u.bs * p.A.site_rows + (int64_t)u.mt * 128;
                const int64_t b0 = (int64_t)u.bs * p.B.site_rows + (int64_t)u.nt * p.N;
                for (int kb = u.kb0; kb < p.kb; ++kb) {
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, wait_limit(p.wait_ns))) {
                        fail();
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + s * STAGE;
                    // a narrower last tile loads only its rows (its own map)
                    const CUtensorMap* mb = u.nc == p.N ? &mapB : &mapBt;
                    mbar_expect_tx(&full[s], NPL * kATile + NPL * u.nc * 64);
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl)
                        tma_2d(st + pl * kATile, &mapA, kb * 32, (int)(a0 + pl * p.A.plane_rows), &full[s]);
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl)
                        tma_2d(st + NPL * kATile + pl * B_TILE, mb, kb * 32, (int)(b0 + pl * p.B.plane_rows),
                               &full[s]);
                    ++issued;
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            if (!ok) {
                // let the copies already issued land before the CTA exits
                for (int k = 0; k < STAGES && k < issued; ++k) {
                    s = (s + STAGES - 1) % STAGES;
                    if (s == STAGES - 1) ph ^= 1;
                    const uint64_t t0 = gtimer();
                    while (!mbar_try(&full[s], ph) && gtimer() - t0 < kTimeoutNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            uint32_t id_pos = 0, id_neg = 0;
            int s = 0, a = 0;
            uint32_t ph = 0, aph = 0;
            bool any = false, ok = true;
            Unit u;
            for (int i = 0; ok && it.get(i, u); ++i) {
                if (u.skip) continue;
                if (!mbar_wait(&acc_empty[a], aph ^ 1, abort_flag, wait_limit(p.wait_ns))) {
                    fail();
                    break;
                }
                tc_fence_after();
                id_pos = F8 ? idesc_e4m3(128, u.nc, false) : idesc(128, u.nc, false);
                id_neg = F8 ? idesc_e4m3(128, u.nc, true) : idesc(128, u.nc, true);
                const uint32_t id_ii = p.conjA ? id_pos : id_neg;   // sign of Ai*Bi in Re
                const uint32_t id_ir = p.conjA ? id_neg : id_pos;   // sign of Ai*Br in Im
                const uint32_t dr = tbase + (uint32_t)(a * 2 * N), di = dr + N;
                for (int kb = u.kb0; kb < p.kb; ++kb) {
                    if (!mbar_wait(&full[s], ph, abort_flag, wait_limit(p.wait_ns))) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + s * STAGE);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        uint64_t ad[NPL], bd[NPL];
#pragma unroll
                        for (int pl = 0; pl < NPL; ++pl) {
                            ad[pl] = sdesc(base + pl * kATile + kk * 32);
                            bd[pl] = sdesc(base + NPL * kATile + pl * B_TILE + kk * 32);
                        }
                        const uint32_t first = (kb == u.kb0 && kk == 0) ? 0u : 1u;
                        if (NPL == 4) {
                            // planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo
                            // Re: Ar Br (+), Ai Bi (-, or + for conj A)
                            mma(dr, ad[0], bd[0], id_pos, first);
                            mma(dr, ad[0], bd[1], id_pos, 1);
                            mma(dr, ad[1], bd[0], id_pos, 1);
                            mma(dr, ad[2], bd[2], id_ii, 1);
                            mma(dr, ad[2], bd[3], id_ii, 1);
                            mma(dr, ad[3], bd[2], id_ii, 1);
                            // Im: Ar Bi (+), Ai Br (+, or - for conj A)
                            mma(di, ad[0], bd[2], id_pos, first);
                            mma(di, ad[0], bd[3], id_pos, 1);
                            mma(di, ad[1], bd[2], id_pos, 1);
                            mma(di, ad[2], bd[0], id_ir, 1);
                            mma(di, ad[2], bd[1], id_ir, 1);
                            mma(di, ad[3], bd[0], id_ir, 1);
                        } else if (F8) {
                            // planes: 0 re, 1 im; K = 32 E4M3 per MMA
                            mma_f8(dr, ad[0], bd[0], id_pos, first);
                            mma_f8(dr, ad[NPL - 1], bd[NPL - 1], id_ii, 1);
                            mma_f8(di, ad[0], bd[NPL - 1], id_pos, first);
                            mma_f8(di, ad[NPL - 1], bd[0], id_ir, 1);
                        } else {
                            // planes: 0 re, 1 im
                            mma(dr, ad[0], bd[0], id_pos, first);
                            mma(dr, ad[NPL - 1], bd[NPL - 1], id_ii, 1);
                            mma(di, ad[0], bd[NPL - 1], id_pos, first);
                            mma(di, ad[NPL - 1], bd[0], id_ir, 1);
                        }
                    }
                    any = true;
                    mma_commit(&empty[s]);
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(&acc_full[a]);
                if (++a == NACC) {
                    a = 0;
                    aph ^= 1;
                }
            }
            if (any) {
                // every MMA issued has finished before TMEM is released
                mma_commit(drain);
                const uint64_t t0 = gtimer();
                while (!mbar_try(drain, 0) && gtimer() - t0 < kTimeoutNs) {
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lane quadrant = warp % 4
        const int q = warp & 3;
        const int et = threadIdx.x - 64;            // 0..127 over the epilogue warps
        int a = 0;
        uint32_t aph = 0;
        Unit u;
        for (int i = 0; it.get(i, u); ++i) {
            if (u.skip) continue;
            // one thread waits; all 128 take the same branch, so no warp can
            // be left alone at a named barrier
            if (et == 0) {
                const bool ok = mbar_wait(&acc_full[a], aph, abort_flag, wait_limit(p.wait_ns));
                *ep_ok = ok ? 1 : 0;
                if (!ok) fail();
            }
            named_sync(1, 128);
            if (!*ep_ok) break;
            tc_fence_after();
            const int row = u.mt * 128 + q * 32 + lane;      // accumulator row of this thread
            const uint32_t tr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 2 * N);
            float sa = 1.f;                                  // F8: the row's scale
            if (F8) sa = __ldg(&p.scaleA[(int64_t)u.bs * p.scaleA_site + row]);
            for (int c0 = 0; c0 < u.nc; c0 += 16) {
                float vr[16], vi[16];
                tmem_ld16(tr + c0, vr);
                tmem_ld16(tr + N + c0, vi);
                tmem_ld_wait();
                const int n0 = u.nt * p.N + c0;                   // first output column
                if (F8) {
                    // the same 16 column scales for every lane (broadcast loads)
                    const float4* sb = reinterpret_cast<const float4*>(p.scaleB + (int64_t)u.bs * p.scaleB_site + n0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float4 s4 = __ldg(&sb[j]);
                        const float s[4] = {s4.x * sa, s4.y * sa, s4.z * sa, s4.w * sa};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            vr[4 * j + k] *= s[k];
                            vi[4 * j + k] *= s[k];
                        }
                    }
                }
                if (EPI == TC_EPI_ROWS) {
                    // A row (ch, b) -> Mt[b][ch * Dp + n]: 16 consecutive columns
                    const int ch = row / p.ep_B, b = row % p.ep_B;
                    uint16_t* o = p.out16 + (int64_t)u.bs * p.out_site + (int64_t)b * p.out_ld +
                                  (int64_t)ch * p.ep_Dp + n0;
                    uint32_t rh[8], ih[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        rh[j] = pack_bf16x2(vr[2 * j], vr[2 * j + 1]);
                        ih[j] = pack_bf16x2(vi[2 * j], vi[2 * j + 1]);
                    }
                    st_v8(o, rh);
                    if (p.out_planes == 4) {
                        uint32_t rl[8], il[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            rl[j] = pack_bf16x2(vr[2 * j] - bf16_lo(rh[j]), vr[2 * j + 1] - bf16_hi(rh[j]));
                            il[j] = pack_bf16x2(vi[2 * j] - bf16_lo(ih[j]), vi[2 * j + 1] - bf16_hi(ih[j]));
                        }
                        st_v8(o + p.out_plane, rl);
                        st_v8(o + 2 * p.out_plane, ih);
                        st_v8(o + 3 * p.out_plane, il);
                    } else {
                        st_v8(o + p.out_plane, ih);
                    }
                } else if (EPI == TC_EPI_C32) {
                    float2* o = p.out32 + (int64_t)u.bs * p.out32_site;
                    if (p.out32_rows) {
                        // A row (ch, b) -> out32[b][ch Dp + n], 16 consecutive columns
                        const int ch = row / p.ep_B, b = row % p.ep_B;
                        o += (int64_t)b * p.out32_ld + (int64_t)ch * p.ep_Dp + n0;
#pragma unroll
                        for (int j = 0; j < 16; ++j) o[j] = make_float2(vr[j], vi[j]);
                    } else if (p.out32_trans) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) o[(int64_t)(n0 + j) * p.out32_ld + row] = make_float2(vr[j], vi[j]);
                    } else {
                        o += (int64_t)row * p.out32_ld + n0;
#pragma unroll
                        for (int j = 0; j < 16; ++j) o[j] = make_float2(vr[j], vi[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[a]);
            if (++a == NACC) {
                a = 0;
                aph ^= 1;
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

template <int N, int EPI, int NPL, bool F8>
cudaError_t launch(const TcArgs& a, const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mbt, int grid,
                   cudaStream_t s) {
    constexpr size_t smem = TcShape<N, NPL>::SMEM;
    static std::atomic<bool> attr{false};
    const cudaError_t e = bip_set_once(attr, [&] {
        return cudaFuncSetAttribute(tc_kernel<N, EPI, NPL, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    });
    if (e != cudaSuccess) return e;
    tc_kernel<N, EPI, NPL, F8><<<grid, kThreads, smem, s>>>(ma, mb, mbt, a);
    return cudaGetLastError();
}

template <int EPI, int NPL, bool F8 = false>
cudaError_t launch_n(const TcArgs& a, const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mbt, int grid,
                     cudaStream_t s) {
    // the template width bounds the shared-memory and TMEM layout; the tile
    // width a.N (a multiple of 16) may be smaller
    return a.N > 128 ? launch<256, EPI, NPL, F8>(a, ma, mb, mbt, grid, s)
                     : launch<128, EPI, NPL, F8>(a, ma, mb, mbt, grid, s);
}

}  // namespace

cudaError_t bip_tc_gemm(const TcArgs& a, cudaStream_t s) {
    if (a.N < 16 || a.N > 256 || a.N % 16) return cudaErrorInvalidValue;
    if (a.A.k != a.B.k || a.kb * 32 != a.A.k) return cudaErrorInvalidValue;
    if (a.npl != 4 && a.npl != 2) return cudaErrorInvalidValue;
    if (a.n_sites < 1 || a.mt_per < 1 || a.nt_per < 1) return cudaErrorInvalidValue;
    // the last tile: 16 .. N columns, a multiple of 16
    const int tail = a.n_cols - (a.nt_per - 1) * a.N;
    if (tail < 16 || tail > a.N || tail % 16) return cudaErrorInvalidValue;
    // every tile must lie inside its operand
    {
        const int64_t pl = a.npl - 1;
        if ((int64_t)(a.n_sites - 1) * a.A.site_rows + pl * a.A.plane_rows + (int64_t)a.mt_per * 128 > a.A.rows)
            return cudaErrorInvalidValue;
        if ((int64_t)(a.n_sites - 1) * a.B.site_rows + pl * a.B.plane_rows + (int64_t)a.n_cols > a.B.rows)
            return cudaErrorInvalidValue;
    }
    CUtensorMap ma, mb, mbt;
    cudaError_t e = make_map_2d(&ma, a.A.base, a.A.rows, a.A.k, 128);
    if (e != cudaSuccess) return e;
    e = make_map_2d(&mb, a.B.base, a.B.rows, a.B.k, a.N);
    if (e != cudaSuccess) return e;
    e = make_map_2d(&mbt, a.B.base, a.B.rows, a.B.k, tail);
    if (e != cudaSuccess) return e;
    const int units = a.n_sites * a.mt_per * a.nt_per;
    const int grid = units < num_sms() ? units : num_sms();
    const bool split = a.npl == 4;
    if (a.f8) {
        // E4M3: two planes (re, im), per-row scales in the epilogue
        if (split || a.conjA || !a.scaleA || !a.scaleB) return cudaErrorInvalidValue;
        if (((uintptr_t)a.scaleB | (size_t)a.scaleB_site * 4 | (size_t)a.N * 4) % 16) return cudaErrorMisalignedAddress;
        switch (a.epi) {
            case TC_EPI_ROWS: return launch_n<TC_EPI_ROWS, 2, true>(a, ma, mb, mbt, grid, s);
            case TC_EPI_C32: return launch_n<TC_EPI_C32, 2, true>(a, ma, mb, mbt, grid, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.epi) {
        case TC_EPI_ROWS: return split ? launch_n<TC_EPI_ROWS, 4>(a, ma, mb, mbt, grid, s)
                                       : launch_n<TC_EPI_ROWS, 2>(a, ma, mb, mbt, grid, s);
        case TC_EPI_C32: return split ? launch_n<TC_EPI_C32, 4>(a, ma, mb, mbt, grid, s)
                                      : launch_n<TC_EPI_C32, 2>(a, ma, mb, mbt, grid, s);
        default: return cudaErrorInvalidValue;
    }
}
