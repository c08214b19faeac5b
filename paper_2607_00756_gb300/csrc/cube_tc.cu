// The 4D cube (Sec. 2.2.6) on the tensor cores: per site, channel and
// detector beam d, a_d(rho) = sum_b M^(n)_{d,b} c_b(rho), and
//   cube[rho][d] += scale sum_n |a_d(rho)|^2
// for the scans of the site's crop mask -- or, in map mode, the same terms
// summed over d into the site's map (the "beam order" of the scan
// contraction: |M c|^2 directly, without the Gram matrix).  Split BF16 (hi + lo, three
// products per real product, twelve per complex one), FP32 accumulation in
// TMEM.  The "probe order" runs the same kernel on other operands:
// a_d(rho) = sum_r S2_d(r) Y^(n)(rho, r) with Y^(n) = H_n x the windowed
// probes, the channel then in B's columns, BF16 planes (four products).
//
// Work item: (site in batch, tile of scans that meets the site's crop
// mask).  K runs over (channel, aperture beam); each channel accumulates
// into its own TMEM pair (re, im), so the epilogue has every channel of an
// element at once.  No floating-point atomics: every output element has one
// writer per launch, and its additions come in a fixed order, so results do
// not depend on scheduling.
//   cube mode: a unit is (group of work items sharing one scan tile, sites
//     in ascending order; tile of 128 detector beams); the CTA that owns it
//     adds each site's channel sum to the cube with a plain read-add-write.
//   map mode: a unit is one work item and one 128-beam tile of d; the
//     detector sum of each scan column is taken by a fixed shuffle tree per
//     warp, then over the four epilogue warps in order, and stored in the
//     unit's own slot; map_reduce_kernel then adds each scan's slots over
//     the d tiles (and, with (scan, channel) columns, over the channels) in
//     order to the site's map.
// The crop mask of a work item's scans is a precomputed 64-bit word per 64
// columns.  Persistent, one CTA per SM, 192 threads: warp 0 TMA producer,
// warp 1 TMEM allocator and MMA issuer, warps 2-5 epilogue.  Every wait is
// bounded; on a timeout the kernel sets *err, drains what it issued and
// frees TMEM.
#include "bip_device.cuh"
#include "tc_common.cuh"

namespace {

constexpr int kThreads = 192;
constexpr int kATile = 128 * 64;                  // bytes: 128 rows x 32 bf16
constexpr int kRing = 4 * (4 * kATile + 4 * 64 * 64);   // bytes of the stage ring
constexpr int kMaxStages = 8;
constexpr int kRed = 4 * 128 * 4;                 // bytes: per-warp column sums (map mode)
constexpr size_t kSmem = 1024 + (size_t)kRing + 256 + kRed;
// A stage holds one 32-wide K block of every plane: split BF16 A re_hi,
// re_lo, im_hi, im_lo then B the same; BF16 (HI) A re, im then B re, im.
// The ring holds as many stages as fit: 4 (split, 64-scan tiles), 3 (split,
// 128), 8 (BF16, 64), 6 (BF16, 128).
template <bool HI, int TN>
struct Shape {
    static constexpr int BTILE = TN * 64;                           // bytes of one B plane
    static constexpr int SBYTES = HI ? 2 * kATile + 2 * BTILE : 4 * kATile + 4 * BTILE;
    static constexpr int NS = kRing / SBYTES;
    static constexpr int BOFF = HI ? 2 * kATile : 4 * kATile;       // B planes in a stage
    static_assert(NS >= 2 && NS <= kMaxStages, "stage ring");
};

// The steps (work item w, d tile mt) of unit u: items w0 .. w1 - 1, tiles
// mt0 .. mt1 - 1 (one of the two ranges has one entry).
struct Steps {
    int w0, w1, mt0, mt1;
};
__device__ __forceinline__ bool unit_steps(const CubeTcArgs& a, int u, Steps& st) {
    if (!a.cube) {
        // map mode: one work item and one d tile per unit
        if (u >= a.n_work * a.mt_per) return false;
        st = Steps{u / a.mt_per, u / a.mt_per + 1, u % a.mt_per, u % a.mt_per + 1};
    } else {
        if (u >= a.n_groups * a.mt_per) return false;
        const int g = u / a.mt_per, mt = u % a.mt_per;
        st = Steps{a.grp[g], a.grp[g + 1], mt, mt + 1};
    }
    return true;
}

// HI: BF16 operands of two planes (four MMAs per K step); TN: scans (B
// rows) per tile, the MMA's N.  Template parameters, so that the issue loop
// carries no branch on them.
template <bool HI, int TN>
__global__ void __launch_bounds__(kThreads, 1)
    cube_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const CubeTcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    using SH = Shape<HI, TN>;
    constexpr int NS = SH::NS, SBYTES = SH::SBYTES, BOFF = SH::BOFF, kBTile = SH::BTILE, kN = TN;
    constexpr int MW = TN / 64;                                  // mask words per work item
    uint64_t* full = (uint64_t*)(smem + kRing);
    uint64_t* empty = full + kMaxStages;
    uint64_t* acc_full = empty + kMaxStages;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* drain = acc_empty + 1;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* ep_ok = abort_flag + 1;
    float* red = (float*)(smem + kRing + 256);              // [4 warps][kN] (map mode)

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 4);
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
    const int kb0 = a.ch0 * a.kb_ch, kb1 = (a.ch0 + a.nacc) * a.kb_ch;

    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(a.err, 1);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            bool ok = true;
            Steps su;
            for (int i = 0; ok && unit_steps(a, blockIdx.x + i * gridDim.x, su); ++i)
            for (int w = su.w0; ok && w < su.w1; ++w)
            for (int mt = su.mt0; ok && mt < su.mt1; ++mt) {
                const int bs = a.work[2 * w], t = a.work[2 * w + 1];
                const int64_t a0 = (int64_t)bs * a.a_site_rows + (int64_t)mt * 128;
                const int64_t b0 = (int64_t)bs * a.b_site_rows + (int64_t)t * kN;
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, wait_limit(a.wait_ns))) {
                        fail();
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + s * SBYTES;
                    // K block within the channel (the operand without channels)
                    // and across channels (the one that has them)
                    const int kx = (kb % a.kb_ch) * 32, kc = kb * 32;
                    const int ax = a.swap_ch ? kx : kc, bx = a.swap_ch ? kc : kx;
                    if constexpr (HI) {
                        mbar_expect_tx(&full[s], SBYTES);
#pragma unroll
                        for (int pl = 0; pl < 2; ++pl) {
                            tma_2d(st + pl * kATile, &mapA, ax, (int)(a0 + pl * a.a_plane_rows), &full[s]);
                            tma_2d(st + BOFF + pl * kBTile, &mapB, bx, (int)(b0 + pl * a.b_plane_rows), &full[s]);
                        }
                    } else {
                        mbar_expect_tx(&full[s], SBYTES);
#pragma unroll
                        for (int pl = 0; pl < 4; ++pl)
                            tma_2d(st + pl * kATile, &mapA, ax, (int)(a0 + pl * a.a_plane_rows), &full[s]);
#pragma unroll
                        for (int pl = 0; pl < 4; ++pl)
                            tma_2d(st + BOFF + pl * kBTile, &mapB, bx, (int)(b0 + pl * a.b_plane_rows), &full[s]);
                    }
                    ++issued;
                    if (++s == NS) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            if (!ok) {
                for (int k = 0; k < NS && k < issued; ++k) {
                    s = (s + NS - 1) % NS;
                    if (s == NS - 1) ph ^= 1;
                    const uint64_t t0 = gtimer();
                    while (!mbar_try(&full[s], ph) && gtimer() - t0 < kTimeoutNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: one accumulator pair per channel
            const uint32_t id_pos = idesc(128, kN, false), id_neg = idesc(128, kN, true);
            int s = 0;
            uint32_t ph = 0, aph = 0;
            bool any = false, ok = true;
            Steps su;
            for (int i = 0; ok && unit_steps(a, blockIdx.x + i * gridDim.x, su); ++i)
            for (int w = su.w0; ok && w < su.w1; ++w)
            for (int mt = su.mt0; ok && mt < su.mt1; ++mt) {
                if (!mbar_wait(acc_empty, aph ^ 1, abort_flag, wait_limit(a.wait_ns))) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(&full[s], ph, abort_flag, wait_limit(a.wait_ns))) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + s * SBYTES);
                    const int ch = (kb - kb0) / a.kb_ch;
                    const uint32_t dr = tbase + (uint32_t)(ch * 2 * kN), di = dr + kN;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint32_t first = (kb % a.kb_ch == 0 && kk == 0) ? 0u : 1u;
                        if constexpr (HI) {
                            const uint64_t ar = sdesc(base + kk * 32), ai = sdesc(base + kATile + kk * 32);
                            const uint64_t br = sdesc(base + BOFF + kk * 32), bi = sdesc(base + BOFF + kBTile + kk * 32);
                            mma(dr, ar, br, id_pos, first);
                            mma(dr, ai, bi, id_neg, 1);
                            mma(di, ar, bi, id_pos, first);
                            mma(di, ai, br, id_pos, 1);
                        } else {
                            uint64_t ad[4], bd[4];
#pragma unroll
                            for (int pl = 0; pl < 4; ++pl) {
                                ad[pl] = sdesc(base + pl * kATile + kk * 32);
                                bd[pl] = sdesc(base + BOFF + pl * kBTile + kk * 32);
                            }
                            // planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo
                            mma(dr, ad[0], bd[0], id_pos, first);
                            mma(dr, ad[0], bd[1], id_pos, 1);
                            mma(dr, ad[1], bd[0], id_pos, 1);
                            mma(dr, ad[2], bd[2], id_neg, 1);
                            mma(dr, ad[2], bd[3], id_neg, 1);
                            mma(dr, ad[3], bd[2], id_neg, 1);
                            mma(di, ad[0], bd[2], id_pos, first);
                            mma(di, ad[0], bd[3], id_pos, 1);
                            mma(di, ad[1], bd[2], id_pos, 1);
                            mma(di, ad[2], bd[0], id_pos, 1);
                            mma(di, ad[2], bd[1], id_pos, 1);
                            mma(di, ad[3], bd[0], id_pos, 1);
                        }
                    }
                    any = true;
                    mma_commit(&empty[s]);
                    if (++s == NS) {
                        s = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(acc_full);
                aph ^= 1;
            }
            if (any) {
                mma_commit(drain);
                const uint64_t t0 = gtimer();
                while (!mbar_try(drain, 0) && gtimer() - t0 < kTimeoutNs) {
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lane quadrant = warp % 4
        const int q = warp & 3;
        const int et = threadIdx.x - 64;
        const bool map_mode = a.mpart != nullptr;
        uint32_t aph = 0;
        bool ok = true;
        Steps su;
        for (int i = 0; ok && unit_steps(a, blockIdx.x + i * gridDim.x, su); ++i) {
            float colacc = 0.f;                 // map mode: thread et's scan column, over the unit
            for (int w = su.w0; ok && w < su.w1; ++w)
            for (int mt = su.mt0; mt < su.mt1; ++mt) {
                if (et == 0) {
                    const bool good = mbar_wait(acc_full, aph, abort_flag, wait_limit(a.wait_ns));
                    *ep_ok = good ? 1 : 0;
                    if (!good) fail();
                }
                named_sync(1, 128);
                if (!*ep_ok) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int t = a.work[2 * w + 1];
                const unsigned long long* mask = a.mask + (size_t)w * MW;
                const int d = mt * 128 + q * 32 + lane;
                const uint32_t tr = tbase + ((uint32_t)(q * 32) << 16);
                for (int c0 = 0; c0 < kN; c0 += 16) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.f;
                    for (int ch = 0; ch < a.nacc; ++ch) {
                        float vr[16], vi[16];
                        tmem_ld16(tr + ch * 2 * kN + c0, vr);
                        tmem_ld16(tr + ch * 2 * kN + kN + c0, vi);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = fmaf(vr[j], vr[j], fmaf(vi[j], vi[j], v[j]));
                    }
                    if (map_mode) {
                        // this warp's 32 beams of each column, by a fixed shuffle tree
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float x = d < a.n_det ? v[j] : 0.f;
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                            if (lane == 0) red[q * kN + c0 + j] = x;
                        }
                    } else if (d < a.n_det) {
                        // the unit owns these cube entries: sites in order, plain adds
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int rho = t * kN + c0 + j;
                            if ((mask[c0 >> 6] >> ((c0 & 63) + j)) & 1ull) {
                                float* e = a.cube + (size_t)rho * a.cube_ld + d;
                                *e += a.scale * v[j];
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
                aph ^= 1;
                if (map_mode) {
                    // the four warps' sums in order, then the d tiles in order
                    named_sync(1, 128);
                    if (et < kN) colacc += ((red[et] + red[kN + et]) + red[2 * kN + et]) + red[3 * kN + et];
                    named_sync(1, 128);
                }
            }
            if (!ok || !map_mode || et >= kN) continue;
            // end of a map-mode unit (one work item, one d tile): its column
            // sums go to the unit's own slot (summed over d tiles, in order,
            // by bip_cube_map_reduce); columns outside the crop mask are 0
            const int w = su.w0;
            const bool in = (a.mask[(size_t)w * MW + (et >> 6)] >> (et & 63)) & 1ull;
            a.mpart[((size_t)w * a.mt_per + su.mt0) * kN + et] = in ? colacc : 0.f;
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

// 64-bit crop masks of the work items' scan tiles, tile/64 words per item
// (bit j of word h: scan tile t + 64 h + j; with (scan, channel) columns,
// the scan of that column).  Sub-item = (work item, word).
__global__ void crop_mask_kernel(CubeTcArgs a, int tn) {
    __shared__ unsigned long long part[4][2];
    const int mw = tn / 64;
    const int sub = blockIdx.x * (blockDim.x / 64) + threadIdx.x / 64;
    const int w = sub / mw, h = sub % mw;
    const int j = threadIdx.x % 64;
    bool in = false;
    if (w < a.n_work) {
        const int bs = a.work[2 * w], t = a.work[2 * w + 1];
        const SiteDev st = a.sites[a.site_ids[bs]];
        const int col = t * tn + h * 64 + j;
        const int rho = a.col_nch ? col / a.col_nch : col;
        in = col < (a.col_nch ? a.P * a.col_nch : a.P) &&
             in_crop(a.scans[2 * rho], a.scans[2 * rho + 1], st.ty, st.tx, a.ny, a.nx, a.fy, a.fx);
    }
    // every lane takes part in the vote and the barrier
    const unsigned bits = __ballot_sync(0xffffffffu, in);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x / 64][(threadIdx.x / 32) & 1] = bits;
    __syncthreads();
    if (j == 0 && w < a.n_work)
        a.mask[sub] = part[threadIdx.x / 64][0] | (part[threadIdx.x / 64][1] << 32);
}

// Map mode, second stage: partial[site][rho] += scale sum_n sum_mt
// mpart[w][mt][c] over the columns (rho ncol + n) of the site's scan,
// w the work item of the column's tile (none: 0), in channel then d-tile
// order -- one thread per (site, scan), so every addition order is fixed.
__global__ void map_reduce_kernel(MapReduceArgs a) {
    const int rho = blockIdx.x * blockDim.x + threadIdx.x;
    const int bs = blockIdx.y;
    if (rho >= a.P) return;
    float v = 0.f;
    for (int n = 0; n < a.ncol; ++n) {
        const int col = rho * a.ncol + n;
        const int w = a.wmap[(size_t)bs * a.n_tiles + col / a.tn];
        if (w < 0) continue;
        const float* m = a.mpart + (size_t)w * a.mt_per * a.tn + col % a.tn;
        for (int mt = 0; mt < a.mt_per; ++mt) v += m[(size_t)mt * a.tn];
    }
    float* e = a.partial + (size_t)a.site_ids[bs] * a.P + rho;
    *e += a.scale * v;
}

template <bool HI, int TN>
cudaError_t launch_cube(const CubeTcArgs& a, const CUtensorMap& ma, const CUtensorMap& mb, cudaStream_t s) {
    static std::atomic<bool> attr{false};
    const cudaError_t e = bip_set_once(attr, [&] {
        return cudaFuncSetAttribute(cube_tc_kernel<HI, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    });
    if (e != cudaSuccess) return e;
    const int units = a.cube ? a.n_groups * a.mt_per : a.n_work * a.mt_per;
    const int grid = units < num_sms() ? units : num_sms();
    cube_tc_kernel<HI, TN><<<grid, kThreads, kSmem, s>>>(ma, mb, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t bip_cube_tc(const CubeTcArgs& a, const void* A, int64_t a_rows, int a_k, const void* B, int64_t b_rows,
                        int b_k, cudaStream_t s) {
    if (a.n_work < 1) return cudaSuccess;
    const int tn = a.tn ? a.tn : 64;
    if (tn != 64 && tn != 128) return cudaErrorInvalidValue;
    // one TMEM accumulator pair (2 tn columns) per channel in 512 columns
    if (a.nacc < 1 || a.nacc * 2 * tn > (int)kTmemCols || a.kb_ch < 1 || a.mt_per < 1 || a.ch0 < 0 || a_k % 32 ||
        b_k % 32)
        return cudaErrorInvalidValue;
    // map mode (mpart: per-unit column sums), or cube mode (groups of items
    // sharing a scan tile)
    if ((a.mpart != nullptr) == (a.cube != nullptr)) return cudaErrorInvalidValue;
    if (a.cube && (a.n_groups < 1 || !a.grp || a.cube_ld < a.n_det)) return cudaErrorInvalidValue;
    if (a.col_nch < 0 || (a.col_nch > 0 && (a.nacc != 1 || a.ch0 != 0 || a.cube))) return cudaErrorInvalidValue;
    // the channel range inside the operand that has channels, one channel's
    // K blocks inside the other
    const int ch_k = a.swap_ch ? b_k : a_k, one_k = a.swap_ch ? a_k : b_k;
    if ((a.ch0 + a.nacc) * a.kb_ch * 32 > ch_k || a.kb_ch * 32 > one_k) return cudaErrorInvalidValue;
    // every tile inside its operand: A rows of the last site, B rows of the
    // last site's last scan tile
    const int64_t pl = a.hi_only ? 1 : 3;
    if ((int64_t)(a.n_sites - 1) * a.a_site_rows + pl * a.a_plane_rows + (int64_t)a.mt_per * 128 > a_rows)
        return cudaErrorInvalidValue;
    if ((int64_t)(a.n_sites - 1) * a.b_site_rows + pl * a.b_plane_rows + (int64_t)a.n_tiles * tn > b_rows)
        return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    cudaError_t e = make_map_2d(&ma, A, a_rows, a_k, 128);
    if (e != cudaSuccess) return e;
    e = make_map_2d(&mb, B, b_rows, b_k, tn);
    if (e != cudaSuccess) return e;
    // the crop masks of the work items (tn / 64 words each, 4 words per
    // 256-thread block)
    const int subs = a.n_work * (tn / 64);
    crop_mask_kernel<<<(subs + 3) / 4, 256, 0, s>>>(a, tn);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.hi_only) return tn == 128 ? launch_cube<true, 128>(a, ma, mb, s) : launch_cube<true, 64>(a, ma, mb, s);
    return tn == 128 ? launch_cube<false, 128>(a, ma, mb, s) : launch_cube<false, 64>(a, ma, mb, s);
}

cudaError_t bip_cube_map_reduce(const MapReduceArgs& a, cudaStream_t s) {
    if (a.n_sites < 1 || a.P < 1) return cudaSuccess;
    if (a.ncol < 1 || a.tn < 1 || a.mt_per < 1 || a.n_tiles * a.tn < a.P * a.ncol) return cudaErrorInvalidValue;
    map_reduce_kernel<<<dim3((a.P + 127) / 128, a.n_sites), 128, 0, s>>>(a);
    return cudaGetLastError();
}
