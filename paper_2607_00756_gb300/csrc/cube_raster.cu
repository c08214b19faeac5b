// The 4D cube's per-beam contraction on a raster scan list, separated over
// the aperture beams' lattice (Sec. 2.2.6, Algorithm 3; the map's raster
// evaluation uses the same property of the probe, Eq. probe).
//
// The aperture beams sit on the lattice h = (f_y k_y, f_x k_x), and on a
// raster rho = (ry[my], rx[mx]) the illumination factorises:
//   c_b(rho) = coef_b Ay[my][k_y] Ax[k_x][mx],
//   Ay = exp(-2 pi i f_y k_y ry / ny),  Ax = exp(-2 pi i f_x k_x rx / nx).
// So a_d(rho) = sum_b M_{d,b} c_b(rho) is two short sums:
//   T[k_y][mx][d] = sum_{k_x} (M_{d,b(k_y,k_x)} coef_b) Ax[k_x][mx]   (stage 1)
//   a_d(my, mx)  = sum_{k_y} Ay[my][k_y] T[k_y][mx][d]                (stage 2)
// and cube[rho][d] += scale sum_n |a_d(rho)|^2 over the crop of each site.
// Per site and channel that is n_d (n_kx + n_ky) My Mx complex products
// instead of n_d B My Mx: about 17x fewer at 512^2, f = 4.  FP32
// throughout.
//
//   stage 1: block = (site, channel, 32 beams d); it walks the k_y rows of
//            the lattice, stages M coef of the row in shared memory and
//            writes T for the scan columns of the site's crop.
//   stage 2: block = (32 beams d, 64 scan rows, 2 scan columns): it owns
//            those cube entries, adds every site of the batch in order
//            (each site's channels: |a|^2 kept in registers) and writes
//            each entry once -- one writer per element, a fixed order, no
//            atomics.
#include "bip_device.cuh"
#include "bip_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kD = 32;        // beams per block (the lanes)
constexpr int kMy = 64;       // scan rows per stage-2 block (8 per thread)
constexpr int kMx = 2;        // scan columns per stage-2 block

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
// the crop mask of site `site` at scan row my / column mx (bits the host
// set from the FP64 crop test of Sec. 2.2.4, per axis)
__device__ __forceinline__ bool crop_row(const CubeRasterArgs& a, int site, int my) {
    return (__ldg(&a.crop_y[(size_t)site * a.wy + (my >> 5)]) >> (my & 31)) & 1u;
}
__device__ __forceinline__ bool crop_col(const CubeRasterArgs& a, int site, int mx) {
    return (__ldg(&a.crop_x[(size_t)site * a.wx + (mx >> 5)]) >> (mx & 31)) & 1u;
}

__global__ void __launch_bounds__(kThreads) cube_raster_t_kernel(CubeRasterArgs a) {
    extern __shared__ float2 sm[];
    float2* ax = sm;                                   // [nkx][Mx]
    float2* mc = ax + (size_t)a.nkx * a.Mx;            // [nkx][kD]
    const int bs = blockIdx.z, ch = blockIdx.y, d0 = blockIdx.x * kD;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int site = a.site_ids[bs];
    const SiteDev st = a.sites[site];
    if (ch >= st.nch) return;                          // (the whole block)
    for (int i = threadIdx.x; i < a.nkx * a.Mx; i += kThreads) ax[i] = a.ax[i];
    const float2* m = a.m + (size_t)bs * a.m_site + (size_t)ch * a.m_ch;
    const int d = d0 + lane;
    float2* tout = a.T + (((size_t)bs * a.nch + ch) * a.nky) * a.Mx * a.nd_pad;
    for (int iy = 0; iy < a.nky; ++iy) {
        __syncthreads();                               // (ax loaded; mc of the last row read)
        for (int i = threadIdx.x; i < a.nkx * kD; i += kThreads) {
            const int ix = i / kD, l = i % kD;
            const int b = __ldg(&a.lat[iy * a.nkx + ix]);
            float2 v = make_float2(0.f, 0.f);
            if (b >= 0 && d0 + l < a.nd) {
                const float2 mv = m[(size_t)b * a.m_b + d0 + l];
                const double2 cf = a.coef[b];
                v = cmul(mv, make_float2((float)cf.x, (float)cf.y));
            }
            mc[i] = v;
        }
        __syncthreads();
        // this warp's scan columns, four at a time: mx = 4 (warp + 8 q) + u,
        // those inside the crop written (each M coef value loaded once for
        // the four)
        for (int m4 = 4 * warp; m4 < a.Mx; m4 += 4 * (kThreads / 32)) {
            bool in[4];
            bool any = false;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                in[u] = m4 + u < a.Mx && crop_col(a, site, m4 + u);
                any |= in[u];
            }
            if (!any) continue;
            float2 acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = make_float2(0.f, 0.f);
            for (int ix = 0; ix < a.nkx; ++ix) {
                const float2 mv = mc[ix * kD + lane];
                const float2* xr = ax + (size_t)ix * a.Mx + m4;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (in[u]) acc[u] = cfma(mv, xr[u], acc[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (in[u]) tout[((size_t)iy * a.Mx + m4 + u) * a.nd_pad + d] = acc[u];
        }
    }
}

constexpr int kTileElems = kMx * kD;     // T values of one (k_y) row of a stage-2 tile
constexpr int kPf = 8;                   // prefetched T values per thread (nky * kTileElems / kThreads <= 8)

__global__ void __launch_bounds__(kThreads) cube_raster_sum_kernel(CubeRasterArgs a) {
    extern __shared__ float2 sm[];
    float2* ay = sm;                                   // [kMy][nky]
    float2* ts = ay + (size_t)kMy * a.nky;             // [2][nky][kMx][kD], double-buffered
    unsigned* meets = (unsigned*)(ts + 2 * (size_t)a.nky * kTileElems);   // [n_sites] (0/1)
    const int d0 = blockIdx.x * kD, my0 = blockIdx.y * kMy, mx0 = blockIdx.z * kMx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = d0 + lane;
    const int tile = a.nky * kTileElems;               // T values per (site, channel)
    for (int i = threadIdx.x; i < kMy * a.nky; i += kThreads) {
        const int r = i / a.nky, iy = i % a.nky;
        ay[i] = my0 + r < a.My ? a.ay[(size_t)(my0 + r) * a.nky + iy] : make_float2(0.f, 0.f);
    }
    // which sites' crops meet this block's entries
    for (int bs = 0; bs < a.n_sites; ++bs) {
        const int site = a.site_ids[bs];
        bool hit = false;
        const int my = my0 + warp * 8 + (lane & 7), mx = mx0 + ((lane >> 3) & 1);
        if (my < a.My && mx < a.Mx) hit = crop_row(a, site, my) && crop_col(a, site, mx);
        hit = __syncthreads_or(hit);
        if (threadIdx.x == 0) meets[bs] = hit ? 1u : 0u;
    }
    __syncthreads();
    // the (site, channel) items in order, and the next one's T values loaded
    // into registers while the current one is summed
    auto next_item = [&](int& bs, int& ch) {
        ++ch;
        while (bs < a.n_sites && (!meets[bs] || ch >= a.sites[a.site_ids[bs]].nch)) {
            ++bs;
            ch = 0;
        }
    };
    auto fetch = [&](int bs, int ch, float2 (&pf)[kPf]) {
        const int site = a.site_ids[bs];
        const float2* tin = a.T + (((size_t)bs * a.nch + ch) * a.nky) * a.Mx * a.nd_pad;
#pragma unroll
        for (int q = 0; q < kPf; ++q) {
            const int i = threadIdx.x + q * kThreads;
            float2 v = make_float2(0.f, 0.f);
            if (i < tile) {
                const int iy = i / kTileElems, r = i % kTileElems, k = r / kD, l = r % kD;
                // T exists only for the crop's columns (stage 1 writes those)
                if (mx0 + k < a.Mx && crop_col(a, site, mx0 + k))
                    v = tin[((size_t)iy * a.Mx + mx0 + k) * a.nd_pad + d0 + l];
            }
            pf[q] = v;
        }
    };
    auto stash = [&](int buf, const float2 (&pf)[kPf]) {
#pragma unroll
        for (int q = 0; q < kPf; ++q) {
            const int i = threadIdx.x + q * kThreads;
            if (i < tile) ts[(size_t)buf * tile + i] = pf[q];
        }
    };
    float acc[8][kMx];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int k = 0; k < kMx; ++k) acc[j][k] = 0.f;
    int bs = 0, ch = -1;
    next_item(bs, ch);
    float2 pf[kPf];
    if (bs < a.n_sites) {
        fetch(bs, ch, pf);
        stash(0, pf);
    }
    __syncthreads();
    int buf = 0;
    while (bs < a.n_sites) {
        int nbs = bs, nch = ch;
        next_item(nbs, nch);
        if (nbs < a.n_sites) fetch(nbs, nch, pf);       // in flight during the sums below
        const int site = a.site_ids[bs];
        bool iny[8], inx[kMx];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int my = my0 + warp * 8 + j;
            iny[j] = my < a.My && crop_row(a, site, my);
        }
#pragma unroll
        for (int k = 0; k < kMx; ++k) inx[k] = mx0 + k < a.Mx && crop_col(a, site, mx0 + k);
        const float2* tb = ts + (size_t)buf * tile;
        float2 am[8][kMx];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int k = 0; k < kMx; ++k) am[j][k] = make_float2(0.f, 0.f);
        // a warp whose eight rows all lie outside the crop skips the sums
        // (the test is the same for all its lanes)
        bool wrow = false;
#pragma unroll
        for (int j = 0; j < 8; ++j) wrow |= iny[j];
        if (wrow)
            for (int iy = 0; iy < a.nky; ++iy) {
                float2 tv[kMx];
#pragma unroll
                for (int k = 0; k < kMx; ++k) tv[k] = tb[(iy * kMx + k) * kD + lane];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float2 y = ay[(warp * 8 + j) * a.nky + iy];
#pragma unroll
                    for (int k = 0; k < kMx; ++k) am[j][k] = cfma(y, tv[k], am[j][k]);
                }
            }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int k = 0; k < kMx; ++k)
                if (iny[j] && inx[k]) acc[j][k] = fmaf(am[j][k].x, am[j][k].x, fmaf(am[j][k].y, am[j][k].y, acc[j][k]));
        // the next item's values into the other buffer (its last reader
        // finished before the barrier that ended the previous item)
        if (nbs < a.n_sites) stash(buf ^ 1, pf);
        __syncthreads();
        buf ^= 1;
        bs = nbs;
        ch = nch;
    }
    if (d >= a.nd) return;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int my = my0 + warp * 8 + j;
        if (my >= a.My) continue;
#pragma unroll
        for (int k = 0; k < kMx; ++k) {
            const int mx = mx0 + k;
            if (mx >= a.Mx) continue;
            float* o = a.cube + ((size_t)my * a.Mx + mx) * a.cube_ld + d;
            *o += a.scale * acc[j][k];
        }
    }
}

}  // namespace

size_t bip_cube_raster_t_bytes(const CubeRasterArgs& a) {
    return (size_t)a.n_sites * a.nch * a.nky * a.Mx * a.nd_pad * sizeof(float2);
}

cudaError_t bip_cube_raster(const CubeRasterArgs& a, cudaStream_t s) {
    if (a.n_sites < 1 || a.nd < 1) return cudaSuccess;
    if (a.nd_pad % kD || a.nd > a.nd_pad || a.nch < 1 || a.nch > 9 || a.nky < 1 || a.nkx < 1 || a.My < 1 || a.Mx < 1)
        return cudaErrorInvalidValue;
    const size_t sm1 = ((size_t)a.nkx * a.Mx + (size_t)a.nkx * kD) * sizeof(float2);
    const size_t sm2 = ((size_t)kMy * a.nky + 2 * (size_t)a.nky * kMx * kD) * sizeof(float2) +
                       (size_t)a.n_sites * sizeof(unsigned);
    if ((size_t)a.nky * kTileElems > (size_t)kPf * kThreads) return cudaErrorInvalidValue;
    if (sm1 > 200 * 1024 || sm2 > 200 * 1024) return cudaErrorInvalidValue;
    if (a.My > 65535 * kMy || a.Mx > 65535 * kMx) return cudaErrorInvalidValue;
    static std::atomic<size_t> attr1{0}, attr2{0};
    cudaError_t e;
    if (sm1 > 48 * 1024) {
        e = bip_raise_once(attr1, sm1, [&] {
            return cudaFuncSetAttribute(cube_raster_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
        });
        if (e != cudaSuccess) return e;
    }
    if (sm2 > 48 * 1024) {
        e = bip_raise_once(attr2, sm2, [&] {
            return cudaFuncSetAttribute(cube_raster_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        });
        if (e != cudaSuccess) return e;
    }
    cube_raster_t_kernel<<<dim3(a.nd_pad / kD, a.nch, a.n_sites), kThreads, sm1, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cube_raster_sum_kernel<<<dim3(a.nd_pad / kD, (a.My + kMy - 1) / kMy, (a.Mx + kMx - 1) / kMx), kThreads, sm2, s>>>(a);
    return cudaGetLastError();
}
