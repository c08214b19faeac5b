// The scan contraction of the map as a trigonometric polynomial.
//
// With c_b(rho) = coef_b exp(-2 pi i h_b.rho/N) and the Gram matrix
// Q = sum_n M^(n)H M^(n) (Hermitian), Eq. map-sum per site is
//   I_tau(rho) = f_y f_x c^H Q c
//              = f_y f_x Re sum_{b <= b'} w_bb' conj(coef_b) Q_bb' coef_b'
//                         exp(2 pi i (h_b - h_b').rho/N),
// w = 1 on the diagonal and 2 above it.  The aperture beams lie on the
// lattice h = f k, so grouping the pairs by their difference
// Delta = k_b - k_b' gives
//   I_tau(rho) = f_y f_x Re sum_Delta G(Delta) exp(2 pi i f Delta.rho/N),
//   G(Delta)   = sum_{b <= b', k_b - k_b' = Delta} w_bb' conj(coef_b) Q_bb' coef_b'.
// Beams are sorted by (h_y, h_x), so b <= b' means Delta <= 0
// lexicographically: Delta_y in [-2K_y, 0], Delta_x in [-2K_x, 2K_x].
// This is an exact regrouping of the sums; it replaces the B x B x scans
// product by a binning of Q (B^2 terms) and ~(2K_y+1)(4K_x+1) terms per scan.
//
//   diff_bin  : warp per (site, Delta), lanes over b, fixed reduction tree
//   diff_eval : persistent; thread per scan of a (site, scan tile) work
//               item; Horner's rule in exp(2 pi i f rho/N) along the
//               lattice rows and over them, start angles reduced to [0, 1)
//               turns in FP64.
//   raster_eval: scans on a raster: the polynomial factorises over the two
//               axes, two small dense stages per site (tables of the phases
//               per scan row and column, angles reduced in FP64 on the host).
#include "bip_device.cuh"
#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

// One warp per difference Delta; the lanes split the beams b and the
// partial sums meet in a fixed shuffle tree, so the result is deterministic.
constexpr int kBinWarps = 8;

__global__ void __launch_bounds__(kBinWarps * 32) diff_bin_kernel(DiffArgs a) {
    extern __shared__ unsigned char smb[];
    int2* kb = reinterpret_cast<int2*>(smb);                         // [B]
    float2* cf = reinterpret_cast<float2*>(kb + a.B);                // [B]
    int* lat = reinterpret_cast<int*>(cf + a.B);                     // [(2Ky+1)(2Kx+1)]
    const int lw = 2 * a.Kx + 1;
    const int nlat = (2 * a.Ky + 1) * lw;
    for (int i = threadIdx.x; i < a.B; i += blockDim.x) {
        kb[i] = __ldg(&a.kb[i]);
        const double2 c = __ldg(&a.coef[i]);
        cf[i] = make_float2((float)c.x, (float)c.y);
    }
    for (int i = threadIdx.x; i < nlat; i += blockDim.x) lat[i] = __ldg(&a.lat[i]);
    __syncthreads();

    const int bs = blockIdx.y;
    const int nd = (2 * a.Ky + 1) * (4 * a.Kx + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int di = blockIdx.x * kBinWarps + warp;
    if (di >= nd) return;
    const int dy = di / (4 * a.Kx + 1) - 2 * a.Ky;       // in [-2Ky, 0]
    const int dx = di % (4 * a.Kx + 1) - 2 * a.Kx;       // in [-2Kx, 2Kx]
    const float2* Q = a.Q + (size_t)bs * a.q_site;
    float gr = 0.f, gi = 0.f;
    if (dy < 0 || dx <= 0) {
        for (int b = lane; b < a.B; b += 32) {
            const int2 k = kb[b];
            const int ky = k.x - dy, kx = k.y - dx;          // partner k_b' = k_b - Delta
            if (ky < -a.Ky || ky > a.Ky || kx < -a.Kx || kx > a.Kx) continue;
            const int bp = lat[(ky + a.Ky) * lw + kx + a.Kx];
            if (bp < 0) continue;
            const float2 q = __ldg(&Q[(size_t)b * a.ldq + bp]);
            const float2 cb = cf[b], cp = cf[bp];
            // w conj(c_b) q c_b', w = 1 on the diagonal, 2 above it
            const float w = (bp == b) ? 1.f : 2.f;
            const float2 t = c_mul(make_float2(cb.x, -cb.y), c_mul(q, cp));
            gr = fmaf(w, t.x, gr);
            gi = fmaf(w, t.y, gi);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gr += __shfl_xor_sync(0xffffffffu, gr, o);
        gi += __shfl_xor_sync(0xffffffffu, gi, o);
    }
    if (lane == 0) a.G[(size_t)bs * nd + di] = make_float2(gr, gi);
}

// exp(2 pi i * turns): the angle is reduced to [0, 1) turns in FP64 (exact
// for the integer part), the rest is FP32 sincospif
__device__ __forceinline__ float2 turn(double t) {
    const float r = (float)(t - floor(t));
    float s, c;
    sincospif(2.0f * r, &s, &c);
    return make_float2(c, s);
}

// Persistent over the (site in batch, scan tile) work items, in a fixed
// round-robin order.  Per scan rho the polynomial
//   sum_{iy, j} G[iy][j] rx^(j - 2K_x) ry^(iy - 2K_y),
//   rx = exp(2 pi i f_x rho_x / N_x), ry = exp(2 pi i f_y rho_y / N_y),
// is evaluated by Horner's rule in rx along each row and in ry over the
// rows (one complex multiply-add per term), then multiplied by the start
// phase rx^(-2K_x) ry^(-2K_y).
__global__ void __launch_bounds__(256) diff_eval_kernel(DiffArgs a) {
    extern __shared__ float2 gs[];
    const int rows = 2 * a.Ky + 1, cols = 4 * a.Kx + 1;
    const int nd = rows * cols;
    for (int w = blockIdx.x; w < a.n_work; w += gridDim.x) {
        const int bs = a.work[2 * w], tile = a.work[2 * w + 1];
        __syncthreads();                           // the previous item's reads of gs are done
        for (int i = threadIdx.x; i < nd; i += blockDim.x) gs[i] = a.G[(size_t)bs * nd + i];
        __syncthreads();
        const int site = a.site_ids[bs];
        const SiteDev st = a.sites[site];
        const int n1 = min((tile + 1) * a.tile, a.P);
        for (int n = tile * a.tile + threadIdx.x; n < n1; n += blockDim.x) {
            const double ry = a.scans[2 * n], rx = a.scans[2 * n + 1];
            if (!in_crop(ry, rx, st.ty, st.tx, a.ny, a.nx, a.fy, a.fx)) {
                a.partial[(size_t)site * a.P + n] = 0.f;
                continue;
            }
            const double ty = (double)a.fy * ry / a.ny, tx = (double)a.fx * rx / a.nx;   // turns per lattice step
            const float2 zy = turn(ty), zx = turn(tx);
            float2 T = make_float2(0.f, 0.f);
            for (int iy = rows - 1; iy >= 0; --iy) {
                const float2* g = gs + iy * cols;
                const int last = iy == rows - 1 ? 2 * a.Kx + 1 : cols;   // Delta_y = 0: Delta_x <= 0 only
                float2 sr = g[last - 1];
#pragma unroll 4
                for (int j = last - 2; j >= 0; --j) {     // sr = sr zx + g[j]
                    const float2 gv = g[j];
                    const float xr = fmaf(sr.x, zx.x, fmaf(-sr.y, zx.y, gv.x));
                    const float xi = fmaf(sr.x, zx.y, fmaf(sr.y, zx.x, gv.y));
                    sr = make_float2(xr, xi);
                }
                // T = T zy + row sum
                const float yr = fmaf(T.x, zy.x, fmaf(-T.y, zy.y, sr.x));
                const float yi = fmaf(T.x, zy.y, fmaf(T.y, zy.x, sr.y));
                T = make_float2(yr, yi);
            }
            const float2 e0 = turn(-2.0 * a.Kx * tx - 2.0 * a.Ky * ty);
            a.partial[(size_t)site * a.P + n] = a.scale * fmaf(e0.x, T.x, -e0.y * T.y);
        }
    }
}

// Raster scans: block = (64 scan rows, site), four warps of 16 rows each;
// stage 1 Y[r][j] = sum_iy Ay[my][iy] G[iy][j] for the block's rows into
// shared memory, stage 2 lane = four adjacent scan columns, 16 rows x 4
// columns of Re(Y Ax) per thread (Ax[j][.] loaded once per j and lane).
constexpr int kRasterWarpRows = 16;
constexpr int kRasterRows = 4 * kRasterWarpRows;
__global__ void __launch_bounds__(128) raster_eval_kernel(DiffArgs a, RasterArgs r) {
    extern __shared__ float2 rs[];
    const int rows = 2 * a.Ky + 1, cols = 4 * a.Kx + 1;
    const int nd = rows * cols;
    float2* gs = rs;                       // [rows][cols]
    float2* ys = rs + nd;                  // [kRasterRows][cols]
    const int bs = blockIdx.y;
    const int my0 = blockIdx.x * kRasterRows;
    const int nr = min(kRasterRows, r.My - my0);
    for (int i = threadIdx.x; i < nd; i += blockDim.x) gs[i] = a.G[(size_t)bs * nd + i];
    __syncthreads();
    for (int i = threadIdx.x; i < nr * cols; i += blockDim.x) {
        const int q = i / cols, j = i % cols;
        const float2* ay = r.Ay + (size_t)(my0 + q) * rows;
        float sx = 0.f, sy = 0.f;
        for (int iy = 0; iy < rows; ++iy) {
            const float2 u = __ldg(&ay[iy]), g = gs[iy * cols + j];
            sx = fmaf(u.x, g.x, fmaf(-u.y, g.y, sx));
            sy = fmaf(u.x, g.y, fmaf(u.y, g.x, sy));
        }
        ys[q * cols + j] = make_float2(sx, sy);
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int q0 = warp * kRasterWarpRows;                 // this warp's first row in the block
    const int wr = min(kRasterWarpRows, nr - q0);          // its rows (may be <= 0)
    if (wr <= 0) return;
    const int site = a.site_ids[bs];
    const SiteDev st = a.sites[site];
    for (int mx0 = 4 * lane; mx0 < r.Mx; mx0 += 128) {
        float acc[kRasterWarpRows][4];
#pragma unroll
        for (int q = 0; q < kRasterWarpRows; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[q][k] = 0.f;
        for (int j = 0; j < cols; ++j) {
            float2 x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = mx0 + k < r.Mx ? __ldg(&r.Ax[(size_t)j * r.Mx + mx0 + k]) : make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < kRasterWarpRows; ++q) {
                const float2 y = ys[(q0 + (q < wr ? q : 0)) * cols + j];
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[q][k] = fmaf(y.x, x[k].x, fmaf(-y.y, x[k].y, acc[q][k]));   // Re(y x)
            }
        }
        for (int q = 0; q < wr; ++q) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int mx = mx0 + k;
                if (mx >= r.Mx) continue;
                const int n = (my0 + q0 + q) * r.Mx + mx;
                if (in_crop(a.scans[2 * n], a.scans[2 * n + 1], st.ty, st.tx, a.ny, a.nx, a.fy, a.fx))
                    a.partial[(size_t)site * a.P + n] = a.scale * acc[q][k];
            }
        }
    }
}

}  // namespace

cudaError_t bip_raster_eval(const DiffArgs& a, const RasterArgs& r, cudaStream_t s) {
    if (a.n_sites < 1 || r.My < 1 || r.Mx < 1 || (int64_t)r.My * r.Mx != a.P) return cudaErrorInvalidValue;
    const size_t nd = (size_t)(2 * a.Ky + 1) * (4 * a.Kx + 1);
    const size_t sm = (nd + (size_t)kRasterRows * (4 * a.Kx + 1)) * sizeof(float2);
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    static std::atomic<size_t> attr{0};
    if (sm > 48 * 1024) {
        const cudaError_t e = bip_raise_once(attr, sm, [&] {
            return cudaFuncSetAttribute(raster_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        });
        if (e != cudaSuccess) return e;
    }
    raster_eval_kernel<<<dim3((r.My + kRasterRows - 1) / kRasterRows, a.n_sites), 128, sm, s>>>(a, r);
    return cudaGetLastError();
}

cudaError_t bip_diff_bin(const DiffArgs& a, cudaStream_t s) {
    const int nd = (2 * a.Ky + 1) * (4 * a.Kx + 1);
    const size_t sm = (size_t)a.B * (sizeof(int2) + sizeof(float2)) +
                      (size_t)(2 * a.Ky + 1) * (2 * a.Kx + 1) * sizeof(int);
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    static std::atomic<size_t> attr{0};
    if (sm > 48 * 1024) {
        const cudaError_t e = bip_raise_once(attr, sm, [&] {
            return cudaFuncSetAttribute(diff_bin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        });
        if (e != cudaSuccess) return e;
    }
    dim3 grid((nd + kBinWarps - 1) / kBinWarps, a.n_sites);
    diff_bin_kernel<<<grid, kBinWarps * 32, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t bip_diff_eval(const DiffArgs& a, cudaStream_t s) {
    if (a.n_work == 0) return cudaSuccess;
    const size_t nd = (size_t)(2 * a.Ky + 1) * (4 * a.Kx + 1);
    const size_t sm = nd * sizeof(float2);
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    static std::atomic<size_t> attr{0};
    if (sm > 48 * 1024) {
        const cudaError_t e = bip_raise_once(attr, sm, [&] {
            return cudaFuncSetAttribute(diff_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        });
        if (e != cudaSuccess) return e;
    }
    // persistent grid: every resident block slot, at most one block per item
    static int per_sm = 0, sms = 0;
    static size_t sm_at = 0;
    int slots;
    {
        std::lock_guard<std::mutex> lk(bip_attr_mutex());
        if (per_sm == 0 || sm_at != sm) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, diff_eval_kernel, 256, sm) != cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            sm_at = sm;
        }
        slots = per_sm * sms;
    }
    const int grid = a.n_work < slots ? a.n_work : slots;
    diff_eval_kernel<<<grid, 256, sm, s>>>(a);
    return cudaGetLastError();
}
