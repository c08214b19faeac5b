// Reverse pass of a map loss through the contraction (the matrices as a
// forward model, Sec. 5): given g(rho) = dL/dI(rho), the derivatives with
// respect to the site occupancies, the transition potentials H and the
// probe aberrations.  FP32 SIMT kernels; per site tau, f = f_y f_x:
//   R_tau     = f o_tau sum_{rho in crop} g(rho) c(rho) c(rho)^H     [B x B]
//   Mbar_n    = M_n R_tau            (stored as GMt = conj(R) Mt, Mt[b][(n, d)])
//   T_n(b, r) = sum_d Mbar_n(d, b) conj S2_d(r)
//   dL/dH_n(r) (as dL/dRe + i dL/dIm) = 2 sum_b conj S1_b(r) T_n(b, r)
//   D_b      += (Q_tau R_tau)_bb,  dL/dtheta = -2 sum_b chi'_b Im D_b
//   dL/do_tau = sum_rho g(rho) I_tau(rho)
//
//   cgemm_gen_kernel : C(m, n) (+)= sum_k opA(A(m, k) s_k) opB(B(k, n)),
//                      arbitrary strides, batched, 64 x 64 tiles
//   crop_weight_kernel, hgrad_kernel, aberr_kernel, aberr_sum_kernel,
//   occ_grad_kernel
#include "bip_device.cuh"
#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int kTile = 64, kKt = 16, kThreads = 256;

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

__global__ void __launch_bounds__(kThreads) cgemm_gen_kernel(CGemmGen a) {
    __shared__ float2 As[kKt][kTile + 1];
    __shared__ float2 Bs[kKt][kTile + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile, z = blockIdx.z;
    const float2* A = a.A + (int64_t)z * a.sab;
    const float2* B = a.B + (int64_t)z * a.sbb;
    const float* dk = a.dk ? a.dk + (int64_t)z * a.sdb : nullptr;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < a.K; k0 += kKt) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int idx = threadIdx.x + l * kThreads;
            // the unit-stride axis runs fastest across the threads
            int m, k;
            if (a.sam == 1) { m = idx % kTile; k = idx / kTile; } else { k = idx % kKt; m = idx / kKt; }
            float2 v = make_float2(0.f, 0.f);
            if (m0 + m < a.M && k0 + k < a.K) {
                v = A[(int64_t)(m0 + m) * a.sam + (int64_t)(k0 + k) * a.sak];
                if (a.conjA) v.y = -v.y;
                if (dk) {
                    const float s = dk[k0 + k];
                    v.x *= s;
                    v.y *= s;
                }
            }
            As[k][m] = v;
            int n;
            if (a.sbn == 1) { n = idx % kTile; k = idx / kTile; } else { k = idx % kKt; n = idx / kKt; }
            float2 w = make_float2(0.f, 0.f);
            if (n0 + n < a.N && k0 + k < a.K) {
                w = B[(int64_t)(k0 + k) * a.sbk + (int64_t)(n0 + n) * a.sbn];
                if (a.conjB) w.y = -w.y;
            }
            Bs[k][n] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKt; ++k) {
            float2 av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(av[i].x, bv[j].x, fmaf(-av[i].y, bv[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(av[i].x, bv[j].y, fmaf(av[i].y, bv[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
    float2* C = a.C + (int64_t)z * a.scb;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= a.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= a.N) continue;
            float2* o = C + (int64_t)m * a.scm + (int64_t)n * a.scn;
            if (a.accumulate) {
                const float2 p = *o;
                *o = make_float2(p.x + acc[i][j].x, p.y + acc[i][j].y);
            } else {
                *o = acc[i][j];
            }
        }
    }
}

// w[bs][rho] = f o_tau g(rho) inside the site's crop window, else 0
__global__ void crop_weight_kernel(GradArgs a, int nb, const int32_t* ids, float* w) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x, bs = blockIdx.y;
    if (p >= a.P) return;
    const int site = ids[bs];
    const SiteDev st = a.sites[site];
    float v = 0.f;
    if (in_crop(a.scans[2 * p], a.scans[2 * p + 1], st.ty, st.tx, a.ny, a.nx, a.fy, a.fx)) {
        const double o = a.occ ? a.occ[site] : 1.0;
        v = (float)(a.scale * o * a.dL_dI[p]);
    }
    w[(size_t)bs * a.P + p] = v;
}

// dL/dH_n(r) = 2 sum_b conj S1_b(r) T_n(b, r); thread = pixel, block row =
// (site, channel)
__global__ void hgrad_kernel(GradArgs a, const int32_t* ids, const float2* S1, int64_t s1_site, const float2* T,
                             int64_t t_site, int64_t t_ch, float2* dH) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int bs = blockIdx.y, n = blockIdx.z;
    if (r >= a.K) return;
    const SiteDev st = a.sites[ids[bs]];
    if (n >= st.nch) return;
    const float2* s1 = S1 + (int64_t)bs * s1_site + r;
    const float2* t = T + (int64_t)bs * t_site + (int64_t)n * t_ch + r;
    float2 acc = make_float2(0.f, 0.f);
    for (int b = 0; b < a.B; ++b) {
        const float2 x = conjf2(__ldg(&s1[(int64_t)b * a.K]));
        const float2 y = __ldg(&t[(int64_t)b * a.K]);
        acc.x = fmaf(x.x, y.x, fmaf(-x.y, y.y, acc.x));
        acc.y = fmaf(x.x, y.y, fmaf(x.y, y.x, acc.y));
    }
    dH[(size_t)st.h_off + (size_t)n * a.K + r] = make_float2(2.f * acc.x, 2.f * acc.y);
}

// D[bs][b] = sum_b' Q[b][b'] R[b'][b]
__global__ void aberr_kernel(int B, int Bpad, const float2* Q, int64_t q_site, const float2* R, int64_t r_site,
                             double2* D) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x, bs = blockIdx.y;
    if (b >= B) return;
    const float2* q = Q + (int64_t)bs * q_site + (int64_t)b * Bpad;
    const float2* rr = R + (int64_t)bs * r_site + b;
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < B; ++k) {
        const float2 x = q[k], y = rr[(int64_t)k * Bpad];
        sx += (double)x.x * y.x - (double)x.y * y.y;
        sy += (double)x.x * y.y + (double)x.y * y.x;
    }
    D[(size_t)bs * B + b] = make_double2(sx, sy);
}

// Dsum[b] += sum over the batch's sites of D[bs][b], in site order
__global__ void aberr_sum_kernel(int B, int nb, const double2* D, double2* Dsum) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double2 s = Dsum[b];
    for (int bs = 0; bs < nb; ++bs) {
        s.x += D[(size_t)bs * B + b].x;
        s.y += D[(size_t)bs * B + b].y;
    }
    Dsum[b] = s;
}

// dL/do_tau = sum_rho g(rho) I_tau(rho); block per site
__global__ void occ_grad_kernel(const float* partial, int P, const double* g, double* out) {
    __shared__ double red[kThreads / 32];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int p = threadIdx.x; p < P; p += kThreads) s += g[p] * (double)partial[(size_t)k * P + p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        out[k] = t;
    }
}

// split into BF16 hi + lo, tile = 32 x 32 of the destination (i, k)
__device__ __forceinline__ uint16_t bf16_rn_u(float x) {
    uint32_t u = __float_as_uint(x);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

__global__ void split_planes_kernel(SplitArgs a) {
    __shared__ float2 tile[32][33];
    const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32, z = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;           // 32 x 8
    const float2* src = a.src + (int64_t)z * a.s_batch;
    // read with the source's contiguous axis across the lanes
    for (int r = ty; r < 32; r += 8) {
        int i, k;
        if (a.s_col == 1) { i = i0 + r; k = k0 + tx; } else { i = i0 + tx; k = k0 + r; }
        float2 v = make_float2(0.f, 0.f);
        if (i < a.rows && k < a.cols) v = __ldg(&src[(int64_t)i * a.s_row + (int64_t)k * a.s_col]);
        if (a.conj) v.y = -v.y;
        if (a.s_col == 1) tile[r][tx] = v; else tile[tx][r] = v;
    }
    __syncthreads();
    const int64_t plane = (int64_t)a.d_rows * a.d_cols;
    uint16_t* dst = a.dst + (int64_t)z * a.d_batch;
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, k = k0 + tx;
        if (i >= a.rows || k >= a.cols) continue;
        const float2 v = tile[r][tx];
        const uint16_t rh = bf16_rn_u(v.x), ih = bf16_rn_u(v.y);
        const uint16_t rl = bf16_rn_u(v.x - __uint_as_float((uint32_t)rh << 16));
        const uint16_t il = bf16_rn_u(v.y - __uint_as_float((uint32_t)ih << 16));
        const int64_t o = (int64_t)i * a.d_cols + a.dcol0 + k;
        dst[o] = rh;
        dst[o + plane] = rl;
        dst[o + 2 * plane] = ih;
        dst[o + 3 * plane] = il;
    }
}

}  // namespace

cudaError_t bip_split_planes(const SplitArgs& a, cudaStream_t s) {
    if (a.rows < 1 || a.cols < 1 || a.batch < 1 || a.rows > a.d_rows || a.dcol0 + a.cols > a.d_cols)
        return cudaErrorInvalidValue;
    if (a.s_col != 1 && a.s_row != 1) return cudaErrorInvalidValue;
    const dim3 grid((a.cols + 31) / 32, (a.rows + 31) / 32, a.batch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    split_planes_kernel<<<grid, dim3(32, 8), 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t bip_cgemm_gen(const CGemmGen& a, cudaStream_t s) {
    if (a.M < 1 || a.N < 1 || a.K < 1 || a.batch < 1) return cudaErrorInvalidValue;
    const dim3 grid((a.N + kTile - 1) / kTile, (a.M + kTile - 1) / kTile, a.batch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    cgemm_gen_kernel<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t bip_grad_crop_weights(const GradArgs& a, int nb, const int32_t* ids, float* w, cudaStream_t s) {
    if (nb < 1 || a.P < 1) return cudaErrorInvalidValue;
    crop_weight_kernel<<<dim3((a.P + 255) / 256, nb), 256, 0, s>>>(a, nb, ids, w);
    return cudaGetLastError();
}

cudaError_t bip_grad_h(const GradArgs& a, int nb, const int32_t* ids, int nch, const float2* S1, int64_t s1_site,
                       const float2* T, int64_t t_site, int64_t t_ch, float2* dH, cudaStream_t s) {
    if (nb < 1 || nch < 1 || nch > 9) return cudaErrorInvalidValue;
    hgrad_kernel<<<dim3((a.K + 255) / 256, nb, nch), 256, 0, s>>>(a, ids, S1, s1_site, T, t_site, t_ch, dH);
    return cudaGetLastError();
}

cudaError_t bip_grad_aberr(int B, int Bpad, int nb, const float2* Q, int64_t q_site, const float2* R, int64_t r_site,
                           double2* D, double2* Dsum, cudaStream_t s) {
    if (nb < 1 || B < 1) return cudaErrorInvalidValue;
    aberr_kernel<<<dim3((B + 127) / 128, nb), 128, 0, s>>>(B, Bpad, Q, q_site, R, r_site, D);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    aberr_sum_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, nb, D, Dsum);
    return cudaGetLastError();
}

cudaError_t bip_grad_occ(const float* partial, int n_sites, int P, const double* g, double* out, cudaStream_t s) {
    if (n_sites < 1) return cudaSuccess;
    occ_grad_kernel<<<n_sites, kThreads, 0, s>>>(partial, P, g, out);
    return cudaGetLastError();
}
