// Multislice sweep of the parent columns of S1 and S2 (Eq. smatrix-advance,
// Eq. s2) with the per-site window stash.
//
// Columns are propagated in the de-tilted frame: a parent h_p of S1 is
// stored as S_p(r) exp(-2 pi i h_p.r/N), which turns its spectrum into a
// cyclic shift of S_p's, so the Fresnel step multiplies by P evaluated at
// the shifted frequency index (k + h_p) mod N.  The start field is then a
// constant (1 for S1, G^{-1/2} for S2) and windows need no de-tilt phase
// when they are stashed.  S2 columns carry exp(-2 pi i h_d.r/N) and use
// the shift -h_d.  P is separable: P(q) = P_y(q_y) P_x(q_x); the tables
// hold exp(-i pi lambda dz q^2) / N per axis, which also normalises the
// unnormalised forward/inverse FFT pair.
//
// One step of a column is two passes over global memory:
//   row pass    [inverse FFT along x] [T_pre] [stash] [T_post] [FFT along x]
//   column pass FFT along y, times the shifted propagator, inverse FFT along y
// with T_j = exp(i sigma V_j) evaluated in-kernel from V (sincosf).
#include <cstdio>

#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int kThreads = 256;

template <int NX>
__global__ void __launch_bounds__(kThreads) row_pass_kernel(MsPlan plan, MsRowArgs a) {
    constexpr int NT = NX / 8;                 // threads per row
    constexpr int RPB = kThreads / NT;         // rows per block
    constexpr int ROWLEN = NX + NX / 16;       // padded
    extern __shared__ float2 smem[];
    float2* tw = smem + RPB * ROWLEN;          // [NX] twiddles
    for (int i = threadIdx.x; i < NX; i += kThreads) tw[i] = __ldg(&plan.twx[i]);
    const int sub = threadIdx.x / NT;
    const int t = threadIdx.x % NT;
    float2* row = smem + sub * ROWLEN;
    const long long pair = (long long)blockIdx.x * RPB + sub;
    const long long npairs = (long long)plan.ncol * plan.ny;
    const bool active = pair < npairs;
    // rows are ordered (y, column) so the rows of a block share V's row
    const int y = active ? (int)(pair / plan.ncol) : 0;
    const int c = active ? (int)(pair % plan.ncol) : 0;
    float2* g = a.cols + ((size_t)c * plan.ny + y) * NX;

    if (active) {
        for (int x = t; x < NX; x += NT)
            row[FFT_PAD(x)] = a.init ? make_float2(a.init_val, 0.f) : g[x];
    }
    __syncthreads();
    if (a.do_ifft) fft_smem<NX, true>(row, t, tw);

    if (active && a.v_pre) {
        const float* v = a.v_pre + (size_t)y * NX;
        for (int x = t; x < NX; x += NT) {
            float s, co;
            sincosf(plan.sigma * __ldg(&v[x]), &s, &co);
            row[FFT_PAD(x)] = c_mul(row[FFT_PAD(x)], make_float2(co, s));
        }
    }
    __syncthreads();
    if (active && a.row_off) {
        const int e1 = __ldg(&a.row_off[y + 1]);
        for (int e = __ldg(&a.row_off[y]); e < e1; ++e) {
            const int4 en = __ldg(&a.row_ent[e]);      // (site, u, ox, -)
            float2* dst = a.stash + (((size_t)en.x * plan.ncol + c) * a.win + en.y) * a.win;
            for (int v = t; v < a.win; v += NT) {
                int x = (en.z + v) % NX;
                if (x < 0) x += NX;
                dst[v] = row[FFT_PAD(x)];
            }
        }
    }
    __syncthreads();
    if (active && a.v_post) {
        const float* v = a.v_post + (size_t)y * NX;
        for (int x = t; x < NX; x += NT) {
            float s, co;
            sincosf(plan.sigma * __ldg(&v[x]), &s, &co);
            row[FFT_PAD(x)] = c_mul(row[FFT_PAD(x)], make_float2(co, s));
        }
    }
    if (a.do_fft) fft_smem<NX, false>(row, t, tw);
    else __syncthreads();
    if (active) {
        for (int x = t; x < NX; x += NT) g[x] = row[FFT_PAD(x)];
    }
}

template <int NY>
__global__ void __launch_bounds__(kThreads) col_pass_kernel(MsPlan plan, float2* cols) {
    constexpr int NT = NY / 8;                  // threads per column FFT
    constexpr int NPAR = kThreads / NT;         // column FFTs in parallel
    constexpr int XB = NPAR > 16 ? NPAR : 16;   // x columns per block
    constexpr int COLLEN = NY + NY / 16 + 1;    // padded, odd stride
    extern __shared__ float2 smem[];
    float2* tw = smem + XB * COLLEN;            // [NY] twiddles
    for (int i = threadIdx.x; i < NY; i += kThreads) tw[i] = __ldg(&plan.twy[i]);
    const int c = blockIdx.y;
    const int x0 = blockIdx.x * XB;
    float2* g = cols + (size_t)c * NY * plan.nx;
    for (int i = threadIdx.x; i < NY * XB; i += kThreads) {
        const int y = i / XB, xx = i % XB;
        smem[xx * COLLEN + FFT_PAD(y)] = g[(size_t)y * plan.nx + x0 + xx];
    }
    const int2 sh = plan.shift[c];
    const int sub = threadIdx.x / NT;
    const int t = threadIdx.x % NT;
    for (int grp = 0; grp < XB; grp += NPAR) {
        const int xx = grp + sub;
        float2* col = smem + xx * COLLEN;
        fft_smem<NY, false>(col, t, tw);
        // shifted propagator at (k_y, k_x = x0 + xx)
        int kx = (x0 + xx + sh.y) % plan.nx;
        if (kx < 0) kx += plan.nx;
        const float2 px = __ldg(&plan.px[kx]);
        for (int ky = t; ky < NY; ky += NT) {
            int iy = (ky + sh.x) % NY;
            if (iy < 0) iy += NY;
            const float2 p = c_mul(__ldg(&plan.py[iy]), px);
            col[FFT_PAD(ky)] = c_mul(col[FFT_PAD(ky)], p);
        }
        fft_smem<NY, true>(col, t, tw);
    }
    for (int i = threadIdx.x; i < NY * XB; i += kThreads) {
        const int y = i / XB, xx = i % XB;
        g[(size_t)y * plan.nx + x0 + xx] = smem[xx * COLLEN + FFT_PAD(y)];
    }
}

template <int NX>
cudaError_t launch_row(const MsPlan& p, const MsRowArgs& a, cudaStream_t s) {
    constexpr int NT = NX / 8, RPB = kThreads / NT, ROWLEN = NX + NX / 16;
    const long long npairs = (long long)p.ncol * p.ny;
    const int blocks = (int)((npairs + RPB - 1) / RPB);
    const size_t sm = ((size_t)RPB * ROWLEN + NX) * sizeof(float2);
    row_pass_kernel<NX><<<blocks, kThreads, sm, s>>>(p, a);
    return cudaGetLastError();
}

template <int NY>
cudaError_t launch_col(const MsPlan& p, float2* cols, cudaStream_t s) {
    constexpr int NT = NY / 8, NPAR = kThreads / NT, XB = NPAR > 16 ? NPAR : 16;
    constexpr int COLLEN = NY + NY / 16 + 1;
    const size_t sm = ((size_t)XB * COLLEN + NY) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(col_pass_kernel<NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    dim3 grid(p.nx / XB, p.ncol);
    col_pass_kernel<NY><<<grid, kThreads, sm, s>>>(p, cols);
    return cudaGetLastError();
}

}  // namespace

cudaError_t bip_ms_row_pass(const MsPlan& p, const MsRowArgs& a, cudaStream_t s) {
    switch (p.nx) {
        case 64: return launch_row<64>(p, a, s);
        case 128: return launch_row<128>(p, a, s);
        case 256: return launch_row<256>(p, a, s);
        case 512: return launch_row<512>(p, a, s);
        case 1024: return launch_row<1024>(p, a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t bip_ms_col_pass(const MsPlan& p, float2* cols, cudaStream_t s) {
    switch (p.ny) {
        case 64: return launch_col<64>(p, cols, s);
        case 128: return launch_col<128>(p, cols, s);
        case 256: return launch_col<256>(p, cols, s);
        case 512: return launch_col<512>(p, cols, s);
        case 1024: return launch_col<1024>(p, cols, s);
        default: return cudaErrorInvalidValue;
    }
}
