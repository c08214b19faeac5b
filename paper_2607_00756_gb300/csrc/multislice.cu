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
// Grid lengths: powers of two 64..1024, and 3 M (192, 384, 768) through
// the radix-3 layer of the register FFT (fft_reg3).
//
// One step of a column is two passes over global memory:
//   row pass    [inverse FFT along x] [T_pre] [stash, save] [T_post] [FFT along x]
//   column pass FFT along y, times the shifted propagator, inverse FFT along y
// with T_j = exp(i sigma V_j) read from a table the build computes once per
// slice (shared by every column and both sweeps), or evaluated in-kernel
// from V (sincosf) where no table is kept.
#include <algorithm>
#include <cstdio>

#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int kThreads = 256;

// Row geometry: a row of NX = S M points (M a power of two; S = 1, or 3
// for the lengths 3 M) is held by NT = M / 8 threads, 8 S values each; a
// block of 256 threads takes RPB rows.  Value (s, m) of thread t is the
// real-space point real(s, m, t) and the frequency freq(s, m, t) (the
// layouts of fft_reg and fft_reg3).
template <int NX>
struct RowShape {
    static constexpr bool THREE = NX % 3 == 0;
    static constexpr int S = THREE ? 3 : 1;
    static constexpr int M = NX / S;
    static constexpr int NT = M / 8;
    static constexpr int RPB = kThreads / NT;
    __device__ __forceinline__ static int real(int s, int m, int t) {
        return THREE ? 3 * (t + m * NT) + s : t + m * NT;
    }
    __device__ __forceinline__ static int freq(int s, int m, int t) { return t + m * NT + s * M; }
};

// forward (INV false) or inverse transform of one row or column held as
// v[S][8], through the two exchange buffers of N entries
template <int N, bool INV>
__device__ __forceinline__ void fft_any(float2 (&v)[RowShape<N>::S][8], float2* b0, float2* b1, int& ph, int t,
                                        const float2* tw) {
    if constexpr (RowShape<N>::THREE)
        fft_reg3<RowShape<N>::M, INV>(v, b0, b1, ph, t, tw);
    else
        fft_reg<N, INV>(v[0], b0, b1, ph, t, tw);
}

// Row pass: a block takes one y and up to RPB consecutive columns, so its
// rows share the transmission exp(i sigma V(y, .)), computed once into
// shared memory.  Each row is held in registers by NT threads in the
// layouts above, so the transmission multiply and the stash act on
// registers and the row crosses shared memory only between FFT passes.
template <int NX>
__global__ void __launch_bounds__(kThreads) row_pass_kernel(MsPlan plan, MsRowArgs a) {
    using RS = RowShape<NX>;
    constexpr int NT = RS::NT, RPB = RS::RPB, S = RS::S;
    constexpr int ROWLEN = NX;
    extern __shared__ float2 smem[];
    const int sub = threadIdx.x / NT;
    const int t = threadIdx.x % NT;
    float2* b0 = smem + 2 * sub * ROWLEN;      // exchange buffers of this row
    float2* b1 = b0 + ROWLEN;
    float2* tw = smem + 2 * RPB * ROWLEN;      // [NX] pass twiddles
    float2* tt = tw + NX;                      // [NX] transmission of this y
    const int gpy = (plan.ncol + RPB - 1) / RPB;
    const int y = blockIdx.x / gpy;
    const int c = (blockIdx.x % gpy) * RPB + sub;
    const bool active = c < plan.ncol;
    float2* g = a.cols + ((size_t)(active ? c : 0) * plan.ny + y) * NX;
    const float* vsl = a.v_pre ? a.v_pre : a.v_post;

    // the row is in frequency order when it arrives for an inverse FFT,
    // in real-space order otherwise
    float2 v[S][8];
#pragma unroll
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 8; ++m)
            v[q][m] = !active ? make_float2(0.f, 0.f)
                              : a.init ? make_float2(a.init_val, 0.f)
                                       : g[a.do_ifft ? RS::freq(q, m, t) : RS::real(q, m, t)];
    for (int i = threadIdx.x; i < NX; i += kThreads) {
        tw[i] = __ldg(&plan.twx[i]);
        if (vsl) {
            if (a.t_slice) {
                tt[i] = __ldg(&a.t_slice[(size_t)y * NX + i]);
            } else {
                float sn, co;
                sincosf(plan.sigma * __ldg(&vsl[(size_t)y * NX + i]), &sn, &co);
                tt[i] = make_float2(co, sn);
            }
        }
    }
    __syncthreads();
    int ph = 0;
    if (a.do_ifft) fft_any<NX, true>(v, b0, b1, ph, t, tw);
    if (a.v_pre) {
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int m = 0; m < 8; ++m) v[q][m] = c_mul(v[q][m], tt[RS::real(q, m, t)]);
    }
    if (active && a.save) {
        float2* o = a.save + ((size_t)c * plan.ny + y) * NX;
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int m = 0; m < 8; ++m) o[RS::real(q, m, t)] = v[q][m];
    }
    if (active && a.row_off) {
        const int e1 = __ldg(&a.row_off[y + 1]);
        for (int e = __ldg(&a.row_off[y]); e < e1; ++e) {
            const int4 en = __ldg(&a.row_ent[e]);      // (site, u, ox, -)
            float2* dst = a.stash + (((size_t)en.x * plan.ncol + c) * a.win + en.y) * a.win;
#pragma unroll
            for (int q = 0; q < S; ++q)
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    int u = (RS::real(q, m, t) - en.z) % NX;   // column of this point in the window
                    if (u < 0) u += NX;
                    if (u < a.win) dst[u] = v[q][m];
                }
        }
    }
    if (a.v_post) {
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int m = 0; m < 8; ++m) v[q][m] = c_mul(v[q][m], tt[RS::real(q, m, t)]);
    }
    if (a.do_fft) fft_any<NX, false>(v, b0, b1, ph, t, tw);
    if (active) {
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int m = 0; m < 8; ++m) g[a.do_fft ? RS::freq(q, m, t) : RS::real(q, m, t)] = v[q][m];
    }
}

// Column pass geometry: XB columns per block, two adjacent columns per
// thread (16-byte loads), NT = M/8 threads per column pair (a column of
// NY = S M points, as a row of RowShape<NY>).
template <int NY>
struct ColShape {
    using RS = RowShape<NY>;
    static constexpr int NT = RS::NT;
    static constexpr int XB = RS::THREE ? (NY == 192 ? 32 : NY == 384 ? 16 : 8)
                                        : (NY <= 256 ? 512 / NT : (NY == 512 ? 16 : 8));
    static constexpr int THREADS = NT * XB / 2;
    // blocks per SM the register budget is set for: 24 values per column
    // and thread for the lengths 3 M
    static constexpr int MINB = RS::THREE ? 3 : 2048 / THREADS / 2;
};

// One exchange of col_fft: pass P of sub-column j of the two columns a, b
// of every thread through the shared [NY][XB] tile (sub-column j in rows
// j M .. j M + M - 1); column pair cp sits at 2 cp, 2 cp + 1, so a warp's
// accesses are runs of 16-byte words.
template <int M, int XB, bool INV, int P, int S>
__device__ __forceinline__ void col_fft_step(float2 (&va)[S][8], float2 (&vb)[S][8], float4* tile, int cp, int t,
                                             const float2* tw) {
    using F = FftReg<M, INV>;
    constexpr int CP = XB / 2;
    __syncthreads();                           // earlier reads of the tile are done
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
        for (int r = 0; r < 8; ++r)
            tile[(j * M + F::out_pos(P, r, t)) * CP + cp] = make_float4(va[j][r].x, va[j][r].y, vb[j][r].x, vb[j][r].y);
    __syncthreads();
    // one column at a time, to keep fewer values live
    const float2* t2 = reinterpret_cast<const float2*>(tile);
#pragma unroll
    for (int j = 0; j < S; ++j) {
        float2 u[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) u[e] = t2[2 * ((j * M + F::template in_pos<P>(e, t)) * CP + cp)];
        F::template pass<P>(u, va[j], t, tw);
#pragma unroll
        for (int e = 0; e < 8; ++e) u[e] = t2[2 * ((j * M + F::template in_pos<P>(e, t)) * CP + cp) + 1];
        F::template pass<P>(u, vb[j], t, tw);
    }
}

template <int NY, int XB, bool INV>
__device__ __forceinline__ void col_fft(float2 (&va)[RowShape<NY>::S][8], float2 (&vb)[RowShape<NY>::S][8],
                                        float4* tile, int cp, int t, const float2* tw) {
    using RS = RowShape<NY>;
    constexpr int M = RS::M, S = RS::S;
    using F = FftReg<M, INV>;
    if constexpr (RS::THREE)
        if (INV) {
            fft3_combine<M, true>(va, t, tw + M);
            fft3_combine<M, true>(vb, t, tw + M);
        }
#pragma unroll
    for (int j = 0; j < S; ++j) {
        F::first(va[j]);
        F::first(vb[j]);
    }
    col_fft_step<M, XB, INV, 1, S>(va, vb, tile, cp, t, tw);
    if constexpr (F::NPASS > 2) col_fft_step<M, XB, INV, 2, S>(va, vb, tile, cp, t, tw);
    if constexpr (F::NPASS > 3) col_fft_step<M, XB, INV, 3, S>(va, vb, tile, cp, t, tw);
    if constexpr (RS::THREE)
        if (!INV) {
            fft3_combine<M, false>(va, t, tw + M);
            fft3_combine<M, false>(vb, t, tw + M);
        }
}

// Column pass: FFT along y, times the shifted propagator, inverse FFT along
// y, for XB adjacent columns x of one parent field; every thread holds two
// adjacent columns at y = real(s, m, t) in registers.
template <int NY>
__global__ void __launch_bounds__(ColShape<NY>::THREADS, ColShape<NY>::MINB) col_pass_kernel(MsPlan plan, float2* cols) {
    using RS = RowShape<NY>;
    constexpr int XB = ColShape<NY>::XB;
    constexpr int CP = XB / 2;
    constexpr int S = RS::S;
    extern __shared__ float4 tile[];                                 // [NY][CP]
    float2* tw = reinterpret_cast<float2*>(tile + NY * CP);          // [NY] twiddles
    const int cp = threadIdx.x % CP, t = threadIdx.x / CP;
    const int c = blockIdx.y;
    const int x = blockIdx.x * XB + 2 * cp;                          // columns x, x + 1
    float2* g = cols + (size_t)c * NY * plan.nx + x;
    float2 va[S][8], vb[S][8];
#pragma unroll
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const float4 v4 = *reinterpret_cast<const float4*>(g + (size_t)RS::real(q, m, t) * plan.nx);
            va[q][m] = make_float2(v4.x, v4.y);
            vb[q][m] = make_float2(v4.z, v4.w);
        }
    for (int i = threadIdx.x; i < NY; i += ColShape<NY>::THREADS) tw[i] = __ldg(&plan.twy[i]);
    __syncthreads();
    col_fft<NY, XB, false>(va, vb, tile, cp, t, tw);
    // shifted propagator at (k_y, k_x) = (freq(s, m, t), x) and (., x + 1)
    const int2 sh = plan.shift[c];
    int kx = (x + sh.y) % plan.nx;
    if (kx < 0) kx += plan.nx;
    const float2 pxa = __ldg(&plan.px[kx]);
    const float2 pxb = __ldg(&plan.px[kx + 1 == plan.nx ? 0 : kx + 1]);
#pragma unroll
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            int iy = (RS::freq(q, m, t) + sh.x) % NY;
            if (iy < 0) iy += NY;
            const float2 py = __ldg(&plan.py[iy]);
            va[q][m] = c_mul(va[q][m], c_mul(py, pxa));
            vb[q][m] = c_mul(vb[q][m], c_mul(py, pxb));
        }
    col_fft<NY, XB, true>(va, vb, tile, cp, t, tw);
#pragma unroll
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 8; ++m)
            *reinterpret_cast<float4*>(g + (size_t)RS::real(q, m, t) * plan.nx) =
                make_float4(va[q][m].x, va[q][m].y, vb[q][m].x, vb[q][m].y);
}

__global__ void transmission_kernel(const float* __restrict__ V, float sigma, size_t n, float2* __restrict__ T) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float sn, co;
        sincosf(sigma * __ldg(&V[i]), &sn, &co);
        T[i] = make_float2(co, sn);
    }
}

template <int NX>
cudaError_t launch_row(const MsPlan& p, const MsRowArgs& a, cudaStream_t s) {
    constexpr int RPB = RowShape<NX>::RPB, ROWLEN = NX;
    const long long blocks = (long long)p.ny * ((p.ncol + RPB - 1) / RPB);
    const size_t sm = ((size_t)2 * RPB * ROWLEN + 2 * NX) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(row_pass_kernel<NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    row_pass_kernel<NX><<<(unsigned)blocks, kThreads, sm, s>>>(p, a);
    return cudaGetLastError();
}

template <int NY>
cudaError_t launch_col(const MsPlan& p, float2* cols, cudaStream_t s) {
    using C = ColShape<NY>;
    if (p.nx % C::XB != 0) return cudaErrorInvalidValue;
    const size_t sm = (size_t)NY * C::XB * sizeof(float2) + NY * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(col_pass_kernel<NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(p.nx / C::XB, p.ncol);
    col_pass_kernel<NY><<<grid, C::THREADS, sm, s>>>(p, cols);
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
        case 192: return launch_row<192>(p, a, s);
        case 384: return launch_row<384>(p, a, s);
        case 768: return launch_row<768>(p, a, s);
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
        case 192: return launch_col<192>(p, cols, s);
        case 384: return launch_col<384>(p, cols, s);
        case 768: return launch_col<768>(p, cols, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t bip_transmission(const float* V, float sigma, int j0, int j1, size_t G, float2* T, cudaStream_t s) {
    if (j1 <= j0) return cudaSuccess;
    const size_t n = (size_t)(j1 - j0) * G;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    transmission_kernel<<<blocks, 256, 0, s>>>(V + (size_t)j0 * G, sigma, n, T + (size_t)j0 * G);
    return cudaGetLastError();
}
