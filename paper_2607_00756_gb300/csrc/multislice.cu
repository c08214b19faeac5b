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
// the radix-3 layer of the register FFT (fft_reg3).  Rows of 512 points
// (the paper-scale grids) take a two-pass form on half-warps when the plan
// carries its twiddle table (row_pass_hw512_kernel).
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
    if (a.row_off) {
        // the stash: the row staged in real-space order in an exchange
        // buffer, then each window crossing row y -- the same entries for
        // every row of the block -- copied from there by the row's threads,
        // NT consecutive pixels per store.  Entries (site, u, ox) are read one
        // per lane and passed round the warp.  The staging buffer is the one
        // the next transform writes only after its first barrier (buffer
        // ph ^ 1); the barrier before staging ends the inverse transform's
        // last reads of it.
        const int e0 = __ldg(&a.row_off[y]), e1 = __ldg(&a.row_off[y + 1]);
        if (e1 > e0) {
            float2* rowbuf = ph ? b0 : b1;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < S; ++q)
#pragma unroll
                for (int m = 0; m < 8; ++m) rowbuf[RS::real(q, m, t)] = v[q][m];
            __syncthreads();
            const int lane = threadIdx.x & 31;
            for (int base = e0; base < e1; base += 32) {
                int4 ent = make_int4(0, 0, 0, 0);
                if (base + lane < e1) ent = __ldg(&a.row_ent[base + lane]);
                const int cnt = min(32, e1 - base);
                for (int k = 0; k < cnt; ++k) {
                    const int site = __shfl_sync(0xffffffffu, ent.x, k);
                    const int wu = __shfl_sync(0xffffffffu, ent.y, k);
                    int ox = __shfl_sync(0xffffffffu, ent.z, k) % NX;
                    if (ox < 0) ox += NX;
                    if (active) {
                        float2* dst = a.stash + (((size_t)site * plan.ncol + c) * a.win + wu) * a.win;
                        for (int u = t; u < a.win; u += NT) {
                            int x = ox + u;
                            if (x >= NX) x -= NX;
                            dst[u] = rowbuf[x];
                        }
                    }
                }
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

// ---------------------------------------------------------------------------
// Rows of 512 points on half-warps.  512 = 32 x 16, so a transform is two
// register passes with one exchange between them: pass 1 a DFT-32 per
// thread over x[t + 16 m] (m = 0..31), pass 2 two DFT-16 per thread, each
// after a twiddle by exp(-+2 pi i e j / 512).  Sixteen threads hold a row in
// the cyclic layout x = t + 16 m in both domains, so the row never leaves
// its half-warp: the exchange needs __syncwarp only, and against the
// radix-8 form above it moves every value through shared memory once per
// transform instead of twice and reads half the twiddles.  A block of 256
// threads takes 16 parent columns at one y.
//
// Local DFTs of length L = 4 B (B = 8 or 4), natural order in and out:
// with n = n1 + 4 n2 and k = B k1 + k2, a DFT-B over n2 for each n1, the
// twiddle W_L^(n1 k2), then a DFT-4 over n1 for each k2.
namespace hw512 {

constexpr int N = 512, NT = 16, NV = 32;
constexpr int RPB = kThreads / NT;                 // rows (parent columns) per block
constexpr int ROWBUF = N + N / 32;                 // exchange entries per row: one pad per 32
constexpr int NTW = 15 * 32;                       // pass-2 twiddles [e - 1][j]

// exp(-2 pi i m / 32)
__constant__ float2 kW32[32] = {
    {1.0f, 0.0f}, {0.9807852506637573f, -0.19509032368659973f}, {0.9238795042037964f, -0.3826834261417389f},
    {0.8314695954322815f, -0.5555702447891235f}, {0.7071067690849304f, -0.7071067690849304f},
    {0.5555702447891235f, -0.8314695954322815f}, {0.3826834261417389f, -0.9238795042037964f},
    {0.19509032368659973f, -0.9807852506637573f}, {0.0f, -1.0f}, {-0.19509032368659973f, -0.9807852506637573f},
    {-0.3826834261417389f, -0.9238795042037964f}, {-0.5555702447891235f, -0.8314695954322815f},
    {-0.7071067690849304f, -0.7071067690849304f}, {-0.8314695954322815f, -0.5555702447891235f},
    {-0.9238795042037964f, -0.3826834261417389f}, {-0.9807852506637573f, -0.19509032368659973f}, {-1.0f, 0.0f},
    {-0.9807852506637573f, 0.19509032368659973f}, {-0.9238795042037964f, 0.3826834261417389f},
    {-0.8314695954322815f, 0.5555702447891235f}, {-0.7071067690849304f, 0.7071067690849304f},
    {-0.5555702447891235f, 0.8314695954322815f}, {-0.3826834261417389f, 0.9238795042037964f},
    {-0.19509032368659973f, 0.9807852506637573f}, {0.0f, 1.0f}, {0.19509032368659973f, 0.9807852506637573f},
    {0.3826834261417389f, 0.9238795042037964f}, {0.5555702447891235f, 0.8314695954322815f},
    {0.7071067690849304f, 0.7071067690849304f}, {0.8314695954322815f, 0.5555702447891235f},
    {0.9238795042037964f, 0.3826834261417389f}, {0.9807852506637573f, 0.19509032368659973f}};

// a W32^m (conjugate for the inverse); m is a constant after unrolling, so
// the branches fold and the quarter turns cost no multiply
template <bool INV>
__device__ __forceinline__ float2 tw32(float2 a, int m) {
    m &= 31;
    if (m == 0) return a;
    if (m == 8) return c_rot<INV>(a);
    if (m == 16) return make_float2(-a.x, -a.y);
    if (m == 24) return c_rot<!INV>(a);
    float2 w = kW32[m];
    if (INV) w.y = -w.y;
    return c_mul(a, w);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2 (&u)[16]) {
    float2 b[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) b[n1][n2] = u[n1 + 4 * n2];
        dft4<INV>(b[n1][0], b[n1][1], b[n1][2], b[n1][3]);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) b[n1][k2] = tw32<INV>(b[n1][k2], 2 * n1 * k2);
    }
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        dft4<INV>(b[0][k2], b[1][k2], b[2][k2], b[3][k2]);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) u[4 * k1 + k2] = b[k1][k2];
    }
}

template <bool INV>
__device__ __forceinline__ void dft32(float2 (&v)[NV]) {
    float2 b[4][8];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) b[n1][n2] = v[n1 + 4 * n2];
        dft8<INV>(b[n1]);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) b[n1][k2] = tw32<INV>(b[n1][k2], n1 * k2);
    }
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        dft4<INV>(b[0][k2], b[1][k2], b[2][k2], b[3][k2]);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) v[8 * k1 + k2] = b[k1][k2];
    }
}

// One length-512 transform of the row held by this half-warp (thread t:
// v[m] = x[t + 16 m] on entry, X[t + 16 m] on exit; unnormalised inverse).
// buf: this row's exchange buffer (entry i at i + i / 32); tw2: the pass-2
// twiddles exp(-2 pi i e j / 512) at (e - 1) 32 + j.  Every lane of the warp
// calls it (the warp's two rows together).
template <bool INV>
__device__ __forceinline__ void fft512(float2 (&v)[NV], float2* buf, int t, const float2* tw2) {
    dft32<INV>(v);
    // pass-1 output r of butterfly t is y[32 t + r]
#pragma unroll
    for (int r = 0; r < 32; ++r) buf[33 * t + r] = v[r];
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = t + 16 * h;                  // pass-2 butterfly: y[j + 32 e], e < 16
        float2 u[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = buf[j + 33 * e];
#pragma unroll
        for (int e = 1; e < 16; ++e) {
            float2 w = tw2[(e - 1) * 32 + j];
            if (INV) w.y = -w.y;
            u[e] = c_mul(u[e], w);
        }
        dft16<INV>(u);
        // output r is X[j + 32 r] = X[t + 16 (2 r + h)]
#pragma unroll
        for (int r = 0; r < 16; ++r) v[2 * r + h] = u[r];
    }
    __syncwarp();                                  // reads done before the buffer is reused
}

}  // namespace hw512

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The row pass of row_pass_kernel<512> on half-warp rows (same arguments,
// same results up to rounding order), persistent over the grid rows: block
// b keeps the column group b % groups and takes the rows y = b / groups,
// + blocks / groups, ...  While a half-warp stores its row it already copies
// its next row into its exchange buffer (idle between transforms) with
// cp.async, and the block copies the next row's transmission into the
// other of two T buffers, so the loads of one row overlap the work of the
// previous one.
__global__ void __launch_bounds__(kThreads, 2) row_pass_hw512_kernel(MsPlan plan, MsRowArgs a, int groups) {
    using namespace hw512;
    extern __shared__ float2 smem[];
    const int sub = threadIdx.x / NT;
    const int t = threadIdx.x % NT;
    float2* buf = smem + sub * ROWBUF;
    float2* tw2 = smem + RPB * ROWBUF;             // [15][32]
    float2* tts = tw2 + NTW;                       // [2][512] transmission of the current / next y
    const int cg = blockIdx.x % groups;
    const int ystep = gridDim.x / groups;          // the launch makes gridDim.x a multiple of groups
    const int c = cg * RPB + sub;
    const bool active = c < plan.ncol;
    const float* vsl = a.v_pre ? a.v_pre : a.v_post;
    const bool table = vsl && a.t_slice;           // T copied from the build's table
    const bool load = active && !a.init;
    float2* gcol = a.cols + (size_t)(active ? c : 0) * plan.ny * N;

    // copies of row y: this half-warp's row into buf (unpadded), the T row
    // into tts[slot]
    auto prefetch = [&](int y, int slot) {
        if (load) {
            const float2* src = gcol + (size_t)y * N;
#pragma unroll
            for (int k = 0; k < 16; ++k) cp_async16(buf + 2 * (t + 16 * k), src + 2 * (t + 16 * k));
        }
        if (table) cp_async16(tts + slot * N + 2 * threadIdx.x, a.t_slice + (size_t)y * N + 2 * threadIdx.x);
        cp_async_commit();
    };

    // windows crossing row y: entries row_off[y] .. row_off[y + 1] - 1 (the
    // same for every column), read one row ahead
    auto entries = [&](int yy, int& o0, int& o1) {
        o0 = o1 = 0;
        if (a.row_off && yy < plan.ny) {
            o0 = __ldg(&a.row_off[yy]);
            o1 = __ldg(&a.row_off[yy + 1]);
        }
    };

    for (int i = threadIdx.x; i < NTW; i += kThreads) tw2[i] = __ldg(&plan.tw512[i]);
    int y = blockIdx.x / groups;
    int slot = 0;
    int e0, e1;
    entries(y, e0, e1);
    if (y < plan.ny) prefetch(y, 0);
    for (; y < plan.ny; y += ystep, slot ^= 1) {
        float2* tt = tts + slot * N;
        // the first 16 entries, one per lane, in flight during the inverse transform
        int4 ent = make_int4(0, 0, 0, 0);
        if (e0 + t < e1) ent = __ldg(&a.row_ent[e0 + t]);
        if (vsl && !a.t_slice) {
            for (int i = threadIdx.x; i < N; i += kThreads) {
                float sn, co;
                sincosf(plan.sigma * __ldg(&vsl[(size_t)y * N + i]), &sn, &co);
                tt[i] = make_float2(co, sn);
            }
        }
        cp_async_wait_all();
        __syncthreads();                           // every copy of this row and its T is visible
        float2 v[NV];
#pragma unroll
        for (int m = 0; m < NV; ++m)
            v[m] = !active ? make_float2(0.f, 0.f) : a.init ? make_float2(a.init_val, 0.f) : buf[t + NT * m];
        __syncwarp();                              // the row is in registers before buf is reused
        if (a.do_ifft) fft512<true>(v, buf, t, tw2);
        if (a.v_pre) {
#pragma unroll
            for (int m = 0; m < NV; ++m) v[m] = c_mul(v[m], tt[t + NT * m]);
        }
        if (active && a.save) {
            float2* o = a.save + ((size_t)c * plan.ny + y) * N;
#pragma unroll
            for (int m = 0; m < NV; ++m) o[t + NT * m] = v[m];
        }
        if (e1 > e0) {
            // the stash: the row in buf (free between the transforms), then each
            // crossing window's segment x = ox .. ox + win - 1 (wrapped) copied
            // from there, 16 consecutive pixels per store; entries (site, u, ox)
            // are read one per lane and passed round the half-warp
#pragma unroll
            for (int m = 0; m < NV; ++m) buf[t + NT * m] = v[m];
            __syncwarp();
            for (int base = e0; base < e1; base += NT) {
                if (base > e0) {
                    ent = make_int4(0, 0, 0, 0);
                    if (base + t < e1) ent = __ldg(&a.row_ent[base + t]);
                }
                const int cnt = min(NT, e1 - base);
                for (int k = 0; k < cnt; ++k) {
                    const int site = __shfl_sync(0xffffffffu, ent.x, k, NT);
                    const int wu = __shfl_sync(0xffffffffu, ent.y, k, NT);
                    const int ox = __shfl_sync(0xffffffffu, ent.z, k, NT);
                    if (active) {
                        float2* dst = a.stash + (((size_t)site * plan.ncol + c) * a.win + wu) * a.win;
                        for (int u = t; u < a.win; u += NT) dst[u] = buf[(ox + u) & (N - 1)];
                    }
                }
            }
            __syncwarp();                          // buf's reads are done before the transform
        }
        if (a.v_post) {
#pragma unroll
            for (int m = 0; m < NV; ++m) v[m] = c_mul(v[m], tt[t + NT * m]);
        }
        if (a.do_fft) fft512<false>(v, buf, t, tw2);
        __syncwarp();                              // buf's last reads are done
        entries(y + ystep, e0, e1);
        if (y + ystep < plan.ny) prefetch(y + ystep, slot ^ 1);
        if (active) {
            float2* g = gcol + (size_t)y * N;
#pragma unroll
            for (int m = 0; m < NV; ++m) g[t + NT * m] = v[m];
        }
    }
    cp_async_wait_all();
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
    static std::atomic<bool> attr{false};
    const cudaError_t e = bip_set_once(attr, [&] {
        return cudaFuncSetAttribute(row_pass_kernel<NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    });
    if (e != cudaSuccess) return e;
    row_pass_kernel<NX><<<(unsigned)blocks, kThreads, sm, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_row_hw512(const MsPlan& p, const MsRowArgs& a, cudaStream_t s) {
    using namespace hw512;
    const int groups = (p.ncol + RPB - 1) / RPB;
    const size_t sm = ((size_t)RPB * ROWBUF + NTW + 2 * N) * sizeof(float2);
    static std::atomic<bool> attr{false};
    static int per_sm = 0, sms = 0;              // written once, before attr is set
    const cudaError_t e0 = bip_set_once(attr, [&] {
        cudaError_t e = cudaFuncSetAttribute(row_pass_hw512_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        int dev = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, row_pass_hw512_kernel, kThreads, sm);
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
        return e;
    });
    if (e0 != cudaSuccess) return e0;
    // persistent: whole rounds of the resident blocks, a multiple of the
    // column groups, at most one block per (group, y)
    long long blocks = (long long)sms * per_sm / groups * groups;
    if (blocks < groups) blocks = groups;
    if (blocks > (long long)groups * p.ny) blocks = (long long)groups * p.ny;
    row_pass_hw512_kernel<<<(unsigned)blocks, kThreads, sm, s>>>(p, a, groups);
    return cudaGetLastError();
}

template <int NY>
cudaError_t launch_col(const MsPlan& p, float2* cols, cudaStream_t s) {
    using C = ColShape<NY>;
    if (p.nx % C::XB != 0) return cudaErrorInvalidValue;
    const size_t sm = (size_t)NY * C::XB * sizeof(float2) + NY * sizeof(float2);
    static std::atomic<bool> attr{false};
    const cudaError_t e = bip_set_once(attr, [&] {
        return cudaFuncSetAttribute(col_pass_kernel<NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    });
    if (e != cudaSuccess) return e;
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
        case 512: return p.tw512 ? launch_row_hw512(p, a, s) : launch_row<512>(p, a, s);
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
