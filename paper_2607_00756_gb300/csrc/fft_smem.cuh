// Shared-memory Stockham FFT for power-of-two lengths 64..1024.
//
// A transform of length N is done by N/8 threads; every pass is a radix-8
// pass while at least 8 points remain per sub-transform, the last one
// radix 4 or 2.  Each thread always holds 8 values per pass (one radix-8,
// two radix-4 or four radix-2 butterflies).  Twiddles W_N^m =
// exp(-2 pi i m / N) come from a table computed on the host in FP64 and
// rounded to FP32 (kept in shared memory by the callers).  Data live in
// shared memory with one padding slot per 16 entries to spread the strided
// accesses over the banks.
#pragma once

#include <cuda_runtime.h>

#define FFT_PAD(i) ((i) + ((i) >> 4))

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 c_rot(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = a;
    a = c_add(t, b);
    b = c_sub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    float2 s02 = c_add(a0, a2), d02 = c_sub(a0, a2);
    float2 s13 = c_add(a1, a3), d13 = c_rot<INV>(c_sub(a1, a3));
    a0 = c_add(s02, s13);
    a2 = c_sub(s02, s13);
    a1 = c_add(d02, d13);
    a3 = c_sub(d02, d13);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
    // even / odd halves
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    const float h = 0.70710678118654752440f;
    // W8^1, W8^2, W8^3 (conjugated for the inverse)
    float2 t1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y))
                    : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
    float2 t2 = c_rot<INV>(o2);
    float2 t3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y))
                    : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    v[0] = c_add(e0, o0);
    v[4] = c_sub(e0, o0);
    v[1] = c_add(e1, t1);
    v[5] = c_sub(e1, t1);
    v[2] = c_add(e2, t2);
    v[6] = c_sub(e2, t2);
    v[3] = c_add(e3, t3);
    v[7] = c_sub(e3, t3);
}

// One in-place Stockham pass of radix R over `buf` (length N, padded).
// Thread t of nt = N/8 handles 8/R butterflies j = t + b*nt.
// Both __syncthreads are block-wide: every thread of the block calls this.
template <int N, int R, bool INV>
__device__ __forceinline__ void stockham_pass(float2* buf, int Ns, int t, const float2* tw) {
    constexpr int NT = N / 8;
    constexpr int NB = 8 / R;
    constexpr int STRIDE = N / R;
    float2 v[8];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * NT;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = buf[FFT_PAD(j + r * STRIDE)];
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * NT;
        const int k = j % Ns;
        if (Ns > 1) {
            const int step = k * (N / (Ns * R));
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * step];
                if (INV) w.y = -w.y;
                v[b * R + r] = c_mul(v[b * R + r], w);
            }
        }
        if (R == 8) dft8<INV>(&v[b * R]);
        if (R == 4) dft4<INV>(v[b * R], v[b * R + 1], v[b * R + 2], v[b * R + 3]);
        if (R == 2) dft2<INV>(v[b * R], v[b * R + 1]);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[FFT_PAD(base + r * Ns)] = v[b * R + r];
    }
    __syncthreads();
}

// Full transform of length N (unnormalised).  `t` in [0, N/8) is the
// thread's rank within this transform; the caller syncs before (data
// written) -- the last pass ends with a block-wide sync.
template <int N, bool INV>
__device__ __forceinline__ void fft_smem(float2* buf, int t, const float2* tw) {
    __syncthreads();
    int Ns = 1;
#pragma unroll
    for (int rem = N; rem >= 8; rem /= 8) {
        stockham_pass<N, 8, INV>(buf, Ns, t, tw);
        Ns *= 8;
    }
    constexpr int LOG = (N == 64) ? 6 : (N == 128) ? 7 : (N == 256) ? 8 : (N == 512) ? 9 : 10;
    if (LOG % 3 == 2) stockham_pass<N, 4, INV>(buf, Ns, t, tw);
    if (LOG % 3 == 1) stockham_pass<N, 2, INV>(buf, Ns, t, tw);
}

// Register-resident transform of length N by NT = N/8 threads.  Thread t
// holds x[t + m NT] in v[m] (m = 0..7) on entry and X[t + m NT] on exit:
// the first radix-8 pass reads exactly that distribution and the last pass
// writes it, so only the data between passes go through shared memory.
// Pass p works on sub-transforms of length Ns = 8^p; for p = 1..NPASS-1 a
// caller stores v at out_pos(p, r, t) (r = 0..7), synchronises, loads
// u[e] from in_pos<p>(e, t) (e = 0..7) and calls pass<p>(u, v, t, tw).
template <int N, bool INV>
struct FftReg {
    static constexpr int NT = N / 8;
    static constexpr int LOG = (N == 64) ? 6 : (N == 128) ? 7 : (N == 256) ? 8 : (N == 512) ? 9 : 10;
    static constexpr int RL = (LOG % 3 == 2) ? 4 : (LOG % 3 == 1) ? 2 : 8;   // radix of the last pass
    static constexpr int NPASS = LOG / 3 + (RL == 8 ? 0 : 1);
    template <int P>
    __host__ __device__ static constexpr int radix() { return P == NPASS - 1 ? RL : 8; }

    __device__ __forceinline__ static void first(float2 (&v)[8]) { dft8<INV>(v); }

    // where output r of pass p-1 goes (that pass has radix 8, butterfly j = t)
    __device__ __forceinline__ static int out_pos(int p, int r, int t) {
        const int Ns = 1 << (3 * (p - 1));
        return (t / Ns) * Ns * 8 + t % Ns + r * Ns;
    }
    // where input e = b R + r of pass P comes from (butterfly j = t + b NT)
    template <int P>
    __device__ __forceinline__ static int in_pos(int e, int t) {
        constexpr int R = radix<P>();
        return t + (e / R) * NT + (e % R) * (N / R);
    }
    // twiddles and butterflies of pass P; the outputs go to v in the
    // order the next pass's put expects, and for the last pass in the
    // cyclic layout: output r of butterfly b is X[t + (b + r NB) NT]
    template <int P>
    __device__ __forceinline__ static void pass(float2 (&u)[8], float2 (&v)[8], int t, const float2* tw) {
        constexpr int R = radix<P>();
        constexpr int NB = 8 / R;
        constexpr int Ns = 1 << (3 * P);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + b * NT;
            const int step = (j % Ns) * (N / (Ns * R));
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * step];
                if (INV) w.y = -w.y;
                u[b * R + r] = c_mul(u[b * R + r], w);
            }
            if (R == 8) dft8<INV>(&u[b * R]);
            if (R == 4) dft4<INV>(u[b * R], u[b * R + 1], u[b * R + 2], u[b * R + 3]);
            if (R == 2) dft2<INV>(u[b * R], u[b * R + 1]);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * NB] = u[b * R + r];
    }
};

// One exchange of fft_reg: pass P through buffer `buf` (padded).
template <int N, bool INV, int P>
__device__ __forceinline__ void fft_reg_step(float2 (&v)[8], float2* buf, int t, const float2* tw) {
    using F = FftReg<N, INV>;
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[FFT_PAD(F::out_pos(P, r, t))] = v[r];
    __syncthreads();
    float2 u[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) u[e] = buf[FFT_PAD(F::template in_pos<P>(e, t))];
    F::template pass<P>(u, v, t, tw);
}

// One transform with two alternating exchange buffers (one barrier per
// exchange).  `ph` selects the buffer of the next exchange and is carried
// across calls, so a buffer is rewritten only after a barrier that follows
// every thread's last read of it.  Every thread of the block calls this.
template <int N, bool INV>
__device__ __forceinline__ void fft_reg(float2 (&v)[8], float2* b0, float2* b1, int& ph, int t, const float2* tw) {
    using F = FftReg<N, INV>;
    F::first(v);
    fft_reg_step<N, INV, 1>(v, ph ? b1 : b0, t, tw);
    ph ^= 1;
    if constexpr (F::NPASS > 2) {
        fft_reg_step<N, INV, 2>(v, ph ? b1 : b0, t, tw);
        ph ^= 1;
    }
    if constexpr (F::NPASS > 3) {
        fft_reg_step<N, INV, 3>(v, ph ? b1 : b0, t, tw);
        ph ^= 1;
    }
}
