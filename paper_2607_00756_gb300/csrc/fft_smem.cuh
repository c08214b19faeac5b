// Register-resident radix-8 Stockham FFT for power-of-two lengths 64..1024.
//
// A transform of length N is done by N/8 threads, each holding 8 values.
// Every pass is a radix-8 pass while at least 8 points remain per
// sub-transform, the last one radix 4 or 2.  The first pass reads and the
// last pass writes the cyclic distribution x[t + m N/8] (thread t, value
// m), so data cross shared memory only between passes.  Twiddles come from
// a table computed on the host in FP64 and rounded to FP32, laid out pass by
// pass so that the threads of a warp read consecutive entries.
#pragma once

#include <cuda_runtime.h>

// Exchange-buffer index: an XOR swizzle inside each 16-entry (128-byte)
// row that keeps both the strided writes and the contiguous reads of every
// pass free of shared-memory bank conflicts (bits 4-6 of the index are
// folded into bits 0-3; it permutes each aligned group of 16).
#define FFT_SWZ(i) ((i) ^ (((i) >> 4) & 7) ^ ((((i) >> 6) & 1) << 3))
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

// Transform of length N by NT = N/8 threads.  Thread t holds x[t + m NT]
// in v[m] (m = 0..7) on entry and X[t + m NT] on exit.  Pass p combines
// sub-transforms of length Ns = 8^p; for p = 1..NPASS-1 a caller stores v
// at out_pos(p, r, t) (r = 0..7), synchronises, loads u[e] from
// in_pos<p>(e, t) (e = 0..7) and calls pass<p>(u, v, t, tw).  The twiddle
// table holds, for each such pass in turn, entry (r - 1) Ns + k =
// exp(-2 pi i r k / (Ns R)), r = 1..R-1, k < Ns (R the pass's radix).
template <int N, bool INV>
struct FftReg {
    static constexpr int NT = N / 8;
    static constexpr int LOG = (N == 64) ? 6 : (N == 128) ? 7 : (N == 256) ? 8 : (N == 512) ? 9 : 10;
    static constexpr int RL = (LOG % 3 == 2) ? 4 : (LOG % 3 == 1) ? 2 : 8;   // radix of the last pass
    static constexpr int NPASS = LOG / 3 + (RL == 8 ? 0 : 1);
    template <int P>
    __host__ __device__ static constexpr int radix() { return P == NPASS - 1 ? RL : 8; }
    // start of pass P's twiddles in the table
    template <int P>
    __host__ __device__ static constexpr int tw_off() {
        if constexpr (P <= 1) return 0;
        else return tw_off<P - 1>() + (radix<P - 1>() - 1) * (1 << (3 * (P - 1)));
    }

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
            const int k = (t + b * NT) % Ns;
            const float2* twp = tw + tw_off<P>() + k;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = twp[(r - 1) * Ns];
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

// One exchange of fft_reg: pass P through buffer `buf` (N entries, swizzled).
template <int N, bool INV, int P>
__device__ __forceinline__ void fft_reg_step(float2 (&v)[8], float2* buf, int t, const float2* tw) {
    using F = FftReg<N, INV>;
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[FFT_SWZ(F::out_pos(P, r, t))] = v[r];
    __syncthreads();
    float2 u[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) u[e] = buf[FFT_SWZ(F::template in_pos<P>(e, t))];
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

// ---------------------------------------------------------------------------
// Length N = 3 M (M a power of two, 64..256): decimation in time by 3.  The
// three interleaved subsequences x[3 p + j] (j = 0, 1, 2) are transformed as
// three length-M transforms on the same threads, in lockstep through one
// exchange buffer of N entries (region j M .. j M + M - 1 for sub-transform
// j), then combined by a radix-3 step:
//   X[k + l M] = sum_j exp(-2 pi i j k / N) exp(-2 pi i j l / 3) Y_j[k].
// Thread t (NT = M / 8 of them) holds x[3 (t + m NT) + j] in v[j][m] on entry
// and X[t + m NT + l M] in v[l][m] on exit; the inverse transform (no 1/N)
// goes the other way.  Its twiddle table holds the length-M table and then
// exp(-2 pi i j k / N) for j = 1, 2 and k < M ([2][M]): N entries in all.

// radix-3 butterfly in place: (a0, a1, a2) -> sum_j a_j W^(j l), W = exp(-+2 pi i / 3)
template <bool INV>
__device__ __forceinline__ void dft3(float2& a0, float2& a1, float2& a2) {
    const float s = 0.86602540378443864676f;   // sin(pi / 3)
    const float2 t1 = c_add(a1, a2);
    const float2 d = c_sub(a1, a2);
    // -i s d (forward) or +i s d (inverse)
    const float2 t2 = INV ? make_float2(-s * d.y, s * d.x) : make_float2(s * d.y, -s * d.x);
    const float2 m = make_float2(fmaf(-0.5f, t1.x, a0.x), fmaf(-0.5f, t1.y, a0.y));
    a0 = c_add(a0, t1);
    a1 = c_add(m, t2);
    a2 = c_sub(m, t2);
}

template <int M, bool INV>
__device__ __forceinline__ void fft3_combine(float2 (&v)[3][8], int t, const float2* tw3) {
    constexpr int NT = M / 8;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int k = t + m * NT;
        float2 w1 = tw3[k], w2 = tw3[M + k];
        if (INV) {
            w1.y = -w1.y;
            w2.y = -w2.y;
            dft3<true>(v[0][m], v[1][m], v[2][m]);
            v[1][m] = c_mul(v[1][m], w1);
            v[2][m] = c_mul(v[2][m], w2);
        } else {
            v[1][m] = c_mul(v[1][m], w1);
            v[2][m] = c_mul(v[2][m], w2);
            dft3<false>(v[0][m], v[1][m], v[2][m]);
        }
    }
}

template <int M, bool INV, int P>
__device__ __forceinline__ void fft3_step(float2 (&v)[3][8], float2* buf, int t, const float2* tw) {
    using F = FftReg<M, INV>;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int r = 0; r < 8; ++r) buf[j * M + FFT_SWZ(F::out_pos(P, r, t))] = v[j][r];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float2 u[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) u[e] = buf[j * M + FFT_SWZ(F::template in_pos<P>(e, t))];
        F::template pass<P>(u, v[j], t, tw);
    }
}

// One length-3M transform with two alternating exchange buffers of 3M
// entries each (as fft_reg); tw: the table described above.
template <int M, bool INV>
__device__ __forceinline__ void fft_reg3(float2 (&v)[3][8], float2* b0, float2* b1, int& ph, int t,
                                         const float2* tw) {
    using F = FftReg<M, INV>;
    if (INV) fft3_combine<M, true>(v, t, tw + M);
#pragma unroll
    for (int j = 0; j < 3; ++j) F::first(v[j]);
    fft3_step<M, INV, 1>(v, ph ? b1 : b0, t, tw);
    ph ^= 1;
    if constexpr (F::NPASS > 2) {
        fft3_step<M, INV, 2>(v, ph ? b1 : b0, t, tw);
        ph ^= 1;
    }
    if constexpr (F::NPASS > 3) {
        fft3_step<M, INV, 3>(v, ph ? b1 : b0, t, tw);
        ph ^= 1;
    }
    if (!INV) fft3_combine<M, false>(v, t, tw + M);
}
