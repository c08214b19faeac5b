// FP32 (SIMT FFMA) complex contractions of the map -- the FP32 path.
//
//   coupling   M^{(n)}_{d,b} = sum_r S2^d(r) [H_n S1^b](r)          (Eq. coupling)
//   Gram       Q_{b,b'} = sum_{n,d} conj(M^{(n)}_{d,b}) M^{(n)}_{d,b'}
// The Gram matrix is an exact regrouping of Eq. map-sum:
//   sum_n sum_d |sum_b M^{(n)}_{d,b} c_b|^2 = c^H (sum_n M^{(n)H} M^{(n)}) c,
// which contracts the detector index once per site instead of once per
// scan; c^H Q c itself is evaluated in difftrans.cu.
//
// cgemm: C[m][n] = sum_k op(A[m][k]) B[n][k], complex64, both operands
// K-contiguous; 64x64 complex tile, 256 threads with 4x4 complex register
// blocks, K step 16, double-buffered shared memory.  4 FFMA per complex MAC.
#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// loads a [64 rows x 16 k] tile of a K-contiguous matrix into s[k][row]
__device__ __forceinline__ void load_tile(float2 (*s)[BM + 1], const float2* __restrict__ g, int64_t ld,
                                          int row0, int nrows, int k0, bool conj) {
    const int tid = threadIdx.x;
    const int row = tid >> 2;             // 0..63
    const int kc = (tid & 3) * 4;         // 0,4,8,12
    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
    if (row0 + row < nrows) {
        const float4* p = reinterpret_cast<const float4*>(g + (size_t)(row0 + row) * ld + k0 + kc);
        v0 = __ldg(p);
        v1 = __ldg(p + 1);
    }
    const float sg = conj ? -1.f : 1.f;
    s[kc + 0][row] = make_float2(v0.x, sg * v0.y);
    s[kc + 1][row] = make_float2(v0.z, sg * v0.w);
    s[kc + 2][row] = make_float2(v1.x, sg * v1.y);
    s[kc + 3][row] = make_float2(v1.z, sg * v1.w);
}

// Accumulates the 64x64 tile (m0, n0) over all of K into acc.
__device__ __forceinline__ void tile_mainloop(float2 acc[TM][TN], const float2* __restrict__ A, int64_t lda,
                                              const float2* __restrict__ B, int64_t ldb, int M, int N, int K,
                                              int m0, int n0, bool conjA, float2 (*As)[BK][BM + 1],
                                              float2 (*Bs)[BK][BN + 1]) {
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    int buf = 0;
    load_tile(As[0], A, lda, m0, M, 0, conjA);
    load_tile(Bs[0], B, ldb, n0, N, 0, false);
    __syncthreads();
    for (int k0 = 0; k0 < K; k0 += BK) {
        if (k0 + BK < K) {
            load_tile(As[buf ^ 1], A, lda, m0, M, k0 + BK, conjA);
            load_tile(Bs[buf ^ 1], B, ldb, n0, N, k0 + BK, false);
        }
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float2 a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) cmac(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
        buf ^= 1;
    }
}

__global__ void __launch_bounds__(256) cgemm_kernel(CGemmArgs p) {
    __shared__ float2 As[2][BK][BM + 1];
    __shared__ float2 Bs[2][BK][BN + 1];
    const int bz = blockIdx.z;
    const float2* A = p.A + (size_t)bz * p.strideA;
    const float2* B = p.Bm + (size_t)bz * p.strideB;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
    tile_mainloop(acc, A, p.lda, B, p.ldb, p.M, p.N, p.K, m0, n0, p.conjA != 0, As, Bs);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float2* C = p.C + (size_t)bz * p.strideC;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= p.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= p.N) continue;
            if (p.epi == 0) {
                C[(size_t)m * p.ldc + n] = acc[i][j];
            } else {
                // coupling -> Gram operand: column n = (ch, b), row m = d
                const int ch = n / p.ep_B, b = n % p.ep_B;
                C[(size_t)b * p.ldc + (size_t)ch * p.ep_Dp + m] = acc[i][j];
            }
        }
    }
}

}  // namespace

cudaError_t bip_cgemm_simt(const CGemmArgs& a, cudaStream_t s) {
    if (a.K % BK != 0 || (a.lda % 2) || (a.ldb % 2)) return cudaErrorInvalidValue;
    dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, a.batch);
    cgemm_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
