// Reverse pass through the window reconstruction and the two multislice
// sweeps: the slice-potential derivative dL/dV_j of a map loss.
//
// In the de-tilted frame of the forward sweep a site's stash is the column
// itself, and the frame factor exp(-+2 pi i h_p.r/N) has unit modulus, so
// the adjoint of a stash is a plain addition of the window's adjoint into
// the adjoint column, and sum_p Im(conj(adjoint) field) is frame-free.
//   S1 (psi_{j+1} = Prop(T_j psi_j)), j descending:
//     mu_j = Prop^H(lambda_{j+1});  dL/dV_j += -2 sigma sum_p Im(conj(mu_j) T_j psi_j);
//     lambda_j = conj(T_j) mu_j + (window adjoints of the sites at plane j)
//   S2 (x_j = T_j Prop(x_{j+1})), j ascending:
//     xbar_j = Prop^H(conj(T_{j-1}) xbar_{j-1}) + (window adjoints at j);
//     dL/dV_j += -2 sigma sum_p Im(conj(xbar_j) x_j)
// Prop^H is the forward column pass run on conjugated propagator tables,
// between two row FFTs, exactly as the forward step splits Prop.
//
// Reconstruction adjoint (Eq. magpreserve, S = phi A U/|U|, u = U/|U|):
//   Ebar = Sbar conj(phi), dL/dA = 2 Re(conj(Ebar) u),
//   Ubar = -(A/|U|) Im(conj(Ebar) u) i u,
//   dtbar_p = sum_t w_tp (Ubar_t + dL/dA_t dt_p / (2 |dt_p|))
// in two deterministic passes: per target (recompute U and A from the
// stash), then per parent over the targets that use it.
#include "bip_device.cuh"
#include "bip_internal.h"
#include "fft_smem.cuh"

namespace {

constexpr int kThreads = 256;

// Row layout of a length-NX row (NX = S M, S = 1 or 3 for the lengths 3 M):
// NT = M / 8 threads per row, value (s, m) of thread t at the real-space
// point real(s, m, t) and the frequency freq(s, m, t) -- the layouts of
// fft_reg and fft_reg3, as the forward row pass holds them.
template <int NX>
struct AdjRow {
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

template <int NX, bool INV>
__device__ __forceinline__ void adj_fft(float2 (&v)[AdjRow<NX>::S][8], float2* b0, float2* b1, int& ph, int t,
                                        const float2* tw) {
    if constexpr (AdjRow<NX>::THREE)
        fft_reg3<AdjRow<NX>::M, INV>(v, b0, b1, ph, t, tw);
    else
        fft_reg<NX, INV>(v[0], b0, b1, ph, t, tw);
}

template <int NX>
__global__ void __launch_bounds__(kThreads) adj_row_kernel(MsPlan plan, MsAdjArgs a) {
    using RS = AdjRow<NX>;
    constexpr int NT = RS::NT, RPB = RS::RPB, S = RS::S;
    extern __shared__ float2 smem[];
    const int sub = threadIdx.x / NT;
    const int t = threadIdx.x % NT;
    float2* b0 = smem + 2 * sub * NX;
    float2* b1 = b0 + NX;
    float2* tw = smem + 2 * RPB * NX;          // [NX]
    float2* tt = tw + NX;                      // [NX] T_j of this y
    float* red = reinterpret_cast<float*>(tt + NX);   // [RPB][NX]
    const int gpy = (plan.ncol + RPB - 1) / RPB;
    const int y = blockIdx.x / gpy;
    const int grp = blockIdx.x % gpy;
    const int c = grp * RPB + sub;
    const bool active = c < plan.ncol;
    float2* g = a.cols + ((size_t)(active ? c : 0) * plan.ny + y) * NX;

    // the row arrives in frequency order for an inverse FFT, in real-space
    // order otherwise, and leaves in frequency order after an FFT
    float2 v[S][8];
#pragma unroll
    for (int q = 0; q < S; ++q)
#pragma unroll
        for (int m = 0; m < 8; ++m)
            v[q][m] = (!active || a.zero_in) ? make_float2(0.f, 0.f)
                                             : g[a.do_ifft ? RS::freq(q, m, t) : RS::real(q, m, t)];
    for (int i = threadIdx.x; i < NX; i += kThreads) {
        tw[i] = __ldg(&plan.twx[i]);
        if (a.v) {
            float s, co;
            sincosf(plan.sigma * __ldg(&a.v[(size_t)y * NX + i]), &s, &co);
            tt[i] = make_float2(co, s);
        }
    }
    __syncthreads();
    int ph = 0;
    if (a.do_ifft && !a.zero_in) adj_fft<NX, true>(v, b0, b1, ph, t, tw);
    auto inject = [&]() {
        if (!active || !a.row_off) return;
        const int e1 = __ldg(&a.row_off[y + 1]);
        for (int e = __ldg(&a.row_off[y]); e < e1; ++e) {
            const int4 en = __ldg(&a.row_ent[e]);      // (site, u, ox, -)
            const float2* src = a.inj + (((size_t)en.x * plan.ncol + c) * a.win + en.y) * a.win;
#pragma unroll
            for (int q = 0; q < S; ++q)
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    int u = (RS::real(q, m, t) - en.z) % NX;
                    if (u < 0) u += NX;
                    if (u < a.win) {
                        const float2 d = __ldg(&src[u]);
                        v[q][m].x += d.x;
                        v[q][m].y += d.y;
                    }
                }
        }
    };
    if (a.inj_before) inject();
    if (a.state) {
        // -2 sigma Im(conj(val) u) of this parent, then summed over the block's
        // parents in order
        const float2* st = a.state + ((size_t)(active ? c : 0) * plan.ny + y) * NX;
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int x = RS::real(q, m, t);
                float r = 0.f;
                if (active) {
                    float2 u = st[x];
                    if (a.state_times_T) u = c_mul(u, tt[x]);
                    // Im(conj(v) u) = v.x u.y - v.y u.x
                    r = -2.f * plan.sigma * (v[q][m].x * u.y - v[q][m].y * u.x);
                }
                red[sub * NX + x] = r;
            }
        __syncthreads();
        for (int i = threadIdx.x; i < NX; i += kThreads) {
            float s = 0.f;
            for (int q = 0; q < RPB; ++q) s += red[q * NX + i];
            a.gv_part[((size_t)grp * plan.ny + y) * NX + i] = s;
        }
    }
    if (a.v) {
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float2 tv = tt[RS::real(q, m, t)];
                v[q][m] = c_mul(v[q][m], make_float2(tv.x, -tv.y));
            }
    }
    if (!a.inj_before) inject();
    if (a.do_fft) adj_fft<NX, false>(v, b0, b1, ph, t, tw);
    if (active) {
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int m = 0; m < 8; ++m) g[a.do_fft ? RS::freq(q, m, t) : RS::real(q, m, t)] = v[q][m];
    }
}

template <int NX>
cudaError_t launch_adj_row(const MsPlan& p, const MsAdjArgs& a, int* groups, cudaStream_t s) {
    constexpr int RPB = AdjRow<NX>::RPB;
    const int gpy = (p.ncol + RPB - 1) / RPB;
    *groups = gpy;
    const long long blocks = (long long)p.ny * gpy;
    const size_t sm = ((size_t)2 * RPB * NX + 2 * NX) * sizeof(float2) + (size_t)RPB * NX * sizeof(float);
    static std::atomic<bool> attr{false};
    const cudaError_t e = bip_set_once(attr, [&] {
        return cudaFuncSetAttribute(adj_row_kernel<NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    });
    if (e != cudaSuccess) return e;
    adj_row_kernel<NX><<<(unsigned)blocks, kThreads, sm, s>>>(p, a);
    return cudaGetLastError();
}

__global__ void gv_reduce_kernel(const float* part, int groups, int G, float* gV) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    float s = gV[i];
    for (int q = 0; q < groups; ++q) s += part[(size_t)q * G + i];
    gV[i] = s;
}

// re-tilt phi_t(r) = exp(sign 2 pi i (h_y iy / ny + h_x ix / nx)) at pixel r
// of the batch's window (win x win, wo pixels into the stashed one)
__device__ __forceinline__ float2 retilt(int2 h, const SiteDev& st, int r, int win, int wo, int ny, int nx,
                                         int sign) {
    const int u = r / win, vv = r - u * win;
    const int iy = wrap_n(st.oy + wo + u, ny), ix = wrap_n(st.ox + wo + vv, nx);
    const float f = (float)(wrap_n(h.x * iy, ny)) / ny + (float)(wrap_n(h.y * ix, nx)) / nx;
    float s, c;
    sincospif(2.f * f, &s, &c);
    return make_float2(c, sign * s);
}

// pass 1: per (target, pixel): Ubar and dL/dA
__global__ void recon_adj_target_kernel(ReconAdjArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y, bs = blockIdx.z;
    if (r >= a.K || t >= a.n_targets) return;
    const int site = a.site_ids[bs];
    const SiteDev st = a.sites[site];
    const size_t sk = (size_t)a.stash_win * a.stash_win;
    const int ru = r / a.win;
    const float2* dt = a.stash + (size_t)site * a.Bp * sk + (size_t)(ru + a.wo) * a.stash_win + (r - ru * a.win) + a.wo;
    float ur = 0.f, ui = 0.f, am = 0.f;
    for (int e = __ldg(&a.w.t_off[t]); e < __ldg(&a.w.t_off[t + 1]); ++e) {
        const int p = __ldg(&a.w.t_par[e]);
        const float w = __ldg(&a.w.t_w[e]);
        const float2 d = __ldg(&dt[(size_t)p * sk]);
        ur = fmaf(w, d.x, ur);
        ui = fmaf(w, d.y, ui);
        am = fmaf(w, sqrtf(d.x * d.x + d.y * d.y), am);
    }
    const float2 phi = retilt(__ldg(&a.h_t[t]), st, r, a.win, a.wo, a.ny, a.nx, a.tilt_sign);
    const float2 sb = a.Sbar[((size_t)bs * a.sbar_rows + t) * a.K + r];
    // Ebar = Sbar conj(phi)
    const float2 eb = make_float2(sb.x * phi.x + sb.y * phi.y, sb.y * phi.x - sb.x * phi.y);
    float2 ubar;
    float dA = 0.f;
    if (!a.magnitude) {
        ubar = eb;
    } else {
        const float m = sqrtf(ur * ur + ui * ui);
        float2 u = make_float2(1.f, 0.f);
        if (m > 0.f) u = make_float2(ur / m, ui / m);
        // conj(Ebar) u
        const float cr = eb.x * u.x + eb.y * u.y, ci = eb.x * u.y - eb.y * u.x;
        dA = 2.f * cr;
        if (m > 0.f) {
            const float k = -(am / m) * ci;          // times i u
            ubar = make_float2(-k * u.y, k * u.x);
        } else {
            ubar = make_float2(0.f, 0.f);
        }
    }
    const size_t o = ((size_t)bs * a.n_targets + t) * a.K + r;
    a.Ubar[o] = ubar;
    a.dA[o] = dA;
}

// pass 2: per (parent, pixel): dtbar_p = sum_t w_tp (Ubar_t + dA_t dt_p / (2|dt_p|))
__global__ void recon_adj_parent_kernel(ReconAdjArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y, bs = blockIdx.z;
    if (r >= a.K || p >= a.Bp) return;
    const int site = a.site_ids[bs];
    const size_t sk = (size_t)a.stash_win * a.stash_win;
    const int ru = r / a.win;
    const size_t sidx = ((size_t)site * a.Bp + p) * sk + (size_t)(ru + a.wo) * a.stash_win + (r - ru * a.win) + a.wo;
    const float2 d = __ldg(&a.stash[sidx]);
    const float md = sqrtf(d.x * d.x + d.y * d.y);
    const float2 unit = md > 0.f ? make_float2(d.x / md, d.y / md) : make_float2(0.f, 0.f);
    float sx = 0.f, sy = 0.f;
    for (int e = __ldg(&a.w.p_off[p]); e < __ldg(&a.w.p_off[p + 1]); ++e) {
        const int t = __ldg(&a.w.p_tgt[e]);
        const float w = __ldg(&a.w.p_w[e]);
        const size_t o = ((size_t)bs * a.n_targets + t) * a.K + r;
        const float2 ub = a.Ubar[o];
        const float h = 0.5f * a.dA[o];
        sx = fmaf(w, fmaf(h, unit.x, ub.x), sx);
        sy = fmaf(w, fmaf(h, unit.y, ub.y), sy);
    }
    a.dtbar[sidx] = make_float2(sx, sy);
}

__global__ void s1bar_kernel(const int32_t* ids, const SiteDev* sites, int B, int K, const float2* H, const float2* T,
                             int64_t t_site, int64_t t_ch, float2* S1bar, int64_t s1_site) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y, bs = blockIdx.z;
    if (r >= K || b >= B) return;
    const SiteDev st = sites[ids[bs]];
    float sx = 0.f, sy = 0.f;
    for (int n = 0; n < st.nch; ++n) {
        const float2 h = __ldg(&H[(size_t)st.h_off + (size_t)n * K + r]);
        const float2 x = T[(int64_t)bs * t_site + (int64_t)n * t_ch + (int64_t)b * K + r];
        // conj(h) x
        sx += h.x * x.x + h.y * x.y;
        sy += h.x * x.y - h.y * x.x;
    }
    S1bar[(int64_t)bs * s1_site + (int64_t)b * K + r] = make_float2(sx, sy);
}

}  // namespace

cudaError_t bip_ms_adj_row_pass(const MsPlan& p, const MsAdjArgs& a, int* groups, cudaStream_t s) {
    switch (p.nx) {
        case 64: return launch_adj_row<64>(p, a, groups, s);
        case 128: return launch_adj_row<128>(p, a, groups, s);
        case 256: return launch_adj_row<256>(p, a, groups, s);
        case 512: return launch_adj_row<512>(p, a, groups, s);
        case 1024: return launch_adj_row<1024>(p, a, groups, s);
        case 192: return launch_adj_row<192>(p, a, groups, s);
        case 384: return launch_adj_row<384>(p, a, groups, s);
        case 768: return launch_adj_row<768>(p, a, groups, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t bip_gv_reduce(const float* part, int groups, int G, float* gV, cudaStream_t s) {
    gv_reduce_kernel<<<(G + 255) / 256, 256, 0, s>>>(part, groups, G, gV);
    return cudaGetLastError();
}

cudaError_t bip_recon_adjoint(const ReconAdjArgs& a, cudaStream_t s) {
    if (a.n_sites < 1 || a.n_targets < 1 || a.Bp < 1 || a.K < 1) return cudaErrorInvalidValue;
    if (a.K != a.win * a.win || a.wo < 0 || a.win + 2 * a.wo != a.stash_win) return cudaErrorInvalidValue;
    if (a.n_targets > 65535 || a.Bp > 65535 || a.n_sites > 65535) return cudaErrorInvalidValue;
    recon_adj_target_kernel<<<dim3((a.K + 255) / 256, a.n_targets, a.n_sites), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    recon_adj_parent_kernel<<<dim3((a.K + 255) / 256, a.Bp, a.n_sites), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t bip_s1bar(int nb, const int32_t* ids, const SiteDev* sites, int B, int K, const float2* H,
                      const float2* T, int64_t t_site, int64_t t_ch, float2* S1bar, int64_t s1_site, cudaStream_t s) {
    if (nb < 1 || B < 1 || B > 65535) return cudaErrorInvalidValue;
    s1bar_kernel<<<dim3((K + 255) / 256, B, nb), 256, 0, s>>>(ids, sites, B, K, H, T, t_site, t_ch, S1bar, s1_site);
    return cudaGetLastError();
}
