// C ABI of the BiP-PRISM library: argument checks, host geometry, device
// tables and the order of the kernels (Algorithm 5).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <new>
#include <numeric>
#include <string>

#include <cuda_fp16.h>
#include <nvtx3/nvToolsExt.h>

#include "bip_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kRowPad = 128;        // aperture-side operand rows: the MMA's 128-row tiles
constexpr int kDetPad = 32;         // detector-side rows: the N of a tile (multiple of 16, K of the Gram a multiple of 32)
constexpr int kScanTile = 256;      // scans per quadratic-form work item
constexpr int kProbeMaxScans = 2048; // the probe order keeps Psi of every scan for a batch of sites

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct bip_ctx {
    bip_config cfg{};
    BipGeometry geo;
    std::string err;
    int prec = 0;
    int Bpad = 0, Dpad = 0;

    // device geometry tables
    bool tables = false;
    DevBuf twy, twx, py, px, ey, ex, shift1, shift2, hbeam, hdet, coef;
    DevBuf grp1_off, grp1_par, grp1_w, grp2_off, grp2_par, grp2_w, ytab, xtab;
    DevBuf kb_d, lat_d;                 // beam lattice of the difference transform
    int Ky = 0, Kx = 0;
    int grp1_n = 0, grp2_n = 0;
    DevBuf wtc, xtc;                    // tensor-core reconstruction: W hi/lo, X planes
    bool recon_tc = false;              // both parent sets fit its K = 64

    // sites of the current builds
    std::vector<SiteDev> sites;
    std::vector<int32_t> plane_ids;     // site ids grouped by plane
    std::vector<int32_t> plane_off;     // [nz + 1]
    DevBuf sites_d, plane_ids_d, seq_ids_d, row_off_d, row_ent_d;
    int n_sites = 0, nch_max = 0, n_ch_total = 0;
    // per-site windows (bip_set_site_windows; empty: every site at win) and
    // the order the maps batch the sites in: by window, descending, stable
    // (seq_ids_d holds it)
    std::vector<int32_t> site_w;
    std::vector<int32_t> batch_order;
    bool uneven = false;                // some site's window is below win
    int64_t h_elems = 0;                // complex elements of H the sites read
    int op_k = 0;                       // row pitch of the coupling operands' current contents
    int xop_k = 0;                      // ... and of the cube's own operands (xopA, xopB)
    int gop_k = 0;                      // ... and of the reverse pass's per-pixel workspaces
    uint64_t sig1 = 0, sig2 = 0;        // site-list signatures of the builds
    bool s1 = false, s2 = false;

    DevBuf stash1, stash2, cols;
    DevBuf cols2;                       // S2's columns while both sweeps run at once (bip_build)
    cudaStream_t side = nullptr;        // bip_build: the stream S2's sweep runs on
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    DevBuf tw512;                       // nx = 512: the half-warp row pass's twiddles

    // map workspaces
    DevBuf scans_d, work_d, partial, gdiff, rsum, illum, cube_scratch, bin_of_d;
    DevBuf opA32, opB32, mt32, q32;     // FP32 path (zeroed at allocation)
    DevBuf opA16, opB16, mt16, q16;     // split-BF16 path (zeroed at allocation)
    DevBuf op8A, op8B;                  // FP8 coupling operands, E4M3 (zeroed at allocation)
    DevBuf occ_d;                       // site occupancies weighting the site sum
    int occ_n = 0;                      // sites they were given for (0: none)
    DevBuf g_s1, g_w, g_R, g_gmt, g_T, g_D, g_Dsum;   // gradient pass workspaces
    DevBuf g_s1bar, g_s2bar, g_ubar, g_dA, g_dt1, g_dt2, g_adj, g_ckpt, g_seg, g_gvp;
    DevBuf g_tA, g_tB, g_sA2, g_sB2;    // split-BF16 operands of the reverse-pass contractions
    DevBuf cubeA, cubeB, cube_work, cube_mask;   // the cube on tcgen05
    DevBuf cube_grp, cube_wmap, mpart;  // cube-mode work groups; map modes' item map and column sums
    std::vector<int32_t> cube_work_h, cube_grp_h, cube_wmap_h;   // what the device copies hold
    DevBuf hcube, shcube, cstash, ccols; // the exact cube: basis, shifts, S2 windows, columns
    DevBuf xopA, xopB, xm32;            // ... its coupling operands and M
    DevBuf tcache;                      // T_j = exp(i sigma V_j) of the slices a sweep crosses
    DevBuf cr_ay, cr_ax, cr_cy, cr_cx, cr_T;   // the cube on a raster: phase tables, crop bits, T
    size_t cube_budget = 0;             // bytes of sweep columns + windows per detector batch (0: auto)
    DevBuf s1t, psi, ybuf;              // the probe order: S1 transposed, Psi, H_n x Psi
    DevBuf pyc, pxc;                    // conjugated propagator tables (adjoint sweeps)
    // capture-safe maps: no host synchronisation, uploads only when the
    // scans or the batching change (so a CUDA graph can hold the launches)
    bool capture_safe = false;
    std::vector<double> scans_cache;
    std::vector<int> batch_off_cache;
    uint64_t work_key = 0;
    // tuned launch parameters (0: the built-in choice)
    int sb_override = 0, cw_override = 0;
    bool raster_eval = true;            // separable evaluation on raster scan lists
    int order = 0;                      // scan contraction: 0 Gram matrix, 1 beam order, 2 probe order
    DevBuf ray, rax;                    // its phase tables
    DevBuf aw1[6], aw2[6];              // per-target / per-parent weights (reconstruction adjoint)
    bool adj_tables = false;
    DevBuf f8pmax, f8inv0, f8inv1, f8hmax, f8H, f8sA, f8sB;   // FP8 per-window scales
    DevBuf errflag;
    std::vector<int32_t> work_h;
    bool check_finite = false;          // scan outputs for NaN / Inf (bip_set_check_finite)
    DevBuf nf_count;

    // per-stage event timing
    uint32_t prof = 0;                  // stages timed (bit s: stage s)
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_rec;
    int64_t launches[BIP_N_STAGES] = {0};
    uint64_t wait_ns = 0;               // give-up limit of the tcgen05 kernels' waits (0: 4 s)
};

namespace {

bip_status fail(bip_ctx* c, bip_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

bip_status fail_cuda(bip_ctx* c, cudaError_t e, const char* what) {
    const bip_status s = (e == cudaErrorMemoryAllocation) ? BIP_ERR_OOM : BIP_ERR_CUDA;
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();   // clear a non-sticky error
    return s;
}

#define CUDA_TRY(c, expr)                                   \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return fail_cuda(c, e_, #expr); \
    } while (0)

// NVTX range over a public call or a stage's launch (host side: under a
// tracing tool the range shows what was enqueued; with no tool attached a
// push or pop is one check of a function pointer).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define BIP_RANGE(name) NvtxRange nvtx_range_(name)

const char* const kStageRange[BIP_N_STAGES] = {
    "bip:ms_row", "bip:ms_col", "bip:reconstruct", "bip:coupling",
    "bip:gram", "bip:quadform", "bip:reduce", "bip:transmission"};

// Brackets one launch with events on its stream when profiling is on, and
// counts it.  Returns the launch's error.
struct StageTimer {
    bip_ctx* c;
    int stage;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEvent_t take() {
        if (c->ev_used == c->ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            c->ev_pool.push_back(e);
        }
        return c->ev_pool[c->ev_used++];
    }
    NvtxRange range;
    StageTimer(bip_ctx* c_, int st, cudaStream_t s_) : c(c_), stage(st), s(s_), range(kStageRange[st]) {
        c->launches[stage]++;
        if (c->prof >> stage & 1u) {
            e0 = take();
            e1 = take();
            if (e0) cudaEventRecord(e0, s);
        }
    }
    ~StageTimer() {
        if (e0 && e1) {
            cudaEventRecord(e1, s);
            c->ev_rec.push_back({stage, {e0, e1}});
        }
    }
};

#define TIMED(c, stage, s, expr)        \
    do {                                 \
        StageTimer t_(c, stage, s);      \
        CUDA_TRY(c, expr);               \
    } while (0)

// Device allocations of the library, counted for tests: the live ones, the
// ones made, and an injected failure (the fail_at-th allocation from the
// moment it is set fails as if the device were out of memory).
std::atomic<int64_t> g_live{0}, g_made{0}, g_fail_at{0};
// bytes of the live allocations and their high-water mark
std::atomic<int64_t> g_bytes{0}, g_peak{0};

void count_bytes(int64_t delta) {
    const int64_t now = g_bytes += delta;
    int64_t peak = g_peak.load();
    while (now > peak && !g_peak.compare_exchange_weak(peak, now)) {
    }
}

cudaError_t ensure(DevBuf& b, size_t bytes, bool zero = false, cudaStream_t s = nullptr) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return cudaSuccess;
    if (b.p) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        cudaFree(b.p);
        --g_live;
        count_bytes(-(int64_t)b.cap);
        b.p = nullptr;
        b.cap = 0;
    }
    const int64_t n = ++g_made;
    const int64_t fail_at = g_fail_at.load();
    if (fail_at > 0 && n == fail_at) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    ++g_live;
    count_bytes((int64_t)bytes);
    b.cap = bytes;
    if (zero) return cudaMemsetAsync(b.p, 0, bytes, s);
    return cudaSuccess;
}

void release(DevBuf& b) {
    if (b.p) {
        cudaFree(b.p);
        --g_live;
        count_bytes(-(int64_t)b.cap);
    }
    b.p = nullptr;
    b.cap = 0;
}

// true while `s` is being captured into a CUDA graph (a host-to-device copy
// from host memory that lives only during the call must not be recorded)
bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

template <class T>
cudaError_t upload(DevBuf& b, const std::vector<T>& h, cudaStream_t s) {
    cudaError_t e = ensure(b, h.size() * sizeof(T), false, s);
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }
// grid lengths the register FFTs take: powers of two 64..1024, and 3 m for m
// a power of two 64..256 (192, 384, 768)
bool grid_len_ok(int n) { return pow2_in(n, 64, 1024) || (n % 3 == 0 && pow2_in(n / 3, 64, 256)); }

int signed_bin(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Twiddles of the register FFT of length n (n a power of two, 64..1024),
// pass by pass: pass p = 1 .. npass-1 combines sub-transforms of length
// Ns = 8^p with radix R (8, or 4 / 2 for the last pass), and its entry
// (r - 1) Ns + k holds exp(-2 pi i r k / (Ns R)), r = 1..R-1, k < Ns.
// Evaluated in FP64, rounded to FP32; the rest of the n entries is zero.
// For n = 3 m (m a power of two): the table of length m, then the radix-3
// step's exp(-2 pi i j k / n) for j = 1, 2 and k < m -- n entries in all.
std::vector<float2> fft_twiddles_pow2(int n);
std::vector<float2> fft_twiddles(int n) {
    if (n % 3 != 0) return fft_twiddles_pow2(n);
    const int m = n / 3;
    std::vector<float2> t = fft_twiddles_pow2(m);
    t.resize(n);
    for (int j = 1; j <= 2; ++j)
        for (int k = 0; k < m; ++k) {
            const double a = -2.0 * kPi * (double)j * k / (double)n;
            t[(size_t)m + (size_t)(j - 1) * m + k] = float2{(float)std::cos(a), (float)std::sin(a)};
        }
    return t;
}

std::vector<float2> fft_twiddles_pow2(int n) {
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    const int rl = lg % 3 == 2 ? 4 : (lg % 3 == 1 ? 2 : 8);
    const int npass = lg / 3 + (rl == 8 ? 0 : 1);
    std::vector<float2> t(n, float2{0.f, 0.f});
    size_t o = 0;
    for (int p = 1; p < npass; ++p) {
        const int ns = 1 << (3 * p), R = p == npass - 1 ? rl : 8;
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < ns; ++k) {
                const double a = -2.0 * kPi * (double)r * k / ((double)ns * R);
                t[o + (size_t)(r - 1) * ns + k] = float2{(float)std::cos(a), (float)std::sin(a)};
            }
        o += (size_t)(R - 1) * ns;
    }
    return t;
}

// Column tile width for n detector rows: as few tiles of at most 256 as
// possible, as even as the multiple-of-16 widths allow.
int tile_width(int n) {
    const int tiles = (n + 255) / 256;
    return round_up((n + tiles - 1) / tiles, 16);
}

// Grouped sparse copy of a dense weight matrix [rows][cols]: rows
// kGatherGroup g .. + kGatherGroup - 1 form group g, whose entries are the
// columns (parents) any of its rows uses, with the rows' weights side by side.
int to_groups(const std::vector<double>& w, int rows, int cols, std::vector<int32_t>& off,
              std::vector<uint16_t>& par, std::vector<float4>& wt) {
    const int ng = (rows + kGatherGroup - 1) / kGatherGroup;
    off.assign(1, 0);
    par.clear();
    wt.clear();
    for (int g = 0; g < ng; ++g) {
        for (int c = 0; c < cols; ++c) {
            float v[kGatherGroup] = {0.f, 0.f, 0.f, 0.f};
            bool any = false;
            for (int i = 0; i < kGatherGroup; ++i) {
                const int r = g * kGatherGroup + i;
                if (r < rows && w[(size_t)r * cols + c] != 0.0) {
                    v[i] = (float)w[(size_t)r * cols + c];
                    any = true;
                }
            }
            if (any) {
                par.push_back((uint16_t)c);
                wt.push_back(float4{v[0], v[1], v[2], v[3]});
            }
        }
        off.push_back((int32_t)par.size());
    }
    return ng;
}

// The map's detector-side factor: dfy dfx, the subsampling of the detector
// beams (a coarse detector sum is 1/(dfy dfx) of the full one for an exit
// wave inside the alias-free window -- the reading that mirrors the
// probe-side PRISM rescale, Sec. 2.2.2).
int det_scale(const bip_ctx* c) { return c->geo.dfy * c->geo.dfx; }

// c_b(rho) coefficients f_y f_x Psi(h_b) / sqrt(G sum |Psi|^2) (Eq. probe)
std::vector<double2> coef_host(const bip_ctx* c) {
    const BipGeometry& geo = c->geo;
    std::vector<double2> coef(geo.B);
    const double fyfx = (double)c->cfg.fy * c->cfg.fx;
    for (int b = 0; b < geo.B; ++b) {
        const std::complex<double> v = fyfx * geo.psi_beam[b] / geo.psi_norm;
        coef[b] = double2{v.real(), v.imag()};
    }
    return coef;
}

bip_status make_tables(bip_ctx* c, cudaStream_t s) {
    if (c->tables) return BIP_OK;
    const bip_config& g = c->cfg;
    const BipGeometry& geo = c->geo;
    auto turn = [](int m, int n, double sign) {
        const double a = sign * 2.0 * kPi * (double)m / (double)n;
        return float2{(float)std::cos(a), (float)std::sin(a)};
    };
    const std::vector<float2> twy = fft_twiddles(g.ny), twx = fft_twiddles(g.nx);
    std::vector<float2> ey(g.ny), ex(g.nx), py(g.ny), px(g.nx);
    for (int m = 0; m < g.ny; ++m) ey[m] = turn(m, g.ny, +1.0);
    for (int m = 0; m < g.nx; ++m) ex[m] = turn(m, g.nx, +1.0);
    // separable propagator exp(-i pi lambda dz q^2) per axis, with the 1/N
    // of the unnormalised inverse FFT folded in
    for (int k = 0; k < g.ny; ++k) {
        const double q = signed_bin(k, g.ny) / g.ly;
        const double a = -kPi * geo.lambda * g.dz * q * q;
        py[k] = float2{(float)(std::cos(a) / g.ny), (float)(std::sin(a) / g.ny)};
    }
    for (int k = 0; k < g.nx; ++k) {
        const double q = signed_bin(k, g.nx) / g.lx;
        const double a = -kPi * geo.lambda * g.dz * q * q;
        px[k] = float2{(float)(std::cos(a) / g.nx), (float)(std::sin(a) / g.nx)};
    }
    std::vector<int2> sh1(geo.Bp1), sh2(geo.Bp2), hb(geo.B), hd(geo.n_det);
    for (int i = 0; i < geo.Bp1; ++i) sh1[i] = int2{geo.h_beam[2 * geo.p1[i]], geo.h_beam[2 * geo.p1[i] + 1]};
    for (int i = 0; i < geo.Bp2; ++i) sh2[i] = int2{-geo.h_det[2 * geo.p2[i]], -geo.h_det[2 * geo.p2[i] + 1]};
    for (int b = 0; b < geo.B; ++b) hb[b] = int2{geo.h_beam[2 * b], geo.h_beam[2 * b + 1]};
    for (int d = 0; d < geo.n_det; ++d) hd[d] = int2{geo.h_det[2 * d], geo.h_det[2 * d + 1]};
    const std::vector<double2> coef = coef_host(c);
    // beam lattice k = h / f of the difference transform
    std::vector<int2> kb(geo.B);
    int Ky = 0, Kx = 0;
    for (int b = 0; b < geo.B; ++b) {
        kb[b] = int2{geo.h_beam[2 * b] / g.fy, geo.h_beam[2 * b + 1] / g.fx};
        Ky = std::max(Ky, std::abs(kb[b].x));
        Kx = std::max(Kx, std::abs(kb[b].y));
    }
    std::vector<int32_t> lat((size_t)(2 * Ky + 1) * (2 * Kx + 1), -1);
    for (int b = 0; b < geo.B; ++b) lat[(size_t)(kb[b].x + Ky) * (2 * Kx + 1) + kb[b].y + Kx] = b;
    c->Ky = Ky;
    c->Kx = Kx;
    CUDA_TRY(c, upload(c->kb_d, kb, s));
    CUDA_TRY(c, upload(c->lat_d, lat, s));
    std::vector<int32_t> o1, o2;
    std::vector<uint16_t> p1, p2;
    std::vector<float4> w1, w2;
    c->grp1_n = to_groups(geo.w1, geo.B, geo.Bp1, o1, p1, w1);
    c->grp2_n = to_groups(geo.w2, geo.n_det, geo.Bp2, o2, p2, w2);
    // separable re-tilt factors exp(+2 pi i h u / n) for window offsets u
    std::vector<float2> yt((size_t)g.ny * g.win), xt((size_t)g.nx * g.win);
    for (int h = 0; h < g.ny; ++h)
        for (int u = 0; u < g.win; ++u) yt[(size_t)h * g.win + u] = turn((int)((int64_t)h * u % g.ny), g.ny, +1.0);
    for (int h = 0; h < g.nx; ++h)
        for (int v = 0; v < g.win; ++v) xt[(size_t)h * g.win + v] = turn((int)((int64_t)h * v % g.nx), g.nx, +1.0);
    CUDA_TRY(c, upload(c->twy, twy, s));
    CUDA_TRY(c, upload(c->twx, twx, s));
    if (g.nx == 512) {
        // twiddles of the half-warp row pass's second pass
        std::vector<float2> t5(15 * 32);
        for (int e = 1; e < 16; ++e)
            for (int j = 0; j < 32; ++j) t5[(size_t)(e - 1) * 32 + j] = turn(e * j, 512, -1.0);
        CUDA_TRY(c, upload(c->tw512, t5, s));
    }
    CUDA_TRY(c, upload(c->ey, ey, s));
    CUDA_TRY(c, upload(c->ex, ex, s));
    CUDA_TRY(c, upload(c->py, py, s));
    CUDA_TRY(c, upload(c->px, px, s));
    CUDA_TRY(c, upload(c->shift1, sh1, s));
    CUDA_TRY(c, upload(c->shift2, sh2, s));
    CUDA_TRY(c, upload(c->hbeam, hb, s));
    CUDA_TRY(c, upload(c->hdet, hd, s));
    CUDA_TRY(c, upload(c->coef, coef, s));
    CUDA_TRY(c, upload(c->grp1_off, o1, s));
    CUDA_TRY(c, upload(c->grp1_par, p1, s));
    CUDA_TRY(c, upload(c->grp1_w, w1, s));
    CUDA_TRY(c, upload(c->grp2_off, o2, s));
    CUDA_TRY(c, upload(c->grp2_par, p2, s));
    CUDA_TRY(c, upload(c->grp2_w, w2, s));
    CUDA_TRY(c, upload(c->ytab, yt, s));
    CUDA_TRY(c, upload(c->xtab, xt, s));
    // NNW weights as dense hi + lo FP16 rows [side][plane][rows_pad][64 parents]
    // for the tensor-core reconstruction (side 0: detector beams, 1: aperture)
    c->recon_tc = geo.Bp1 <= 64 && geo.Bp2 <= 64;
    if (c->recon_tc) {
        const int Dw = round_up(geo.n_det, kRowPad);
        std::vector<uint16_t> wt((size_t)(2 * Dw + 2 * c->Bpad) * 64, 0);
        auto fill = [&](const std::vector<double>& w, int n, int bp, int row0, int rows_pad) {
            for (int t = 0; t < n; ++t)
                for (int p = 0; p < bp; ++p) {
                    const float x = (float)w[(size_t)t * bp + p];
                    const __half hi = __float2half_rn(x);
                    const __half lo = __float2half_rn(x - __half2float(hi));
                    wt[(size_t)(row0 + t) * 64 + p] = __half_as_ushort(hi);
                    wt[(size_t)(row0 + rows_pad + t) * 64 + p] = __half_as_ushort(lo);
                }
        };
        fill(geo.w2, geo.n_det, geo.Bp2, 0, Dw);
        fill(geo.w1, geo.B, geo.Bp1, 2 * Dw, c->Bpad);
        CUDA_TRY(c, upload(c->wtc, wt, s));
    }
    // the cube's complete basis: beams and the sweep's propagator shifts -h
    std::vector<int2> hc(geo.n_cube), shc(geo.n_cube);
    for (int d = 0; d < geo.n_cube; ++d) {
        hc[d] = int2{geo.h_cube[2 * d], geo.h_cube[2 * d + 1]};
        shc[d] = int2{-hc[d].x, -hc[d].y};
    }
    CUDA_TRY(c, upload(c->hcube, hc, s));
    CUDA_TRY(c, upload(c->shcube, shc, s));
    CUDA_TRY(c, ensure(c->errflag, 64, true, s));
    c->tables = true;
    return BIP_OK;
}

uint64_t site_signature(const std::vector<SiteDev>& v) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    };
    for (const SiteDev& s : v) {
        mix(&s.ty, sizeof(double));
        mix(&s.tx, sizeof(double));
        mix(&s.plane, sizeof(int32_t));
        mix(&s.nch, sizeof(int32_t));
    }
    return h;
}

// host part: validates the atoms and computes the site list (no CUDA call)
bip_status parse_sites(bip_ctx* c, const bip_atom* atoms, int32_t n_atoms, std::vector<SiteDev>& sites,
                       int& nmax, int& total) {
    const bip_config& g = c->cfg;
    if (!atoms || n_atoms < 1) return fail(c, BIP_ERR_INVALID_ARG, "atoms is null or n_atoms < 1");
    const double dy = g.ly / g.ny, dx = g.lx / g.nx;
    int off = 0;
    nmax = 0;
    for (int i = 0; i < n_atoms; ++i) {
        const bip_atom& a = atoms[i];
        if (a.nch < 0 || a.nch > 9)
            return fail(c, BIP_ERR_INVALID_ARG, "atom nch must lie in [0, 9]");
        if (a.nch == 0) continue;
        if (a.slice < 0 || a.slice >= g.nz)
            return fail(c, BIP_ERR_INVALID_ARG, "ionized atom slice outside [0, nz)");
        if (!std::isfinite(a.y) || !std::isfinite(a.x))
            return fail(c, BIP_ERR_INVALID_ARG, "atom position is not finite");
        SiteDev sd{};
        sd.ty = a.y / dy;
        sd.tx = a.x / dx;
        sd.oy = (int32_t)std::floor(sd.ty + 0.5) - g.win / 2;
        sd.ox = (int32_t)std::floor(sd.tx + 0.5) - g.win / 2;
        sd.plane = a.slice;
        sd.nch = a.nch;
        sd.ch_off = off;
        sd.w = g.win;
        sd.wo = 0;
        if ((int64_t)(off + a.nch) * g.win * g.win > INT32_MAX)
            return fail(c, BIP_ERR_INVALID_ARG, "H would exceed 2^31 complex elements");
        sd.h_off = off * g.win * g.win;
        off += a.nch;
        nmax = std::max(nmax, (int)a.nch);
        sites.push_back(sd);
    }
    if (sites.empty()) return fail(c, BIP_ERR_INVALID_ARG, "no ionized atom (every nch is 0)");
    total = off;
    return BIP_OK;
}

// Windows crossing each grid row, per plane: row_off[j * (ny + 1) + y] ..
// row_off[j * (ny + 1) + y + 1] - 1 index (site, window row, window x
// origin, 0) entries; the multislice row pass stashes exactly those.
void row_windows(const bip_config& g, const std::vector<SiteDev>& sites, std::vector<int32_t>& off,
                 std::vector<int4>& ent) {
    const int ny1 = g.ny + 1;
    std::vector<int32_t> cnt((size_t)g.nz * ny1, 0);
    for (const SiteDev& sd : sites)
        for (int u = 0; u < g.win; ++u) {
            int y = (sd.oy + u) % g.ny;
            if (y < 0) y += g.ny;
            cnt[(size_t)sd.plane * ny1 + y + 1]++;
        }
    off.assign((size_t)g.nz * ny1, 0);
    int32_t run = 0;
    for (int j = 0; j < g.nz; ++j) {
        for (int y = 0; y < g.ny; ++y) {
            off[(size_t)j * ny1 + y] = run;
            run += cnt[(size_t)j * ny1 + y + 1];
        }
        off[(size_t)j * ny1 + g.ny] = run;
    }
    ent.assign(run, int4{0, 0, 0, 0});
    std::vector<int32_t> fill(off);
    for (int s = 0; s < (int)sites.size(); ++s) {
        const SiteDev& sd = sites[s];
        for (int u = 0; u < g.win; ++u) {
            int y = (sd.oy + u) % g.ny;
            if (y < 0) y += g.ny;
            ent[fill[(size_t)sd.plane * ny1 + y]++] = int4{s, u, sd.ox, 0};
        }
    }
}

// Per-site windows onto the site list: w, wo and the H offsets, the batch
// order (sites by window, descending; ties in site order), and both to the
// device.  site_w empty: every site at the context's win.
bip_status apply_windows(bip_ctx* c, cudaStream_t s) {
    const int win = c->cfg.win;
    const int n = (int)c->sites.size();
    int64_t h = 0;
    c->uneven = false;
    for (int k = 0; k < n; ++k) {
        SiteDev& sd = c->sites[k];
        sd.w = c->site_w.empty() ? win : c->site_w[k];
        sd.wo = (win - sd.w) / 2;
        sd.h_off = (int32_t)h;
        h += (int64_t)sd.nch * sd.w * sd.w;
        if (sd.w != win) c->uneven = true;
    }
    c->h_elems = h;
    c->batch_order.resize(n);
    std::iota(c->batch_order.begin(), c->batch_order.end(), 0);
    std::stable_sort(c->batch_order.begin(), c->batch_order.end(),
                     [&](int32_t a, int32_t b) { return c->sites[a].w > c->sites[b].w; });
    c->work_key = 0;                    // the batches may have changed
    CUDA_TRY(c, upload(c->sites_d, c->sites, s));
    CUDA_TRY(c, upload(c->seq_ids_d, c->batch_order, s));
    return BIP_OK;
}

bip_status set_sites(bip_ctx* c, std::vector<SiteDev>& sites, int nmax, int total, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const uint64_t sig = site_signature(sites);
    if (sig != c->sig1 && sig != c->sig2) {
        c->s1 = c->s2 = false;
    }
    if (sig != site_signature(c->sites)) {
        c->occ_n = 0;                   // occupancies and windows belong to a site list
        c->site_w.clear();
    }
    c->sites = sites;
    c->n_sites = (int)sites.size();
    c->nch_max = nmax;
    c->n_ch_total = total;
    c->plane_off.assign(g.nz + 1, 0);
    for (auto& sd : sites) c->plane_off[sd.plane + 1]++;
    for (int j = 0; j < g.nz; ++j) c->plane_off[j + 1] += c->plane_off[j];
    c->plane_ids.assign(sites.size(), 0);
    std::vector<int32_t> fill(c->plane_off.begin(), c->plane_off.end() - 1);
    for (int i = 0; i < (int)sites.size(); ++i) c->plane_ids[fill[sites[i].plane]++] = i;
    bip_status st = apply_windows(c, s);
    if (st != BIP_OK) return st;
    CUDA_TRY(c, upload(c->plane_ids_d, c->plane_ids, s));
    std::vector<int32_t> roff;
    std::vector<int4> rent;
    row_windows(g, c->sites, roff, rent);
    CUDA_TRY(c, upload(c->row_off_d, roff, s));
    CUDA_TRY(c, upload(c->row_ent_d, rent, s));
    return BIP_OK;
}

MsPlan plan_for(bip_ctx* c, int ncol, const DevBuf& shift) {
    MsPlan p{};
    p.ny = c->cfg.ny;
    p.nx = c->cfg.nx;
    p.ncol = ncol;
    p.sigma = (float)c->geo.sigma;
    p.twy = (const float2*)c->twy.p;
    p.twx = (const float2*)c->twx.p;
    p.py = (const float2*)c->py.p;
    p.px = (const float2*)c->px.p;
    p.shift = (const int2*)shift.p;
    p.tw512 = c->cfg.nx == 512 ? (const float2*)c->tw512.p : nullptr;
    return p;
}

bip_status build_common(bip_ctx* c, const float* V, const bip_atom* atoms, int32_t n_atoms, cudaStream_t s) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!V) return fail(c, BIP_ERR_INVALID_ARG, "V is null");
    std::vector<SiteDev> sites;
    int nmax = 0, total = 0;
    bip_status st = parse_sites(c, atoms, n_atoms, sites, nmax, total);
    if (st != BIP_OK) return st;
    st = make_tables(c, s);
    if (st != BIP_OK) return st;
    return set_sites(c, sites, nmax, total, s);
}


// Workspaces of the S1 build: its stash, the column set, the transmissions.
bip_status alloc_s1(bip_ctx* c, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const size_t win2 = (size_t)g.win * g.win, G = (size_t)g.ny * g.nx;
    CUDA_TRY(c, ensure(c->stash1, (size_t)c->n_sites * c->geo.Bp1 * win2 * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->cols, (size_t)std::max(c->geo.Bp1, c->geo.Bp2) * G * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->tcache, (size_t)g.nz * G * sizeof(float2), false, s));
    return BIP_OK;
}

// ... of the S2 build, its columns in `cols`.
bip_status alloc_s2(bip_ctx* c, DevBuf& cols, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const size_t win2 = (size_t)g.win * g.win, G = (size_t)g.ny * g.nx;
    CUDA_TRY(c, ensure(c->stash2, (size_t)c->n_sites * c->geo.Bp2 * win2 * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(cols, (size_t)std::max(c->geo.Bp1, c->geo.Bp2) * G * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->tcache, (size_t)g.nz * G * sizeof(float2), false, s));
    return BIP_OK;
}

// S1's forward sweep (Eq. smatrix-advance) on columns `cols`, stashing the
// windows of each plane's sites; with `transmission` it first computes T_j
// of the slices it crosses into the table.
bip_status sweep_s1(bip_ctx* c, const float* V, float2* cols, bool transmission, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const size_t G = (size_t)g.ny * g.nx;
    const MsPlan plan = plan_for(c, c->geo.Bp1, c->shift1);
    int last = 0;
    for (auto& sd : c->sites) last = std::max(last, (int)sd.plane);
    if (transmission)
        TIMED(c, BIP_STAGE_TRANSMISSION, s, bip_transmission(V, (float)c->geo.sigma, 0, last, G, (float2*)c->tcache.p, s));
    for (int j = 0; j <= last; ++j) {
        MsRowArgs a{};
        a.cols = cols;
        a.init = j == 0;
        a.init_val = 1.0f;
        a.do_ifft = j > 0;
        a.v_pre = nullptr;
        a.v_post = j < last ? V + (size_t)j * G : nullptr;
        a.t_slice = j < last ? (const float2*)c->tcache.p + (size_t)j * G : nullptr;
        a.do_fft = j < last;
        if (c->plane_off[j + 1] > c->plane_off[j]) {
            a.row_off = (const int32_t*)c->row_off_d.p + (size_t)j * (g.ny + 1);
            a.row_ent = (const int4*)c->row_ent_d.p;
        }
        a.win = g.win;
        a.stash = (float2*)c->stash1.p;
        TIMED(c, BIP_STAGE_MS_ROW, s, bip_ms_row_pass(plan, a, s));
        if (j < last) TIMED(c, BIP_STAGE_MS_COL, s, bip_ms_col_pass(plan, cols, s));
    }
    return BIP_OK;
}

// S2's backward sweep (Eq. s2) on columns `cols` from the exit surface to
// the shallowest plane with a site.
bip_status sweep_s2(bip_ctx* c, const float* V, float2* cols, bool transmission, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const size_t G = (size_t)g.ny * g.nx;
    const MsPlan plan = plan_for(c, c->geo.Bp2, c->shift2);
    int first = g.nz - 1;
    for (auto& sd : c->sites) first = std::min(first, (int)sd.plane);
    // start: G^{-1/2} constant, forward row FFT, then the first propagator
    {
        MsRowArgs a{};
        a.cols = cols;
        a.init = 1;
        a.init_val = (float)(1.0 / std::sqrt((double)G));
        a.do_fft = 1;
        a.win = g.win;
        a.stash = (float2*)c->stash2.p;
        TIMED(c, BIP_STAGE_MS_ROW, s, bip_ms_row_pass(plan, a, s));
        TIMED(c, BIP_STAGE_MS_COL, s, bip_ms_col_pass(plan, cols, s));
    }
    if (transmission)
        TIMED(c, BIP_STAGE_TRANSMISSION, s, bip_transmission(V, (float)c->geo.sigma, first, g.nz, G, (float2*)c->tcache.p, s));
    for (int j = g.nz - 1; j >= first; --j) {
        MsRowArgs a{};
        a.cols = cols;
        a.do_ifft = 1;
        a.v_pre = V + (size_t)j * G;
        a.t_slice = (const float2*)c->tcache.p + (size_t)j * G;
        a.do_fft = j > first;
        if (c->plane_off[j + 1] > c->plane_off[j]) {
            a.row_off = (const int32_t*)c->row_off_d.p + (size_t)j * (g.ny + 1);
            a.row_ent = (const int4*)c->row_ent_d.p;
        }
        a.win = g.win;
        a.stash = (float2*)c->stash2.p;
        TIMED(c, BIP_STAGE_MS_ROW, s, bip_ms_row_pass(plan, a, s));
        if (j > first) TIMED(c, BIP_STAGE_MS_COL, s, bip_ms_col_pass(plan, cols, s));
    }
    return BIP_OK;
}

}  // namespace

// ===========================================================================

extern "C" {

bip_status bip_create(const bip_config* cfg, bip_ctx** out) {
    BIP_RANGE("bip_create");
    if (!cfg || !out) return BIP_ERR_INVALID_ARG;
    *out = nullptr;
    const bip_config& g = *cfg;
    bip_ctx* c = new (std::nothrow) bip_ctx();
    if (!c) return BIP_ERR_OOM;
    auto bad = [&](bip_status s, const char*) {
        delete c;
        return s;
    };
    if (!grid_len_ok(g.ny) || !grid_len_ok(g.nx)) return bad(BIP_ERR_SHAPE, "grid");
    if (!(g.ly > 0) || !(g.lx > 0) || g.nz < 1 || !(g.dz >= 0) || !(g.e0 > 0) || !(g.alpha > 0) ||
        !(g.theta_det > 0) || !std::isfinite(g.defocus) || !std::isfinite(g.cs))
        return bad(BIP_ERR_INVALID_ARG, "optics");
    if (g.fy < 1 || g.fx < 1 || g.ny % g.fy || g.nx % g.fx) return bad(BIP_ERR_SHAPE, "f");
    if (g.dfy < 0 || g.dfx < 0 || (g.dfy > 0 && g.ny % g.dfy) || (g.dfx > 0 && g.nx % g.dfx))
        return bad(BIP_ERR_SHAPE, "detector subsampling");
    if (g.cube_ky < 0 || g.cube_kx < 0 || g.cube_ky > g.ny || g.cube_kx > g.nx || ((g.cube_ky > 0) != (g.cube_kx > 0)))
        return bad(BIP_ERR_SHAPE, "cube box");
    if (g.win < 16 || g.win % 16 || g.win > g.ny / g.fy || g.win > g.nx / g.fx) return bad(BIP_ERR_SHAPE, "win");
    if (g.nrad1 < 0 || g.nrad2 < 0 || g.nang1 < 1 || g.nang2 < 1) return bad(BIP_ERR_INVALID_ARG, "rings");
    if (g.recon != BIP_RECON_COMPLEX && g.recon != BIP_RECON_MAGNITUDE) return bad(BIP_ERR_INVALID_ARG, "recon");
    if (g.prec != BIP_PREC_FP32 && g.prec != BIP_PREC_SPLIT_BF16 && g.prec != BIP_PREC_MIXED &&
        g.prec != BIP_PREC_FP8_TILE)
        return bad(BIP_ERR_INVALID_ARG, "prec");
    c->cfg = g;
    c->prec = g.prec;
    std::string err;
    bip_status st = bip_geometry_cached(g, c->geo, err);
    if (st != BIP_OK) {
        delete c;
        return st;
    }
    c->Bpad = round_up(c->geo.B, kRowPad);
    c->Dpad = round_up(c->geo.n_det, kDetPad);
    *out = c;
    return BIP_OK;
}

bip_status bip_destroy(bip_ctx* c) {
    if (!c) return BIP_ERR_INVALID_ARG;
    DevBuf* all[] = {&c->twy, &c->twx, &c->py, &c->px, &c->ey, &c->ex, &c->shift1, &c->shift2, &c->hbeam,
                     &c->hdet, &c->coef, &c->grp1_off, &c->grp1_par, &c->grp1_w, &c->grp2_off, &c->grp2_par, &c->grp2_w, &c->ytab,
                     &c->xtab, &c->sites_d,
                     &c->plane_ids_d, &c->seq_ids_d, &c->row_off_d, &c->row_ent_d, &c->stash1, &c->stash2, &c->cols, &c->scans_d,
                     &c->gdiff, &c->kb_d, &c->lat_d, &c->work_d, &c->partial, &c->opA32, &c->opB32, &c->mt32, &c->q32, &c->opA16,
                     &c->opB16, &c->mt16, &c->q16, &c->errflag, &c->rsum, &c->wtc, &c->xtc, &c->illum,
                     &c->cube_scratch, &c->bin_of_d, &c->op8A, &c->op8B, &c->f8pmax, &c->f8inv0, &c->f8inv1,
                     &c->f8hmax, &c->f8H, &c->f8sA, &c->f8sB, &c->occ_d, &c->g_s1, &c->g_w, &c->g_R,
                     &c->g_gmt, &c->g_T, &c->g_D, &c->g_Dsum, &c->g_s1bar, &c->g_s2bar, &c->g_ubar, &c->g_dA,
                     &c->g_dt1, &c->g_dt2, &c->g_adj, &c->g_ckpt, &c->g_seg, &c->g_gvp, &c->pyc, &c->pxc,
                     &c->ray, &c->rax, &c->g_tA, &c->g_tB, &c->g_sA2, &c->g_sB2, &c->cubeA, &c->cubeB,
                     &c->cube_work, &c->cube_mask, &c->s1t, &c->psi, &c->ybuf, &c->cube_grp, &c->cube_wmap, &c->mpart,
                     &c->hcube, &c->shcube, &c->cstash, &c->ccols, &c->xopA, &c->xopB, &c->xm32, &c->tcache,
                     &c->cr_ay, &c->cr_ax, &c->cr_cy, &c->cr_cx, &c->cr_T, &c->nf_count, &c->tw512, &c->cols2};
    for (DevBuf* b : all) release(*b);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    for (int i = 0; i < 6; ++i) {
        release(c->aw1[i]);
        release(c->aw2[i]);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
    return BIP_OK;
}

bip_status bip_query(const bip_ctx* c, int32_t* B, int32_t* n_det, int32_t* Bp1, int32_t* Bp2, int32_t* n_sites) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (B) *B = c->geo.B;
    if (n_det) *n_det = c->geo.n_det;
    if (Bp1) *Bp1 = c->geo.Bp1;
    if (Bp2) *Bp2 = c->geo.Bp2;
    if (n_sites) *n_sites = (c->s1 || c->s2) ? c->n_sites : 0;
    return BIP_OK;
}

bip_status bip_get_geometry(const bip_ctx* c, int32_t* h_beam, int32_t* h_det, int32_t* p1, int32_t* p2,
                            double* w1, double* w2) {
    if (!c) return BIP_ERR_INVALID_ARG;
    const BipGeometry& g = c->geo;
    if (h_beam) std::memcpy(h_beam, g.h_beam.data(), g.h_beam.size() * sizeof(int32_t));
    if (h_det) std::memcpy(h_det, g.h_det.data(), g.h_det.size() * sizeof(int32_t));
    if (p1) std::memcpy(p1, g.p1.data(), g.p1.size() * sizeof(int32_t));
    if (p2) std::memcpy(p2, g.p2.data(), g.p2.size() * sizeof(int32_t));
    if (w1) std::memcpy(w1, g.w1.data(), g.w1.size() * sizeof(double));
    if (w2) std::memcpy(w2, g.w2.data(), g.w2.size() * sizeof(double));
    return BIP_OK;
}

bip_status bip_get_config(const bip_ctx* c, bip_config* out) {
    if (!c || !out) return BIP_ERR_INVALID_ARG;
    *out = c->cfg;
    return BIP_OK;
}

bip_status bip_set_precision(bip_ctx* c, int32_t prec) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (prec != BIP_PREC_FP32 && prec != BIP_PREC_SPLIT_BF16 && prec != BIP_PREC_MIXED &&
        prec != BIP_PREC_FP8_TILE)
        return fail(c, BIP_ERR_INVALID_ARG, "unknown precision");
    c->prec = prec;
    return BIP_OK;
}

const char* bip_last_error(const bip_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

bip_status bip_build_s1(bip_ctx* c, const float* V, const bip_atom* atoms, int32_t n_atoms, void* stream) {
    BIP_RANGE("bip_build_s1");
    cudaStream_t s = (cudaStream_t)stream;
    bip_status st = build_common(c, V, atoms, n_atoms, s);
    if (st != BIP_OK) return st;
    st = alloc_s1(c, s);
    if (st != BIP_OK) return st;
    st = sweep_s1(c, V, (float2*)c->cols.p, true, s);
    if (st != BIP_OK) return st;
    c->s1 = true;
    c->sig1 = site_signature(c->sites);
    return BIP_OK;
}

bip_status bip_build_s2(bip_ctx* c, const float* V, const bip_atom* atoms, int32_t n_atoms, void* stream) {
    BIP_RANGE("bip_build_s2");
    cudaStream_t s = (cudaStream_t)stream;
    bip_status st = build_common(c, V, atoms, n_atoms, s);
    if (st != BIP_OK) return st;
    st = alloc_s2(c, c->cols, s);
    if (st != BIP_OK) return st;
    st = sweep_s2(c, V, (float2*)c->cols.p, true, s);
    if (st != BIP_OK) return st;
    c->s2 = true;
    c->sig2 = site_signature(c->sites);
    return BIP_OK;
}

bip_status bip_build(bip_ctx* c, const float* V, const bip_atom* atoms, int32_t n_atoms, void* stream) {
    BIP_RANGE("bip_build");
    cudaStream_t s = (cudaStream_t)stream;
    if (!c) return BIP_ERR_INVALID_ARG;
    if (capturing(s)) return fail(c, BIP_ERR_INVALID_ARG, "bip_build is not capturable");
    bip_status st = build_common(c, V, atoms, n_atoms, s);
    if (st != BIP_OK) return st;
    // everything the two sweeps write is allocated before they fork
    st = alloc_s1(c, s);
    if (st == BIP_OK) st = alloc_s2(c, c->cols2, s);
    if (st != BIP_OK) return st;
    if (!c->side) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    if (!c->ev_fork) CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    if (!c->ev_join) CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    // the transmissions of every slice, once, before the fork (both sweeps read them)
    const size_t G = (size_t)c->cfg.ny * c->cfg.nx;
    TIMED(c, BIP_STAGE_TRANSMISSION, s, bip_transmission(V, (float)c->geo.sigma, 0, c->cfg.nz, G,
                                                         (float2*)c->tcache.p, s));
    c->s1 = c->s2 = false;
    CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));
    CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    // S1 on the caller's stream, S2 on the side stream; the caller's stream
    // waits for S2 whatever happened, so nothing of it runs on unjoined
    const bip_status st1 = sweep_s1(c, V, (float2*)c->cols.p, false, s);
    const bip_status st2 = st1 == BIP_OK ? sweep_s2(c, V, (float2*)c->cols2.p, false, c->side) : st1;
    const cudaError_t e1 = cudaEventRecord(c->ev_join, c->side);
    const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(s, c->ev_join, 0) : e1;
    if (st2 != BIP_OK) return st2;
    CUDA_TRY(c, e2);
    c->s1 = c->s2 = true;
    c->sig1 = c->sig2 = site_signature(c->sites);
    return BIP_OK;
}

}  // extern "C"

// ===========================================================================
// the map (Algorithm 5, per-site part)

namespace {

// Frees the map's batch-sized workspaces (operands, M, the cube kernel's
// operands and partial sums, the probe order's buffers, FP8 scales) after
// the stream has drained; the next map allocates what its batching needs.
// Tables, builds, scans and work lists stay.
void release_map_workspaces(bip_ctx* c, cudaStream_t s) {
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    for (DevBuf* b : {&c->opA32, &c->opB32, &c->mt32, &c->q32, &c->opA16, &c->opB16, &c->mt16, &c->q16,
                      &c->op8A, &c->op8B, &c->gdiff, &c->cubeA, &c->cubeB, &c->cube_mask, &c->mpart,
                      &c->s1t, &c->psi, &c->ybuf, &c->xtc, &c->f8pmax, &c->f8inv0, &c->f8inv1, &c->f8sA,
                      &c->f8sB})
        release(*b);
}

// Gather arguments of one side (1: S1 windows of the aperture beams,
// 2: S2 windows of the detector beams) for sites ids[0 .. n).
// w: the batch's window (0: the context's win), the central w x w block of
// the stashed windows.
GatherArgs gather_args(const bip_ctx* c, int side, const int32_t* ids, int n, int w = 0) {
    const bip_config& g = c->cfg;
    if (w <= 0) w = g.win;
    GatherArgs a{};
    a.n_sites = n;
    a.site_ids = ids;
    a.sites = (const SiteDev*)c->sites_d.p;
    a.win = w; a.ny = g.ny; a.nx = g.nx; a.K = w * w;
    a.stash_win = g.win;
    a.wo = (g.win - w) / 2;
    a.magnitude = g.recon == BIP_RECON_MAGNITUDE;
    a.ey = (const float2*)c->ey.p;
    a.ex = (const float2*)c->ex.p;
    a.ytab = (const float2*)c->ytab.p;
    a.xtab = (const float2*)c->xtab.p;
    a.fx = g.fx;
    if (side == 1) {
        a.Bp = c->geo.Bp1; a.n_targets = c->geo.B; a.rows_pad = c->geo.B;
        a.stash = (const float2*)c->stash1.p;
        a.grp = GroupDev{c->grp1_n, (const int32_t*)c->grp1_off.p, (const uint16_t*)c->grp1_par.p, (const float4*)c->grp1_w.p};
        a.h_t = (const int2*)c->hbeam.p;
        a.tilt_sign = +1;
    } else {
        a.Bp = c->geo.Bp2; a.n_targets = c->geo.n_det; a.rows_pad = c->geo.n_det;
        a.stash = (const float2*)c->stash2.p;
        a.grp = GroupDev{c->grp2_n, (const int32_t*)c->grp2_off.p, (const uint16_t*)c->grp2_par.p, (const float4*)c->grp2_w.p};
        a.h_t = (const int2*)c->hdet.p;
        a.tilt_sign = -1;
        a.fx = c->geo.dfx;      // the detector beams' lattice step along x
    }
    return a;
}

// Tensor-core reconstruction of one batch (mixed and FP8 paths): X planes
// from the stashes, then W X with the epilogue writing both coupling
// operands -- BF16, or E4M3 with the per-window scales computed in between
// from the parents' window maxima (which the X preparation takes).
// probe: the aperture side written transposed and without H_n, the probe
// order's operand: [site][4 planes][K][Bpad], re in plane 0 and im in plane 2
// (the split-BF16 layout with zero lo planes)
// w: the batch's window (0: the context's win; operand rows of w^2).
bip_status recon_tc_batch(bip_ctx* c, const int32_t* ids, int nb, const void* H, void* opA, void* opB,
                          cudaStream_t s, bool probe = false, bool s2_side = true, int w = 0) {
    const bip_config& g = c->cfg;
    const BipGeometry& geo = c->geo;
    if (w <= 0) w = g.win;
    const int K = w * w, Dpad = c->Dpad, Bpad = c->Bpad, nch = c->nch_max;
    const bool f8 = c->prec == BIP_PREC_FP8_TILE;
    CUDA_TRY(c, ensure(c->xtc, (size_t)2 * nb * 3 * K * 64 * sizeof(uint16_t), false, s));
    if (f8) {
        CUDA_TRY(c, ensure(c->f8pmax, (size_t)2 * nb * 64 * sizeof(unsigned), false, s));
        CUDA_TRY(c, ensure(c->f8inv0, (size_t)nb * Dpad * sizeof(float), false, s));
        CUDA_TRY(c, ensure(c->f8inv1, (size_t)nb * Bpad * sizeof(float), false, s));
        CUDA_TRY(c, ensure(c->f8sA, (size_t)nb * nch * Bpad * sizeof(float), false, s));
        CUDA_TRY(c, ensure(c->f8sB, (size_t)nb * Dpad * sizeof(float), false, s));
        CUDA_TRY(c, cudaMemsetAsync(c->f8pmax.p, 0, (size_t)2 * nb * 64 * sizeof(unsigned), s));
    }
    XprepArgs x{};
    x.n_sites = nb;
    x.site_ids = ids;
    x.K = K;
    x.w = w;
    x.stash_win = g.win;
    x.wo = (g.win - w) / 2;
    x.X = (uint16_t*)c->xtc.p;
    x.side[0] = XprepSide{s2_side ? (const float2*)c->stash2.p : nullptr, s2_side ? geo.Bp2 : 0, 0};
    x.side[1] = XprepSide{(const float2*)c->stash1.p, geo.Bp1, 3 * nb};
    x.pmax = f8 ? (unsigned*)c->f8pmax.p : nullptr;
    TIMED(c, BIP_STAGE_GATHER, s, bip_xprep(x, s));
    const int Dw = round_up(geo.n_det, kRowPad);
    if (f8) {
        F8ScaleArgs f{};
        f.n_sites = nb;
        f.site_ids = ids;
        f.sites = (const SiteDev*)c->sites_d.p;
        f.nch = nch;
        f.hmax = (const float*)c->f8hmax.p;
        f.W = (const uint16_t*)c->wtc.p;
        f.w_row0[0] = 0; f.w_pad[0] = Dw; f.n_targets[0] = geo.n_det; f.rows_pad[0] = Dpad;
        f.w_row0[1] = 2 * Dw; f.w_pad[1] = Bpad; f.n_targets[1] = geo.B; f.rows_pad[1] = Bpad;
        f.pmax = (const unsigned*)c->f8pmax.p;
        f.inv_row[0] = (float*)c->f8inv0.p;
        f.inv_row[1] = (float*)c->f8inv1.p;
        f.scaleB = (float*)c->f8sB.p;
        f.scaleA = (float*)c->f8sA.p;
        TIMED(c, BIP_STAGE_GATHER, s, bip_f8_scales(f, s));
    }
    ReconArgs r{};
    r.n_sites = nb;
    r.site_ids = ids;
    r.sites = (const SiteDev*)c->sites_d.p;
    r.K = K; r.win = w; r.ny = g.ny; r.nx = g.nx;
    r.stash_win = g.win;
    r.wo = (g.win - w) / 2;
    // work units of the largest multiple of 64 pixels up to 1024 that divides K
    r.chunk_px = 64;
    for (int cp = std::min(K, 1024) / 64 * 64; cp >= 64; cp -= 64)
        if (K % cp == 0) {
            r.chunk_px = cp;
            break;
        }
    r.chunks = K / r.chunk_px;
    r.magnitude = g.recon == BIP_RECON_MAGNITUDE;
    r.ey = (const float2*)c->ey.p;
    r.ex = (const float2*)c->ex.p;
    r.ytab = (const float2*)c->ytab.p;
    r.xtab = (const float2*)c->xtab.p;
    r.H = f8 ? (const float2*)c->f8H.p : (const float2*)H;
    r.W = (const uint16_t*)c->wtc.p;
    r.w_rows = 2 * Dw + 2 * Bpad;
    r.Xb = (const uint16_t*)c->xtc.p;
    r.x_rows = (int64_t)2 * nb * 3 * K;
    r.out[0] = (uint16_t*)opA;
    r.out[1] = (uint16_t*)opB;
    r.side[0] = ReconSide{geo.n_det, Dpad, Dw, Dw / 128, 0, -1, (const int2*)c->hdet.p, 0, 0,
                          (int64_t)2 * Dpad * K, (int64_t)Dpad * K};
    if (!s2_side) r.side[0] = ReconSide{0, 0, 0, 0, 0, -1, (const int2*)c->hdet.p, 0, 0, 0, 0};
    r.side[1] = ReconSide{geo.B, Bpad, Bpad, Bpad / 128, nch, +1, (const int2*)c->hbeam.p, 2 * Dw, 3 * nb,
                          (int64_t)2 * nch * Bpad * K, (int64_t)nch * Bpad * K};
    if (probe) {
        r.side[1].nch = 0;
        r.side[1].site_stride = (int64_t)4 * K * Bpad;
        r.side[1].plane_stride = (int64_t)2 * K * Bpad;
        r.side[1].trans = 1;
        r.side[1].ld = Bpad;
    }
    r.err = (int*)c->errflag.p;
    r.wait_ns = c->wait_ns;
    if (f8) {
        r.f8 = 1;
        r.inv_row[0] = (const float*)c->f8inv0.p;
        r.inv_row[1] = (const float*)c->f8inv1.p;
    }
    TIMED(c, BIP_STAGE_GATHER, s, bip_recon_tc(r, s));
    return BIP_OK;
}

// ---- reverse pass through the reconstruction and the sweeps

// per-target and per-parent lists of the non-zero weights of one side
bip_status adj_tables(bip_ctx* c, cudaStream_t s) {
    if (c->adj_tables) return BIP_OK;
    const BipGeometry& geo = c->geo;
    const bip_config& g = c->cfg;
    auto build = [&](const std::vector<double>& w, int nt, int bp, DevBuf* out) -> bip_status {
        std::vector<int32_t> toff(1, 0), tpar, poff(1, 0), ptgt;
        std::vector<float> tw, pw;
        for (int t = 0; t < nt; ++t) {
            for (int p = 0; p < bp; ++p)
                if (w[(size_t)t * bp + p] != 0.0) {
                    tpar.push_back(p);
                    tw.push_back((float)w[(size_t)t * bp + p]);
                }
            toff.push_back((int32_t)tpar.size());
        }
        for (int p = 0; p < bp; ++p) {
            for (int t = 0; t < nt; ++t)
                if (w[(size_t)t * bp + p] != 0.0) {
                    ptgt.push_back(t);
                    pw.push_back((float)w[(size_t)t * bp + p]);
                }
            poff.push_back((int32_t)ptgt.size());
        }
        CUDA_TRY(c, upload(out[0], toff, s));
        CUDA_TRY(c, upload(out[1], tpar, s));
        CUDA_TRY(c, upload(out[2], tw, s));
        CUDA_TRY(c, upload(out[3], poff, s));
        CUDA_TRY(c, upload(out[4], ptgt, s));
        CUDA_TRY(c, upload(out[5], pw, s));
        return BIP_OK;
    };
    bip_status st = build(geo.w1, geo.B, geo.Bp1, c->aw1);
    if (st != BIP_OK) return st;
    st = build(geo.w2, geo.n_det, geo.Bp2, c->aw2);
    if (st != BIP_OK) return st;
    // conj(P): the propagator tables of the forward sweep, conjugated
    std::vector<float2> py(g.ny), px(g.nx);
    CUDA_TRY(c, cudaMemcpyAsync(py.data(), c->py.p, g.ny * sizeof(float2), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaMemcpyAsync(px.data(), c->px.p, g.nx * sizeof(float2), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    for (auto& v : py) v.y = -v.y;
    for (auto& v : px) v.y = -v.y;
    CUDA_TRY(c, upload(c->pyc, py, s));
    CUDA_TRY(c, upload(c->pxc, px, s));
    c->adj_tables = true;
    return BIP_OK;
}

AdjWeights adj_weights(DevBuf* w) {
    return AdjWeights{(const int32_t*)w[0].p, (const int32_t*)w[1].p, (const float*)w[2].p,
                      (const int32_t*)w[3].p, (const int32_t*)w[4].p, (const float*)w[5].p};
}

int isqrt_up(int n) {
    int k = 1;
    while (k * k < n) ++k;
    return k;
}

// dL/dV_j through the S1 sweep (psi_{j+1} = Prop(T_j psi_j)), j < the last
// ionization plane, from the window adjoints dtbar1 of every site; forward
// states recomputed from checkpoints every ceil(sqrt(n)) slices
bip_status adjoint_s1(bip_ctx* c, const float* V, float* dV, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const size_t G = (size_t)g.ny * g.nx;
    const int ncol = c->geo.Bp1;
    int jmax = 0;
    for (auto& sd : c->sites) jmax = std::max(jmax, (int)sd.plane);
    if (jmax == 0) return BIP_OK;
    const int n = jmax, k = isqrt_up(n), nck = (n + k - 1) / k;
    const size_t state = (size_t)ncol * G;
    CUDA_TRY(c, ensure(c->g_adj, state * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->g_ckpt, (size_t)nck * state * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->g_seg, (size_t)k * state * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->g_gvp, (size_t)ncol * G * sizeof(float), false, s));
    MsPlan fp = plan_for(c, ncol, c->shift1), cp = fp;
    cp.py = (const float2*)c->pyc.p;
    cp.px = (const float2*)c->pxc.p;
    float2* cols = (float2*)c->cols.p;
    float2* adj = (float2*)c->g_adj.p;
    auto row_off = [&](int j) -> const int32_t* {
        return c->plane_off[j + 1] > c->plane_off[j] ? (const int32_t*)c->row_off_d.p + (size_t)j * (g.ny + 1) : nullptr;
    };
    auto fwd_row = [&](int j, float2* save, bool fft) -> cudaError_t {
        MsRowArgs a{};
        a.cols = cols;
        a.init = j == 0;
        a.init_val = 1.0f;
        a.do_ifft = j > 0;
        a.v_post = V + (size_t)j * G;
        a.do_fft = fft;
        a.win = g.win;
        a.save = save;
        return bip_ms_row_pass(fp, a, s);
    };
    // forward sweep, keeping the field at the start of every k-th step
    const int last_ck = (nck - 1) * k;
    for (int j = 0; j < last_ck; ++j) {
        if (j % k == 0 && j > 0)
            CUDA_TRY(c, cudaMemcpyAsync((float2*)c->g_ckpt.p + (size_t)(j / k) * state, cols, state * sizeof(float2),
                                        cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(c, fwd_row(j, nullptr, true));
        CUDA_TRY(c, bip_ms_col_pass(fp, cols, s));
    }
    if (last_ck > 0)
        CUDA_TRY(c, cudaMemcpyAsync((float2*)c->g_ckpt.p + (size_t)(last_ck / k) * state, cols, state * sizeof(float2),
                                    cudaMemcpyDeviceToDevice, s));
    int groups = 0;
    auto adj_row = [&](int j, bool zero_in, const float2* st, bool fft) -> bip_status {
        MsAdjArgs a{};
        a.cols = adj;
        a.zero_in = zero_in;
        a.do_ifft = !zero_in;
        a.v = zero_in ? nullptr : V + (size_t)j * G;
        a.state = st;
        a.state_times_T = 1;
        a.inj_before = 0;
        a.row_off = row_off(j);
        a.row_ent = (const int4*)c->row_ent_d.p;
        a.win = g.win;
        a.inj = (const float2*)c->g_dt1.p;
        a.gv_part = (float*)c->g_gvp.p;
        a.do_fft = fft;
        CUDA_TRY(c, bip_ms_adj_row_pass(fp, a, &groups, s));
        if (st) CUDA_TRY(c, bip_gv_reduce((const float*)c->g_gvp.p, groups, (int)G, dV + (size_t)j * G, s));
        return BIP_OK;
    };
    // lambda at the last plane: its window adjoints only
    bip_status st = adj_row(jmax, true, nullptr, true);
    if (st != BIP_OK) return st;
    CUDA_TRY(c, bip_ms_col_pass(cp, adj, s));
    for (int m = nck - 1; m >= 0; --m) {
        const int j0 = m * k, j1 = std::min(j0 + k, n) - 1;
        if (m > 0)
            CUDA_TRY(c, cudaMemcpyAsync(cols, (float2*)c->g_ckpt.p + (size_t)m * state, state * sizeof(float2),
                                        cudaMemcpyDeviceToDevice, s));
        for (int j = j0; j <= j1; ++j) {
            CUDA_TRY(c, fwd_row(j, (float2*)c->g_seg.p + (size_t)(j - j0) * state, j < j1));
            if (j < j1) CUDA_TRY(c, bip_ms_col_pass(fp, cols, s));
        }
        for (int j = j1; j >= j0; --j) {
            st = adj_row(j, false, (const float2*)c->g_seg.p + (size_t)(j - j0) * state, j > 0);
            if (st != BIP_OK) return st;
            if (j > 0) CUDA_TRY(c, bip_ms_col_pass(cp, adj, s));
        }
    }
    return BIP_OK;
}

// dL/dV_j through the S2 sweep (x_j = T_j Prop(x_{j+1})), j >= the first
// ionization plane, ascending, from the window adjoints dtbar2
bip_status adjoint_s2(bip_ctx* c, const float* V, float* dV, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const size_t G = (size_t)g.ny * g.nx;
    const int ncol = c->geo.Bp2;
    int first = g.nz;
    for (auto& sd : c->sites) first = std::min(first, (int)sd.plane);
    if (first >= g.nz) return BIP_OK;
    const int n = g.nz - first, k = isqrt_up(n), nck = (n + k - 1) / k;
    const size_t state = (size_t)ncol * G;
    CUDA_TRY(c, ensure(c->g_adj, state * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->g_ckpt, (size_t)nck * state * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->g_seg, (size_t)k * state * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->g_gvp, (size_t)ncol * G * sizeof(float), false, s));
    MsPlan fp = plan_for(c, ncol, c->shift2), cp = fp;
    cp.py = (const float2*)c->pyc.p;
    cp.px = (const float2*)c->pxc.p;
    float2* cols = (float2*)c->cols.p;
    float2* adj = (float2*)c->g_adj.p;
    auto row_off = [&](int j) -> const int32_t* {
        return c->plane_off[j + 1] > c->plane_off[j] ? (const int32_t*)c->row_off_d.p + (size_t)j * (g.ny + 1) : nullptr;
    };
    auto fwd_row = [&](int j, float2* save, bool fft) -> cudaError_t {
        MsRowArgs a{};
        a.cols = cols;
        a.do_ifft = 1;
        a.v_pre = V + (size_t)j * G;
        a.do_fft = fft;
        a.win = g.win;
        a.save = save;
        return bip_ms_row_pass(fp, a, s);
    };
    // forward: the start column, then j = nz-1 down, keeping the field at the
    // start of row pass j for j = nz-1 - m k
    {
        MsRowArgs a{};
        a.cols = cols;
        a.init = 1;
        a.init_val = (float)(1.0 / std::sqrt((double)G));
        a.do_fft = 1;
        a.win = g.win;
        CUDA_TRY(c, bip_ms_row_pass(fp, a, s));
        CUDA_TRY(c, bip_ms_col_pass(fp, cols, s));
    }
    const int lowest_ck = g.nz - 1 - (nck - 1) * k;
    for (int j = g.nz - 1; j >= lowest_ck; --j) {
        if ((g.nz - 1 - j) % k == 0)
            CUDA_TRY(c, cudaMemcpyAsync((float2*)c->g_ckpt.p + (size_t)((g.nz - 1 - j) / k) * state, cols,
                                        state * sizeof(float2), cudaMemcpyDeviceToDevice, s));
        if (j == lowest_ck) break;
        CUDA_TRY(c, fwd_row(j, nullptr, true));
        CUDA_TRY(c, bip_ms_col_pass(fp, cols, s));
    }
    int groups = 0;
    for (int m = nck - 1; m >= 0; --m) {
        const int jhi = g.nz - 1 - m * k, jlo = std::max(first, jhi - k + 1);
        CUDA_TRY(c, cudaMemcpyAsync(cols, (float2*)c->g_ckpt.p + (size_t)m * state, state * sizeof(float2),
                                    cudaMemcpyDeviceToDevice, s));
        for (int j = jhi; j >= jlo; --j) {
            CUDA_TRY(c, fwd_row(j, (float2*)c->g_seg.p + (size_t)(j - jlo) * state, j > jlo));
            if (j > jlo) CUDA_TRY(c, bip_ms_col_pass(fp, cols, s));
        }
        for (int j = jlo; j <= jhi; ++j) {
            MsAdjArgs a{};
            a.cols = adj;
            a.zero_in = j == first;
            a.do_ifft = j > first;
            a.v = V + (size_t)j * G;
            a.state = (const float2*)c->g_seg.p + (size_t)(j - jlo) * state;
            a.state_times_T = 0;
            a.inj_before = 1;
            a.row_off = row_off(j);
            a.row_ent = (const int4*)c->row_ent_d.p;
            a.win = g.win;
            a.inj = (const float2*)c->g_dt2.p;
            a.gv_part = (float*)c->g_gvp.p;
            a.do_fft = j < g.nz - 1;
            CUDA_TRY(c, bip_ms_adj_row_pass(fp, a, &groups, s));
            CUDA_TRY(c, bip_gv_reduce((const float*)c->g_gvp.p, groups, (int)G, dV + (size_t)j * G, s));
            if (j < g.nz - 1) CUDA_TRY(c, bip_ms_col_pass(cp, adj, s));
        }
    }
    return BIP_OK;
}

// FP8 path: max_r |H_n| of every channel of every site and H_n divided by
// it, once per call
bip_status f8_hmax(bip_ctx* c, const void* H, cudaStream_t s) {
    CUDA_TRY(c, ensure(c->f8hmax, (size_t)c->n_sites * 9 * sizeof(float), false, s));
    CUDA_TRY(c, ensure(c->f8H, (size_t)c->h_elems * sizeof(float2), false, s));
    F8HmaxArgs h{c->n_sites, (const SiteDev*)c->sites_d.p, (const float2*)H, (float*)c->f8hmax.p,
                 (float2*)c->f8H.p};
    TIMED(c, BIP_STAGE_GATHER, s, bip_f8_hmax(h, s));
    return BIP_OK;
}

// BF16 planes of the coupling output and the Gram operands: split BF16
// keeps hi and lo (4), the mixed and FP8 paths one BF16 value (2)
int gram_planes(int prec) { return prec == BIP_PREC_SPLIT_BF16 ? 4 : 2; }

// Sites per batch of the tensor-core map path: the batch whose tile counts
// fill whole rounds of the SMs best (the coupling, the reconstruction and
// the Gram launch one CTA per SM and walk their tiles in rounds), weighted
// by the stages' usual shares of the map time, between 16 and 32 sites, and
// -- above 16 -- small enough that the batch's coupling output (which the
// Gram re-reads several times) stays within 1.2 x the L2 cache.
int tc_batch(const bip_ctx* c) {
    // the device's SM count and L2 size, read once (thread-safe
    // initialisation; one GPU per process)
    static const int2 dev_info = [] {
        int dev = 0, sms = 0, l2 = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 148;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 < 1) l2 = 64 << 20;
        return int2{sms, l2};
    }();
    const int sms = dev_info.x, l2 = dev_info.y;
    const int npl = gram_planes(c->prec);
    const double mt_site = 2.0 * npl * c->Bpad * (double)c->nch_max * c->Dpad;   // bytes of Mt per site
    // at least 16 sites: fewer leave the Gram (a few tiles per site) without
    // enough tiles to fill the SMs
    const int sb_max = std::max(16, std::min(32, (int)(1.2 * l2 / mt_site)));
    const int K = c->cfg.win * c->cfg.win, nch = c->nch_max;
    const int cw = tile_width(c->Dpad);
    const int coupling = (nch * c->Bpad / 128) * ((c->Dpad + cw - 1) / cw);
    const int recon = (round_up(c->geo.n_det, kRowPad) / 128 + c->Bpad / 128) * (K / std::min(K, 1024));
    int gram = 0;
    for (int mt = 0; mt < c->Bpad / 128; ++mt)
        for (int nt = 0; nt < c->Bpad / 256; ++nt) gram += (nt + 1) * 256 > mt * 128;
    auto eff = [&](int per, int sb) {
        const int units = per * sb;
        return (double)units / ((double)((units + sms - 1) / sms) * sms);
    };
    int best = 16;
    double best_e = -1.0;
    for (int sb = 16; sb <= sb_max; ++sb) {
        const double e = 0.6 * eff(coupling, sb) + 0.3 * eff(recon, sb) + 0.1 * eff(gram, sb);
        if (e > best_e + 1e-9) {
            best_e = e;
            best = sb;
        }
    }
    return std::min(c->n_sites, best);
}

bip_status check_map_args(bip_ctx* c, const void* H, const double* scans, int32_t P, const void* out) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!c->s1 || !c->s2 || c->sig1 != c->sig2)
        return fail(c, BIP_ERR_INVALID_ARG, "bip_build_s1 and bip_build_s2 must run first on the same sites");
    if (!H || !scans || !out) return fail(c, BIP_ERR_INVALID_ARG, "null pointer argument");
    if ((reinterpret_cast<uintptr_t>(H) & 15) != 0) return fail(c, BIP_ERR_INVALID_ARG, "H must be 16-byte aligned");
    if (P < 1) return fail(c, BIP_ERR_INVALID_ARG, "P must be >= 1");
    for (int i = 0; i < 2 * P; ++i)
        if (!std::isfinite(scans[i])) return fail(c, BIP_ERR_INVALID_ARG, "scan position is not finite");
    return BIP_OK;
}

// A scan list that is a raster: scan my Mx + mx at (y_my, x_mx), rows of
// equal y, the x of every row the same sequence (equal within 1e-9 px).
struct Raster {
    bool ok = false;
    int My = 0, Mx = 0;
};
Raster detect_raster(const double* sc, int P) {
    Raster r;
    if (P < 1) return r;
    int Mx = 1;
    while (Mx < P && sc[2 * Mx] == sc[0]) ++Mx;
    if (P % Mx) return r;
    const int My = P / Mx;
    for (int p = 0; p < P; ++p) {
        const int i = p / Mx, j = p % Mx;
        if (std::fabs(sc[2 * p] - sc[2 * (size_t)i * Mx]) > 1e-9 || std::fabs(sc[2 * p + 1] - sc[2 * j + 1]) > 1e-9)
            return r;
    }
    r.ok = true;
    r.My = My;
    r.Mx = Mx;
    return r;
}

// exp(2 pi i t), t reduced to [0, 1) turns in FP64
float2 turn_d(double t) {
    t -= std::floor(t);
    return float2{(float)std::cos(2.0 * kPi * t), (float)std::sin(2.0 * kPi * t)};
}

// conservative test: can any scan with y in [y0, y1] and x in [x0, x1] lie
// inside the crop window of site (ty, tx)?
bool box_meets_crop(double y0, double y1, double x0, double x1, double ty, double tx, const bip_config& g) {
    auto axis = [](double lo, double hi, double t, int n, int f) {
        const double half = 0.5 * n / f;
        for (int k = -2; k <= 2; ++k) {
            const double a = t - half + (double)k * n, b = t + half + (double)k * n;
            if (hi >= a && lo < b) return true;
        }
        return false;
    };
    return axis(y0, y1, ty, g.ny, g.fy) && axis(x0, x1, tx, g.nx, g.fx);
}

// Cube accumulation arguments of one batch (the coupling's format is set by
// the caller).
CubeArgs cube_args(const bip_ctx* c, const int32_t* ids, int nb, int P, float* cube) {
    const bip_config& g = c->cfg;
    CubeArgs a{};
    a.n_sites = nb;
    a.site_ids = ids;
    a.sites = (const SiteDev*)c->sites_d.p;
    a.n_det = c->geo.n_det;
    a.Bpad = c->Bpad;
    a.nch = c->nch_max;
    a.Dp = c->Dpad;
    a.m_ld = (int64_t)c->nch_max * c->Dpad;
    a.C = (const float2*)c->illum.p;
    a.P = P;
    a.scans = (const double*)c->scans_d.p;
    a.ny = g.ny; a.nx = g.nx; a.fy = g.fy; a.fx = g.fx;
    a.scale = (float)det_scale(c);
    a.cube = cube;
    a.cube_ld = c->geo.n_det;
    return a;
}

// The coupling operands' rows past a side's targets (the padding up to
// Dpad / Bpad) must read as zero: the Gram contraction runs over every
// detector row (and the probe order's operands are cleared with them).  The buffers are zeroed when allocated and every writer
// packs target rows only, at pitch K = w^2; after a batch packed at another
// pitch, rows that are padding at pitch K may hold values, so the buffers
// are cleared before the pitch changes (never while every site has the
// context's window).
bip_status operand_layout(bip_ctx* c, int K, cudaStream_t s) {
    if (c->op_k == K) return BIP_OK;
    if (c->op_k != 0)
        for (DevBuf* b : {&c->opA16, &c->opB16, &c->op8A, &c->op8B, &c->opA32, &c->opB32, &c->s1t, &c->psi, &c->ybuf})
            if (b->p) CUDA_TRY(c, cudaMemsetAsync(b->p, 0, b->cap, s));
    c->op_k = K;
    return BIP_OK;
}

// Batches of the map: at most SB consecutive sites of the batch order, a
// batch never spanning two window sizes (its contractions run at K = w^2).
// With every site at the context's window these are the sites 0..SB-1,
// SB..2SB-1, ...
std::vector<std::pair<int, int>> map_batches(const bip_ctx* c, int SB) {
    std::vector<std::pair<int, int>> out;
    for (int b0 = 0; b0 < c->n_sites;) {
        const int w = c->sites[c->batch_order[b0]].w;
        int nb = 1;
        while (nb < SB && b0 + nb < c->n_sites && c->sites[c->batch_order[b0 + nb]].w == w) ++nb;
        out.push_back({b0, nb});
        b0 += nb;
    }
    return out;
}

bip_status raster_cube_setup(bip_ctx* c, const double* scans, int P, int SB, int nd_pad, int64_t m_b, int64_t m_ch,
                             int64_t m_site, int64_t cube_ld, float scale, CubeRasterArgs& cra, bool& sep,
                             cudaStream_t s);
// The map, its per-site contributions, or the 4D cube (cube_out [P][n_det]):
// the reconstruction and the coupling are shared, then either the Gram
// matrix and the scan polynomial or the per-beam contraction.
bip_status run_map(bip_ctx* c, const void* H, const double* scans, int32_t P, float* partial_out,
                   double* map_out, float* cube_out, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const BipGeometry& geo = c->geo;
    const int K = g.win * g.win;
    const int Bpad = c->Bpad, Dpad = c->Dpad;
    const int nch = c->nch_max;
    const bool tc = c->prec != BIP_PREC_FP32;
    // planes of the coupling and Gram operands: split BF16 (4) or BF16 (2);
    // the FP8 coupling reads two E4M3 planes and writes BF16 for the Gram
    const int npl = gram_planes(c->prec);
    const bool f8 = c->prec == BIP_PREC_FP8_TILE;
    if (f8 && !c->recon_tc)
        return fail(c, BIP_ERR_UNSUPPORTED, "the FP8 coupling needs at most 64 parents per side");
    const int tile = kScanTile;
    const int n_tiles = (P + tile - 1) / tile;
    const int nd = (2 * c->Ky + 1) * (4 * c->Kx + 1);

    // the scan list, uploaded unless a capture-safe context already holds it
    const bool same_scans = c->capture_safe && c->scans_cache.size() == (size_t)P * 2 &&
                            std::equal(scans, scans + 2 * P, c->scans_cache.begin());
    if (!same_scans) {
        if (capturing(s))
            return fail(c, BIP_ERR_INVALID_ARG,
                        "a captured map must repeat the scans of the capture-safe warm-up call");
        CUDA_TRY(c, ensure(c->scans_d, (size_t)P * 2 * sizeof(double), false, s));
        CUDA_TRY(c, cudaMemcpyAsync(c->scans_d.p, scans, (size_t)P * 2 * sizeof(double), cudaMemcpyHostToDevice, s));
        c->scans_cache.assign(scans, scans + 2 * P);
    }
    float* partial = partial_out;
    // beam order: the map as |M c|^2 summed over the detector beams on the
    // cube kernel, without the Gram matrix (tensor-core precisions)
    const bool beam = !cube_out && tc && c->order == 1;
    // probe order: the windowed probes Psi = C^T S1 of every scan, then
    // |S2^T (H_n x Psi)|^2 summed over d and n on the cube kernel (mixed)
    const bool probe = !cube_out && c->order == 2;
    if (probe && (c->prec != BIP_PREC_MIXED || !c->recon_tc))
        return fail(c, BIP_ERR_UNSUPPORTED, "the probe order needs the mixed precision and at most 64 parents per side");
    if (probe && P > kProbeMaxScans) return fail(c, BIP_ERR_UNSUPPORTED, "the probe order takes at most 2048 scans");
    if (cube_out || beam || probe) {
        // c_b(rho) for every scan
        CUDA_TRY(c, ensure(c->illum, (size_t)Bpad * P * sizeof(float2), false, s));
        IllumArgs ia{P, geo.B, Bpad, (const int2*)c->hbeam.p, (const double2*)c->coef.p, (const double*)c->scans_d.p,
                     g.ny, g.nx, (float2*)c->illum.p};
        CUDA_TRY(c, bip_illum(ia, s));
    }
    if (cube_out) {
        // the cube cleared
        CUDA_TRY(c, cudaMemsetAsync(cube_out, 0, (size_t)P * geo.n_det * sizeof(float), s));
    } else {
        if (!partial) {
            CUDA_TRY(c, ensure(c->partial, (size_t)c->n_sites * P * sizeof(float), false, s));
            partial = (float*)c->partial.p;
        }
        // scans outside a site's crop mask stay 0: the evaluation writes only
        // the scan tiles that can meet the mask
        CUDA_TRY(c, cudaMemsetAsync(partial, 0, (size_t)c->n_sites * P * sizeof(float), s));
    }

    // raster scan lists take the separable evaluation: phase tables per scan
    // row and column, angles reduced in FP64
    Raster raster;
    RasterArgs rargs{};
    if (!cube_out && !beam && !probe && c->raster_eval) raster = detect_raster(scans, P);
    if (raster.ok) {
        const int rows = 2 * c->Ky + 1, cols = 4 * c->Kx + 1;
        if (!same_scans) {
            std::vector<float2> ay((size_t)raster.My * rows), ax((size_t)cols * raster.Mx);
            for (int my = 0; my < raster.My; ++my) {
                const double ry = scans[2 * (size_t)my * raster.Mx];
                for (int iy = 0; iy < rows; ++iy)
                    ay[(size_t)my * rows + iy] = turn_d((double)g.fy * (iy - 2 * c->Ky) * ry / g.ny);
            }
            for (int mx = 0; mx < raster.Mx; ++mx) {
                const double rx = scans[2 * (size_t)mx + 1];
                for (int j = 0; j < cols; ++j) ax[(size_t)j * raster.Mx + mx] = turn_d((double)g.fx * (j - 2 * c->Kx) * rx / g.nx);
            }
            CUDA_TRY(c, upload(c->ray, ay, s));
            CUDA_TRY(c, upload(c->rax, ax, s));
        }
        rargs = RasterArgs{raster.My, raster.Mx, (const float2*)c->ray.p, (const float2*)c->rax.p};
    }

    // scan-tile bounding boxes (host)
    std::vector<double> bb((size_t)n_tiles * 4);
    for (int t = 0; t < n_tiles; ++t) {
        double y0 = INFINITY, y1 = -INFINITY, x0 = INFINITY, x1 = -INFINITY;
        for (int p = t * tile; p < std::min(P, (t + 1) * tile); ++p) {
            y0 = std::min(y0, scans[2 * p]);
            y1 = std::max(y1, scans[2 * p]);
            x0 = std::min(x0, scans[2 * p + 1]);
            x1 = std::max(x1, scans[2 * p + 1]);
        }
        bb[4 * t] = y0; bb[4 * t + 1] = y1; bb[4 * t + 2] = x0; bb[4 * t + 3] = x1;
    }

    const int SB = c->sb_override > 0 ? std::min(c->n_sites, c->sb_override)
                                      : (tc ? tc_batch(c) : std::min(c->n_sites, 8));
    const std::vector<std::pair<int, int>> batches = map_batches(c, SB);
    // workspaces for the context's window (the largest); a batch of smaller
    // windows uses the front of each
    const size_t rowsA = Dpad, rowsB = (size_t)nch * Bpad;
    const size_t perA = rowsA * K, perB = rowsB * K;
    const size_t perMt = (size_t)Bpad * nch * Dpad, perQ = (size_t)Bpad * Bpad;
    if (!tc) {
        CUDA_TRY(c, ensure(c->opA32, SB * perA * sizeof(float2), true, s));
        CUDA_TRY(c, ensure(c->opB32, SB * perB * sizeof(float2), true, s));
        CUDA_TRY(c, ensure(c->mt32, SB * perMt * sizeof(float2), true, s));
    } else {
        // up to four bf16 planes per complex element: 8 bytes, as complex64
        if (f8) {
            // two E4M3 planes per complex element
            CUDA_TRY(c, ensure(c->op8A, SB * perA * 2, true, s));
            CUDA_TRY(c, ensure(c->op8B, SB * perB * 2, true, s));
        } else {
            CUDA_TRY(c, ensure(c->opA16, SB * perA * 8, true, s));
            CUDA_TRY(c, ensure(c->opB16, SB * perB * 8, true, s));
        }
        CUDA_TRY(c, ensure(c->mt16, SB * perMt * 8, true, s));
        if (cube_out || beam) CUDA_TRY(c, ensure(c->mt32, SB * perMt * sizeof(float2), true, s));
        if (probe) {
            const size_t P128 = round_up(P, 128), P64r = round_up(P, 64);
            CUDA_TRY(c, ensure(c->s1t, SB * 4 * (size_t)K * Bpad * sizeof(uint16_t), true, s));
            // zeroed when allocated: rows of scans beyond the last 16-scan tile
            // are never written and reach only masked columns of the cube kernel
            CUDA_TRY(c, ensure(c->psi, SB * P128 * K * sizeof(float2), true, s));
            CUDA_TRY(c, ensure(c->ybuf, SB * 2 * P64r * nch * K * sizeof(uint16_t), true, s));
        }
        CUDA_TRY(c, cudaMemsetAsync(c->errflag.p, 0, sizeof(int), s));
    }
    CUDA_TRY(c, ensure(c->q32, SB * perQ * sizeof(float2), true, s));
    // G(Delta) of every site when the raster evaluation runs once at the end,
    // else of one batch
    CUDA_TRY(c, ensure(c->gdiff, (size_t)(raster.ok ? c->n_sites : SB) * nd * sizeof(float2), false, s));

    if (f8 && c->n_sites > 0) {
        bip_status st = f8_hmax(c, H, s);
        if (st != BIP_OK) return st;
    }

    // work lists (site in batch, scan tile) for all batches, uploaded once
    // (kept across calls of a capture-safe context while scans, sites and
    // batching are unchanged)
    const uint64_t work_key = (c->sig1 * 1000003ull) ^ ((uint64_t)SB << 32) ^ (uint64_t)P;
    const bool same_work = same_scans && c->work_key == work_key;
    std::vector<int32_t>& work = c->work_h;
    std::vector<int>& batch_off = c->batch_off_cache;
    if (!same_work) {
    work.clear();
    batch_off.clear();
    for (const auto& bt : batches) {
        batch_off.push_back((int)work.size() / 2);
        for (int bs = 0; bs < bt.second; ++bs) {
            const SiteDev& sd = c->sites[c->batch_order[bt.first + bs]];
            for (int t = 0; t < n_tiles; ++t)
                if (box_meets_crop(bb[4 * t], bb[4 * t + 1], bb[4 * t + 2], bb[4 * t + 3], sd.ty, sd.tx, g)) {
                    work.push_back(bs);
                    work.push_back(t);
                }
        }
    }
    batch_off.push_back((int)work.size() / 2);
    if (capturing(s))
        return fail(c, BIP_ERR_INVALID_ARG, "a captured map must repeat the arguments of the capture-safe warm-up call");
    CUDA_TRY(c, upload(c->work_d, work, s));
    c->work_key = work_key;
    }

    // the cube on tcgen05: c_b(rho) as split planes [4][crow][Bpad] once, and
    // work lists of (site in batch, scan tile meeting its crop mask)
    // the per-beam cube of qEELS on a raster scan list: the separated
    // contraction of cube_raster.cu instead of the cube kernel
    CubeRasterArgs cra{};
    bool sepq = false;
    if (cube_out) {
        bip_status st = raster_cube_setup(c, scans, P, SB, Dpad, tc ? (int64_t)Dpad : (int64_t)nch * Dpad,
                                          tc ? (int64_t)Bpad * Dpad : (int64_t)Dpad, (int64_t)perMt, geo.n_det,
                                          (float)det_scale(c), cra, sepq, s);
        if (st != BIP_OK) return st;
    }
    const bool cube_tc = (cube_out || beam || probe) && tc && !sepq;
    // scans per tile of the cube kernel (its MMA's N) for the cube and the
    // beam order: 128 once there are that many scans, else 64; the probe
    // order's last contraction keeps 64
    const int ctn = (cube_out || beam) && P >= 128 ? 128 : 64;
    // the probe order's last contraction: the channels in the tile's columns
    // ((scan, channel) pairs, one accumulator) when that takes fewer 64-wide
    // tiles than a 64-scan tile with one accumulator per channel (few scans)
    const bool probe_cols = probe && (P * nch + 63) / 64 < nch * ((P + 63) / 64);
    const int P64 = round_up(P, 64), D128 = round_up(Dpad, 128);
    // rows of each plane of C^T: whole scan tiles of the cube kernel, or (probe
    // order) whole 128-row tiles
    const int crow = probe ? round_up(P, 128) : round_up(P, ctn);
    const size_t KB = (size_t)nch * Bpad;
    std::vector<int> cube_off, cube_goff;
    int n_ct_map = 0;                   // map modes: scan tiles per site (the wmap rows)
    if (cube_tc) {
        CUDA_TRY(c, ensure(c->cubeB, (size_t)4 * crow * Bpad * sizeof(uint16_t), true, s));
        if (!probe) CUDA_TRY(c, ensure(c->cubeA, (size_t)SB * 4 * D128 * KB * sizeof(uint16_t), true, s));
        SplitArgs sc{(const float2*)c->illum.p, 1, P, 0, P, Bpad, 1, (uint16_t*)c->cubeB.p, 0, crow, Bpad, 0, 0};
        CUDA_TRY(c, bip_split_planes(sc, s));
        // tiles of ctn scans -- or, for the probe order with fewer columns that
        // way, of 64 (scan, channel) columns -- and their scans' bounding boxes
        const int ncol = probe_cols ? nch : 1;
        const int tile = probe ? 64 : ctn;
        const int n_ct = (P * ncol + tile - 1) / tile;
        std::vector<double> bb64;
        for (int t = 0; t < n_ct; ++t) {
            double y0 = INFINITY, y1 = -INFINITY, x0 = INFINITY, x1 = -INFINITY;
            for (int p = t * tile / ncol; p < std::min(P, ((t + 1) * tile + ncol - 1) / ncol); ++p) {
                y0 = std::min(y0, scans[2 * p]);
                y1 = std::max(y1, scans[2 * p]);
                x0 = std::min(x0, scans[2 * p + 1]);
                x1 = std::max(x1, scans[2 * p + 1]);
            }
            bb64.insert(bb64.end(), {y0, y1, x0, x1});
        }
        // work items per batch; for the per-beam output (cube mode) ordered by
        // scan tile, then site, with one group per tile: a group's items
        // write the same cube entries, in site order, from one CTA
        std::vector<int32_t> cw, cg, wm;
        int max_items = 0;
        for (const auto& bt : batches) {
            const int b0 = bt.first, nbb = bt.second;
            cube_off.push_back((int)cw.size() / 2);
            cube_goff.push_back((int)cg.size());
            const int first = (int)cw.size() / 2;
            auto meets = [&](int bs, int t) {
                const SiteDev& sd = c->sites[c->batch_order[b0 + bs]];
                return box_meets_crop(bb64[4 * t], bb64[4 * t + 1], bb64[4 * t + 2], bb64[4 * t + 3], sd.ty, sd.tx, g);
            };
            if (cube_out) {
                for (int t = 0; t < n_ct; ++t) {
                    const int g0 = (int)cw.size() / 2 - first;
                    for (int bs = 0; bs < nbb; ++bs)
                        if (meets(bs, t)) {
                            cw.push_back(bs);
                            cw.push_back(t);
                        }
                    if ((int)cw.size() / 2 - first > g0) cg.push_back(g0);
                }
                cg.push_back((int)cw.size() / 2 - first);
            } else {
                // map modes: each (site, tile)'s work item, or -1
                for (int bs = 0; bs < nbb; ++bs)
                    for (int t = 0; t < n_ct; ++t) {
                        const bool m = meets(bs, t);
                        wm.push_back(m ? (int)cw.size() / 2 - first : -1);
                        if (m) {
                            cw.push_back(bs);
                            cw.push_back(t);
                        }
                    }
                max_items = std::max(max_items, (int)cw.size() / 2 - first);
            }
        }
        cube_off.push_back((int)cw.size() / 2);
        cube_goff.push_back((int)cg.size());
        // uploaded only when they differ from the device copies (so that a
        // capture-safe map repeated with its warm-up arguments records no copy)
        auto sync_list = [&](DevBuf& d, std::vector<int32_t>& held, const std::vector<int32_t>& v) -> bip_status {
            if (held == v && d.p) return BIP_OK;
            if (capturing(s))
                return fail(c, BIP_ERR_INVALID_ARG,
                            "a captured map must repeat the arguments of the capture-safe warm-up call");
            CUDA_TRY(c, upload(d, v, s));
            held = v;
            return BIP_OK;
        };
        bip_status sl = sync_list(c->cube_work, c->cube_work_h, cw);
        if (sl == BIP_OK && cube_out) sl = sync_list(c->cube_grp, c->cube_grp_h, cg);
        if (sl == BIP_OK && !cube_out) sl = sync_list(c->cube_wmap, c->cube_wmap_h, wm);
        if (sl != BIP_OK) return sl;
        if (!cube_out)
            CUDA_TRY(c, ensure(c->mpart, std::max<size_t>(1, (size_t)max_items * (D128 / 128) * tile) * sizeof(float),
                               false, s));
        n_ct_map = n_ct;
        CUDA_TRY(c, ensure(c->cube_mask, std::max<size_t>(1, cw.size() / 2 * (tile / 64)) * sizeof(unsigned long long),
                           false, s));
    }

    for (int bi = 0; bi < (int)batches.size(); ++bi) {
        const int b0 = batches[bi].first, nb = batches[bi].second;
        const int32_t* ids = (const int32_t*)c->seq_ids_d.p + b0;
        // the batch's window: its contractions run over K = w^2 pixels, the
        // operands packed at that row length (these shadow the context-wide
        // sizes the workspaces were allocated for)
        const int wb = c->sites[c->batch_order[b0]].w;
        const int K = wb * wb;
        const size_t perA = rowsA * K, perB = rowsB * K;
        {
            bip_status st = operand_layout(c, K, s);
            if (st != BIP_OK) return st;
        }
        // S2 windows -> coupling A operand, S1 windows x H_n -> B operand
        GatherArgs g2 = gather_args(c, 2, ids, nb, wb);
        g2.rows_pad = Dpad;
        GatherArgs g1 = gather_args(c, 1, ids, nb, wb);
        g1.rows_pad = Bpad;
        g1.nch = nch;
        g1.H = (const float2*)H;
        if (tc) {
            g2.out_bf16 = (uint16_t*)c->opA16.p;
            g2.out_planes = npl;
            g2.site_stride = (int64_t)(npl * perA);
            g1.out_bf16 = (uint16_t*)c->opB16.p;
            g1.out_planes = npl;
            g1.site_stride = (int64_t)(npl * perB);
        } else {
            g2.out_c64 = (float2*)c->opA32.p;
            g2.site_stride = (int64_t)perA;
            g1.out_c64 = (float2*)c->opB32.p;
            g1.site_stride = (int64_t)perB;
        }
        if (probe) {
            bip_status st = recon_tc_batch(c, ids, nb, H, c->opA16.p, c->s1t.p, s, true, true, wb);
            if (st != BIP_OK) return st;
            // Psi[rho][r] = sum_b c_b(rho) S1_b(r): A = S1 transposed (pixels in
            // 128-row tiles; BF16, zero lo planes), B = C^T (the scans as the
            // tile's columns, so that few scans cost few columns; split BF16,
            // c exact to FP32), written transposed as complex64 Psi[rho][r]
            const int P128 = crow, P16 = round_up(P, 16);
            TcArgs G1{};
            G1.epi = TC_EPI_C32;
            G1.N = std::min(256, P16);
            G1.npl = 4;
            G1.A = TcOperand{c->s1t.p, (int64_t)SB * 4 * K, Bpad, (int64_t)4 * K, (int64_t)K};
            G1.B = TcOperand{c->cubeB.p, (int64_t)4 * crow, Bpad, 0, (int64_t)crow};
            G1.kb = Bpad / 32;
            G1.n_sites = nb;
            G1.mt_per = K / 128;
            G1.nt_per = (P16 + G1.N - 1) / G1.N;
            G1.n_cols = P16;
            G1.out32 = (float2*)c->psi.p;
            G1.out32_site = (int64_t)P128 * K;
            G1.out32_ld = K;
            G1.out32_trans = 1;
            G1.err = (int*)c->errflag.p;
            G1.wait_ns = c->wait_ns;
            TIMED(c, BIP_STAGE_COUPLING, s, bip_tc_gemm(G1, s));
            // Y^(n) = H_n x Psi, then a^(n)_d(rho) = sum_r S2_d(r) Y^(n)(rho, r)
            // and the |.|^2 sums over d and n into the sites' maps
            ProbeYArgs y{};
            y.n_sites = nb;
            y.rows = P64;
            y.K = K;
            y.nch = nch;
            y.site_ids = ids;
            y.sites = (const SiteDev*)c->sites_d.p;
            y.psi = (const float2*)c->psi.p;
            y.psi_rows = P128;
            y.H = (const float2*)H;
            y.Y = (uint16_t*)c->ybuf.p;
            y.y_rows = P64;
            TIMED(c, BIP_STAGE_QUADFORM, s, bip_probe_y(y, s));
            // B = Y: rows rho with the channel in the columns (n K + r), one
            // accumulator per channel -- or, with few scans, seen as rows
            // (rho, n) of K, every channel of a scan in the tile's columns and
            // the channel sum taken over columns
            CubeTcArgs ct{};
            ct.n_work = cube_off[bi + 1] - cube_off[bi];
            ct.work = (const int32_t*)c->cube_work.p + 2 * (size_t)cube_off[bi];
            ct.mask = (unsigned long long*)c->cube_mask.p + cube_off[bi];
            ct.n_sites = nb;
            ct.n_tiles = probe_cols ? (P * nch + 63) / 64 : P64 / 64;
            ct.mt_per = D128 / 128;
            ct.kb_ch = K / 32;
            ct.a_site_rows = 2 * (int64_t)Dpad;
            ct.a_plane_rows = Dpad;
            ct.b_site_rows = 2 * (int64_t)P64 * (probe_cols ? nch : 1);
            ct.b_plane_rows = (int64_t)P64 * (probe_cols ? nch : 1);
            ct.swap_ch = 1;
            ct.hi_only = 1;
            ct.col_nch = probe_cols ? nch : 0;
            ct.n_det = geo.n_det;
            ct.P = P;
            ct.scans = (const double*)c->scans_d.p;
            ct.sites = (const SiteDev*)c->sites_d.p;
            ct.site_ids = ids;
            ct.ny = g.ny; ct.nx = g.nx; ct.fy = g.fy; ct.fx = g.fx;
            ct.scale = (float)det_scale(c);
            ct.mpart = (float*)c->mpart.p;
            ct.err = (int*)c->errflag.p;
            ct.wait_ns = c->wait_ns;
            // the per-unit column sums added to the sites' maps, in order
            MapReduceArgs mr{(const float*)c->mpart.p, (const int32_t*)c->cube_wmap.p + (size_t)b0 * n_ct_map, nb,
                             n_ct_map, 64, ct.mt_per, probe_cols ? nch : 1, P, ids, (float)det_scale(c), partial};
            // A: the S2 windows (opA16 holds four planes' room: 4 SB Dpad rows of K)
            if (probe_cols) {
                ct.ch0 = 0;
                ct.nacc = 1;
                TIMED(c, BIP_STAGE_QUADFORM, s,
                      bip_cube_tc(ct, c->opA16.p, (int64_t)SB * 4 * Dpad, K, c->ybuf.p, (int64_t)SB * 2 * P64 * nch,
                                  K, s));
                TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_map_reduce(mr, s));
            } else {
                for (int ch0 = 0; ch0 < nch; ch0 += 4) {
                    ct.ch0 = ch0;
                    ct.nacc = std::min(4, nch - ch0);
                    TIMED(c, BIP_STAGE_QUADFORM, s,
                          bip_cube_tc(ct, c->opA16.p, (int64_t)SB * 4 * Dpad, K, c->ybuf.p, (int64_t)SB * 2 * P64,
                                      nch * K, s));
                    TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_map_reduce(mr, s));
                }
            }
            continue;
        }
        if (f8) {
            bip_status st = recon_tc_batch(c, ids, nb, H, c->op8A.p, c->op8B.p, s, false, true, wb);
            if (st != BIP_OK) return st;
        } else if (c->prec == BIP_PREC_MIXED && c->recon_tc) {
            bip_status st = recon_tc_batch(c, ids, nb, H, c->opA16.p, c->opB16.p, s, false, true, wb);
            if (st != BIP_OK) return st;
        } else {
            TIMED(c, BIP_STAGE_GATHER, s, bip_gather(g2, s));
            TIMED(c, BIP_STAGE_GATHER, s, bip_gather(g1, s));
        }
        if (tc) {
            // coupling M = S2^T diag(H) S1 with the aperture side (rows (ch, b),
            // 128-row tiles) as A and the detector side (columns d, 256-wide
            // tiles and a narrower last one) as B; written as Mt[b][ch Dp + d]
            TcArgs A{};
            A.epi = TC_EPI_ROWS;
            A.N = c->cw_override > 0 ? std::min(c->cw_override, Dpad) : tile_width(Dpad);
            A.npl = npl;
            A.out_planes = npl;
            A.A = TcOperand{c->opB16.p, (int64_t)SB * npl * (int64_t)rowsB, K, npl * (int64_t)rowsB, (int64_t)rowsB};
            A.B = TcOperand{c->opA16.p, (int64_t)SB * npl * (int64_t)rowsA, K, npl * (int64_t)rowsA, (int64_t)rowsA};
            A.kb = K / 32;
            A.n_sites = nb;
            A.mt_per = (int)(rowsB / 128);
            A.nt_per = (Dpad + A.N - 1) / A.N;
            A.n_cols = Dpad;
            A.out16 = (uint16_t*)c->mt16.p;
            A.out_site = npl * (int64_t)perMt;
            A.out_plane = (int64_t)perMt;
            A.out_ld = (int64_t)nch * Dpad;
            A.ep_B = Bpad;
            A.ep_Dp = Dpad;
            A.err = (int*)c->errflag.p;
            A.wait_ns = c->wait_ns;
            if (f8) {
                // E4M3 rows of K bytes, seen by the tensor maps as K / 2 bf16
                A.f8 = 1;
                A.A = TcOperand{c->op8B.p, (int64_t)SB * 2 * (int64_t)rowsB, K / 2, 2 * (int64_t)rowsB, (int64_t)rowsB};
                A.B = TcOperand{c->op8A.p, (int64_t)SB * 2 * (int64_t)rowsA, K / 2, 2 * (int64_t)rowsA, (int64_t)rowsA};
                A.kb = K / 64;
                A.scaleA = (const float*)c->f8sA.p;
                A.scaleA_site = (int64_t)rowsB;
                A.scaleB = (const float*)c->f8sB.p;
                A.scaleB_site = Dpad;
            }
            if (cube_out || beam) {
                // per-beam values want M itself to FP32: complex64 rows (ch, b)
                A.epi = TC_EPI_C32;
                A.out32 = (float2*)c->mt32.p;
                A.out32_site = (int64_t)perMt;
                A.out32_ld = Dpad;
            }
            TIMED(c, BIP_STAGE_COUPLING, s, bip_tc_gemm(A, s));
            if (sepq) {
                CubeRasterArgs r = cra;
                r.n_sites = nb;
                r.site_ids = ids;
                r.m = (const float2*)c->mt32.p;
                r.nd = geo.n_det;
                r.cube = cube_out;
                TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_raster(r, s));
                continue;
            }
            if (cube_out || beam) {
                // A = M transposed to rows d, K = (ch, b), as split planes; then
                // the per-beam contraction and |.|^2 channel sum on tcgen05
                SplitArgs sa{(const float2*)c->mt32.p, 1, Dpad, (int64_t)perMt, Dpad, (int)KB, nb,
                             (uint16_t*)c->cubeA.p, (int64_t)(4 * D128 * KB), D128, (int)KB, 0, 0};
                TIMED(c, BIP_STAGE_QUADFORM, s, bip_split_planes(sa, s));
                CubeTcArgs ct{};
                ct.n_work = cube_off[bi + 1] - cube_off[bi];
                ct.work = (const int32_t*)c->cube_work.p + 2 * (size_t)cube_off[bi];
                ct.mask = (unsigned long long*)c->cube_mask.p + (size_t)cube_off[bi] * (ctn / 64);
                ct.n_sites = nb;
                ct.tn = ctn;
                ct.n_tiles = crow / ctn;
                ct.mt_per = D128 / 128;
                ct.kb_ch = Bpad / 32;
                ct.a_site_rows = 4 * (int64_t)D128;
                ct.a_plane_rows = D128;
                ct.b_plane_rows = crow;
                ct.n_det = geo.n_det;
                ct.P = P;
                ct.scans = (const double*)c->scans_d.p;
                ct.sites = (const SiteDev*)c->sites_d.p;
                ct.site_ids = ids;
                ct.ny = g.ny; ct.nx = g.nx; ct.fy = g.fy; ct.fx = g.fx;
                ct.scale = (float)det_scale(c);
                MapReduceArgs mr{};
                if (beam) {
                    ct.mpart = (float*)c->mpart.p;
                    mr = MapReduceArgs{(const float*)c->mpart.p, (const int32_t*)c->cube_wmap.p + (size_t)b0 * n_ct_map,
                                       nb, n_ct_map, ctn, ct.mt_per, 1, P, ids, (float)det_scale(c), partial};
                } else {
                    ct.cube = cube_out;
                    ct.cube_ld = geo.n_det;
                    ct.n_groups = cube_goff[bi + 1] - cube_goff[bi] - 1;
                    ct.grp = (const int32_t*)c->cube_grp.p + cube_goff[bi];
                }
                ct.err = (int*)c->errflag.p;
                ct.wait_ns = c->wait_ns;
                // channels per launch: one TMEM accumulator pair (2 ctn columns)
                // each in 512 columns
                const int per = 512 / (2 * ctn);
                for (int ch0 = 0; ch0 < nch; ch0 += per) {
                    ct.ch0 = ch0;
                    ct.nacc = std::min(per, nch - ch0);
                    TIMED(c, BIP_STAGE_QUADFORM, s,
                          bip_cube_tc(ct, c->cubeA.p, (int64_t)nb * 4 * D128, (int)KB, c->cubeB.p, (int64_t)4 * crow,
                                      Bpad, s));
                    if (beam) TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_map_reduce(mr, s));
                }
                continue;
            }
            // Gram Q = sum_n M^(n)H M^(n), upper triangle, FP32
            TcArgs Gq{};
            Gq.epi = TC_EPI_C32;
            Gq.N = (Bpad % 256 == 0) ? 256 : 128;
            Gq.npl = npl;
            Gq.A = TcOperand{c->mt16.p, (int64_t)SB * npl * Bpad, nch * Dpad, npl * (int64_t)Bpad, Bpad};
            Gq.B = Gq.A;
            Gq.kb = nch * Dpad / 32;
            Gq.n_sites = nb;
            Gq.mt_per = Bpad / 128;
            Gq.nt_per = Bpad / Gq.N;
            Gq.n_cols = Bpad;
            Gq.conjA = 1;
            Gq.tri = 1;
            Gq.out32 = (float2*)c->q32.p;
            Gq.out32_site = (int64_t)perQ;
            Gq.out32_ld = Bpad;
            Gq.err = (int*)c->errflag.p;
            Gq.wait_ns = c->wait_ns;
            TIMED(c, BIP_STAGE_GRAM, s, bip_tc_gemm(Gq, s));
        } else {
            // coupling M = S2^T diag(H) S1, stored transposed for the Gram step
            CGemmArgs A{};
            A.M = geo.n_det; A.N = (int)rowsB; A.K = K;
            A.A = (const float2*)c->opA32.p; A.lda = K; A.strideA = (int64_t)perA;
            A.Bm = (const float2*)c->opB32.p; A.ldb = K; A.strideB = (int64_t)perB;
            A.batch = nb;
            A.epi = 1;
            A.C = (float2*)c->mt32.p; A.ldc = (int64_t)nch * Dpad; A.strideC = (int64_t)perMt;
            A.ep_B = Bpad; A.ep_Dp = Dpad;
            TIMED(c, BIP_STAGE_COUPLING, s, bip_cgemm_simt(A, s));
            if (sepq) {
                CubeRasterArgs r = cra;
                r.n_sites = nb;
                r.site_ids = ids;
                r.m = (const float2*)c->mt32.p;
                r.nd = geo.n_det;
                r.cube = cube_out;
                TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_raster(r, s));
                continue;
            }
            if (cube_out) {
                CubeArgs ca = cube_args(c, ids, nb, P, cube_out);
                ca.m32 = (const float2*)c->mt32.p;
                ca.m_site = (int64_t)perMt;
                TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_accumulate(ca, s));
                continue;
            }
            // Gram Q = sum_n M^(n)H M^(n)
            CGemmArgs Bq{};
            Bq.M = Bpad; Bq.N = Bpad; Bq.K = nch * Dpad;
            Bq.A = (const float2*)c->mt32.p; Bq.lda = (int64_t)nch * Dpad; Bq.strideA = (int64_t)perMt;
            Bq.Bm = Bq.A; Bq.ldb = Bq.lda; Bq.strideB = Bq.strideA;
            Bq.conjA = 1;
            Bq.batch = nb;
            Bq.epi = 0;
            Bq.C = (float2*)c->q32.p; Bq.ldc = Bpad; Bq.strideC = (int64_t)perQ;
            TIMED(c, BIP_STAGE_GRAM, s, bip_cgemm_simt(Bq, s));
        }
        // I_tau(rho) = f_y f_x c^H Q c as a trigonometric polynomial over
        // beam-lattice differences, on the site's crop-window scan tiles
        DiffArgs d{};
        d.n_sites = nb;
        d.Q = (const float2*)c->q32.p;
        d.q_site = (int64_t)perQ;
        d.ldq = Bpad;
        d.B = geo.B;
        d.kb = (const int2*)c->kb_d.p;
        d.coef = (const double2*)c->coef.p;
        d.Ky = c->Ky;
        d.Kx = c->Kx;
        d.lat = (const int32_t*)c->lat_d.p;
        d.G = (float2*)c->gdiff.p + (raster.ok ? (size_t)b0 * nd : 0);
        d.work = (const int32_t*)c->work_d.p + 2 * batch_off[bi];
        d.n_work = batch_off[bi + 1] - batch_off[bi];
        d.tile = tile;
        d.P = P;
        d.scans = (const double*)c->scans_d.p;
        d.sites = (const SiteDev*)c->sites_d.p;
        d.site_ids = ids;
        d.ny = g.ny; d.nx = g.nx; d.fy = g.fy; d.fx = g.fx;
        d.scale = (float)det_scale(c);
        d.partial = partial;
        TIMED(c, BIP_STAGE_QUADFORM, s, bip_diff_bin(d, s));
        if (!raster.ok && d.n_work > 0) TIMED(c, BIP_STAGE_QUADFORM, s, bip_diff_eval(d, s));
    }
    if (raster.ok && c->n_sites > 0 && !cube_out && !beam && !probe) {
        // the scan polynomial of every site at once (sites in order)
        DiffArgs d{};
        d.n_sites = c->n_sites;
        d.Ky = c->Ky;
        d.Kx = c->Kx;
        d.G = (float2*)c->gdiff.p;
        d.P = P;
        d.scans = (const double*)c->scans_d.p;
        d.sites = (const SiteDev*)c->sites_d.p;
        d.site_ids = (const int32_t*)c->seq_ids_d.p;
        d.ny = g.ny; d.nx = g.nx; d.fy = g.fy; d.fx = g.fx;
        d.scale = (float)det_scale(c);
        d.partial = partial;
        TIMED(c, BIP_STAGE_QUADFORM, s, bip_raster_eval(d, rargs, s));
    }
    if (tc && !c->capture_safe) {
        int flag = 0;
        CUDA_TRY(c, cudaMemcpyAsync(&flag, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (flag) return fail(c, BIP_ERR_TIMEOUT, "a tensor-core contraction gave up waiting (device timeout)");
    }
    if (map_out && !cube_out) {
        CUDA_TRY(c, ensure(c->rsum, bip_reduce_scratch_bytes(c->n_sites, P), false, s));
        const double* occ = c->occ_n == c->n_sites ? (const double*)c->occ_d.p : nullptr;
        TIMED(c, BIP_STAGE_REDUCE, s, bip_reduce_sites(partial, c->n_sites, P, c->rsum.p, map_out, s, occ));
        if (c->n_sites > 0) c->launches[BIP_STAGE_REDUCE]++;   // two kernels: chunks, then their sum
    }
    return BIP_OK;
}

// Setup of the cube's separated per-beam contraction on a raster scan list
// (cube_raster.cu): the raster test, the phase tables per scan row and
// column (angles reduced in FP64), each site's crop per axis as bits (the
// FP64 test of in_crop, one axis at a time), and the stage-1 workspace T
// for batches of SB sites and nd_pad beams.  M(n, b, d) of a batch lies at
// m[bs m_site + b m_b + n m_ch + d].  sep is false, and nothing is set up,
// when the scans are no raster or the lattice is too large for the kernels.
bip_status raster_cube_setup(bip_ctx* c, const double* scans, int P, int SB, int nd_pad, int64_t m_b, int64_t m_ch,
                             int64_t m_site, int64_t cube_ld, float scale, CubeRasterArgs& cra, bool& sep,
                             cudaStream_t s) {
    const bip_config& g = c->cfg;
    const Raster rr = detect_raster(scans, P);
    const int nky = 2 * c->Ky + 1, nkx = 2 * c->Kx + 1;
    // (stage 2 prefetches a tile of nky x 64 values with 8 per thread: nky <= 32)
    sep = rr.ok && nky <= 32 && nkx <= 128 && (size_t)nkx * (rr.Mx + 32) * 8 <= 200 * 1024;
    if (!sep) return BIP_OK;
    const int nch = c->nch_max;
    std::vector<double> ry(rr.My), rx(rr.Mx);
    for (int my = 0; my < rr.My; ++my) ry[my] = scans[2 * (size_t)my * rr.Mx];
    for (int mx = 0; mx < rr.Mx; ++mx) rx[mx] = scans[2 * (size_t)mx + 1];
    std::vector<float2> ay((size_t)rr.My * nky), ax((size_t)nkx * rr.Mx);
    for (int my = 0; my < rr.My; ++my)
        for (int iy = 0; iy < nky; ++iy)
            ay[(size_t)my * nky + iy] = turn_d(-(double)g.fy * (iy - c->Ky) * ry[my] / g.ny);
    for (int ix = 0; ix < nkx; ++ix)
        for (int mx = 0; mx < rr.Mx; ++mx)
            ax[(size_t)ix * rr.Mx + mx] = turn_d(-(double)g.fx * (ix - c->Kx) * rx[mx] / g.nx);
    auto axis = [](double r, double t, int n, int f) {
        double d = r - t;
        d -= n * std::floor((d + 0.5 * n) / n);
        const double h = 0.5 * n / f;
        return d >= -h && d < h;
    };
    const int wy = (rr.My + 31) / 32, wx = (rr.Mx + 31) / 32;
    std::vector<uint32_t> cy((size_t)c->n_sites * wy, 0u), cx((size_t)c->n_sites * wx, 0u);
    for (int k = 0; k < c->n_sites; ++k) {
        const SiteDev& sd = c->sites[k];
        for (int my = 0; my < rr.My; ++my)
            if (axis(ry[my], sd.ty, g.ny, g.fy)) cy[(size_t)k * wy + my / 32] |= 1u << (my % 32);
        for (int mx = 0; mx < rr.Mx; ++mx)
            if (axis(rx[mx], sd.tx, g.nx, g.fx)) cx[(size_t)k * wx + mx / 32] |= 1u << (mx % 32);
    }
    CUDA_TRY(c, upload(c->cr_cy, cy, s));
    CUDA_TRY(c, upload(c->cr_cx, cx, s));
    CUDA_TRY(c, upload(c->cr_ay, ay, s));
    CUDA_TRY(c, upload(c->cr_ax, ax, s));
    cra = CubeRasterArgs{};
    cra.crop_y = (const uint32_t*)c->cr_cy.p;
    cra.crop_x = (const uint32_t*)c->cr_cx.p;
    cra.wy = wy;
    cra.wx = wx;
    cra.nch = nch;
    cra.nd_pad = nd_pad;
    cra.nky = nky;
    cra.nkx = nkx;
    cra.lat = (const int32_t*)c->lat_d.p;
    cra.coef = (const double2*)c->coef.p;
    cra.ay = (const float2*)c->cr_ay.p;
    cra.ax = (const float2*)c->cr_ax.p;
    cra.My = rr.My;
    cra.Mx = rr.Mx;
    cra.n_sites = SB;
    CUDA_TRY(c, ensure(c->cr_T, bip_cube_raster_t_bytes(cra), false, s));
    cra.T = (float2*)c->cr_T.p;
    cra.cube_ld = cube_ld;
    cra.scale = scale;
    cra.sites = (const SiteDev*)c->sites_d.p;
    cra.m_site = m_site;
    cra.m_b = m_b;
    cra.m_ch = m_ch;
    return BIP_OK;
}

// The energy-filtered 4D cube (Sec. 2.2.6, Algorithm 3): S1 partitioned
// (the context's S1 stash, rebuilt on each window), the exit side exact on
// the complete basis: batches of the cube's beams are taken back from the
// exit surface as unpartitioned S2 columns (one sweep per batch, windows of
// every site stashed), re-tilted into the coupling's detector operand, and
// cube[rho][d] += sum_n |sum_b M_{d,b} c_b(rho)|^2 site by site in order.
bip_status run_cube_exact(bip_ctx* c, const float* V, const void* H, const double* scans, int32_t P,
                          float* cube_out, cudaStream_t s) {
    const bip_config& g = c->cfg;
    const BipGeometry& geo = c->geo;
    if (c->prec == BIP_PREC_FP8_TILE)
        return fail(c, BIP_ERR_UNSUPPORTED, "the cube has no FP8 path (its exit side has no per-window scales)");
    const int K = g.win * g.win, Bpad = c->Bpad, nch = c->nch_max;
    const bool tc = c->prec != BIP_PREC_FP32;
    const int npl = gram_planes(c->prec);
    const size_t G = (size_t)g.ny * g.nx;
    const int n_cube = geo.n_cube;

    CUDA_TRY(c, ensure(c->scans_d, (size_t)P * 2 * sizeof(double), false, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->scans_d.p, scans, (size_t)P * 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    c->scans_cache.clear();
    CUDA_TRY(c, ensure(c->illum, (size_t)Bpad * P * sizeof(float2), false, s));
    IllumArgs ia{P, geo.B, Bpad, (const int2*)c->hbeam.p, (const double2*)c->coef.p, (const double*)c->scans_d.p,
                 g.ny, g.nx, (float2*)c->illum.p};
    CUDA_TRY(c, bip_illum(ia, s));
    CUDA_TRY(c, cudaMemsetAsync(cube_out, 0, (size_t)P * n_cube * sizeof(float), s));

    // beams per sweep: the windows of every site plus the columns, within
    // half the free device memory (at most 96 GB), a multiple of 32
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(c, cudaMemGetInfo(&free_b, &total_b));
    const size_t per_beam = (size_t)c->n_sites * K * sizeof(float2) + G * sizeof(float2);
    size_t budget = c->cube_budget ? c->cube_budget : std::min(free_b / 2, (size_t)96 << 30);
    int nbd = (int)std::min<size_t>((size_t)round_up(n_cube, kDetPad), budget / per_beam / kDetPad * kDetPad);
    nbd = std::min(nbd, 2048);
    if (nbd < kDetPad)
        return fail(c, BIP_ERR_OOM, "not enough device memory for 32 exact S2 columns and their windows");
    const int Dpb = nbd, D128 = round_up(Dpb, 128);
    CUDA_TRY(c, ensure(c->cstash, (size_t)c->n_sites * nbd * K * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->ccols, (size_t)nbd * G * sizeof(float2), false, s));

    // site batches and their buffers (as the map's)
    const int SB = c->sb_override > 0 ? std::min(c->n_sites, c->sb_override)
                                      : (tc ? tc_batch(c) : std::min(c->n_sites, 8));
    const std::vector<std::pair<int, int>> batches = map_batches(c, SB);   // (one window size each)
    const size_t rowsB = (size_t)nch * Bpad, perA = (size_t)Dpb * K, perB = rowsB * K;
    const size_t perMt = (size_t)Bpad * nch * Dpb, KB = (size_t)nch * Bpad;
    // the cube's own operand and coupling buffers: the map's keep zero
    // padding in their own row layout, which these rows would overwrite
    // (8 bytes per element: complex64, or up to four BF16 planes)
    CUDA_TRY(c, ensure(c->xopA, SB * perA * 8, true, s));
    CUDA_TRY(c, ensure(c->xopB, SB * perB * 8, true, s));
    CUDA_TRY(c, ensure(c->xm32, SB * perMt * sizeof(float2), true, s));
    if (tc) CUDA_TRY(c, cudaMemsetAsync(c->errflag.p, 0, sizeof(int), s));

    // On a raster scan list the per-beam contraction separates over the
    // aperture beams' lattice (cube_raster.cu)
    CubeRasterArgs cra{};
    bool sep = false;
    {
        bip_status st = raster_cube_setup(c, scans, P, SB, Dpb, tc ? (int64_t)Dpb : (int64_t)nch * Dpb,
                                          tc ? (int64_t)Bpad * Dpb : (int64_t)Dpb, (int64_t)perMt, n_cube, 1.0f,
                                          cra, sep, s);
        if (st != BIP_OK) return st;
    }

    // tcgen05 per-beam contraction: c_b(rho) as split planes, and work items
    // grouped by scan tile (sites ascending), one CTA per cube tile
    const int ctn = P >= 128 ? 128 : 64;
    const int crow = round_up(P, ctn), n_ct = crow / ctn;
    std::vector<int> cube_off, cube_goff;
    if (tc && !sep) {
        CUDA_TRY(c, ensure(c->cubeB, (size_t)4 * crow * Bpad * sizeof(uint16_t), true, s));
        CUDA_TRY(c, ensure(c->cubeA, (size_t)SB * 4 * D128 * KB * sizeof(uint16_t), true, s));
        SplitArgs sc{(const float2*)c->illum.p, 1, P, 0, P, Bpad, 1, (uint16_t*)c->cubeB.p, 0, crow, Bpad, 0, 0};
        CUDA_TRY(c, bip_split_planes(sc, s));
        std::vector<double> bb;
        for (int t = 0; t < n_ct; ++t) {
            double y0 = INFINITY, y1 = -INFINITY, x0 = INFINITY, x1 = -INFINITY;
            for (int p = t * ctn; p < std::min(P, (t + 1) * ctn); ++p) {
                y0 = std::min(y0, scans[2 * p]);
                y1 = std::max(y1, scans[2 * p]);
                x0 = std::min(x0, scans[2 * p + 1]);
                x1 = std::max(x1, scans[2 * p + 1]);
            }
            bb.insert(bb.end(), {y0, y1, x0, x1});
        }
        std::vector<int32_t> cw, cg;
        for (const auto& bt : batches) {
            const int b0 = bt.first, nbb = bt.second;
            cube_off.push_back((int)cw.size() / 2);
            cube_goff.push_back((int)cg.size());
            const int first = (int)cw.size() / 2;
            for (int t = 0; t < n_ct; ++t) {
                const int g0 = (int)cw.size() / 2 - first;
                for (int bs = 0; bs < nbb; ++bs) {
                    const SiteDev& sd = c->sites[c->batch_order[b0 + bs]];
                    if (box_meets_crop(bb[4 * t], bb[4 * t + 1], bb[4 * t + 2], bb[4 * t + 3], sd.ty, sd.tx, g)) {
                        cw.push_back(bs);
                        cw.push_back(t);
                    }
                }
                if ((int)cw.size() / 2 - first > g0) cg.push_back(g0);
            }
            cg.push_back((int)cw.size() / 2 - first);
        }
        cube_off.push_back((int)cw.size() / 2);
        cube_goff.push_back((int)cg.size());
        CUDA_TRY(c, upload(c->cube_work, cw, s));
        CUDA_TRY(c, upload(c->cube_grp, cg, s));
        c->cube_work_h = cw;                // what the device copies now hold
        c->cube_grp_h = cg;
        CUDA_TRY(c, ensure(c->cube_mask, std::max<size_t>(1, cw.size() / 2 * (ctn / 64)) * sizeof(unsigned long long),
                           false, s));
    }

    int first_plane = g.nz - 1;
    for (auto& sd : c->sites) first_plane = std::min(first_plane, (int)sd.plane);
    CUDA_TRY(c, ensure(c->tcache, (size_t)g.nz * G * sizeof(float2), false, s));
    TIMED(c, BIP_STAGE_TRANSMISSION, s, bip_transmission(V, (float)geo.sigma, first_plane, g.nz, G, (float2*)c->tcache.p, s));
    for (int d0 = 0; d0 < n_cube; d0 += nbd) {
        const int nd = std::min(nbd, n_cube - d0);
        // the batch's exact S2 columns, exit surface to the first site plane
        MsPlan plan = plan_for(c, nd, c->shcube);
        plan.shift = (const int2*)c->shcube.p + d0;
        {
            MsRowArgs a{};
            a.cols = (float2*)c->ccols.p;
            a.init = 1;
            a.init_val = (float)(1.0 / std::sqrt((double)G));
            a.do_fft = 1;
            a.win = g.win;
            a.stash = (float2*)c->cstash.p;
            TIMED(c, BIP_STAGE_MS_ROW, s, bip_ms_row_pass(plan, a, s));
            TIMED(c, BIP_STAGE_MS_COL, s, bip_ms_col_pass(plan, (float2*)c->ccols.p, s));
        }
        for (int j = g.nz - 1; j >= first_plane; --j) {
            MsRowArgs a{};
            a.cols = (float2*)c->ccols.p;
            a.do_ifft = 1;
            a.v_pre = V + (size_t)j * G;
            a.t_slice = (const float2*)c->tcache.p + (size_t)j * G;
            a.do_fft = j > first_plane;
            if (c->plane_off[j + 1] > c->plane_off[j]) {
                a.row_off = (const int32_t*)c->row_off_d.p + (size_t)j * (g.ny + 1);
                a.row_ent = (const int4*)c->row_ent_d.p;
            }
            a.win = g.win;
            a.stash = (float2*)c->cstash.p;
            TIMED(c, BIP_STAGE_MS_ROW, s, bip_ms_row_pass(plan, a, s));
            if (j > first_plane) TIMED(c, BIP_STAGE_MS_COL, s, bip_ms_col_pass(plan, (float2*)c->ccols.p, s));
        }
        for (int bi = 0; bi < (int)batches.size(); ++bi) {
            const int b0 = batches[bi].first, nb = batches[bi].second;
            const int32_t* ids = (const int32_t*)c->seq_ids_d.p + b0;
            // the batch's window: its operands packed at K = w^2 (shadowing the
            // context-wide sizes the buffers were allocated for); after a
            // batch at another pitch the operands' padding rows are cleared
            const int wb = c->sites[c->batch_order[b0]].w;
            const int K = wb * wb;
            const size_t perA = (size_t)Dpb * K, perB = rowsB * K;
            if (c->xop_k != K) {
                if (c->xop_k != 0) {
                    CUDA_TRY(c, cudaMemsetAsync(c->xopA.p, 0, c->xopA.cap, s));
                    CUDA_TRY(c, cudaMemsetAsync(c->xopB.p, 0, c->xopB.cap, s));
                }
                c->xop_k = K;
            }
            // aperture side H_n S1 (partitioned, rebuilt on the windows)
            if (c->prec == BIP_PREC_MIXED && c->recon_tc) {
                bip_status st = recon_tc_batch(c, ids, nb, H, nullptr, c->xopB.p, s, false, false, wb);
                if (st != BIP_OK) return st;
            } else {
                GatherArgs g1 = gather_args(c, 1, ids, nb, wb);
                g1.rows_pad = Bpad;
                g1.nch = nch;
                g1.H = (const float2*)H;
                if (tc) {
                    g1.out_bf16 = (uint16_t*)c->xopB.p;
                    g1.out_planes = npl;
                    g1.site_stride = (int64_t)(npl * perB);
                } else {
                    g1.out_c64 = (float2*)c->xopB.p;
                    g1.site_stride = (int64_t)perB;
                }
                TIMED(c, BIP_STAGE_GATHER, s, bip_gather(g1, s));
            }
            // detector side: the exact S2 windows re-tilted
            RetiltArgs ra{};
            ra.n_sites = nb;
            ra.site_ids = ids;
            ra.sites = (const SiteDev*)c->sites_d.p;
            ra.win = wb; ra.ny = g.ny; ra.nx = g.nx; ra.K = K;
            ra.stash_win = g.win;
            ra.wo = (g.win - wb) / 2;
            ra.nd = nd;
            ra.stash = (const float2*)c->cstash.p;
            ra.h = (const int2*)c->hcube.p + d0;
            ra.ey = (const float2*)c->ey.p;
            ra.ex = (const float2*)c->ex.p;
            ra.rows_pad = Dpb;
            if (tc) {
                ra.out_bf16 = (uint16_t*)c->xopA.p;
                ra.out_planes = npl;
                ra.site_stride = (int64_t)npl * perA;
            } else {
                ra.out_c64 = (float2*)c->xopA.p;
                ra.site_stride = (int64_t)perA;
            }
            TIMED(c, BIP_STAGE_GATHER, s, bip_retilt(ra, s));
            if (tc) {
                // M with rows (ch, b) and columns d, complex64
                TcArgs A{};
                A.epi = TC_EPI_C32;
                A.N = tile_width(Dpb);
                A.npl = npl;
                A.out_planes = npl;
                A.A = TcOperand{c->xopB.p, (int64_t)SB * npl * (int64_t)rowsB, K, npl * (int64_t)rowsB, (int64_t)rowsB};
                A.B = TcOperand{c->xopA.p, (int64_t)SB * npl * (int64_t)Dpb, K, npl * (int64_t)Dpb, (int64_t)Dpb};
                A.kb = K / 32;
                A.n_sites = nb;
                A.mt_per = (int)(rowsB / 128);
                A.nt_per = (Dpb + A.N - 1) / A.N;
                A.n_cols = Dpb;
                A.out32 = (float2*)c->xm32.p;
                A.out32_site = (int64_t)perMt;
                A.out32_ld = Dpb;
                A.ep_B = Bpad;
                A.ep_Dp = Dpb;
                A.err = (int*)c->errflag.p;
                A.wait_ns = c->wait_ns;
                TIMED(c, BIP_STAGE_COUPLING, s, bip_tc_gemm(A, s));
                if (sep) {
                    CubeRasterArgs r = cra;
                    r.n_sites = nb;
                    r.site_ids = ids;
                    r.m = (const float2*)c->xm32.p;
                    r.nd = nd;
                    r.cube = cube_out + d0;
                    TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_raster(r, s));
                    continue;
                }
                SplitArgs sa{(const float2*)c->xm32.p, 1, Dpb, (int64_t)perMt, Dpb, (int)KB, nb,
                             (uint16_t*)c->cubeA.p, (int64_t)(4 * D128 * KB), D128, (int)KB, 0, 0};
                TIMED(c, BIP_STAGE_QUADFORM, s, bip_split_planes(sa, s));
                CubeTcArgs ct{};
                ct.n_work = cube_off[bi + 1] - cube_off[bi];
                ct.work = (const int32_t*)c->cube_work.p + 2 * (size_t)cube_off[bi];
                ct.mask = (unsigned long long*)c->cube_mask.p + (size_t)cube_off[bi] * (ctn / 64);
                ct.n_sites = nb;
                ct.tn = ctn;
                ct.n_tiles = n_ct;
                ct.mt_per = D128 / 128;
                ct.kb_ch = Bpad / 32;
                ct.a_site_rows = 4 * (int64_t)D128;
                ct.a_plane_rows = D128;
                ct.b_plane_rows = crow;
                ct.n_det = nd;
                ct.P = P;
                ct.scans = (const double*)c->scans_d.p;
                ct.sites = (const SiteDev*)c->sites_d.p;
                ct.site_ids = ids;
                ct.ny = g.ny; ct.nx = g.nx; ct.fy = g.fy; ct.fx = g.fx;
                ct.scale = 1.0f;
                ct.cube = cube_out + d0;
                ct.cube_ld = n_cube;
                ct.n_groups = cube_goff[bi + 1] - cube_goff[bi] - 1;
                ct.grp = (const int32_t*)c->cube_grp.p + cube_goff[bi];
                ct.err = (int*)c->errflag.p;
                ct.wait_ns = c->wait_ns;
                const int per = 512 / (2 * ctn);
                for (int ch0 = 0; ch0 < nch; ch0 += per) {
                    ct.ch0 = ch0;
                    ct.nacc = std::min(per, nch - ch0);
                    TIMED(c, BIP_STAGE_QUADFORM, s,
                          bip_cube_tc(ct, c->cubeA.p, (int64_t)nb * 4 * D128, (int)KB, c->cubeB.p, (int64_t)4 * crow,
                                      Bpad, s));
                }
            } else {
                CGemmArgs A{};
                A.M = nd; A.N = (int)rowsB; A.K = K;
                A.A = (const float2*)c->xopA.p; A.lda = K; A.strideA = (int64_t)perA;
                A.Bm = (const float2*)c->xopB.p; A.ldb = K; A.strideB = (int64_t)perB;
                A.batch = nb;
                A.epi = 1;
                A.C = (float2*)c->xm32.p; A.ldc = (int64_t)nch * Dpb; A.strideC = (int64_t)perMt;
                A.ep_B = Bpad; A.ep_Dp = Dpb;
                TIMED(c, BIP_STAGE_COUPLING, s, bip_cgemm_simt(A, s));
                if (sep) {
                    CubeRasterArgs r = cra;
                    r.n_sites = nb;
                    r.site_ids = ids;
                    r.m = (const float2*)c->xm32.p;
                    r.nd = nd;
                    r.cube = cube_out + d0;
                    TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_raster(r, s));
                    continue;
                }
                CubeArgs ca = cube_args(c, ids, nb, P, cube_out + d0);
                ca.n_det = nd;
                ca.Dp = Dpb;
                ca.m_ld = (int64_t)nch * Dpb;
                ca.m32 = (const float2*)c->xm32.p;
                ca.m_site = (int64_t)perMt;
                ca.scale = 1.0f;
                ca.cube_ld = n_cube;
                TIMED(c, BIP_STAGE_QUADFORM, s, bip_cube_accumulate(ca, s));
            }
        }
    }
    if (tc && !c->capture_safe) {
        int flag = 0;
        CUDA_TRY(c, cudaMemcpyAsync(&flag, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (flag) return fail(c, BIP_ERR_TIMEOUT, "a tensor-core contraction gave up waiting (device timeout)");
    }
    return BIP_OK;
}

// Optional scan of a call's outputs for NaN or infinite values
// (bip_set_check_finite).  Synchronises the stream.
struct OutSpan {
    const void* p;
    int64_t n;
    int bytes;
};

bip_status finite_check(bip_ctx* c, std::initializer_list<OutSpan> spans, cudaStream_t s) {
    if (!c->check_finite) return BIP_OK;
    CUDA_TRY(c, ensure(c->nf_count, sizeof(unsigned long long), false, s));
    CUDA_TRY(c, cudaMemsetAsync(c->nf_count.p, 0, sizeof(unsigned long long), s));
    for (const OutSpan& o : spans)
        if (o.p && o.n > 0)
            CUDA_TRY(c, bip_count_nonfinite(o.p, o.n, o.bytes, (unsigned long long*)c->nf_count.p, s));
    unsigned long long bad = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&bad, c->nf_count.p, sizeof(bad), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (bad) return fail(c, BIP_ERR_NUMERIC, std::to_string(bad) + " output values are NaN or infinite");
    return BIP_OK;
}

bip_status refuse_check_under_capture(bip_ctx* c, cudaStream_t s) {
    if (c && c->check_finite && capturing(s))
        return fail(c, BIP_ERR_INVALID_ARG, "the finite check synchronises the stream: turn it off to capture");
    return BIP_OK;
}

}  // namespace

extern "C" {

bip_status bip_coreloss_map(bip_ctx* c, const void* H, const double* scan_px, int32_t P, double* map_out,
                            void* stream) {
    BIP_RANGE("bip_coreloss_map");
    bip_status st = check_map_args(c, H, scan_px, P, map_out);
    if (st == BIP_OK) st = refuse_check_under_capture(c, (cudaStream_t)stream);
    if (st != BIP_OK) return st;
    st = run_map(c, H, scan_px, P, nullptr, map_out, nullptr, (cudaStream_t)stream);
    if (st != BIP_OK) return st;
    return finite_check(c, {{map_out, P, 8}}, (cudaStream_t)stream);
}

bip_status bip_coreloss_sites(bip_ctx* c, const void* H, const double* scan_px, int32_t P, float* partial_out,
                              void* stream) {
    BIP_RANGE("bip_coreloss_sites");
    bip_status st = check_map_args(c, H, scan_px, P, partial_out);
    if (st == BIP_OK) st = refuse_check_under_capture(c, (cudaStream_t)stream);
    if (st != BIP_OK) return st;
    st = run_map(c, H, scan_px, P, partial_out, nullptr, nullptr, (cudaStream_t)stream);
    if (st != BIP_OK) return st;
    return finite_check(c, {{partial_out, (int64_t)c->n_sites * P, 4}}, (cudaStream_t)stream);
}

bip_status bip_coreloss_cube(bip_ctx* c, const float* V, const void* H, const double* scan_px, int32_t P,
                             float* cube_out, void* stream) {
    BIP_RANGE("bip_coreloss_cube");
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!c->s1 || site_signature(c->sites) != c->sig1)
        return fail(c, BIP_ERR_INVALID_ARG, "bip_build_s1 must run first (the cube's sites are its sites)");
    if (!V || !H || !scan_px || !cube_out) return fail(c, BIP_ERR_INVALID_ARG, "null pointer argument");
    if ((reinterpret_cast<uintptr_t>(H) & 15) != 0) return fail(c, BIP_ERR_INVALID_ARG, "H must be 16-byte aligned");
    if (P < 1) return fail(c, BIP_ERR_INVALID_ARG, "P must be >= 1");
    for (int i = 0; i < 2 * P; ++i)
        if (!std::isfinite(scan_px[i])) return fail(c, BIP_ERR_INVALID_ARG, "scan position is not finite");
    bip_status st = refuse_check_under_capture(c, (cudaStream_t)stream);
    if (st != BIP_OK) return st;
    st = run_cube_exact(c, V, H, scan_px, P, cube_out, (cudaStream_t)stream);
    if (st != BIP_OK) return st;
    return finite_check(c, {{cube_out, (int64_t)P * c->geo.n_cube, 4}}, (cudaStream_t)stream);
}

bip_status bip_cube_beams(const bip_ctx* c, int32_t* n_cube, int32_t* h) {
    if (!c || !n_cube) return BIP_ERR_INVALID_ARG;
    *n_cube = c->geo.n_cube;
    if (h) std::memcpy(h, c->geo.h_cube.data(), c->geo.h_cube.size() * sizeof(int32_t));
    return BIP_OK;
}

bip_status bip_set_wait_limit(bip_ctx* c, int64_t ns) {
    if (!c || ns < 0) return BIP_ERR_INVALID_ARG;
    c->wait_ns = (uint64_t)ns;
    return BIP_OK;
}

bip_status bip_debug_fail_alloc(int64_t k) {
    if (k < 0) return BIP_ERR_INVALID_ARG;
    g_made = 0;
    g_fail_at = k;
    return BIP_OK;
}

bip_status bip_debug_allocs(int64_t* live, int64_t* made) {
    if (live) *live = g_live.load();
    if (made) *made = g_made.load();
    return BIP_OK;
}

bip_status bip_set_cube_memory(bip_ctx* c, int64_t bytes) {
    if (!c || bytes < 0) return BIP_ERR_INVALID_ARG;
    c->cube_budget = (size_t)bytes;
    return BIP_OK;
}

// qEELS bins: the distinct components of the detector beams along `axis`,
// ascending, and each beam's bin.
static bool qeels_bins(const bip_ctx* c, int axis, std::vector<int32_t>& bins, std::vector<int32_t>& bin_of) {
    if (axis != 0 && axis != 1) return false;
    const BipGeometry& geo = c->geo;
    bins.clear();
    for (int d = 0; d < geo.n_det; ++d) bins.push_back(geo.h_det[2 * d + axis]);
    std::sort(bins.begin(), bins.end());
    bins.erase(std::unique(bins.begin(), bins.end()), bins.end());
    bin_of.resize(geo.n_det);
    for (int d = 0; d < geo.n_det; ++d)
        bin_of[d] = (int32_t)(std::lower_bound(bins.begin(), bins.end(), geo.h_det[2 * d + axis]) - bins.begin());
    return true;
}

bip_status bip_qeels_bins(const bip_ctx* c, int32_t axis, int32_t* n_bins, int32_t* h_values) {
    if (!c || !n_bins) return BIP_ERR_INVALID_ARG;
    std::vector<int32_t> bins, bin_of;
    if (!qeels_bins(c, axis, bins, bin_of)) return BIP_ERR_INVALID_ARG;
    *n_bins = (int32_t)bins.size();
    if (h_values) std::copy(bins.begin(), bins.end(), h_values);
    return BIP_OK;
}

bip_status bip_coreloss_qeels(bip_ctx* c, const void* H, const double* scan_px, int32_t P, int32_t axis,
                              float* qeels_out, void* stream) {
    BIP_RANGE("bip_coreloss_qeels");
    bip_status st = check_map_args(c, H, scan_px, P, qeels_out);
    if (st != BIP_OK) return st;
    std::vector<int32_t> bins, bin_of;
    if (!qeels_bins(c, axis, bins, bin_of)) return fail(c, BIP_ERR_INVALID_ARG, "axis must be 0 (q_y) or 1 (q_x)");
    if ((axis == 0 ? c->geo.dfy : c->geo.dfx) != 1)
        return fail(c, BIP_ERR_INVALID_ARG,
                    "qEELS needs the resolved axis sampled at f = 1: create the context with dfy = 1 (axis 0) "
                    "or dfx = 1 (axis 1)");
    cudaStream_t s = (cudaStream_t)stream;
    st = refuse_check_under_capture(c, s);
    if (st != BIP_OK) return st;
    CUDA_TRY(c, ensure(c->cube_scratch, (size_t)P * c->geo.n_det * sizeof(float), false, s));
    CUDA_TRY(c, upload(c->bin_of_d, bin_of, s));
    st = run_map(c, H, scan_px, P, nullptr, nullptr, (float*)c->cube_scratch.p, s);
    if (st != BIP_OK) return st;
    CUDA_TRY(c, bip_qeels_bin((const float*)c->cube_scratch.p, P, c->geo.n_det, (const int32_t*)c->bin_of_d.p,
                              (int)bins.size(), qeels_out, s));
    return finite_check(c, {{qeels_out, (int64_t)P * (int64_t)bins.size(), 4}}, s);
}

bip_status bip_set_capture_safe(bip_ctx* c, int32_t on) {
    if (!c) return BIP_ERR_INVALID_ARG;
    c->capture_safe = on != 0;
    c->scans_cache.clear();
    c->work_key = 0;
    return BIP_OK;
}

bip_status bip_check_errors(bip_ctx* c, void* stream) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!c->errflag.p) return BIP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int flag = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&flag, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (flag) {
        CUDA_TRY(c, cudaMemsetAsync(c->errflag.p, 0, sizeof(int), s));
        return fail(c, BIP_ERR_TIMEOUT, "a tensor-core contraction gave up waiting (device timeout)");
    }
    return BIP_OK;
}

bip_status bip_set_raster_eval(bip_ctx* c, int32_t on) {
    if (!c) return BIP_ERR_INVALID_ARG;
    c->raster_eval = on != 0;
    c->scans_cache.clear();      // the phase tables follow the next call's scans
    return BIP_OK;
}

bip_status bip_set_order(bip_ctx* c, int32_t order) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (order < 0 || order > 2) return fail(c, BIP_ERR_INVALID_ARG, "order must be 0 (Gram), 1 (beam) or 2 (probe)");
    if (order == 2 && c->prec != BIP_PREC_MIXED)
        return fail(c, BIP_ERR_UNSUPPORTED, "the probe order runs in the mixed precision only");
    c->order = order;
    return BIP_OK;
}

bip_status bip_set_launch(bip_ctx* c, int32_t sites_per_batch, int32_t coupling_tile) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (sites_per_batch < 0 || coupling_tile < 0 || coupling_tile > 256 || coupling_tile % 16)
        return fail(c, BIP_ERR_INVALID_ARG, "sites_per_batch >= 0, coupling_tile a multiple of 16 in 0..256");
    c->sb_override = sites_per_batch;
    c->cw_override = coupling_tile;
    return BIP_OK;
}

bip_status bip_autotune(bip_ctx* c, const void* H, const double* scan_px, int32_t P, double* map_out, void* stream,
                        int32_t* sites_per_batch, int32_t* coupling_tile, int32_t* order, double* best_ms) {
    BIP_RANGE("bip_autotune");
    bip_status st = check_map_args(c, H, scan_px, P, map_out);
    if (st != BIP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool tc = c->prec != BIP_PREC_FP32;
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, BIP_ERR_CUDA, "cudaEventCreate");
    }
    // mean device time of two maps after one warm-up map (allocations, uploads)
    auto time_map = [&](int sb, int cw, double* ms) -> bip_status {
        c->sb_override = sb;
        c->cw_override = cw;
        bip_status r = run_map(c, H, scan_px, P, nullptr, map_out, nullptr, s);
        if (r != BIP_OK) return r;
        CUDA_TRY(c, cudaEventRecord(e0, s));
        for (int i = 0; i < 2 && r == BIP_OK; ++i) r = run_map(c, H, scan_px, P, nullptr, map_out, nullptr, s);
        if (r != BIP_OK) return r;
        CUDA_TRY(c, cudaEventRecord(e1, s));
        CUDA_TRY(c, cudaEventSynchronize(e1));
        float t = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&t, e0, e1));
        *ms = t / 2.0;
        return BIP_OK;
    };
    std::vector<int> sbs;
    const int base = tc ? tc_batch(c) : std::min(c->n_sites, 8);
    for (int v : tc ? std::vector<int>{base, 16, 19, 20, 24, 28, 32} : std::vector<int>{base, 4, 8, 16})
        if (v >= 1 && v <= std::max(1, c->n_sites) && std::find(sbs.begin(), sbs.end(), v) == sbs.end())
            sbs.push_back(v);
    int best_sb = base, best_cw = 0;
    double best = 1e300, t = 0.0;
    for (int sb : sbs) {
        st = time_map(sb, 0, &t);
        if (st == BIP_ERR_OOM && sb != base) {
            release_map_workspaces(c, s);
            st = BIP_OK;
            continue;
        }
        if (st != BIP_OK) break;
        if (t < best) {
            best = t;
            best_sb = sb;
        }
    }
    if (st == BIP_OK && tc) {
        // coupling tile width: the built-in even split, or fixed widths
        for (int cw : {128, 160, 192, 224, 256}) {
            if (cw > c->Dpad) continue;
            st = time_map(best_sb, cw, &t);
            if (st != BIP_OK) break;
            if (t < best) {
                best = t;
                best_cw = cw;
            }
        }
    }
    // the scan contraction's order: the Gram matrix, |M c|^2 per beam, or
    // the windowed probes (mixed precision, up to kProbeMaxScans scans)
    const int order0 = c->order;
    int best_order = order0;
    if (st == BIP_OK && tc) {
        const bool probe_ok = c->prec == BIP_PREC_MIXED && c->recon_tc && P <= kProbeMaxScans;
        for (int o : {0, 1, 2}) {
            if (o == order0 || (o == 2 && !probe_ok)) continue;
            c->order = o;
            st = time_map(best_sb, best_cw, &t);
            if (st == BIP_ERR_OOM) {
                // this order's workspaces do not fit: not a candidate
                release_map_workspaces(c, s);
                st = BIP_OK;
                continue;
            }
            if (st != BIP_OK) break;
            if (t < best) {
                best = t;
                best_order = o;
            }
        }
    }
    if (st == BIP_OK && best_order != order0) {
        // the batch size again under the chosen order (the beam and probe
        // orders' last contraction has its own work units per site)
        c->order = best_order;
        for (int sb : {8, 12, 13, 14, 16, 19, 24, 27, 28, 32}) {
            if (sb == best_sb || sb > std::max(1, c->n_sites)) continue;
            st = time_map(sb, best_cw, &t);
            if (st == BIP_ERR_OOM) {
                release_map_workspaces(c, s);
                st = BIP_OK;
                continue;
            }
            if (st != BIP_OK) break;
            if (t < best) {
                best = t;
                best_sb = sb;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->sb_override = best_sb;
    c->cw_override = best_cw;
    c->order = best_order;
    // the trials' largest workspaces are not kept: the next map allocates
    // what the chosen settings need
    release_map_workspaces(c, s);
    if (st != BIP_OK) return st;
    if (sites_per_batch) *sites_per_batch = best_sb;
    if (coupling_tile) *coupling_tile = best_cw;
    if (order) *order = best_order;
    if (best_ms) *best_ms = best;
    return BIP_OK;
}

bip_status bip_set_occupancy(bip_ctx* c, const double* occ) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!occ) {
        c->occ_n = 0;
        return BIP_OK;
    }
    if (c->n_sites < 1) return fail(c, BIP_ERR_INVALID_ARG, "no sites: build the matrices first");
    for (int k = 0; k < c->n_sites; ++k)
        if (!std::isfinite(occ[k])) return fail(c, BIP_ERR_INVALID_ARG, "occupancy is not finite");
    CUDA_TRY(c, ensure(c->occ_d, (size_t)c->n_sites * sizeof(double), false, nullptr));
    CUDA_TRY(c, cudaMemcpy(c->occ_d.p, occ, (size_t)c->n_sites * sizeof(double), cudaMemcpyHostToDevice));
    c->occ_n = c->n_sites;
    return BIP_OK;
}

bip_status bip_set_site_windows(bip_ctx* c, const int32_t* win, void* stream) {
    BIP_RANGE("bip_set_site_windows");
    if (!c) return BIP_ERR_INVALID_ARG;
    if (c->n_sites < 1) return fail(c, BIP_ERR_INVALID_ARG, "no sites: build the matrices first");
    std::vector<int32_t> w;
    if (win) {
        w.assign(win, win + c->n_sites);
        int64_t h = 0;
        for (int k = 0; k < c->n_sites; ++k) {
            if (w[k] == 0) w[k] = c->cfg.win;
            if (w[k] < 16 || w[k] % 16 || w[k] > c->cfg.win)
                return fail(c, BIP_ERR_INVALID_ARG, "a site window must be a multiple of 16 in [16, win] (or 0)");
            h += (int64_t)c->sites[k].nch * w[k] * w[k];
        }
        if (h > INT32_MAX) return fail(c, BIP_ERR_INVALID_ARG, "H would exceed 2^31 complex elements");
    }
    c->site_w = w;
    return apply_windows(c, (cudaStream_t)stream);
}

bip_status bip_set_aberrations(bip_ctx* c, double defocus, double cs, void* stream) {
    BIP_RANGE("bip_set_aberrations");
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!std::isfinite(defocus) || !std::isfinite(cs)) return fail(c, BIP_ERR_INVALID_ARG, "aberration not finite");
    c->cfg.defocus = defocus;
    c->cfg.cs = cs;
    bip_set_psi(c->cfg, c->geo);
    if (c->tables) CUDA_TRY(c, upload(c->coef, coef_host(c), (cudaStream_t)stream));
    return BIP_OK;
}

static bip_status coreloss_grad(bip_ctx* c, const float* V, const void* H, const double* scan_px, int32_t P,
                                const double* dL_dI, double* d_occ, void* d_H, double* d_aberr, float* d_V,
                                void* stream) {
    bip_status st = check_map_args(c, H, scan_px, P, dL_dI);
    if (st != BIP_OK) return st;
    if (d_V && !V) return fail(c, BIP_ERR_INVALID_ARG, "d_V needs the V the matrices were built from");
    if ((reinterpret_cast<uintptr_t>(d_H) & 7) != 0) return fail(c, BIP_ERR_INVALID_ARG, "d_H must be 8-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const bip_config& g = c->cfg;
    const BipGeometry& geo = c->geo;
    const int K = g.win * g.win, Bpad = c->Bpad, Dpad = c->Dpad, nch = c->nch_max, B = geo.B;
    const double* occ = c->occ_n == c->n_sites ? (const double*)c->occ_d.p : nullptr;
    if (d_occ) {
        // dL/do_tau = sum_rho g I_tau with the forward partials
        CUDA_TRY(c, ensure(c->partial, (size_t)c->n_sites * P * sizeof(float), false, s));
        st = run_map(c, H, scan_px, P, (float*)c->partial.p, nullptr, nullptr, s);
        if (st != BIP_OK) return st;
        CUDA_TRY(c, bip_grad_occ((const float*)c->partial.p, c->n_sites, P, dL_dI, d_occ, s));
    }
    if (!d_H && !d_aberr && !d_V) return BIP_OK;
    if (d_V) {
        st = adj_tables(c, s);
        if (st != BIP_OK) return st;
        CUDA_TRY(c, ensure(c->g_dt1, (size_t)c->n_sites * geo.Bp1 * K * sizeof(float2), false, s));
        CUDA_TRY(c, ensure(c->g_dt2, (size_t)c->n_sites * geo.Bp2 * K * sizeof(float2), false, s));
        CUDA_TRY(c, ensure(c->g_s1bar, (size_t)std::min(c->n_sites, 8) * Bpad * K * sizeof(float2), true, s));
        CUDA_TRY(c, ensure(c->g_s2bar, (size_t)std::min(c->n_sites, 8) * round_up(Dpad, 128) * K * sizeof(float2),
                           true, s));
        const size_t rows = (size_t)std::max(Bpad, Dpad);
        CUDA_TRY(c, ensure(c->g_ubar, (size_t)std::min(c->n_sites, 8) * rows * K * sizeof(float2), false, s));
        CUDA_TRY(c, ensure(c->g_dA, (size_t)std::min(c->n_sites, 8) * rows * K * sizeof(float), false, s));
    }
    // FP32 contraction per batch of sites: S2, H_n S1 and S1 windows, M (as
    // Mt[b][(n, d)]), Q, then the reverse steps
    CUDA_TRY(c, ensure(c->scans_d, (size_t)P * 2 * sizeof(double), false, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->scans_d.p, scan_px, (size_t)P * 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, ensure(c->illum, (size_t)Bpad * P * sizeof(float2), false, s));
    IllumArgs ia{P, B, Bpad, (const int2*)c->hbeam.p, (const double2*)c->coef.p, (const double*)c->scans_d.p, g.ny,
                 g.nx, (float2*)c->illum.p};
    CUDA_TRY(c, bip_illum(ia, s));
    const int SB = std::min(c->n_sites, 8);
    const size_t perA = (size_t)Dpad * K, perB = (size_t)nch * Bpad * K, perS1 = (size_t)Bpad * K;
    const size_t ldm = (size_t)nch * Dpad, perMt = (size_t)Bpad * ldm, perQ = (size_t)Bpad * Bpad;
    const size_t perT = (size_t)nch * Bpad * K;
    // contractions of the reverse pass on the tensor cores (split BF16, three
    // products) for the tensor-core precisions, FP32 SIMT for FP32
    const bool tcg = c->prec != BIP_PREC_FP32;
    const int D128 = round_up(Dpad, 128);
    const size_t KB = (size_t)nch * Bpad;
    const size_t perS2bar = (size_t)(tcg ? D128 : Dpad) * K;
    if (tcg) {
        CUDA_TRY(c, ensure(c->opA16, SB * perA * 8, true, s));
        CUDA_TRY(c, ensure(c->opB16, SB * perB * 8, true, s));
        CUDA_TRY(c, ensure(c->g_tA, SB * 4 * (size_t)Bpad * Dpad * sizeof(uint16_t), true, s));
        CUDA_TRY(c, ensure(c->g_tB, SB * 4 * (size_t)K * Dpad * sizeof(uint16_t), true, s));
        if (d_V) {
            CUDA_TRY(c, ensure(c->g_sA2, SB * 4 * (size_t)D128 * KB * sizeof(uint16_t), true, s));
            CUDA_TRY(c, ensure(c->g_sB2, SB * 4 * (size_t)K * KB * sizeof(uint16_t), true, s));
        }
        CUDA_TRY(c, cudaMemsetAsync(c->errflag.p, 0, sizeof(int), s));
    }
    CUDA_TRY(c, ensure(c->opA32, SB * perA * sizeof(float2), true, s));
    CUDA_TRY(c, ensure(c->opB32, SB * perB * sizeof(float2), true, s));
    st = operand_layout(c, K, s);
    if (st != BIP_OK) return st;
    CUDA_TRY(c, ensure(c->g_s1, SB * perS1 * sizeof(float2), true, s));
    CUDA_TRY(c, ensure(c->mt32, SB * perMt * sizeof(float2), true, s));
    CUDA_TRY(c, ensure(c->q32, SB * perQ * sizeof(float2), true, s));
    CUDA_TRY(c, ensure(c->g_w, (size_t)SB * P * sizeof(float), false, s));
    CUDA_TRY(c, ensure(c->g_R, SB * perQ * sizeof(float2), true, s));
    CUDA_TRY(c, ensure(c->g_gmt, SB * perMt * sizeof(float2), true, s));
    CUDA_TRY(c, ensure(c->g_T, SB * perT * sizeof(float2), false, s));
    CUDA_TRY(c, ensure(c->g_D, (size_t)SB * B * sizeof(double2), false, s));
    CUDA_TRY(c, ensure(c->g_Dsum, (size_t)B * sizeof(double2), false, s));
    CUDA_TRY(c, cudaMemsetAsync(c->g_Dsum.p, 0, (size_t)B * sizeof(double2), s));
    if (d_H) CUDA_TRY(c, cudaMemsetAsync(d_H, 0, (size_t)c->h_elems * sizeof(float2), s));
    // window adjoints of sites with smaller windows than the stash: zero
    // outside their block (the sweeps inject the whole stashed window)
    if (d_V && c->uneven) {
        CUDA_TRY(c, cudaMemsetAsync(c->g_dt1.p, 0, (size_t)c->n_sites * geo.Bp1 * K * sizeof(float2), s));
        CUDA_TRY(c, cudaMemsetAsync(c->g_dt2.p, 0, (size_t)c->n_sites * geo.Bp2 * K * sizeof(float2), s));
    }
    GradArgs ga{};
    ga.P = P; ga.K = K; ga.B = B;
    ga.scans = (const double*)c->scans_d.p;
    ga.dL_dI = dL_dI;
    ga.occ = occ;
    ga.sites = (const SiteDev*)c->sites_d.p;
    ga.ny = g.ny; ga.nx = g.nx; ga.fy = g.fy; ga.fx = g.fx;
    ga.scale = (double)det_scale(c);
    for (const auto& bt : map_batches(c, SB)) {
        const int b0 = bt.first, nb = bt.second;
        const int32_t* ids = (const int32_t*)c->seq_ids_d.p + b0;
        // the batch's window (one size per batch): every per-pixel buffer at
        // pitch K = w^2, shadowing the context-wide sizes the workspaces were
        // allocated for; a pitch change clears them first (their padding
        // rows must read as zero)
        const int wb = c->sites[c->batch_order[b0]].w;
        const int K = wb * wb;
        const size_t perA = (size_t)Dpad * K, perB = (size_t)nch * Bpad * K, perS1 = (size_t)Bpad * K;
        const size_t perT = (size_t)nch * Bpad * K, perS2bar = (size_t)(tcg ? D128 : Dpad) * K;
        st = operand_layout(c, K, s);
        if (st != BIP_OK) return st;
        if (c->gop_k != K) {
            if (c->gop_k != 0)
                for (DevBuf* b : {&c->g_s1, &c->g_T, &c->g_tB, &c->g_sB2, &c->g_s1bar, &c->g_s2bar, &c->g_ubar, &c->g_dA})
                    if (b->p) CUDA_TRY(c, cudaMemsetAsync(b->p, 0, b->cap, s));
            c->gop_k = K;
        }
        GradArgs gab = ga;
        gab.K = K;
        GatherArgs g2 = gather_args(c, 2, ids, nb, wb);
        g2.rows_pad = Dpad;
        g2.out_c64 = (float2*)c->opA32.p;
        g2.site_stride = (int64_t)perA;
        CUDA_TRY(c, bip_gather(g2, s));
        GatherArgs g1 = gather_args(c, 1, ids, nb, wb);
        g1.rows_pad = Bpad;
        g1.nch = nch;
        g1.H = (const float2*)H;
        g1.out_c64 = (float2*)c->opB32.p;
        g1.site_stride = (int64_t)perB;
        CUDA_TRY(c, bip_gather(g1, s));
        GatherArgs g0 = gather_args(c, 1, ids, nb, wb);
        g0.rows_pad = Bpad;
        g0.out_c64 = (float2*)c->g_s1.p;
        g0.site_stride = (int64_t)perS1;
        CUDA_TRY(c, bip_gather(g0, s));
        if (tcg) {
            // operands as split planes, then M on tcgen05 written as Mt[b][(n, d)]
            SplitArgs sa{(const float2*)c->opA32.p, K, 1, (int64_t)perA, Dpad, K, nb, (uint16_t*)c->opA16.p,
                         (int64_t)(4 * perA), Dpad, K, 0, 0};
            CUDA_TRY(c, bip_split_planes(sa, s));
            SplitArgs sb{(const float2*)c->opB32.p, K, 1, (int64_t)perB, (int)KB, K, nb, (uint16_t*)c->opB16.p,
                         (int64_t)(4 * perB), (int)KB, K, 0, 0};
            CUDA_TRY(c, bip_split_planes(sb, s));
            TcArgs A{};
            A.epi = TC_EPI_C32;
            A.N = tile_width(Dpad);
            A.npl = 4;
            A.A = TcOperand{c->opB16.p, (int64_t)nb * 4 * (int64_t)KB, K, 4 * (int64_t)KB, (int64_t)KB};
            A.B = TcOperand{c->opA16.p, (int64_t)nb * 4 * (int64_t)Dpad, K, 4 * (int64_t)Dpad, (int64_t)Dpad};
            A.kb = K / 32;
            A.n_sites = nb;
            A.mt_per = (int)(KB / 128);
            A.nt_per = (Dpad + A.N - 1) / A.N;
            A.n_cols = Dpad;
            A.out32 = (float2*)c->mt32.p;
            A.out32_site = (int64_t)perMt;
            A.out32_ld = (int64_t)ldm;
            A.out32_rows = 1;
            A.ep_B = Bpad;
            A.ep_Dp = Dpad;
            A.err = (int*)c->errflag.p;
            A.wait_ns = c->wait_ns;
            CUDA_TRY(c, bip_tc_gemm(A, s));
        } else {
            CGemmArgs A{};
            A.M = geo.n_det; A.N = nch * Bpad; A.K = K;
            A.A = (const float2*)c->opA32.p; A.lda = K; A.strideA = (int64_t)perA;
            A.Bm = (const float2*)c->opB32.p; A.ldb = K; A.strideB = (int64_t)perB;
            A.batch = nb;
            A.epi = 1;
            A.C = (float2*)c->mt32.p; A.ldc = (int64_t)ldm; A.strideC = (int64_t)perMt;
            A.ep_B = Bpad; A.ep_Dp = Dpad;
            CUDA_TRY(c, bip_cgemm_simt(A, s));
        }
        // R_tau = f o_tau sum_{rho in crop} g c c^H
        CUDA_TRY(c, bip_grad_crop_weights(gab, nb, ids, (float*)c->g_w.p, s));
        CGemmGen r{};
        r.M = B; r.N = B; r.K = P; r.batch = nb;
        r.A = (const float2*)c->illum.p; r.sam = P; r.sak = 1; r.sab = 0;
        r.dk = (const float*)c->g_w.p; r.sdb = P;
        r.B = (const float2*)c->illum.p; r.sbk = 1; r.sbn = P; r.sbb = 0; r.conjB = 1;
        r.C = (float2*)c->g_R.p; r.scm = Bpad; r.scn = 1; r.scb = (int64_t)perQ;
        CUDA_TRY(c, bip_cgemm_gen(r, s));
        if (d_aberr) {
            // Q = sum_n M_n^H M_n, then D_b += (Q R)_bb
            CGemmArgs Bq{};
            Bq.M = Bpad; Bq.N = Bpad; Bq.K = (int)ldm;
            Bq.A = (const float2*)c->mt32.p; Bq.lda = (int64_t)ldm; Bq.strideA = (int64_t)perMt;
            Bq.Bm = Bq.A; Bq.ldb = Bq.lda; Bq.strideB = Bq.strideA;
            Bq.conjA = 1;
            Bq.batch = nb;
            Bq.epi = 0;
            Bq.C = (float2*)c->q32.p; Bq.ldc = Bpad; Bq.strideC = (int64_t)perQ;
            CUDA_TRY(c, bip_cgemm_simt(Bq, s));
            CUDA_TRY(c, bip_grad_aberr(B, Bpad, nb, (const float2*)c->q32.p, (int64_t)perQ, (const float2*)c->g_R.p,
                                       (int64_t)perQ, (double2*)c->g_D.p, (double2*)c->g_Dsum.p, s));
        }
        if (d_H || d_V) {
            // Mbar_n = M_n R, kept as GMt = conj(R) Mt (R Hermitian)
            CGemmGen m{};
            m.M = B; m.N = (int)ldm; m.K = B; m.batch = nb;
            m.A = (const float2*)c->g_R.p; m.sam = Bpad; m.sak = 1; m.sab = (int64_t)perQ; m.conjA = 1;
            m.B = (const float2*)c->mt32.p; m.sbk = (int64_t)ldm; m.sbn = 1; m.sbb = (int64_t)perMt;
            m.C = (float2*)c->g_gmt.p; m.scm = (int64_t)ldm; m.scn = 1; m.scb = (int64_t)perMt;
            CUDA_TRY(c, bip_cgemm_gen(m, s));
            // T_n(b, r) = sum_d Mbar_n(d, b) conj S2_d(r)
            if (tcg) {
                // B operand: conj(S2) transposed to rows r, K = d (once per batch)
                SplitArgs st{(const float2*)c->opA32.p, 1, K, (int64_t)perA, K, Dpad, nb, (uint16_t*)c->g_tB.p,
                             (int64_t)4 * K * Dpad, K, Dpad, 0, 1};
                CUDA_TRY(c, bip_split_planes(st, s));
            }
            for (int n = 0; n < nch; ++n) {
                if (tcg) {
                    SplitArgs sg{(const float2*)c->g_gmt.p + (size_t)n * Dpad, (int64_t)ldm, 1, (int64_t)perMt, Bpad,
                                 Dpad, nb, (uint16_t*)c->g_tA.p, (int64_t)4 * Bpad * Dpad, Bpad, Dpad, 0, 0};
                    CUDA_TRY(c, bip_split_planes(sg, s));
                    TcArgs t{};
                    t.epi = TC_EPI_C32;
                    t.N = 256;
                    t.npl = 4;
                    t.A = TcOperand{c->g_tA.p, (int64_t)nb * 4 * Bpad, Dpad, 4 * (int64_t)Bpad, Bpad};
                    t.B = TcOperand{c->g_tB.p, (int64_t)nb * 4 * K, Dpad, 4 * (int64_t)K, K};
                    t.kb = Dpad / 32;
                    t.n_sites = nb;
                    t.mt_per = Bpad / 128;
                    t.nt_per = (K + 255) / 256;
                    t.n_cols = K;
                    t.out32 = (float2*)c->g_T.p + (size_t)n * Bpad * K;
                    t.out32_site = (int64_t)perT;
                    t.out32_ld = K;
                    t.err = (int*)c->errflag.p;
                    t.wait_ns = c->wait_ns;
                    CUDA_TRY(c, bip_tc_gemm(t, s));
                } else {
                    CGemmGen t{};
                    t.M = B; t.N = K; t.K = geo.n_det; t.batch = nb;
                    t.A = (const float2*)c->g_gmt.p + (size_t)n * Dpad; t.sam = (int64_t)ldm; t.sak = 1;
                    t.sab = (int64_t)perMt;
                    t.B = (const float2*)c->opA32.p; t.sbk = K; t.sbn = 1; t.sbb = (int64_t)perA; t.conjB = 1;
                    t.C = (float2*)c->g_T.p + (size_t)n * Bpad * K; t.scm = K; t.scn = 1; t.scb = (int64_t)perT;
                    CUDA_TRY(c, bip_cgemm_gen(t, s));
                }
            }
            if (d_H)
                CUDA_TRY(c, bip_grad_h(gab, nb, ids, nch, (const float2*)c->g_s1.p, (int64_t)perS1,
                                       (const float2*)c->g_T.p, (int64_t)perT, (int64_t)Bpad * K, (float2*)d_H, s));
        }
        if (d_V) {
            // S1bar_b(r) = sum_n conj H_n(r) T_n(b, r);
            // S2bar_d(r) = sum_n sum_b Mbar_n(d, b) conj(H_n(r) S1_b(r))
            CUDA_TRY(c, bip_s1bar(nb, ids, (const SiteDev*)c->sites_d.p, B, K, (const float2*)H,
                                  (const float2*)c->g_T.p, (int64_t)perT, (int64_t)Bpad * K, (float2*)c->g_s1bar.p,
                                  (int64_t)perS1, s));
            if (tcg) {
                // one contraction over K = (n, b): A = Mbar^T rows d, B = conj(H S1)^T rows r
                for (int n = 0; n < nch; ++n) {
                    SplitArgs sg{(const float2*)c->g_gmt.p + (size_t)n * Dpad, 1, (int64_t)ldm, (int64_t)perMt, Dpad,
                                 Bpad, nb, (uint16_t*)c->g_sA2.p, (int64_t)(4 * D128 * KB), D128, (int)KB, n * Bpad, 0};
                    CUDA_TRY(c, bip_split_planes(sg, s));
                }
                SplitArgs sx{(const float2*)c->opB32.p, 1, K, (int64_t)perB, K, (int)KB, nb, (uint16_t*)c->g_sB2.p,
                             (int64_t)(4 * K * KB), K, (int)KB, 0, 1};
                CUDA_TRY(c, bip_split_planes(sx, s));
                TcArgs u{};
                u.epi = TC_EPI_C32;
                u.N = 256;
                u.npl = 4;
                u.A = TcOperand{c->g_sA2.p, (int64_t)nb * 4 * D128, (int)KB, 4 * (int64_t)D128, D128};
                u.B = TcOperand{c->g_sB2.p, (int64_t)nb * 4 * K, (int)KB, 4 * (int64_t)K, K};
                u.kb = (int)(KB / 32);
                u.n_sites = nb;
                u.mt_per = D128 / 128;
                u.nt_per = (K + 255) / 256;
                u.n_cols = K;
                u.out32 = (float2*)c->g_s2bar.p;
                u.out32_site = (int64_t)perS2bar;
                u.out32_ld = K;
                u.err = (int*)c->errflag.p;
                u.wait_ns = c->wait_ns;
                CUDA_TRY(c, bip_tc_gemm(u, s));
            } else {
                for (int n = 0; n < nch; ++n) {
                    CGemmGen u{};
                    u.M = geo.n_det; u.N = K; u.K = B; u.batch = nb;
                    u.A = (const float2*)c->g_gmt.p + (size_t)n * Dpad; u.sam = 1; u.sak = (int64_t)ldm;
                    u.sab = (int64_t)perMt;
                    u.B = (const float2*)c->opB32.p + (size_t)n * Bpad * K; u.sbk = K; u.sbn = 1;
                    u.sbb = (int64_t)perB;
                    u.conjB = 1;
                    u.C = (float2*)c->g_s2bar.p; u.scm = K; u.scn = 1; u.scb = (int64_t)perS2bar;
                    u.accumulate = n > 0;
                    CUDA_TRY(c, bip_cgemm_gen(u, s));
                }
            }
            // back through the reconstructions into the window adjoints
            for (int side = 1; side <= 2; ++side) {
                ReconAdjArgs ra{};
                ra.n_sites = nb;
                ra.site_ids = ids;
                ra.sites = (const SiteDev*)c->sites_d.p;
                ra.K = K; ra.win = wb; ra.ny = g.ny; ra.nx = g.nx;
                ra.stash_win = g.win;
                ra.wo = (g.win - wb) / 2;
                ra.magnitude = g.recon == BIP_RECON_MAGNITUDE;
                if (side == 1) {
                    ra.Bp = geo.Bp1; ra.n_targets = B; ra.tilt_sign = +1;
                    ra.h_t = (const int2*)c->hbeam.p;
                    ra.stash = (const float2*)c->stash1.p;
                    ra.w = adj_weights(c->aw1);
                    ra.Sbar = (const float2*)c->g_s1bar.p; ra.sbar_rows = Bpad;
                    ra.dtbar = (float2*)c->g_dt1.p;
                } else {
                    ra.Bp = geo.Bp2; ra.n_targets = geo.n_det; ra.tilt_sign = -1;
                    ra.h_t = (const int2*)c->hdet.p;
                    ra.stash = (const float2*)c->stash2.p;
                    ra.w = adj_weights(c->aw2);
                    ra.Sbar = (const float2*)c->g_s2bar.p; ra.sbar_rows = (int)(perS2bar / K);
                    ra.dtbar = (float2*)c->g_dt2.p;
                }
                ra.Ubar = (float2*)c->g_ubar.p;
                ra.dA = (float*)c->g_dA.p;
                CUDA_TRY(c, bip_recon_adjoint(ra, s));
            }
        }
    }
    if (tcg) {
        int flag = 0;
        CUDA_TRY(c, cudaMemcpyAsync(&flag, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (flag) return fail(c, BIP_ERR_TIMEOUT, "a tensor-core contraction gave up waiting (device timeout)");
    }
    if (d_V) {
        CUDA_TRY(c, cudaMemsetAsync(d_V, 0, (size_t)g.nz * g.ny * g.nx * sizeof(float), s));
        st = adjoint_s1(c, V, d_V, s);
        if (st != BIP_OK) return st;
        st = adjoint_s2(c, V, d_V, s);
        if (st != BIP_OK) return st;
    }
    if (d_aberr) {
        std::vector<double2> D(B);
        CUDA_TRY(c, cudaMemcpyAsync(D.data(), c->g_Dsum.p, (size_t)B * sizeof(double2), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        // dL/dtheta = -2 sum_b chi'_b Im D_b
        double gdf = 0.0, gcs = 0.0;
        for (int b = 0; b < B; ++b) {
            double ddf = 0.0, dcs = 0.0;
            bip_aberration_phase(g, geo.lambda, geo.h_beam[2 * b], geo.h_beam[2 * b + 1], nullptr, &ddf, &dcs);
            gdf += -2.0 * ddf * D[b].y;
            gcs += -2.0 * dcs * D[b].y;
        }
        d_aberr[0] = gdf;
        d_aberr[1] = gcs;
    }
    return BIP_OK;
}

bip_status bip_coreloss_grad(bip_ctx* c, const float* V, const void* H, const double* scan_px, int32_t P,
                             const double* dL_dI, double* d_occ, void* d_H, double* d_aberr, float* d_V,
                             void* stream) {
    BIP_RANGE("bip_coreloss_grad");
    bip_status st = refuse_check_under_capture(c, (cudaStream_t)stream);
    if (st != BIP_OK) return st;
    st = coreloss_grad(c, V, H, scan_px, P, dL_dI, d_occ, d_H, d_aberr, d_V, stream);
    if (st != BIP_OK || !c->check_finite) return st;
    if (d_aberr && !(std::isfinite(d_aberr[0]) && std::isfinite(d_aberr[1])))
        return fail(c, BIP_ERR_NUMERIC, "the aberration derivatives are NaN or infinite");
    const int64_t G = (int64_t)c->cfg.ny * c->cfg.nx;
    return finite_check(c,
                        {{d_occ, c->n_sites, 8}, {d_H, 2 * c->h_elems, 4}, {d_V, (int64_t)c->cfg.nz * G, 4}},
                        (cudaStream_t)stream);
}

bip_status bip_copy_stash(bip_ctx* c, int32_t which, int32_t site, void* out, void* stream) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!out) return fail(c, BIP_ERR_INVALID_ARG, "out is null");
    if (which != 1 && which != 2) return fail(c, BIP_ERR_INVALID_ARG, "which must be 1 or 2");
    if ((which == 1 && !c->s1) || (which == 2 && !c->s2)) return fail(c, BIP_ERR_INVALID_ARG, "matrix not built");
    if (site < 0 || site >= c->n_sites) return fail(c, BIP_ERR_INVALID_ARG, "site out of range");
    const int ncol = which == 1 ? c->geo.Bp1 : c->geo.Bp2;
    const size_t n = (size_t)ncol * c->cfg.win * c->cfg.win;
    const float2* src = (const float2*)(which == 1 ? c->stash1.p : c->stash2.p) + (size_t)site * n;
    CUDA_TRY(c, cudaMemcpyAsync(out, src, n * sizeof(float2), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return BIP_OK;
}

bip_status bip_export_stash(bip_ctx* c, int32_t which, void* dst, int64_t bytes, void* stream) {
    if (!c) return BIP_ERR_INVALID_ARG;
    if (which != 1 && which != 2) return fail(c, BIP_ERR_INVALID_ARG, "which must be 1 or 2");
    if ((which == 1 && !c->s1) || (which == 2 && !c->s2)) return fail(c, BIP_ERR_INVALID_ARG, "matrix not built");
    if (!dst) return fail(c, BIP_ERR_INVALID_ARG, "dst is null");
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return fail(c, BIP_ERR_INVALID_ARG, "bip_export_stash is not capturable");
    const size_t need = (size_t)c->n_sites * (which == 1 ? c->geo.Bp1 : c->geo.Bp2) * c->cfg.win * c->cfg.win *
                        sizeof(float2);
    if (bytes < 0 || (size_t)bytes != need)
        return fail(c, BIP_ERR_SHAPE, "the stash is " + std::to_string(need) + " bytes, not " + std::to_string(bytes));
    const void* src = which == 1 ? c->stash1.p : c->stash2.p;
    CUDA_TRY(c, cudaMemcpyAsync(dst, src, need, cudaMemcpyDefault, s));
    return BIP_OK;
}

bip_status bip_import_stash(bip_ctx* c, int32_t which, const bip_atom* atoms, int32_t n_atoms, const void* src,
                            int64_t bytes, void* stream) {
    BIP_RANGE("bip_import_stash");
    if (!c) return BIP_ERR_INVALID_ARG;
    if (which != 1 && which != 2) return fail(c, BIP_ERR_INVALID_ARG, "which must be 1 or 2");
    if (!src) return fail(c, BIP_ERR_INVALID_ARG, "src is null");
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return fail(c, BIP_ERR_INVALID_ARG, "bip_import_stash is not capturable");
    std::vector<SiteDev> sites;
    int nmax = 0, total = 0;
    bip_status st = parse_sites(c, atoms, n_atoms, sites, nmax, total);
    if (st != BIP_OK) return st;
    const int ncol = which == 1 ? c->geo.Bp1 : c->geo.Bp2;
    const size_t need = sites.size() * ncol * c->cfg.win * c->cfg.win * sizeof(float2);
    if (bytes < 0 || (size_t)bytes != need)
        return fail(c, BIP_ERR_SHAPE, "a stash of these sites is " + std::to_string(need) + " bytes, not " +
                                          std::to_string(bytes));
    st = make_tables(c, s);
    if (st != BIP_OK) return st;
    st = set_sites(c, sites, nmax, total, s);
    if (st != BIP_OK) return st;
    DevBuf& stash = which == 1 ? c->stash1 : c->stash2;
    const size_t G = (size_t)c->cfg.ny * c->cfg.nx;
    CUDA_TRY(c, ensure(stash, need, false, s));
    // the reverse pass's sweeps use the builds' column workspace
    CUDA_TRY(c, ensure(c->cols, (size_t)std::max(c->geo.Bp1, c->geo.Bp2) * G * sizeof(float2), false, s));
    CUDA_TRY(c, cudaMemcpyAsync(stash.p, src, need, cudaMemcpyDefault, s));
    if (which == 1) {
        c->s1 = true;
        c->sig1 = site_signature(c->sites);
    } else {
        c->s2 = true;
        c->sig2 = site_signature(c->sites);
    }
    return BIP_OK;
}

bip_status bip_set_check_finite(bip_ctx* c, int32_t on) {
    if (!c) return BIP_ERR_INVALID_ARG;
    c->check_finite = on != 0;
    return BIP_OK;
}

bip_status bip_mem_stats(int64_t* live_bytes, int64_t* peak_bytes, int32_t reset_peak) {
    if (live_bytes) *live_bytes = g_bytes.load();
    if (peak_bytes) *peak_bytes = g_peak.load();
    if (reset_peak) g_peak = g_bytes.load();
    return BIP_OK;
}

bip_status bip_site_windows(bip_ctx* c, int32_t site, void* s1_out, void* s2_out, void* stream) {
    BIP_RANGE("bip_site_windows");
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!c->s1 || !c->s2 || c->sig1 != c->sig2)
        return fail(c, BIP_ERR_INVALID_ARG, "bip_build_s1 and bip_build_s2 must run first on the same sites");
    if (site < 0 || site >= c->n_sites) return fail(c, BIP_ERR_INVALID_ARG, "site out of range");
    if (c->uneven) return fail(c, BIP_ERR_UNSUPPORTED, "site windows are given at the context's window only");
    if (((reinterpret_cast<uintptr_t>(s1_out) | reinterpret_cast<uintptr_t>(s2_out)) & 15) != 0)
        return fail(c, BIP_ERR_INVALID_ARG, "window outputs must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const bip_config& g = c->cfg;
    const int K = g.win * g.win;
    const int32_t* ids = (const int32_t*)c->seq_ids_d.p + site;
    if (s1_out) {
        GatherArgs a = gather_args(c, 1, ids, 1);
        a.out_c64 = (float2*)s1_out;
        a.site_stride = (int64_t)c->geo.B * K;
        CUDA_TRY(c, bip_gather(a, s));
    }
    if (s2_out) {
        GatherArgs a = gather_args(c, 2, ids, 1);
        a.out_c64 = (float2*)s2_out;
        a.site_stride = (int64_t)c->geo.n_det * K;
        CUDA_TRY(c, bip_gather(a, s));
    }
    return BIP_OK;
}

bip_status bip_set_profiling(bip_ctx* c, int32_t on) {
    if (!c) return BIP_ERR_INVALID_ARG;
    c->prof = on < 0 ? (1u << BIP_N_STAGES) - 1u : (uint32_t)on & ((1u << BIP_N_STAGES) - 1u);
    c->ev_used = 0;
    c->ev_rec.clear();
    for (int i = 0; i < BIP_N_STAGES; ++i) c->launches[i] = 0;
    return BIP_OK;
}

bip_status bip_get_profile(bip_ctx* c, double* ms, int64_t* launches) {
    if (!c) return BIP_ERR_INVALID_ARG;
    double acc[BIP_N_STAGES] = {0};
    for (auto& r : c->ev_rec) {
        CUDA_TRY(c, cudaEventSynchronize(r.second.second));
        float t = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&t, r.second.first, r.second.second));
        acc[r.first] += t;
    }
    for (int i = 0; i < BIP_N_STAGES; ++i) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = c->launches[i];
    }
    return BIP_OK;
}

bip_status bip_site_coupling(bip_ctx* c, const void* H, int32_t site, void* m_out, void* stream) {
    BIP_RANGE("bip_site_coupling");
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!c->s1 || !c->s2 || c->sig1 != c->sig2)
        return fail(c, BIP_ERR_INVALID_ARG, "bip_build_s1 and bip_build_s2 must run first on the same sites");
    if (!H || !m_out) return fail(c, BIP_ERR_INVALID_ARG, "null pointer argument");
    if ((reinterpret_cast<uintptr_t>(H) & 15) != 0) return fail(c, BIP_ERR_INVALID_ARG, "H must be 16-byte aligned");
    if (site < 0 || site >= c->n_sites) return fail(c, BIP_ERR_INVALID_ARG, "site out of range");
    if (c->uneven) return fail(c, BIP_ERR_UNSUPPORTED, "the site coupling is given at the context's window only");
    cudaStream_t s = (cudaStream_t)stream;
    const bip_config& g = c->cfg;
    const BipGeometry& geo = c->geo;
    const int K = g.win * g.win, Bpad = c->Bpad, Dpad = c->Dpad, nch = c->nch_max;
    const bool tc = c->prec != BIP_PREC_FP32;
    const bool f8 = c->prec == BIP_PREC_FP8_TILE;
    if (f8 && !c->recon_tc)
        return fail(c, BIP_ERR_UNSUPPORTED, "the FP8 coupling needs at most 64 parents per side");
    const int npl = gram_planes(c->prec);
    const size_t perA = (size_t)Dpad * K, perB = (size_t)nch * Bpad * K;
    const size_t ldc = (size_t)nch * Bpad;
    DevBuf& opA = f8 ? c->op8A : tc ? c->opA16 : c->opA32;
    DevBuf& opB = f8 ? c->op8B : tc ? c->opB16 : c->opB32;
    CUDA_TRY(c, ensure(opA, perA * (f8 ? 2 : 8), true, s));
    CUDA_TRY(c, ensure(opB, perB * (f8 ? 2 : 8), true, s));
    CUDA_TRY(c, ensure(c->partial, (size_t)Dpad * ldc * sizeof(float2), false, s));
    const int32_t* ids = (const int32_t*)c->seq_ids_d.p + site;
    GatherArgs g2 = gather_args(c, 2, ids, 1);
    g2.rows_pad = Dpad;
    GatherArgs g1 = gather_args(c, 1, ids, 1);
    g1.rows_pad = Bpad;
    g1.nch = nch;
    g1.H = (const float2*)H;
    if (tc) {
        g2.out_bf16 = (uint16_t*)opA.p; g2.out_planes = npl; g2.site_stride = (int64_t)(npl * perA);
        g1.out_bf16 = (uint16_t*)opB.p; g1.out_planes = npl; g1.site_stride = (int64_t)(npl * perB);
    } else {
        g2.out_c64 = (float2*)opA.p; g2.site_stride = (int64_t)perA;
        g1.out_c64 = (float2*)opB.p; g1.site_stride = (int64_t)perB;
    }
    if (tc) CUDA_TRY(c, cudaMemsetAsync(c->errflag.p, 0, sizeof(int), s));
    if (f8) {
        bip_status st = f8_hmax(c, H, s);
        if (st != BIP_OK) return st;
    }
    if ((c->prec == BIP_PREC_MIXED || f8) && c->recon_tc) {
        bip_status st = recon_tc_batch(c, ids, 1, H, opA.p, opB.p, s);
        if (st != BIP_OK) return st;
    } else {
        TIMED(c, BIP_STAGE_GATHER, s, bip_gather(g2, s));
        TIMED(c, BIP_STAGE_GATHER, s, bip_gather(g1, s));
    }
    float2* tmp = (float2*)c->partial.p;      // [Dpad][nch * Bpad] complex64
    if (tc) {
        // the map's orientation: aperture side (ch, b) as A, detector side as
        // B; the C32 epilogue writes tmp[d][(ch, b)]
        TcArgs A{};
        A.epi = TC_EPI_C32;
        A.N = tile_width(Dpad);
        A.npl = npl;
        A.A = TcOperand{opB.p, npl * (int64_t)ldc, K, npl * (int64_t)ldc, (int64_t)ldc};
        A.B = TcOperand{opA.p, npl * (int64_t)Dpad, K, npl * (int64_t)Dpad, Dpad};
        A.kb = K / 32;
        A.n_sites = 1;
        A.mt_per = (int)(ldc / 128);
        A.nt_per = (Dpad + A.N - 1) / A.N;
        A.n_cols = Dpad;
        A.out32 = tmp;
        A.out32_site = 0;
        A.out32_ld = (int64_t)ldc;
        A.out32_trans = 1;
        A.err = (int*)c->errflag.p;
        A.wait_ns = c->wait_ns;
        if (f8) {
            A.f8 = 1;
            A.A = TcOperand{opB.p, 2 * (int64_t)ldc, K / 2, 2 * (int64_t)ldc, (int64_t)ldc};
            A.B = TcOperand{opA.p, 2 * (int64_t)Dpad, K / 2, 2 * (int64_t)Dpad, Dpad};
            A.kb = K / 64;
            A.scaleA = (const float*)c->f8sA.p;
            A.scaleA_site = (int64_t)ldc;
            A.scaleB = (const float*)c->f8sB.p;
            A.scaleB_site = Dpad;
        }
        TIMED(c, BIP_STAGE_COUPLING, s, bip_tc_gemm(A, s));
    } else {
        CGemmArgs A{};
        A.M = geo.n_det; A.N = (int)ldc; A.K = K;
        A.A = (const float2*)opA.p; A.lda = K; A.strideA = (int64_t)perA;
        A.Bm = (const float2*)opB.p; A.ldb = K; A.strideB = (int64_t)perB;
        A.batch = 1;
        A.epi = 0;
        A.C = tmp; A.ldc = (int64_t)ldc; A.strideC = 0;
        TIMED(c, BIP_STAGE_COUPLING, s, bip_cgemm_simt(A, s));
    }
    // [n_det][(ch, b)] -> m_out[ch][n_det][B]
    for (int ch = 0; ch < nch; ++ch)
        CUDA_TRY(c, cudaMemcpy2DAsync((float2*)m_out + (size_t)ch * geo.n_det * geo.B, geo.B * sizeof(float2),
                                      tmp + (size_t)ch * Bpad, ldc * sizeof(float2), geo.B * sizeof(float2),
                                      geo.n_det, cudaMemcpyDeviceToDevice, s));
    if (tc) {
        int flag = 0;
        CUDA_TRY(c, cudaMemcpyAsync(&flag, c->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (flag) return fail(c, BIP_ERR_TIMEOUT, "a tensor-core contraction gave up waiting (device timeout)");
    }
    return BIP_OK;
}

}  // extern "C"

// ===========================================================================
// S1 build without any allocation: parent columns and device tables in the
// library's static scratch array, windows written to the caller's buffer.

extern "C" bip_status bip_build_s1_noalloc(bip_ctx* c, const float* V, const bip_atom* atoms, int32_t n_atoms,
                                           void* stash, void* stream) {
    BIP_RANGE("bip_build_s1_noalloc");
    if (!c) return BIP_ERR_INVALID_ARG;
    if (!V) return fail(c, BIP_ERR_INVALID_ARG, "V is null");
    if (!stash) return fail(c, BIP_ERR_INVALID_ARG, "stash is null");
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s))
        return fail(c, BIP_ERR_INVALID_ARG, "bip_build_s1_noalloc copies from call-local host memory: not capturable");
    const bip_config& g = c->cfg;
    const BipGeometry& geo = c->geo;
    std::vector<SiteDev> sites;
    int nmax = 0, total = 0;
    bip_status st = parse_sites(c, atoms, n_atoms, sites, nmax, total);
    if (st != BIP_OK) return st;
    const int ncol = geo.Bp1;
    const size_t G = (size_t)g.ny * g.nx;

    // layout of the scratch array, every region 256-byte aligned
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_cols = 0;
    const size_t o_twy = o_cols + al((size_t)ncol * G * sizeof(float2));
    const size_t o_twx = o_twy + al((size_t)g.ny * sizeof(float2));
    const size_t o_py = o_twx + al((size_t)g.nx * sizeof(float2));
    const size_t o_px = o_py + al((size_t)g.ny * sizeof(float2));
    const size_t o_sh = o_px + al((size_t)g.nx * sizeof(float2));
    std::vector<int32_t> roff;
    std::vector<int4> rent;
    row_windows(g, sites, roff, rent);
    const size_t o_roff = o_sh + al((size_t)ncol * sizeof(int2));
    const size_t o_rent = o_roff + al(roff.size() * sizeof(int32_t));
    const size_t need = o_rent + al(rent.size() * sizeof(int4));
    if (need > kNoallocScratchBytes)
        return fail(c, BIP_ERR_SHAPE,
                    "bip_build_s1_noalloc needs " + std::to_string(need) + " bytes of scratch (" +
                        std::to_string(ncol) + " parent columns of " + std::to_string(g.ny) + "x" +
                        std::to_string(g.nx) + "); the static scratch holds " +
                        std::to_string(kNoallocScratchBytes) + " bytes");

    void* base = nullptr;
    CUDA_TRY(c, bip_noalloc_scratch_ptr(&base));
    unsigned char* sc = (unsigned char*)base;

    // host tables (same definitions as the context's: FP64 then rounded)
    const std::vector<float2> twy = fft_twiddles(g.ny), twx = fft_twiddles(g.nx);
    std::vector<float2> py(g.ny), px(g.nx);
    for (int k = 0; k < g.ny; ++k) {
        const double q = signed_bin(k, g.ny) / g.ly;
        const double a = -kPi * geo.lambda * g.dz * q * q;
        py[k] = float2{(float)(std::cos(a) / g.ny), (float)(std::sin(a) / g.ny)};
    }
    for (int k = 0; k < g.nx; ++k) {
        const double q = signed_bin(k, g.nx) / g.lx;
        const double a = -kPi * geo.lambda * g.dz * q * q;
        px[k] = float2{(float)(std::cos(a) / g.nx), (float)(std::sin(a) / g.nx)};
    }
    std::vector<int2> sh(ncol);
    for (int i = 0; i < ncol; ++i) sh[i] = int2{geo.h_beam[2 * geo.p1[i]], geo.h_beam[2 * geo.p1[i] + 1]};
    // planes that hold sites
    std::vector<int32_t> off(g.nz + 1, 0);
    for (auto& sd : sites) off[sd.plane + 1]++;
    for (int j = 0; j < g.nz; ++j) off[j + 1] += off[j];
    auto put = [&](size_t o, const void* h, size_t bytes) {
        return cudaMemcpyAsync(sc + o, h, bytes, cudaMemcpyHostToDevice, s);
    };
    CUDA_TRY(c, put(o_twy, twy.data(), twy.size() * sizeof(float2)));
    CUDA_TRY(c, put(o_twx, twx.data(), twx.size() * sizeof(float2)));
    CUDA_TRY(c, put(o_py, py.data(), py.size() * sizeof(float2)));
    CUDA_TRY(c, put(o_px, px.data(), px.size() * sizeof(float2)));
    CUDA_TRY(c, put(o_sh, sh.data(), sh.size() * sizeof(int2)));
    CUDA_TRY(c, put(o_roff, roff.data(), roff.size() * sizeof(int32_t)));
    CUDA_TRY(c, put(o_rent, rent.data(), rent.size() * sizeof(int4)));

    MsPlan plan{};
    plan.ny = g.ny;
    plan.nx = g.nx;
    plan.ncol = ncol;
    plan.sigma = (float)geo.sigma;
    plan.twy = (const float2*)(sc + o_twy);
    plan.twx = (const float2*)(sc + o_twx);
    plan.py = (const float2*)(sc + o_py);
    plan.px = (const float2*)(sc + o_px);
    plan.shift = (const int2*)(sc + o_sh);
    float2* cols = (float2*)(sc + o_cols);
    int last = 0;
    for (auto& sd : sites) last = std::max(last, (int)sd.plane);
    for (int j = 0; j <= last; ++j) {
        MsRowArgs a{};
        a.cols = cols;
        a.init = j == 0;
        a.init_val = 1.0f;
        a.do_ifft = j > 0;
        a.v_post = j < last ? V + (size_t)j * G : nullptr;
        a.do_fft = j < last;
        if (off[j + 1] > off[j]) {
            a.row_off = (const int32_t*)(sc + o_roff) + (size_t)j * (g.ny + 1);
            a.row_ent = (const int4*)(sc + o_rent);
        }
        a.win = g.win;
        a.stash = (float2*)stash;
        CUDA_TRY(c, bip_ms_row_pass(plan, a, s));
        if (j < last) CUDA_TRY(c, bip_ms_col_pass(plan, cols, s));
    }
    return BIP_OK;
}
