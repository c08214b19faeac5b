// Internal declarations of the BiP-PRISM library: context, geometry and the
// launchers of every CUDA kernel.  Host code only (no device code here).
#pragma once

#include <atomic>
#include <complex>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bip.h"

// ---------------------------------------------------------------------------
// host geometry (FP64), built once per context

// Runs `set` (a kernel's launch attributes, set once per process: the
// library serves one GPU per process) until it first succeeds, safely when
// several host threads launch at once.
inline std::mutex& bip_attr_mutex() {
    static std::mutex m;
    return m;
}
template <class F>
cudaError_t bip_set_once(std::atomic<bool>& done, F&& set) {
    if (done.load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lk(bip_attr_mutex());
    if (done.load(std::memory_order_relaxed)) return cudaSuccess;
    const cudaError_t e = set();
    if (e == cudaSuccess) done.store(true, std::memory_order_release);
    return e;
}
// Runs `set` (raising a kernel's dynamic shared-memory limit to `bytes`)
// when `bytes` is above the largest size it succeeded for so far (`cur`),
// safely when several host threads launch at once.
template <class F>
cudaError_t bip_raise_once(std::atomic<size_t>& cur, size_t bytes, F&& set) {
    if (bytes <= cur.load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lk(bip_attr_mutex());
    if (bytes <= cur.load(std::memory_order_relaxed)) return cudaSuccess;
    const cudaError_t e = set();
    if (e == cudaSuccess) cur.store(bytes, std::memory_order_release);
    return e;
}

struct BipGeometry {
    double lambda = 0.0;      // electron wavelength, Angstrom
    double sigma = 0.0;       // interaction constant, rad/(V*Angstrom)
    int n_full = 0;           // aperture beams before subsampling
    int B = 0, n_det = 0, Bp1 = 0, Bp2 = 0;
    int dfy = 1, dfx = 1;                          // detector-side subsampling in effect
    std::vector<int32_t> h_beam, h_det;            // [B*2], [n_det*2]  (y, x)
    std::vector<int32_t> h_cube;                   // [n_cube*2]: the cube's complete basis
    int n_cube = 0;
    std::vector<int32_t> p1, p2;                   // parent positions in the lists
    std::vector<double> w1, w2;                    // [B*Bp1], [n_det*Bp2]
    std::vector<std::complex<double>> psi_beam;    // Psi(h_b)
    double psi_norm = 0.0;                         // sqrt(G sum_aperture |Psi|^2)
};

bip_status bip_build_geometry(const bip_config& cfg, BipGeometry& g, std::string& err);
// bip_build_geometry through the on-disk cache when one is set (geom_cache.cpp)
bip_status bip_geometry_cached(const bip_config& cfg, BipGeometry& g, std::string& err);
// chi(q) = pi lambda df |q|^2 + (pi/2) Cs lambda^3 |q|^4 of beam h (Psi = exp(-i chi))
// and its derivatives with respect to df and Cs (each output optional)
void bip_aberration_phase(const bip_config& c, double lambda, int hy, int hx, double* chi, double* d_defocus,
                          double* d_cs);
// Psi(h_b) of the aperture beams for the configuration's df and Cs
void bip_set_psi(const bip_config& c, BipGeometry& g);

// Sibson weights of `queries` against `parents` (integer beam indices,
// physical scale 1/ly, 1/lx); dense [nq * np] row-major.
void bip_sibson_weights(const std::vector<int32_t>& parents, const std::vector<int32_t>& queries,
                        double ly, double lx, std::vector<double>& w);

// ---------------------------------------------------------------------------
// device-side tables shared by several kernels

struct SiteDev {            // one ionized site, as the kernels see it
    int32_t oy, ox;         // origin of its stashed window (the context's win; unwrapped pixel index)
    int32_t plane;          // slice index
    int32_t nch;            // channels
    int32_t ch_off;         // first channel in H
    int32_t h_off;          // first element of its channels in H (channels of w x w each)
    int32_t w;              // its own window (<= win, a multiple of 16): the central
    int32_t wo;             // w x w block of the stashed window, at offset wo = (win - w) / 2
    double ty, tx;          // position in pixels
};

// Natural-neighbour weights of consecutive target groups: the targets
// kGatherGroup g .. kGatherGroup g + kGatherGroup - 1 share one list of
// parents (the union of their neighbours), each entry with the weights of
// all the group's targets (0 where the parent is not a neighbour).
constexpr int kGatherGroup = 4;
struct GroupDev {
    int32_t n_groups;
    const int32_t* off;     // [n_groups + 1] entry range of each group
    const uint16_t* par;    // [entries] parent index
    const float4* w;        // [entries] weights of the group's targets
};

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)

// multislice.cu
struct MsPlan {
    int ny, nx, ncol;
    float sigma;                    // interaction constant (FP32)
    const float2* twy;              // [ny] register-FFT twiddles, pass by pass
    const float2* twx;              // [nx]
    const float2* py;               // [ny] exp(-i pi lambda dz qy^2) / ny
    const float2* px;               // [nx]
    const int2* shift;              // [ncol] propagator shift (sy, sx)
    const float2* tw512;            // nx = 512: exp(-2 pi i e j / 512) at (e - 1) 32 + j,
                                    // e = 1..15, j < 32 (the half-warp row pass); else null
};
// row pass: [inverse row FFT] -> [T_pre] -> [stash] -> [T_post] -> [row FFT]
struct MsRowArgs {
    float2* cols;                   // [ncol, ny, nx]
    const float* v_pre;             // V slice applied before the stash (or null)
    const float* v_post;            // V slice applied after the stash (or null);
                                    // at most one of the two is set
    const float2* t_slice;          // the slice's T = exp(i sigma V) [ny][nx], when
                                    // precomputed (else evaluated from V)
    int init;                       // 1: start from a constant field `init_val`
    float init_val;
    int do_ifft, do_fft;
    // windows crossing each row of this plane: entries row_off[y] ..
    // row_off[y+1]-1 of row_ent, each (site, window row u, window x origin)
    const int32_t* row_off;         // [ny + 1] (null: no stash at this pass)
    const int4* row_ent;
    int win;
    float2* stash;                  // [n_sites_total, ncol, win, win]
    float2* save;                   // the real-space field at the stash point,
                                    // [ncol, ny, nx] (null: not kept)
};
cudaError_t bip_ms_row_pass(const MsPlan& plan, const MsRowArgs& a, cudaStream_t s);
// T_j = exp(i sigma V_j) of slices j0 .. j1 - 1 into T [nz][ny][nx] (the same
// slice offsets as V), once per build, for the row passes of both sweeps
cudaError_t bip_transmission(const float* V, float sigma, int j0, int j1, size_t G, float2* T, cudaStream_t s);
cudaError_t bip_ms_col_pass(const MsPlan& plan, float2* cols, cudaStream_t s);

// gather.cu : window reconstruction into GEMM operands
struct GatherArgs {
    int n_sites;                    // sites in this batch
    const int32_t* site_ids;        // [n_sites] global site index
    const SiteDev* sites;           // all sites
    int win, ny, nx;                // win: the batch's window (K = win^2 pixels)
    int stash_win, wo;              // stashed windows (and the tables' rows) of stash_win pixels;
                                    // the batch's window starts wo pixels in on both axes
    int Bp, n_targets, rows_pad;    // parents, targets, padded rows
    const float2* stash;            // [n_sites_total, Bp, stash_win, stash_win]
    GroupDev grp;                   // weights of the targets
    const int2* h_t;                // [n_targets] target beams (y, x)
    int tilt_sign;                  // +1 (S1) or -1 (S2)
    int magnitude;                  // 1: magnitude-preserving
    const float2* ey;               // [ny] exp(+2 pi i m / ny)
    const float2* ex;               // [nx]
    const float2* ytab;             // [ny][stash_win] exp(+2 pi i h u / ny), row h mod ny
    const float2* xtab;             // [nx][stash_win] exp(+2 pi i h v / nx), row h mod nx
    int fx;                         // lattice step of the targets along x
    // channel expansion (S1 side): out row (n * rows_pad + t) = H_n * S
    int nch;                        // 0: no channel product (S2 side)
    const float2* H;                // site channels from SiteDev::h_off, win x win each
    // outputs (one of the two layouts)
    float2* out_c64;                // [n_sites][rows_total][K] complex64
    uint16_t* out_bf16;             // [n_sites][planes][rows_total][K]: 4 planes (re_hi, re_lo,
                                    // im_hi, im_lo) or 2 planes (re, im)
    int out_planes;                 // 4 or 2
    int64_t site_stride;            // elements per site in the output
    int K;                          // window pixels (row length)
};
cudaError_t bip_gather(const GatherArgs& a, cudaStream_t s);

// recon_tc.cu : window reconstruction on the tensor cores (mixed path).
// X [site-plane rows][K px][64 parents] bf16: row (x_site0 + 3 bs + plane) K
// + px, planes re, im, magnitude of the de-tilted stash.
// cube_raster.cu : the cube's per-beam contraction on a raster scan list,
// separated over the aperture beams' lattice (two short sums, FP32)
struct CubeRasterArgs {
    int n_sites;                    // sites of the batch
    const int32_t* site_ids;
    const SiteDev* sites;
    const float2* m;                // M(n, b, d) = m[bs m_site + b m_b + n m_ch + d], complex64
    int64_t m_site, m_b, m_ch;
    int nch;                        // channel slots of M (a site uses its first nch)
    int nd, nd_pad;                 // beams d of the batch; row pitch of T (multiple of 32)
    int nky, nkx;                   // lattice rows 2 Ky + 1 and columns 2 Kx + 1
    const int32_t* lat;             // [nky][nkx] aperture beam at (k_y, k_x), or -1
    const double2* coef;            // [B] c_b(rho) = coef_b exp(-2 pi i h_b.rho / N)
    const float2* ay;               // [My][nky] exp(-2 pi i f_y k_y ry[my] / ny)
    const float2* ax;               // [nkx][Mx] exp(-2 pi i f_x k_x rx[mx] / nx)
    const uint32_t* crop_y;         // [all sites][wy] bit my: row my inside the site's crop (one axis)
    const uint32_t* crop_x;         // [all sites][wx] bit mx: column mx inside it
    int wy, wx;                     // words per site: ceil(My / 32), ceil(Mx / 32)
    int My, Mx;                     // scan (my, mx) is scan my Mx + mx
    float2* T;                      // workspace, bip_cube_raster_t_bytes
    float* cube;                    // cube[(my Mx + mx) cube_ld + d] += scale sum_n |a_d|^2
    int64_t cube_ld;
    float scale;
};
size_t bip_cube_raster_t_bytes(const CubeRasterArgs& a);
cudaError_t bip_cube_raster(const CubeRasterArgs& a, cudaStream_t s);

struct XprepSide {
    const float2* stash;            // [n_sites_total][Bp][stash_win^2]
    int Bp;                         // parents (<= 64)
    int x_site0;                    // first site-plane row block of this side
};
struct XprepArgs {
    int n_sites;                    // sites in this batch
    const int32_t* site_ids;        // [n_sites]
    int K;                          // window pixels (w^2)
    int w, stash_win, wo;           // the batch's window inside the stashed ones
    uint16_t* X;
    XprepSide side[2];              // 0: S2 (detector), 1: S1 (aperture)
    // FP8 path: largest |dt_p(r)| over the window of each parent, as float
    // bits, [2 sides][n_sites][64] (cleared by the caller); null: not taken
    unsigned* pmax;
};
cudaError_t bip_xprep(const XprepArgs& a, cudaStream_t s);

struct ReconSide {
    int n_targets;
    int rows_pad;                   // output rows per channel plane (>= n_targets)
    int w_pad;                      // rows of each W plane, = 128 mt_tiles
    int mt_tiles;
    int nch;                        // 0: no channel product (S2 side)
    int tilt_sign;                  // +1 (S1) or -1 (S2)
    const int2* h_t;                // [n_targets] target beams
    int w_row0;                     // first row of this side's W planes (hi, lo)
    int x_site0;                    // as in XprepSide
    int64_t site_stride;            // output elements per site
    int64_t plane_stride;           // output elements per plane (re, im)
    // transposed output (BF16, nch = 0): element (t, px) at px ld + t, so
    // that the targets are the contiguous index (the probe order's S1)
    int trans;
    int64_t ld;
};
struct ReconArgs {
    int n_sites;
    const int32_t* site_ids;
    const SiteDev* sites;
    int K, win, ny, nx;             // win: the batch's window, K = win^2
    int stash_win, wo;              // the tables' row length; offset of the batch's window
    int chunk_px, chunks;           // pixels per work unit, units per target tile
    int magnitude;
    const float2* ey;               // [ny] exp(+2 pi i m / ny)
    const float2* ex;               // [nx]
    const float2* ytab;             // [ny][stash_win]
    const float2* xtab;             // [nx][stash_win]
    const float2* H;                // site channels from SiteDev::h_off, K each; 16-byte aligned
    const uint16_t* W;              // [w_rows][64] bf16: per side hi then lo planes
    int w_rows;
    const uint16_t* Xb;             // X of XprepArgs
    int64_t x_rows;
    uint16_t* out[2];               // coupling operands (2 bf16 planes each)
    ReconSide side[2];
    int* err;                       // set to 1 on a device timeout
    uint64_t wait_ns;               // give-up limit of each wait (0: the built-in 4 s)
    // FP8 path: the operands are E4M3 bytes (out[] then holds bytes, same
    // element strides), each row scaled by inv_row[side][bs rows_pad + t];
    // H is then H_n / max_r |H_n| (F8HmaxArgs::Hs)
    int f8;
    const float* inv_row[2];
};
cudaError_t bip_recon_tc(const ReconArgs& a, cudaStream_t s);

// fp8.cu : per-window scales of the E4M3 coupling operands.  For target t
// of a side, bound_t = kappa sum_p w_tp pmax_p (kappa = 1 + 2^-6; w = the
// hi + lo BF16 weights of the W tensor); S1 rows are further scaled by
// max_r |H_n(r)| of their channel.
struct F8HmaxArgs {
    int n_sites;                    // all sites of the context
    const SiteDev* sites;
    const float2* H;                // site channels from SiteDev::h_off, w^2 each
    float* hmax;                    // [n_sites][9]: max_r |H_n(r)| (0 past the site's channels)
    float2* Hs;                     // H's layout: H_n / max_r |H_n| (0 where the max is 0)
};
cudaError_t bip_f8_hmax(const F8HmaxArgs& a, cudaStream_t s);
struct F8ScaleArgs {
    int n_sites;                    // sites of the batch
    const int32_t* site_ids;
    const SiteDev* sites;
    int nch;                        // channel planes of the S1 operand
    const float* hmax;              // of F8HmaxArgs, by site id
    const uint16_t* W;              // [w_rows][64] bf16
    int w_row0[2], w_pad[2], n_targets[2], rows_pad[2];
    const unsigned* pmax;           // [2][n_sites][64] (float bits)
    float* inv_row[2];              // [n_sites][rows_pad[side]]: 448 / bound (0 for empty rows)
    float* scaleB;                  // S2 rows: [n_sites][rows_pad[0]] bound / 448
    float* scaleA;                  // S1 rows (ch, b): [n_sites][nch rows_pad[1]] max|H_n| bound / 448
};
cudaError_t bip_f8_scales(const F8ScaleArgs& a, cudaStream_t s);

// gemm_simt.cu : FP32 complex GEMMs, C[m][n] = sum_k op(A[m][k]) B[n][k]
struct CGemmArgs {
    int M, N, K;                    // complex sizes (K multiple of 16)
    const float2* A; int64_t lda, strideA;   // row-major [M][lda], batch stride
    const float2* Bm; int64_t ldb, strideB;
    int conjA;
    int batch;
    // epilogue
    int epi;                        // 0: C row-major; 1: transposed to Mt[n%Bp][(n/Bp)*Dp + m]
    float2* C; int64_t ldc, strideC;
    int ep_B, ep_Dp;                // epilogue 1 geometry
};
cudaError_t bip_cgemm_simt(const CGemmArgs& a, cudaStream_t s);

// difftrans.cu : the per-site quadratic form c^H Q c as a trigonometric
// polynomial over beam-lattice differences (see the file's header)
struct DiffArgs {
    int n_sites;                    // binning: sites in the batch
    const float2* Q;                // FP32 Gram matrices [site][B..][ldq], upper triangle valid
    int64_t q_site;
    int ldq;
    int B;
    const int2* kb;                 // [B] beam lattice coordinates h / f (y, x)
    const double2* coef;            // [B] probe coefficients f_y f_x Psi / norm
    int Ky, Kx;                     // largest |k| on each axis
    const int32_t* lat;             // [(2Ky+1)(2Kx+1)] beam at each lattice point, -1 if none
    float2* G;                      // [site][(2Ky+1)(4Kx+1)] coefficients, Delta <= 0 (lex)
    // evaluation over (site, scan tile) work items
    const int32_t* work;
    int n_work, tile, P;
    const double* scans;
    const SiteDev* sites;
    const int32_t* site_ids;
    int ny, nx, fy, fx;
    float scale;                    // f_y f_x
    float* partial;                 // [n_sites_total][P]
};
cudaError_t bip_diff_bin(const DiffArgs& a, cudaStream_t s);
cudaError_t bip_diff_eval(const DiffArgs& a, cudaStream_t s);
// Raster scans rho(my, mx) = (y0 + sy my, x0 + sx mx), scan index my Mx + mx:
// the same polynomial as two separable stages per site,
//   I(my, mx) = f Re sum_iy Ay[my][iy] sum_j G[iy][j] Ax[j][mx],
//   Ay[my][iy] = exp(2 pi i f_y (iy - 2K_y) rho_y(my) / N_y)   [My][rows]
//   Ax[j][mx]  = exp(2 pi i f_x (j - 2K_x) rho_x(mx) / N_x)    [cols][Mx]
// written for the scans inside each site's crop mask (others stay 0).
struct RasterArgs {
    int My, Mx;
    const float2* Ay;
    const float2* Ax;
};
cudaError_t bip_raster_eval(const DiffArgs& a, const RasterArgs& r, cudaStream_t s);

// reduce.cu : map[rho] = FP64 Neumaier sum over sites of the partials
// (already zero outside each site's crop mask), in a fixed order; scratch
// of bip_reduce_scratch_bytes(n_sites, P) bytes.
size_t bip_reduce_scratch_bytes(int n_sites, int P);
// adds to *count the NaN or infinite values among n values of elem_bytes (4: float, 8: double)
cudaError_t bip_count_nonfinite(const void* v, int64_t n, int elem_bytes, unsigned long long* count, cudaStream_t s);
// occ (optional, [n_sites]): each site's contribution is weighted by its
// occupancy before the sum
cudaError_t bip_reduce_sites(const float* partial, int n_sites, int P, void* scratch, double* map_out,
                             cudaStream_t s, const double* occ = nullptr);

// gemm_tc.cu : tcgen05 complex contractions in split BF16 or BF16.
// Operands are bf16 planes, K contiguous -- four (re_hi, re_lo, im_hi,
// im_lo) or two (re, im) -- seen by TMA as one 2-D tensor [rows][K]; row
// (site, plane, r) is at site * site_rows + plane * plane_rows + r.
enum TcEpilogue { TC_EPI_ROWS = 0, TC_EPI_C32 = 2 };
struct TcOperand {
    const void* base;               // bf16 planes, 16-byte aligned
    int64_t rows;                   // rows of the 2-D tensor
    int k;                          // row length (multiple of 32)
    int64_t site_rows, plane_rows;  // row offsets of a site and of a plane
};
struct TcArgs {
    int epi;                        // TcEpilogue
    int N;                          // 128 or 256 (tile columns)
    int npl;                        // operand planes: 4 (split BF16) or 2 (BF16: re, im)
    int out_planes;                 // ROWS epilogue: planes written (4 or 2)
    TcOperand A, B;                 // A tiles of 128 rows, B tiles of N rows
    int kb;                         // K blocks of 32
    int n_sites, mt_per, nt_per;    // tiles per site
    int n_cols;                     // B rows per site in use: the last tile has
                                    // n_cols - (nt_per - 1) N columns (multiple of 16)
    int conjA;
    // E4M3 operands (kind::f8f6f4): rows of 2 k bytes, seen by the tensor
    // maps as k bf16; the products are scaled by scaleA[site][row] and
    // scaleB[site][column] in the epilogue
    int f8;
    const float* scaleA;
    const float* scaleB;
    int64_t scaleA_site, scaleB_site;
    // Hermitian output: tiles entirely below the diagonal are skipped
    int tri;
    // ROWS epilogue: A row r = (ch, b) = (r / ep_B, r % ep_B), output column n
    // -> out16[site][plane][b][ch * ep_Dp + n] (bf16 planes)
    uint16_t* out16;
    int64_t out_site, out_plane, out_ld;
    int ep_B, ep_Dp;
    // C32 epilogue: complex64 out32[site][row][n] (or [n][row] when transposed)
    float2* out32;
    int64_t out32_site, out32_ld;
    int out32_trans;
    int out32_rows;                 // A row (ch, b) -> out32[site][b][ch ep_Dp + n] (as ROWS)
    int* err;                       // device flag: set when a wait gives up
    uint64_t wait_ns;               // give-up limit of each wait (0: the built-in 4 s)
};
cudaError_t bip_tc_gemm(const TcArgs& a, cudaStream_t s);

// cube.cu : the 4D cube (the detector sum of Eq. map-sum left open)
struct IllumArgs {
    int P, B, Bpad;                 // scans, aperture beams, padded rows
    const int2* h;                  // [B] aperture beams (h_y, h_x)
    const double2* coef;            // [B] f_y f_x Psi / sqrt(G sum |Psi|^2)
    const double* scans;            // [P][2] pixels
    int ny, nx;
    float2* C;                      // [Bpad][P] c_b(rho), rows >= B zero
};
cudaError_t bip_illum(const IllumArgs& a, cudaStream_t s);

struct CubeArgs {
    int n_sites;                    // sites of this batch, added in order
    const int32_t* site_ids;
    const SiteDev* sites;
    int n_det, Bpad, nch, Dp;       // M^(n)_{d,b} at element b m_ld + n Dp + d
    int64_t m_ld, m_site;           // row stride, site stride
    const float2* m32;              // the coupling, complex64
    const float2* C;                // [Bpad][P]
    int P;
    const double* scans;
    int ny, nx, fy, fx;
    float scale;                    // the detector-side factor (1 for the exact cube)
    float* cube;                    // [P][cube_ld], rows d accumulated
    int64_t cube_ld;                // (>= n_det)
};
cudaError_t bip_cube_accumulate(const CubeArgs& a, cudaStream_t s);
// cube_tc.cu : the cube on tcgen05 (split BF16).  A = M transposed to rows d,
// K = (channel, b): [site][4 planes][rows (128 multiple)][nch Bpad] bf16;
// B = c_b(rho): [4 planes][scans (64 multiple)][Bpad] bf16.  Work items (site
// in batch, scan tile meeting its crop mask) x 128-row tiles of d, grouped
// so that every output element has one writer per launch (no atomics);
// channels ch0 .. ch0 + nacc - 1 per launch.
struct CubeTcArgs {
    int n_work;
    const int32_t* work;            // [n_work][2] (site in batch, scan tile)
    unsigned long long* mask;       // [n_work][tn / 64] crop masks (written by the launch)
    int n_sites, n_tiles;           // sites in the batch, scan tiles of B
    int mt_per, kb_ch, ch0, nacc;   // d tiles, K blocks per channel, channel range
    int64_t a_site_rows, a_plane_rows, b_plane_rows;
    int n_det, P;
    const double* scans;
    const SiteDev* sites;
    const int32_t* site_ids;
    int ny, nx, fy, fx;
    float scale;                    // the detector-side factor (1 for the exact cube)
    float* cube;                    // cube mode: [P][cube_ld], rows d added to; or
    float* mpart;                   // map mode: [n_work][mt_per][tn] column sums over each
                                    // unit's 128 beams (bip_cube_map_reduce adds them up)
    int64_t cube_ld;                // cube row stride (>= n_det)
    // units: cube mode, (group g of work items grp[g] .. grp[g+1]-1 -- one
    // scan tile, sites ascending -- x d tile); map mode, (work item, d tile)
    int n_groups;
    const int32_t* grp;
    // probe order: B rows per site (0: one B for every site), the channel in
    // B's columns instead of A's (A = S2 windows, B = H_n x windowed probes),
    // and operands of two BF16 planes (re, im) instead of four (split BF16)
    int64_t b_site_rows;
    int swap_ch;
    int hi_only;
    // map mode with B's rows (scan, channel) pairs, col_nch of them per scan
    // (one accumulator: the channel sum is taken over columns); 0: off
    int col_nch;
    // scans (B rows) per tile and the MMA's N: 64 (0 means 64) or 128; the
    // crop masks then take tn / 64 words per work item
    int tn;
    int* err;
    uint64_t wait_ns;               // give-up limit of each wait (0: the built-in 4 s)
};
// a_k, b_k: row lengths of A and B (bf16 elements)
cudaError_t bip_cube_tc(const CubeTcArgs& a, const void* A, int64_t a_rows, int a_k, const void* B, int64_t b_rows,
                        int b_k, cudaStream_t s);
// map mode's second stage: partial[site][rho] += scale sum over the scan's
// columns (rho ncol + n) and the d tiles of mpart, in order
struct MapReduceArgs {
    const float* mpart;             // [n_work][mt_per][tn]
    const int32_t* wmap;            // [n_sites][n_tiles]: work item of (site, tile), or -1
    int n_sites, n_tiles, tn, mt_per, ncol, P;
    const int32_t* site_ids;
    float scale;
    float* partial;                 // [n_sites_total][P]
};
cudaError_t bip_cube_map_reduce(const MapReduceArgs& a, cudaStream_t s);

// probe.cu : the probe order of the scan contraction.  Y[site][plane][rho][n K
// + r] = H_n(r) Psi(rho, r) as BF16 planes (re, im), from the windowed probes
// Psi = C^T S1 (complex64 [site][rho][K]); channels a site lacks are zero
struct ProbeYArgs {
    int n_sites, rows, K, nch;      // rows: scans per site (Psi and Y)
    const int32_t* site_ids;
    const SiteDev* sites;
    const float2* psi;              // [n_sites][psi_rows][K]
    int64_t psi_rows;
    const float2* H;                // [sum nch][K]
    uint16_t* Y;                    // [n_sites][2][y_rows][nch K]
    int64_t y_rows;
};
cudaError_t bip_probe_y(const ProbeYArgs& a, cudaStream_t s);
// qEELS: out[rho][bin_of[d]] = sum of cube[rho][d] over the beams of a bin
cudaError_t bip_qeels_bin(const float* cube, int P, int n_det, const int32_t* bin_of, int n_bins, float* out,
                          cudaStream_t s);

// adjoint_ms.cu : the reverse pass through the reconstruction and the two
// multislice sweeps, in the de-tilted frame of the forward sweep (where a
// site's stash is the column itself, so window adjoints enter unchanged).
// Adjoint row pass: [inverse row FFT] [+inj if inj_before] [gV] [x conj T]
// [+inj if after] [row FFT]; with a column pass on conjugated propagator
// tables it applies Prop^H.  gV: -2 sigma sum_p Im(conj(val) u), val the
// adjoint field at that point and u = T_j state (S1) or state (S2), summed
// over the block's parents into gv_part[group][y][x].
struct MsAdjArgs {
    float2* cols;                   // adjoint field [ncol, ny, nx]
    int zero_in;                    // 1: the incoming field is zero
    int do_ifft, do_fft;
    const float* v;                 // V_j: multiply by conj(T_j) (null: none)
    const float2* state;            // forward state [ncol, ny, nx] real space (null: no gV)
    int state_times_T;              // 1: u = T_j state (S1), 0: u = state (S2)
    int inj_before;                 // 1: inject before gV and conj(T_j) (S2)
    const int32_t* row_off;         // injection windows of this plane (as MsRowArgs)
    const int4* row_ent;
    int win;
    const float2* inj;              // [n_sites_total, ncol, win, win]
    float* gv_part;                 // [groups][ny][nx]
};
cudaError_t bip_ms_adj_row_pass(const MsPlan& plan, const MsAdjArgs& a, int* groups, cudaStream_t s);
// gV[y][x] += sum_g part[g][y][x] (groups in order)
cudaError_t bip_gv_reduce(const float* part, int groups, int G, float* gV, cudaStream_t s);
// per-target / per-parent transposed weights of one side
struct AdjWeights {
    const int32_t* t_off;           // [n_targets + 1]
    const int32_t* t_par;           // parents of each target
    const float* t_w;
    const int32_t* p_off;           // [Bp + 1]
    const int32_t* p_tgt;           // targets of each parent
    const float* p_w;
};
struct ReconAdjArgs {
    int n_sites;                    // batch
    const int32_t* site_ids;
    const SiteDev* sites;
    int K, win, ny, nx, Bp, n_targets;   // win: the batch's window, K = win^2
    int stash_win, wo;              // the stashed windows' size; offset of the batch's window
    int magnitude, tilt_sign;
    const int2* h_t;
    const float2* stash;            // [n_sites_total][Bp][stash_win^2]
    AdjWeights w;
    const float2* Sbar;             // [bs][rows][K] dL/dS*, row stride sbar_rows
    int sbar_rows;
    float2* Ubar;                   // scratch [bs][n_targets][K]
    float* dA;                      // scratch [bs][n_targets][K]
    float2* dtbar;                  // out [n_sites_total][Bp][stash_win^2]: the batch's sites' blocks
};
cudaError_t bip_recon_adjoint(const ReconAdjArgs& a, cudaStream_t s);
// S1bar[bs][b][r] = sum_n conj H_n(r) T[bs][n][b][r]
cudaError_t bip_s1bar(int nb, const int32_t* ids, const SiteDev* sites, int B, int K, const float2* H,
                      const float2* T, int64_t t_site, int64_t t_ch, float2* S1bar, int64_t s1_site, cudaStream_t s);

// grad.cu : reverse pass of a map loss through the contraction
// generic complex GEMM: C(m, n) (+)= sum_k opA(A(m, k) dk[k]) opB(B(k, n)),
// X(i, j) = X[z sXb + i sXi + j sXj] for batch z
struct CGemmGen {
    int M, N, K, batch;
    const float2* A; int64_t sam, sak, sab;
    const float2* B; int64_t sbk, sbn, sbb;
    float2* C; int64_t scm, scn, scb;
    const float* dk; int64_t sdb;   // optional real scale of each k (null: 1)
    int conjA, conjB, accumulate;
};
cudaError_t bip_cgemm_gen(const CGemmGen& a, cudaStream_t s);
struct GradArgs {
    int P, K, B;
    const double* scans;            // [P][2] pixels (device)
    const double* dL_dI;            // [P] g(rho)
    const double* occ;              // [n_sites] occupancies (null: 1)
    const SiteDev* sites;
    int ny, nx, fy, fx;
    double scale;                   // f_y f_x
};
// w[bs][rho] = f o g(rho) on the site's crop window, 0 elsewhere
cudaError_t bip_grad_crop_weights(const GradArgs& a, int nb, const int32_t* ids, float* w, cudaStream_t s);
// dH[ch_off + n][r] = 2 sum_b conj S1[bs][b][r] T[bs][n][b][r]
cudaError_t bip_grad_h(const GradArgs& a, int nb, const int32_t* ids, int nch, const float2* S1, int64_t s1_site,
                       const float2* T, int64_t t_site, int64_t t_ch, float2* dH, cudaStream_t s);
// D[bs][b] = sum_b' Q[bs][b][b'] R[bs][b'][b]; Dsum[b] += sum_bs D[bs][b]
cudaError_t bip_grad_aberr(int B, int Bpad, int nb, const float2* Q, int64_t q_site, const float2* R, int64_t r_site,
                           double2* D, double2* Dsum, cudaStream_t s);
// out[k] = sum_rho g(rho) partial[k][rho]
cudaError_t bip_grad_occ(const float* partial, int n_sites, int P, const double* g, double* out, cudaStream_t s);
// complex64 matrix -> the four split-BF16 planes (re_hi, re_lo, im_hi, im_lo)
// of a tensor-core operand: dst[z][plane][i][dcol0 + k] (row length d_cols,
// plane stride d_rows d_cols, batch stride d_batch) = split(op(src[z s_batch
// + i s_row + k s_col])), op = conj when conj; i < rows, k < cols (the rest
// of the destination is left as it is).  Tiled through shared memory, so
// either source stride may be the contiguous one.
struct SplitArgs {
    const float2* src;
    int64_t s_row, s_col, s_batch;
    int rows, cols, batch;
    uint16_t* dst;
    int64_t d_batch;
    int d_rows, d_cols, dcol0;
    int conj;
};
cudaError_t bip_split_planes(const SplitArgs& a, cudaStream_t s);

// cube_exact.cu : the cube's exit side.  stash [n_sites_total][nd][K] holds
// the windows of nd unpartitioned S2 columns (beams h[0 .. nd)) in the
// de-tilted frame; the kernel writes S2_d(r) = stash exp(-2 pi i h_d.r/N) as
// the coupling's detector operand, row d of [site in batch][rows_pad][K].
struct RetiltArgs {
    int n_sites;                    // sites of this batch
    const int32_t* site_ids;
    const SiteDev* sites;
    int win, ny, nx, K;             // win: the batch's window, K = win^2
    int stash_win, wo;              // the stashed windows' size; offset of the batch's
    int nd;                         // beams in the stash
    const float2* stash;            // [all sites][nd][stash_win^2]
    const int2* h;                  // [nd] (h_y, h_x)
    const float2* ey;               // [ny] exp(+2 pi i m / ny)
    const float2* ex;               // [nx]
    int rows_pad;                   // output rows per plane (>= nd)
    float2* out_c64;                // complex64 output, or
    uint16_t* out_bf16;             // BF16 planes (out_planes: 2 re, im; 4 split hi + lo)
    int out_planes;
    int64_t site_stride;            // output elements per site
};
cudaError_t bip_retilt(const RetiltArgs& a, cudaStream_t s);

// noalloc.cu : the static device scratch used by bip_build_s1_noalloc
constexpr size_t kNoallocScratchBytes = size_t(32) << 20;   // 32 MiB per GPU
// Device address of that array on the current device; the first call on a
// device looks it up (cudaGetSymbolAddress), later calls reuse it.
cudaError_t bip_noalloc_scratch_ptr(void** ptr);
