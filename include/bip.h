/*
 * bip.h -- C ABI of the GB300 BiP-PRISM core-loss evaluation library.
 *
 * The library evaluates the detector-integrated core-loss (EELS) elemental
 * map of the BiP-PRISM method (arxiv 2607.00756, Algorithm 5): both
 * scattering matrices are partitioned onto hex-ring parent beams, rebuilt
 * by natural-neighbour interpolation on each ionized atom's window, and
 * contracted with the transition potentials and the probe illumination.
 *
 * Conventions used by every call
 *   grid      pixel r = (r_y, r_x), corner origin, N_y x N_x pixels over
 *             L_y x L_x Angstrom; slices 0..nz-1 of thickness dz.
 *   beams     signed integer index h in [-N/2, N/2) per axis, spatial
 *             frequency q = (h_y/L_y, h_x/L_x); lists are ordered by
 *             (h_y, h_x) ascending.
 *   complex   interleaved (re, im) float32 pairs ("complex64").
 *   window    the win x win pixel block of a site at pixel position
 *             t = position / pixel size starting at floor(t + 1/2) - win/2
 *             on each axis, wrapped periodically.
 *   sites     the atoms with nch > 0, in the order they appear in the atom
 *             array passed to bip_build_s1 / bip_build_s2.
 *   memory    device pointers are owned by the caller and never freed by the
 *             library; host pointers are read (or written) only during the
 *             call.  The library's own device workspaces (window stashes,
 *             GEMM operands) belong to the context and are released by
 *             bip_destroy.
 *   streams   `stream` is a cudaStream_t (NULL: the legacy default stream).
 *             Work is enqueued on it; host-visible outputs are complete when
 *             the call returns, device outputs when the stream reaches the
 *             end of the enqueued work.
 *   errors    every call returns a bip_status and never aborts; argument
 *             checks run before any launch; bip_last_error(ctx) gives the
 *             text of the last failure on that context.  Calls on one
 *             context are not thread-safe; distinct contexts are
 *             independent.
 *   devices   one GPU per process (the current device when a context is
 *             created and used): the kernels' shared-memory launch limits
 *             are raised once per process, on the device of their first
 *             launch.  Several GPUs take one process each.
 */
#ifndef BIP_H
#define BIP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bip_ctx bip_ctx;

typedef enum {
    BIP_OK = 0,
    BIP_ERR_INVALID_ARG = 1,   /* null pointer, bad value, wrong call order   */
    BIP_ERR_SHAPE = 2,         /* sizes inconsistent with the configuration   */
    BIP_ERR_OOM = 3,           /* a device or host allocation failed          */
    BIP_ERR_CUDA = 4,          /* a CUDA call failed (text in bip_last_error) */
    BIP_ERR_TIMEOUT = 5,       /* a device-side wait gave up                  */
    BIP_ERR_UNSUPPORTED = 6,   /* valid request the library does not implement */
    BIP_ERR_NUMERIC = 7        /* an output holds NaN or Inf (only with
                                  bip_set_check_finite on)                    */
} bip_status;

typedef enum {
    BIP_PREC_FP32 = 0,         /* FP32 SIMT complex GEMMs                     */
    BIP_PREC_SPLIT_BF16 = 1,   /* tcgen05, every contraction in BF16 hi+lo
                                  (3 products per real product), FP32 acc.    */
    BIP_PREC_MIXED = 2,        /* tcgen05, coupling and Gram in BF16 (one
                                  product); the window reconstruction's sums
                                  on tcgen05 in FP16 (weights hi+lo, parent
                                  values rounded once) when both parent sets
                                  are <= 64, else the FP32 SIMT gather; the
                                  scan polynomial in FP32; FP32 accumulation
                                  throughout                                 */
    BIP_PREC_FP8_TILE = 3      /* as MIXED, but the coupling's operands in
                                  FP8 E4M3 with one scale per 64x64 window
                                  (operand row): the scale is an a-priori
                                  bound of the row, kappa sum_p w_tp
                                  max_r |dt_p(r)| (times max_r |H_n| on the
                                  S1 side; kappa = 1 + 2^-6), applied to the
                                  FP32 products in the epilogue.  Needs both
                                  parent sets <= 64 (else UNSUPPORTED).    */
} bip_precision;

typedef enum {
    BIP_RECON_COMPLEX = 0,     /* plain convex average (Eq. window-recon)     */
    BIP_RECON_MAGNITUDE = 1    /* magnitude-preserving (Eq. magpreserve)      */
} bip_recon;

/* An atom site: position in Angstrom, slice index, number of transition
 * channels (0: not ionized). */
typedef struct {
    double y, x;
    int32_t slice;
    int32_t nch;
} bip_atom;

/* Simulation parameters (lengths in Angstrom, angles in rad, energy in eV).
 * Constraints checked by bip_create: ny, nx powers of two in [64, 1024] or
 * 3 times a power of two in [64, 256] (192, 384, 768 -- for f = 3);
 * fy | ny and fx | nx; dfy, dfx 0 or dividing ny, nx; win a multiple of
 * 16 with 16 <= win <=
 * min(ny/fy, nx/fx); nz >= 1;
 * e0 > 0; 0 < alpha; 0 < theta_det; nrad >= 0; nang >= 1; the aperture and
 * detector discs fit inside the grid's Nyquist band. */
typedef struct {
    int32_t ny, nx;
    double ly, lx;
    int32_t nz;
    double dz;
    double e0, alpha, theta_det;
    double defocus, cs;
    int32_t fy, fx;
    int32_t nrad1, nang1, nrad2, nang2;
    int32_t win;
    int32_t recon;             /* bip_recon     */
    int32_t prec;              /* bip_precision */
    /* detector-side subsampling of the beams S2 carries (h_y = 0 mod dfy,
     * h_x = 0 mod dfx); 0 takes the probe's fy, fx.  qEELS resolved along
     * q_x needs dfx = 1 (along q_y: dfy = 1); the map's detector factor is
     * dfy dfx. */
    int32_t dfy, dfx;
    /* the 4D cube's output basis: 0, 0 -- every beam with |q| lambda <=
     * theta_det; else a box of cube_ky x cube_kx k-pixels centred on the
     * zero beam, -cube_ky/2 <= h_y < cube_ky/2 (and likewise for x), at most
     * ny x nx. */
    int32_t cube_ky, cube_kx;
} bip_config;

/* Host geometry (Algorithm 5 build steps; Sec. 2.2.2-2.2.3, Eq. nnw):
 * aperture beams |q| lambda <= alpha with h = 0 mod f, detector beams
 * |q| lambda <= theta_det with h = 0 mod (dfy, dfx), hex-ring parents for
 * both and FP64 Sibson natural-neighbour weights, computed once and cached
 * in the context; and the 4D cube's complete output basis, every beam with
 * |q| lambda <= theta_det (no subsampling), or the box of k-pixels the
 * configuration names.  Host only: touches no GPU.
 * *out receives the new context. */
bip_status bip_create(const bip_config* cfg, bip_ctx** out);

/* Releases the context and every device workspace it holds.  The caller
 * must make sure no work enqueued with this context is still running. */
bip_status bip_destroy(bip_ctx* ctx);

/* Sizes of the cached geometry: B aperture beams, n_det detector beams,
 * Bp1 probe parents, Bp2 detector parents; n_sites after a build (else 0).
 * Any pointer may be NULL. */
bip_status bip_query(const bip_ctx* ctx, int32_t* B, int32_t* n_det,
                     int32_t* Bp1, int32_t* Bp2, int32_t* n_sites);

/* Copies the cached geometry to host buffers (any may be NULL):
 * h_beam [B,2], h_det [n_det,2] beam indices; p1 [Bp1], p2 [Bp2] parent
 * positions within those lists; w1 [B,Bp1], w2 [n_det,Bp2] dense FP64
 * weights (row = target beam). */
bip_status bip_get_geometry(const bip_ctx* ctx, int32_t* h_beam, int32_t* h_det,
                            int32_t* p1, int32_t* p2, double* w1, double* w2);

/* Copies the configuration the context was created with to *out. */
bip_status bip_get_config(const bip_ctx* ctx, bip_config* out);

/* On-disk cache of the host geometry (the natural-neighbour weights depend
 * only on the aperture, the detector and the rings, so, as in the paper's
 * Sec. 2.2.3, they are computed once per such geometry): with a directory
 * set, bip_create looks there for its geometry's file -- named by a 64-bit
 * hash of the configuration fields the geometry reads (grid, cell, energy,
 * angles, defocus, Cs, f, rings, detector subsampling, cube box) -- and
 * reads it instead of recomputing, after checking its format version, the
 * configuration fields stored in it and its checksum.  A missing file, or
 * one that fails a check, is recomputed and written again (under a
 * temporary name, then renamed into place).  A directory that cannot be
 * written only costs the recomputation; bip_create's result is the same
 * either way.
 * bip_set_geometry_cache(dir): process-wide; NULL or "" turns the cache
 *   off.  Until it is first called, the environment variable
 *   BIP_GEOMETRY_CACHE (read once) names the directory.
 * bip_geometry_cache_stats: since the process started, geometries read from
 *   the cache (hits), computed and written with the cache on (misses), and
 *   files that failed a check (rejected); any pointer may be NULL. */
bip_status bip_set_geometry_cache(const char* dir);
bip_status bip_geometry_cache_stats(int64_t* hits, int64_t* misses, int64_t* rejected);

/* Chooses the contraction arithmetic for later bip_coreloss_* calls. */
bip_status bip_set_precision(bip_ctx* ctx, int32_t prec);

/* Probe-forming matrix S1 (Eq. smatrix-advance; Algorithm 5 first and
 * fourth steps): the Bp1 parent plane waves are advanced through
 * T_j = exp(i sigma V_j) and the Fresnel propagator to every plane that
 * holds a site, and each site's window of every parent, de-tilted by
 * exp(-2 pi i h_p.r/N) (Eq. part-basis), is kept in the context.
 *   V      [nz, ny, nx] float32 device: projected potential in V*Angstrom.
 *   atoms  [n_atoms] host; sites are the entries with nch > 0, their slice
 *          must lie in [0, nz); n_atoms >= 1.
 * Errors: BIP_ERR_INVALID_ARG (null, bad slice/nch), BIP_ERR_OOM,
 * BIP_ERR_CUDA. */
bip_status bip_build_s1(bip_ctx* ctx, const float* V, const bip_atom* atoms,
                        int32_t n_atoms, void* stream);

/* Detector matrix S2 (Eq. s2, Algorithm 4 second step): the conjugate
 * detector plane waves G^{-1/2} exp(-2 pi i h_d.r/N) of the Bp2 detector
 * parents are back-propagated from the exit surface by the transposed
 * multislice (P, then T_j, for j = nz-1 down to 0), and each site's
 * window at its plane, de-tilted by exp(+2 pi i h_p.r/N), is kept.  Same
 * arguments and errors as bip_build_s1; the atom array must describe the
 * same sites as the S1 build when both are used by one map. */
bip_status bip_build_s2(bip_ctx* ctx, const float* V, const bip_atom* atoms,
                        int32_t n_atoms, void* stream);

/* Both builds at once: the S1 and S2 sweeps of bip_build_s1 and
 * bip_build_s2 with the same arguments, S1 on `stream` and S2 on a stream
 * the context creates at its first use (non-blocking, on the current
 * device), forked from and joined back into `stream` by events, so that the
 * two sweeps' kernels share the GPU.  The stashes are bit-identical to
 * those of the two separate calls, and the context is afterwards as after
 * them.  S2's sweep gets its own column workspace (Bp2 x ny x nx complex64
 * more device memory than the separate calls).  On an error the side
 * stream's work is still joined into `stream`.  Not capturable into a CUDA
 * graph (BIP_ERR_INVALID_ARG on a capturing stream; the builds upload host
 * tables).  Errors as bip_build_s1. */
bip_status bip_build(bip_ctx* ctx, const float* V, const bip_atom* atoms, int32_t n_atoms,
                     void* stream);

/* Elemental map (Algorithm 5; Eq. window-recon, magpreserve, coupling,
 * map-sum): for every site the windows of S1 and S2 are rebuilt from the
 * parents, M^{(n)} = S2^T diag(H_n) S1 is formed, and
 *   I(rho) = f_y f_x sum_sites sum_n sum_d |sum_b M^{(n)}_{d,b} c_b(rho)|^2,
 *   c_b(rho) = f_y f_x Psi(h_b) / sqrt(G sum_aperture |Psi|^2)
 *              exp(-2 pi i h_b.rho/N),
 * each site contributing only at scans whose minimum-image offset from it
 * lies in [-N/(2f), N/(2f)) on both axes (crop mask).  Sites are summed in
 * a fixed order in FP64 with Neumaier compensation.
 *   H        complex64 device: transition potentials of each site's
 *            channels sampled on its window, sites in order, each channel
 *            [w, w] (w = win, or the site's own window after
 *            bip_set_site_windows: [sum_sites nch w^2] in all); 16-byte
 *            aligned (else BIP_ERR_INVALID_ARG).
 *   scan_px  [P, 2] float64 host: scan positions in pixels (y, x).
 *   map_out  [P] float64 device.
 * Requires both builds on this context (else BIP_ERR_INVALID_ARG). */
bip_status bip_coreloss_map(bip_ctx* ctx, const void* H, const double* scan_px,
                            int32_t P, double* map_out, void* stream);

/* Per-site contributions I_tau(rho) of the map above, [n_sites, P] float32
 * device; entries outside a site's crop mask are written as 0.  The map is
 * their FP64 sum over sites. */
bip_status bip_coreloss_sites(bip_ctx* ctx, const void* H, const double* scan_px,
                              int32_t P, float* partial_out, void* stream);

/* Energy-filtered 4D cube I(q, rho) (Sec. 2.2.6; Algorithm 3): the cube
 * keeps every output beam, so S2 is not reduced.  S1 stays partitioned (the
 * context's bip_build_s1 windows, rebuilt per site as for the map); the exit
 * side is exact on the complete basis -- every beam with |q| lambda <=
 * theta_det, unsubsampled, or the configuration's box of k-pixels
 * (bip_cube_beams) -- through unpartitioned S2
 * columns (Eq. s2, the reciprocity form of Algorithm 3's exit multislice):
 *   cube[rho][q] = sum_sites sum_n |sum_b M^(n)_{q,b} c_b(rho)|^2,
 *   M^(n)_{q,b} = sum_{r in window} S2^q(r) H_n(r) S~1^b(r),
 * over the sites whose crop mask holds rho; no detector-side factor.  The
 * call builds the S2 columns itself, in batches of beams (one backward
 * sweep each, every site's window kept for the batch), sized to half the
 * free device memory (at most 96 GB; bip_set_cube_memory sets the bytes);
 * it needs bip_build_s1 on this context (bip_build_s2 is not used).  Sites
 * are added in a fixed order and every element has one writer per launch:
 * the result does not depend on scheduling.
 *   V        [nz, ny, nx] float32 device, the potential S1 was built from.
 *   H, scan_px as bip_coreloss_map.
 *   cube_out [P, n_cube] float32 device, overwritten; beams in the order of
 *            bip_cube_beams.
 * Precisions: the coupling M in the context's precision -- FP32 (SIMT),
 * SPLIT_BF16 and MIXED (tcgen05); FP8 contexts return BIP_ERR_UNSUPPORTED.
 * The per-beam sum over b: on a raster scan list (scan p = my Mx + mx at
 * (ry[my], rx[mx])) separated over the aperture beams' lattice, two short
 * FP32 sums (c_b(rho) factorises over the axes); on any other list in the
 * context's precision (tcgen05, or FP32 SIMT).  The same holds for qEELS.
 * BIP_ERR_OOM when not even 32 beams fit.
 * bip_cube_beams: n_cube and (h, nullable host int32 [n_cube, 2]) the
 *   basis's beams (h_y, h_x), ordered by (h_y, h_x).  Host only. */
bip_status bip_coreloss_cube(bip_ctx* ctx, const float* V, const void* H, const double* scan_px,
                             int32_t P, float* cube_out, void* stream);
bip_status bip_cube_beams(const bip_ctx* ctx, int32_t* n_cube, int32_t* h);
bip_status bip_set_cube_memory(bip_ctx* ctx, int64_t bytes);

/* Momentum-resolved output (qEELS, Sec. 2.2.6): one diffraction axis
 * resolved, the perpendicular one summed,
 *   qeels[rho][i] = dfy dfx sum_sites sum_n sum_{d : h_d[axis] = bins[i]}
 *                   |sum_b M^(n)_{d,b} c_b(rho)|^2,
 * with S2 partitioned as for the map -- which the paper allows only with
 * the resolved axis sampled at f = 1: axis 0 (q_y resolved) needs a context
 * created with dfy = 1, axis 1 (q_x) with dfx = 1 (else
 * BIP_ERR_INVALID_ARG).  The bins partition the detector beams, so their
 * sum is the map of the same context.  Sites are added in a fixed order.
 *   bip_qeels_bins: the number of bins and (h_values, nullable host int32
 *   [n_bins]) their h components, ascending.  Host only.
 *   qeels_out [P, n_bins] float32 device, overwritten.
 * Other requirements as bip_coreloss_map. */
bip_status bip_qeels_bins(const bip_ctx* ctx, int32_t axis, int32_t* n_bins, int32_t* h_values);
bip_status bip_coreloss_qeels(bip_ctx* ctx, const void* H, const double* scan_px, int32_t P,
                              int32_t axis, float* qeels_out, void* stream);

/* Launch control.
 * bip_set_capture_safe(ctx, on): the map calls issue no host
 *   synchronisation and upload the scan list and work lists only when they
 *   change, so that after one warm-up call with the same arguments a CUDA
 *   graph can capture them (several contexts -- specimens of uneven size --
 *   into one graph).  Device timeouts are then reported by
 *   bip_check_errors (which synchronises the stream) instead of by the map.
 * bip_set_launch: sites per batch and coupling tile width (multiple of 16,
 *   <= 256) of the tensor-core path; 0 restores the built-in choice (tile
 *   counts against the SM count and the L2 size).
 * bip_autotune: times maps (two after a warm-up, CUDA events) over sites per
 *   batch, then coupling tile widths, then the contraction order (see
 *   bip_set_order) -- and, when another order wins, the sites per batch
 *   again under it -- keeps the fastest in the context and returns it;
 *   map_out holds the last map.  Results do not depend on
 *   these choices (each site's arithmetic and the site-sum order are fixed). */
bip_status bip_set_capture_safe(bip_ctx* ctx, int32_t on);
/* bip_set_raster_eval(ctx, on): with on (the default) a scan list that is a
 * raster (rows of equal y, every row the same x sequence) takes the
 * separable evaluation of the scan polynomial (two small dense stages per
 * site); off, or for any other list, Horner's rule per scan. */
bip_status bip_set_raster_eval(bip_ctx* ctx, int32_t on);
bip_status bip_check_errors(bip_ctx* ctx, void* stream);
bip_status bip_set_launch(bip_ctx* ctx, int32_t sites_per_batch, int32_t coupling_tile);
bip_status bip_autotune(bip_ctx* ctx, const void* H, const double* scan_px, int32_t P, double* map_out,
                        void* stream, int32_t* sites_per_batch, int32_t* coupling_tile, int32_t* order,
                        double* best_ms);
/* bip_set_order: the scan contraction of the map, 0 (default) through the
 * Gram matrix Q = sum_n M^H M and the lattice-difference polynomial
 * (Algorithm 4's c^H Q c), 1 "beam order": |sum_b M_{d,b} c_b(rho)|^2 for
 * every detector beam on tcgen05 (split BF16) with the detector sum taken in
 * the epilogue -- cheaper when few scans meet each site; tensor-core
 * precisions only (FP32 contexts keep the Gram route); 2 "probe order":
 * the windowed probes Psi(rho, r) = sum_b c_b(rho) S1_b(r) of every scan
 * (one tcgen05 GEMM per site), then a^(n)_d(rho) = sum_r S2_d(r) H_n(r)
 * Psi(rho, r) and |a|^2 summed over d and n as in beam order -- the cheapest
 * order when few scans meet each site (work ~ P instead of the coupling's
 * n_det nch B); mixed precision only (else BIP_ERR_UNSUPPORTED), at most
 * 2048 scans per map (BIP_ERR_UNSUPPORTED from the map).  Every order
 * sums in a fixed order (no floating-point atomics), so a map does not
 * depend on scheduling.  bip_autotune also times the other orders. */
bip_status bip_set_order(bip_ctx* ctx, int32_t order);

/* Model parameters of the map beyond the specimen (for fitting; Sec. 5
 * names the matrices as a forward model for simulation-constrained
 * reconstruction).
 * bip_set_occupancy: per-site occupancies o_tau weighting the site sum,
 *   I = sum_tau o_tau I_tau (Eq. map-sum); occ: host float64 [n_sites] in the
 *   order of the built sites, or NULL for all 1.  Kept until the next build
 *   with another site list.  BIP_ERR_INVALID_ARG before a build or for a
 *   non-finite value.
 * bip_set_aberrations: probe defocus and Cs (Angstrom) of Psi(h) =
 *   exp(-i chi), chi = pi lambda df |q|^2 + (pi/2) Cs lambda^3 |q|^4, for
 *   the following maps (the matrices do not depend on them). */
bip_status bip_set_occupancy(bip_ctx* ctx, const double* occ);
bip_status bip_set_aberrations(bip_ctx* ctx, double defocus, double cs, void* stream);

/* Windows of their own for the sites (Eq. coupling: the sum over the crop
 * window Omega_tau of each site, whose size follows the support of its
 * H_n; sites of several edges batched in one map).  win: host int32
 * [n_sites] in the order of the built sites, each a multiple of 16 in
 * [16, the context's win] or 0 (the context's win); NULL: every site at the
 * context's win again.  Site k's window is the w_k x w_k block starting at
 * floor(t + 1/2) - w_k/2 on each axis -- the central block of the window
 * the builds stash, so the builds need not be repeated.  The map then takes
 * its sites in batches of one window size each, every contraction of a
 * batch over its w_k^2 pixels, and H holds each site's channels on its own
 * window (see bip_coreloss_map).  Kept until the next build with another
 * site list.  The maps (every contraction order, bip_coreloss_sites,
 * bip_autotune), qEELS, the cube and the reverse pass take such sites
 * (d_H then has H's layout); bip_site_windows and bip_site_coupling return
 * BIP_ERR_UNSUPPORTED while a site's window is below win.  BIP_ERR_INVALID_ARG before a build, for a
 * bad size, or when H would exceed 2^31 complex elements. */
bip_status bip_set_site_windows(bip_ctx* ctx, const int32_t* win, void* stream);

/* Reverse pass of a scalar loss L of the map: given g = dL/dI(rho) on the
 * scans, the derivatives at the context's current state (occupancies,
 * aberrations, built matrices):
 *   d_occ [n_sites] float64 device: dL/do_tau = sum_rho g I_tau;
 *   d_H   H's layout, complex64 device: dL/dRe H + i dL/dIm H of every
 *         channel sample (for transition amplitudes a with H = a H0:
 *         dL/dRe a + i dL/dIm a = sum_r d_H(r) conj(H0(r)));
 *   d_aberr [2] float64 host: dL/d defocus, dL/d Cs;
 *   d_V [nz, ny, nx] float32 device: dL/dV_j of every slice potential,
 *         through the reconstruction (Eq. magpreserve) and both sweeps
 *         (Eq. smatrix-advance, Eq. s2); V (device, the potential the
 *         matrices were built from) is then required (every grid length
 *         bip_create takes).  The sweeps' forward states are recomputed
 *         from checkpoints every ceil(sqrt(n)) slices.
 * Any output may be NULL (not computed).  Steps: R_tau = f_y f_x o_tau
 * sum_{rho in crop} g c c^H; Mbar = M R; dL/dH_n(r) = 2 sum_{d,b}
 * Mbar_n(d,b) conj(S2_d(r) S1_b(r)); dL/dtheta = -2 sum_b chi'_b Im
 * sum_tau (Q_tau R_tau)_bb -- the contractions in FP32 on every precision;
 * d_occ uses the context's precision for I_tau.
 *   dL_dI [P] float64 device; other requirements as bip_coreloss_map;
 *   d_H 8-byte aligned.  Synchronises the stream when d_aberr is given. */
bip_status bip_coreloss_grad(bip_ctx* ctx, const float* V, const void* H, const double* scan_px,
                             int32_t P, const double* dL_dI, double* d_occ, void* d_H,
                             double* d_aberr, float* d_V, void* stream);

/* Stage access for validation.
 * bip_copy_stash: the de-tilted parent windows of one site, which = 1 (S1,
 *   [Bp1, win, win]) or 2 (S2, [Bp2, win, win]) complex64, to device `out`.
 * bip_site_windows: the reconstructed windows of one site, S1 [B, win, win]
 *   and S2 [n_det, win, win] complex64 device (Eq. window-recon).
 * bip_site_coupling: the coupling matrices of one site, [nch_max, n_det, B]
 *   complex64 device (Eq. coupling), nch_max the largest channel count of
 *   the built sites (missing channels of a site come out zero), computed in
 *   the context's precision.
 * H, s1_out and s2_out must be 16-byte aligned (else BIP_ERR_INVALID_ARG). */
bip_status bip_copy_stash(bip_ctx* ctx, int32_t which, int32_t site, void* out,
                          void* stream);
bip_status bip_site_windows(bip_ctx* ctx, int32_t site, void* s1_out, void* s2_out,
                            void* stream);
bip_status bip_site_coupling(bip_ctx* ctx, const void* H, int32_t site, void* m_out,
                             void* stream);

/* Saving and restoring the builds, so that maps can be rerun without the
 * multislice: the map, the per-site and qEELS calls and the autotuner read
 * only the window stashes, the site list, the geometry and H.
 * bip_export_stash(ctx, which, dst, bytes): the whole stash of S1
 *   (which = 1) or S2 (2), [n_sites, Bp, win, win] complex64 in site order
 *   (per site the layout of bip_copy_stash), to dst -- device, pinned or
 *   pageable host memory (the copy direction follows the pointers).  bytes
 *   must equal the stash's size, n_sites * Bp * win * win * 8 (else
 *   BIP_ERR_SHAPE, nothing copied).  A pageable dst is complete when the
 *   call returns, others when the stream reaches the copy.
 * bip_import_stash(ctx, which, atoms, n_atoms, src, bytes): the reverse.
 *   It takes the site list from the atoms as bip_build_s<which> would,
 *   checks bytes against that list (else BIP_ERR_SHAPE before any other
 *   effect) and copies the stash in; afterwards the context is as after
 *   bip_build_s<which> with those atoms.  The stash must come from a
 *   context with the same configuration (geometry, window, grid), which the
 *   library cannot check from the bytes: the caller keeps them together
 *   (the Python binding stores the configuration with the stash and
 *   compares it).  The source may be reused when the stream reaches the
 *   copy (pageable host memory: when the call returns).
 * Neither call may be captured into a CUDA graph (BIP_ERR_INVALID_ARG on a
 * capturing stream). */
bip_status bip_export_stash(bip_ctx* ctx, int32_t which, void* dst, int64_t bytes, void* stream);
bip_status bip_import_stash(bip_ctx* ctx, int32_t which, const bip_atom* atoms, int32_t n_atoms,
                            const void* src, int64_t bytes, void* stream);

/* bip_set_check_finite(ctx, on): with on, bip_coreloss_map, _sites, _cube,
 *   _qeels and _grad scan their outputs for NaN or infinite values once
 *   they are computed and return BIP_ERR_NUMERIC (with the count in
 *   bip_last_error) if any is found; the outputs are written either way.
 *   The scan synchronises the stream, so with the check on these calls
 *   refuse a capturing stream (BIP_ERR_INVALID_ARG).  Off by default.
 * bip_mem_stats: bytes of device memory the library's contexts hold now
 *   (every context's workspaces; bip_build_s1_noalloc's static array and
 *   caller-owned buffers excluded) and the high-water mark since the
 *   process started or the last reset (reset_peak != 0 sets it to the live
 *   bytes after reading).  Either pointer may be NULL. */
bip_status bip_set_check_finite(bip_ctx* ctx, int32_t on);
bip_status bip_mem_stats(int64_t* live_bytes, int64_t* peak_bytes, int32_t reset_peak);

/* Per-stage timing of the library's own kernels.  With profiling on, every
 * launch is bracketed by CUDA events recorded on the stream it runs on;
 * bip_get_profile waits for them and returns, per stage, the summed device
 * time in ms and the number of launches since profiling was (re)enabled.
 * Stages: multislice row pass, multislice column pass, window
 * reconstruction, coupling GEMM, Gram GEMM, quadratic form, illumination +
 * site sum, the slices' transmissions exp(i sigma V) (once per build).  ms / launches: [BIP_N_STAGES] host arrays (either may be
 * NULL).  bip_set_profiling(ctx, on): on = 0 stops timing, on < 0 times
 * every stage, on > 0 times the stages whose bit (1 << stage) is set; the
 * launch counts cover every stage.  Each call clears earlier records. */
enum {
    BIP_STAGE_MS_ROW = 0, BIP_STAGE_MS_COL = 1, BIP_STAGE_GATHER = 2, BIP_STAGE_COUPLING = 3,
    BIP_STAGE_GRAM = 4, BIP_STAGE_QUADFORM = 5, BIP_STAGE_REDUCE = 6, BIP_STAGE_TRANSMISSION = 7,
    BIP_N_STAGES = 8
};
bip_status bip_set_profiling(bip_ctx* ctx, int32_t on);
bip_status bip_get_profile(bip_ctx* ctx, double* ms, int64_t* launches);

/* bip_build_s1 for callers that cannot allocate device memory: a host
 * framework that owns every device allocation through its own pool, a
 * process whose device-memory budget is fixed up front, or a pipeline that
 * cannot afford cudaMalloc/cudaFree because they synchronize the device and
 * would stall its other streams.  (This entry point has no counterpart in
 * the paper; it is the same S1 build as bip_build_s1.)
 *
 * It allocates nothing.  The caller passes the inputs of bip_build_s1 and
 * the output `stash` [n_sites, Bp1, win, win] complex64 (device): the
 * de-tilted S1 parent windows of every site, the layout bip_copy_stash
 * returns per site.  The parent columns and the device tables live in a
 * static array of 32 MiB inside the library, which every GPU that loads
 * the library holds until the process exits.  The context only supplies
 * its host geometry (bip_create allocates no device memory); this call does
 * not touch the context's own device buffers or mark S1 as built.
 *
 * Each call looks up the array's address in the current device context and
 * copies its tables and site lists from host memory that lives only during
 * the call, so the call must not be captured into a CUDA graph: on a stream
 * that is being captured it returns BIP_ERR_INVALID_ARG.  Requests that
 * need more than 32 MiB -- Bp1 * ny * nx * 8 bytes of parent columns plus a
 * few KB of tables and site lists -- return BIP_ERR_SHAPE with the sizes in
 * bip_last_error.  All calls share the one array and keep the last call's
 * contents; calls that overlap on the GPU (on different streams, or from
 * different threads) race and corrupt each other's results. */
bip_status bip_build_s1_noalloc(bip_ctx* ctx, const float* V, const bip_atom* atoms,
                                int32_t n_atoms, void* stash, void* stream);

/* Failure handling, for tests and for callers that want short limits.
 * bip_set_wait_limit: the give-up limit (ns) of every wait inside the
 *   tensor-core kernels of this context (0: the built-in 4 s).  A wait that
 *   gives up makes the kernel stop issuing work, let its copies and MMAs in
 *   flight finish (bounded by the built-in limit), free its tensor memory
 *   and set a flag, which the call returns as BIP_ERR_TIMEOUT (capture-safe
 *   contexts: bip_check_errors).  The context stays usable.
 * bip_debug_fail_alloc(k): the k-th device allocation the library makes
 *   from now on (in any context) fails as if the device were out of memory,
 *   so that the call returns BIP_ERR_OOM; 0 turns it off.  Resets the count
 *   bip_debug_allocs reports as made.
 * bip_debug_allocs: the device allocations of the library alive now (every
 *   context's workspaces) and made since the last bip_debug_fail_alloc
 *   (either pointer may be NULL). */
bip_status bip_set_wait_limit(bip_ctx* ctx, int64_t ns);
bip_status bip_debug_fail_alloc(int64_t k);
bip_status bip_debug_allocs(int64_t* live, int64_t* made);

/* Text of the last error on this context ("" if none; static text if ctx
 * is NULL). */
const char* bip_last_error(const bip_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BIP_H */
