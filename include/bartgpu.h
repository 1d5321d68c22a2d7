/*
 * bartgpu.h -- C ABI of the GB300 (sm_103a) forward-model library for the
 * BART retrieval method (Harrington et al. 2022, "An Open-Source Bayesian
 * Atmospheric Radiative Transfer (BART) Code: I", arXiv:2104.12522).
 *
 * The library computes the data-parallel hot path that the paper's sampler
 * calls for every proposal (Sec. 3, Fig. 1 "BART chart"; Sec. 4, the list of
 * optimisations):
 *   1. the line-by-line opacity grid (Sec. 3 "computes the opacities on the
 *      spot ... or interpolates from a pre-calculated table"; Sec. 4 items 3-4),
 *   2. the per-proposal spectrum: temperature interpolation of the grid,
 *      abundance scaling, optical depth, emission at Gauss-Legendre angles or
 *      the transit ray geometry (Sec. 3, Sec. 6.1),
 *   3. integration over filter bandpasses (the spectrum integrator, Sec. 3).
 *
 * Conventions shared by every entry point:
 *   - Every array argument named "device" is a pointer into the memory of the
 *     context's GPU and is owned by the caller.  Arrays named "host" are read
 *     during the call only.  The context owns scratch space only.
 *   - Calls are asynchronous on the context's stream: results are ready after
 *     bart_sync() or any later stream-ordered operation.
 *   - Errors that can be detected on the host (NULL pointers, sizes out of
 *     range, non-monotonic axes) return before any launch, and
 *     bart_last_error() describes them.  Errors found on the device (a
 *     watchdog that expired, a device-side range check) set a status word that
 *     bart_sync() returns.  Nothing throws across the ABI.
 *   - Floating-point arithmetic is FP32 unless stated; no sum uses atomics
 *     except where an entry point says so.
 */
#ifndef BARTGPU_H
#define BARTGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BART_ABI_VERSION 4

typedef enum {
  BART_OK = 0,
  BART_EINVAL = 1,       /* invalid argument (NULL, size, ordering) */
  BART_ENOMEM = 2,       /* scratch allocation failed */
  BART_ECUDA = 3,        /* CUDA runtime error; see bart_last_error */
  BART_ETIMEOUT = 4,     /* a device watchdog expired */
  BART_ERANGE = 5,       /* a device-side range check failed */
  BART_EUNSUPPORTED = 6  /* valid request this build does not support */
} bart_status;

typedef struct bart_ctx bart_ctx;

/* Library ABI version (BART_ABI_VERSION of the build). */
int bart_abi_version(void);

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context, or NULL on failure.  No kernel is launched. */
bart_status bart_create(bart_ctx** out, int device, void* cuda_stream);

/* Release the context's scratch memory and CUDA graphs.  NULL is ignored. */
void bart_destroy(bart_ctx* ctx);

/* Change the stream later calls are issued on. */
bart_status bart_set_stream(bart_ctx* ctx, void* cuda_stream);

/* Message describing the last error returned on this context ("" if none).
 * The string is owned by the context and valid until its next call. */
const char* bart_last_error(const bart_ctx* ctx);

/* Wait for the context's stream, then read and clear the device status word.
 * Returns BART_OK, BART_ETIMEOUT, BART_ERANGE or BART_ECUDA. */
bart_status bart_sync(bart_ctx* ctx);

/* Tile autotuning of the batched forward model (on by default): the first
 * eager call of each launch shape times every candidate wavenumber-tile width
 * with CUDA events on the context's stream and keeps the fastest for later
 * calls; during a stream capture only a cached or the default width is used.
 * enable = 0 turns it off and forgets the choices. */
bart_status bart_set_autotune(bart_ctx* ctx, int enable);

/* Wavenumber-tile width (threads per CTA) of the emission forward model:
 * 64, 128 or 256 fixes it for later calls of this context; 0 (the default)
 * leaves the choice to the autotuner (or the default width when autotuning is
 * off).  Spectra do not depend on the width, band values only through the
 * order of their partial sums.  Other values return BART_EINVAL. */
bart_status bart_set_emission_tile(bart_ctx* ctx, int tile);

/* Launch structure of an emission batch in bart_forward_spectra_batch.
 *   BART_LAUNCH_FUSED (default): one persistent kernel per batch.  CTAs (as
 *     many as fit on the SMs) take (wavenumber tile, proposal) units from a
 *     device counter in tile-major order, so the CTAs in flight read the same
 *     grid rows and share them through L2; each unit evaluates its proposal's
 *     T(P) profile and abundances, the column and the band partial sums, and
 *     the CTA finishing a proposal's last tile reduces its band values.  The
 *     counters reset themselves at the end of the launch, so a captured graph
 *     replays it unchanged.
 *     A CTA thread takes two wavenumbers and their arithmetic runs on packed
 *     FP32 pairs.  It addresses grid rows by 32-bit element offsets: grids
 *     with n_species * n_layers * n_temps * n_nu + n_nu >= 2^32 (16 GiB and
 *     more) take the BART_LAUNCH_SPLIT path instead.
 *   BART_LAUNCH_SPLIT: three launches (per-proposal profile kernel, one CTA
 *     per (proposal, tile) column kernel, band reduction), kept for
 *     comparison.
 *   BART_LAUNCH_FUSED_TMA: the fused kernel with the grid rows of each layer
 *     staged in shared memory by bulk copies (a producer warp, a ring of
 *     mbarrier-tracked buffers) instead of per-thread loads; used where
 *     nu.n_nu is a multiple of 4 and the grid is 16-byte aligned (else the
 *     fused kernel runs; the same grid-size limit).  Kept for comparison: it
 *     measures slower on GB300.
 * Results agree to FP32 rounding (band values through the order of partial
 * sums).  Other values return BART_EINVAL. */
#define BART_LAUNCH_FUSED 0
#define BART_LAUNCH_SPLIT 1
#define BART_LAUNCH_FUSED_TMA 2
bart_status bart_set_emission_launch(bart_ctx* ctx, int mode);

/* Graph capture of library calls.  bart_capture_begin starts capturing the
 * work of later calls on this context (they run nothing until the graph is
 * launched; the capture goes to a private stream ordered after the context's
 * stream); bart_capture_end stops it and instantiates the graph into *out.
 * bart_graph_launch replays it on the context's stream; bart_graph_destroy
 * frees it.  Calls inside a capture must not need new scratch or changed
 * constant tables: make one eager call of the same shape and arguments first
 * (otherwise they return BART_EINVAL and bart_capture_end fails).  A graph
 * keeps the device pointers it was captured with: replaying it recomputes
 * from whatever those buffers hold then (CUDA Graphs; the paper's sampler
 * calls the same forward model once per generation, Sec. 3). */
typedef struct bart_graph bart_graph;
bart_status bart_capture_begin(bart_ctx* ctx);
bart_status bart_capture_end(bart_ctx* ctx, bart_graph** out);
bart_status bart_graph_launch(bart_ctx* ctx, const bart_graph* graph);
void bart_graph_destroy(bart_graph* graph);

/* Writes "shape -> tile" lines of the autotuner's choices into buf (len bytes,
 * NUL-terminated, truncated if short); returns the full length, -1 for NULL. */
int bart_autotune_report(const bart_ctx* ctx, char* buf, int len);

/* ------------------------------------------------------------ line lists */

/* One species' line list, structure of arrays, all DEVICE pointers, sorted by
 * line centre ascending (the order the opacity kernels rely on).
 *   nu0_cm       line centre, cm^-1 (FP64)
 *   log10_s296   log10 line strength at 296 K, cm molecule^-1 (HITRAN units)
 *   elow_cm      lower-state energy E'', cm^-1
 *   gamma_ref_cm Lorentz half width at 1 bar and 296 K, cm^-1
 *   mass_amu     molecular mass (host value), amu
 */
typedef struct {
  int64_t n_lines;
  const double* nu0_cm;
  const float* log10_s296;
  const float* elow_cm;
  const float* gamma_ref_cm;
  double mass_amu;
} bart_linelist;

/* Uniform wavenumber grid nu_j = nu_start_cm + j * dnu_cm, j = 0 .. n_nu-1.
 * The opacity is sampled at these points (Sec. 4: profiles are sampled at the
 * output-grid wavenumbers, not averaged over bins).  1 <= n_nu < 2^31. */
typedef struct {
  double nu_start_cm;
  double dnu_cm;
  int64_t n_nu;
} bart_nugrid;

/* ---------------------------------------------------------- opacity build */

/* Line-by-line opacity computed directly at explicit (P, T) cells (Sec. 3):
 *   out[s][c][j] = sum_i S_i(T_c) V(nu_j - nu0_i; sigma_i(T_c), gamma_i(P_c, T_c))
 * in cm^2 molecule^-1, for species s < n_species, cell c < n_cells.
 * V is the Voigt profile of Sec. 6.1.1 (Eqs. 2-11), evaluated through the
 * Faddeeva function in FP32 with region-dependent approximations (relative
 * error <= 1e-5).  S(T): HITRAN convention, T_ref = 296 K, partition ratio
 * (T/T_ref)^1.5.  sigma = (nu0/c) sqrt(kT/m) (Gaussian standard deviation of
 * Eq. 2).  gamma = gamma_ref (P/1 bar) (296/T)^0.5.  A line contributes at
 * grid points with |nu_j - nu0| <= cutoff_cm, the difference taken in FP64 as
 * (nu_start + j*dnu) - nu0.  Lines are summed in FP32 with compensation
 * (partial sums over 128 lines folded with TwoSum) in a fixed order: the
 * result does not vary between runs.  With a line-strength threshold set
 * (bart_set_line_threshold) lines below it are left out.
 *   species  host array [n_species] of line lists (device arrays inside)
 *   p_bar    host [n_cells] pressures, bar, > 0
 *   t_K      host [n_cells] temperatures, K, > 0
 *   out      device [n_species][n_cells][nu.n_nu] FP32, written entirely
 * Returns BART_EINVAL for NULL pointers, n_species < 1, n_cells < 1,
 * non-positive P, T, dnu or cutoff, or n_nu outside [1, 2^31). */
bart_status bart_opacity_cells(bart_ctx* ctx, const bart_linelist* species, int n_species,
                               const double* p_bar, const double* t_K, int n_cells,
                               bart_nugrid nu, double cutoff_cm, float* out);

/* The precomputed opacity table of Sec. 3 and Sec. 4 item 3: the opacity of
 * each species on the output grid over the layer pressures and a grid of
 * temperatures,
 *   grid[s][k][m][j] = opacity at (p_bar[k], t_K[m]) as in bart_opacity_cells.
 *   p_bar  host [n_layers], strictly increasing (top of atmosphere first)
 *   t_K    host [n_temps], strictly increasing
 *   grid   device [n_species][n_layers][n_temps][nu.n_nu] FP32
 * Same error behaviour as bart_opacity_cells, plus BART_EINVAL for
 * non-increasing axes. */
bart_status bart_build_opacity_grid(bart_ctx* ctx, const bart_linelist* species, int n_species,
                                    const double* p_bar, int n_layers,
                                    const double* t_K, int n_temps,
                                    bart_nugrid nu, double cutoff_cm, float* grid);

/* ------------------------------------------- the paper's Voigt-table scheme */

/* The opacity scheme of Sec. 4 items 4-5 and Sec. 6.1.1 (test f04broadening):
 * Voigt profiles tabulated once for a grid of widths and read by every line.
 *   n_sigma Doppler widths (Gaussian standard deviations, cm^-1) log-spaced
 *   from sigma_lo to sigma_hi, n_gamma Lorentz half widths (cm^-1) log-spaced
 *   from gamma_lo to gamma_hi; each profile sampled `oversample` times per grid
 *   interval dnu_cm, aligned to the grid, out to cutoff_cm (plus one interval).
 * A line at a cell uses the profile of the nearest widths in ln sigma and
 * ln gamma (clamped to the bounds), its centre rounded to the nearest fine
 * sample, read at the grid points within |nu_j - nu0| <= cutoff of its exact
 * centre; strengths as in bart_opacity_cells.  The profile values come from
 * the same FP32 Faddeeva evaluation as the direct sum.  The table occupies
 * n_sigma n_gamma oversample (2 ceil(cutoff/dnu) + 3) x 4 bytes of device
 * memory on the context's device, owned by the table until
 * bart_voigt_table_destroy.  The line-strength bound is not applied on this
 * path.  Returns BART_EINVAL for non-positive or inverted bounds, counts < 1
 * or a table above 200 GB, BART_ENOMEM if the device memory is missing. */
typedef struct bart_voigt_table bart_voigt_table;
bart_status bart_voigt_table_create(bart_ctx* ctx, int n_sigma, double sigma_lo, double sigma_hi,
                                    int n_gamma, double gamma_lo, double gamma_hi, int oversample,
                                    double dnu_cm, double cutoff_cm, bart_voigt_table** out);
void bart_voigt_table_destroy(bart_voigt_table* table);
/* Device bytes held by the table (-1 for NULL). */
int64_t bart_voigt_table_bytes(const bart_voigt_table* table);

/* bart_opacity_cells and bart_build_opacity_grid with the table scheme; same
 * arguments and layouts plus the table, which must have been built on this
 * context's device for the same dnu and a cutoff >= cutoff_cm (else
 * BART_EINVAL). */
bart_status bart_opacity_cells_table(bart_ctx* ctx, const bart_voigt_table* table,
                                     const bart_linelist* species, int n_species, const double* p_bar,
                                     const double* t_K, int n_cells, bart_nugrid nu, double cutoff_cm,
                                     float* out);
bart_status bart_build_opacity_grid_table(bart_ctx* ctx, const bart_voigt_table* table,
                                          const bart_linelist* species, int n_species,
                                          const double* p_bar, int n_layers, const double* t_K, int n_temps,
                                          bart_nugrid nu, double cutoff_cm, float* grid);

/* Line-strength lower bound of Sec. 4 item 6 for the following
 * bart_opacity_cells / bart_build_opacity_grid calls on this context: at each
 * (P, T) cell, a line whose strength S_i(T) is below rel times the strongest
 * line of its species at that cell is left out of the sum (the comparison is
 * made on ln S in FP32).  rel <= 0 turns the bound off (the default).
 * Returns BART_EINVAL for NULL ctx or a non-finite rel. */
bart_status bart_set_line_threshold(bart_ctx* ctx, double rel);

/* Re w(x + i y) of the Faddeeva function (Sec. 6.1.1, Eqs. 4-11) as the
 * opacity kernels evaluate it, for y >= 0.  x, y, out: device [n] FP32.
 * Exposed so the profile evaluation can be checked on its own. */
bart_status bart_faddeeva_re(bart_ctx* ctx, const float* x, const float* y, int64_t n, float* out);

/* ----------------------------------------------------------- forward model */

/* Opacity grid as produced by bart_build_opacity_grid.
 *   grid   device [n_species][n_layers][n_temps][nu.n_nu]
 *   p_bar  host [n_layers] strictly increasing, t_K host [n_temps] strictly
 *          increasing (n_temps may be 1: a per-layer opacity with no T axis). */
typedef struct {
  const float* grid;
  int n_species, n_layers, n_temps;
  const double* p_bar;
  const double* t_K;
  bart_nugrid nu;
} bart_grid_desc;

enum { BART_EMISSION = 0, BART_TRANSMISSION = 1 };

/* Forward-model constants (Sec. 3; Sec. 6.2 for the HD 189733 b-like values).
 *   geometry      BART_EMISSION or BART_TRANSMISSION
 *   n_angles      emission: Gauss-Legendre points on mu in [0, 1], 1..16
 *   g_cgs         gravity, cm s^-2 (at r_planet for transmission)
 *   mu_amu        mean molecular mass of the atmosphere, amu
 *   t_int_K, t_star_K, r_star_tp_cm, a_orbit_cm
 *                 constants of the T(P) profile (internal temperature,
 *                 stellar temperature and radius, orbital distance)
 *   t_min_K, t_max_K  clamp of the profile temperature
 *   p_ref_bar     transmission: pressure at r_planet
 *   p_top_bar, p_bot_bar  transmission: instance levels are log-spaced
 *                 between these (n_levels[i] of them)
 *   x0            host [n_species] base volume mixing ratios X0_s
 *   tau_max       emission: Sec. 4 item 7, stop the layer integration at a
 *                 wavenumber once the vertical optical depth from the top
 *                 exceeds tau_max; the level reached is then the bottom
 *                 (blackbody) boundary.  <= 0 turns it off.
 *   p_cloud_bar   gray cloud deck (Sec. 3): an opaque surface on the first
 *                 level with P >= p_cloud_bar (grid layers for emission, the
 *                 instance's levels for transmission; a deck between levels
 *                 acts at the deeper one, at least two levels remain).
 *                 Emission takes that level's blackbody as the bottom
 *                 boundary; transmission takes the planet as opaque below it
 *                 (altitudes stay those of the whole column).  <= 0: no deck.
 *   rayleigh_coef Rayleigh scattering (Sec. 3) by the bulk gas: cross-section
 *                 per molecule a nu^4 in cm^2, a in cm^2 (cm^-1)^-4 (about
 *                 8.4e-45 for H2), added to every level as extinction
 *                 (mass opacity a nu^4 / (mu m_u)).  0: off; must be finite
 *                 and >= 0 (BART_EINVAL otherwise).
 * (tau_max was added in ABI version 2, p_cloud_bar and rayleigh_coef in
 * version 3, each at the end of the struct.) */
typedef struct {
  int32_t geometry;
  int32_t n_angles;
  double g_cgs, mu_amu;
  double t_int_K, t_star_K, r_star_tp_cm, a_orbit_cm;
  double t_min_K, t_max_K;
  double p_ref_bar, p_top_bar, p_bot_bar;
  const double* x0;
  double tau_max;
  double p_cloud_bar;
  double rayleigh_coef;
} bart_fwd_cfg;

/* A batch of proposals (emission) or instances (transmission).
 *   n            number of entries, >= 1
 *   theta        device [n][5 + n_species]: log10 kappa, log10 gamma1,
 *                log10 gamma2, alpha, beta (the five T(P) parameters), then
 *                the log10 abundance scalings a_s (X_s = X0_s 10^a_s)
 *                (Sec. 7, nine free parameters)
 *   t_profile    device [n][n_layers] or NULL; if set, emission uses these
 *                layer temperatures instead of the T(P) profile of theta
 *   n_levels     transmission: device [n] level counts in [2, 192]
 *   nu_lo, nu_hi device [n] grid index span [lo, hi) of each entry, or NULL
 *                for the whole grid
 *   spec_offsets device [n+1] start of entry i's spectrum in the packed output
 *                (NULL: entry i starts at i * nu.n_nu)
 *   r_planet_cm, r_star_cm  transmission: device [n] radii
 *   active       device [n] or NULL: entries with active[i] == 0 are skipped
 *                and their spectra and band values are left untouched (used by
 *                the screened sampler to evaluate survivors only) */
typedef struct {
  int32_t n;
  const float* theta;
  const float* t_profile;
  const int32_t* n_levels;
  const int64_t* nu_lo;
  const int64_t* nu_hi;
  const int64_t* spec_offsets;
  const float* r_planet_cm;
  const float* r_star_cm;
  const int32_t* active;
} bart_batch;

/* Filter transmission curves on the grid: device [n_bands][nu.n_nu] FP32. */
typedef struct {
  int32_t n_bands;
  const float* weights;
} bart_filters;

/* Spectra of a batch of proposals from the opacity grid, optionally with
 * their band values (the second pass of Sec. 4; Fig. 1 transit + spectrum
 * integrator).  Emission returns the planetary flux F(nu) in
 * erg s^-1 cm^-2 (cm^-1)^-1 (layer-averaged source, blackbody interior, no
 * stellar light); transmission returns the transit depth (R_p,eff/R_star)^2.
 *   spectra  device packed output (see spec_offsets) or NULL
 *   filters  bands to integrate, or NULL
 *   bands    device [n][filters->n_bands] or NULL (needs filters)
 * Band values are the trapezoid-weighted means of bart_band_integrate; a band
 * with no weight on an entry's span yields 0.  An entry whose span is invalid
 * (lo < 0, hi > nu.n_nu or lo >= hi) keeps its spectrum untouched, gets band
 * values 0 and makes bart_sync() return BART_ERANGE. */
bart_status bart_forward_spectra_batch(bart_ctx* ctx, const bart_grid_desc* grid,
                                       const bart_fwd_cfg* cfg, const bart_batch* batch,
                                       float* spectra, const bart_filters* filters,
                                       float* bands);

/* Spectrum integrator (Sec. 3): for spectrum i on grid span [lo_i, hi_i),
 *   out[i][b] = sum_j W_bj F_ij dw_j / sum_j W_bj dw_j,
 * dw_j the trapezoid weights of the span (half weight at both ends), W the
 * filter curves on the full grid.  A band with zero weight gives 0.
 *   spectra       device packed spectra (spec_offsets as in bart_batch)
 *   spec_offsets  device [n_spec+1] or NULL (spectrum i at i * nu.n_nu)
 *   nu_lo, nu_hi  device [n_spec] spans or NULL (whole grid)
 *   out           device [n_spec][filters->n_bands] FP32 */
bart_status bart_band_integrate(bart_ctx* ctx, const float* spectra, const int64_t* spec_offsets,
                                const int64_t* nu_lo, const int64_t* nu_hi, int n_spec,
                                bart_nugrid nu, const bart_filters* filters, float* out);

/* Contribution functions of emission spectra (the post-processing of Sec. 3
 * computes them per bandpass).  Each proposal's flux is split into one term
 * per layer plus the bottom boundary, with the layer-averaged source of
 * bart_forward_spectra_batch:
 *   C_k(nu) = 2 pi sum_i w_i mu_i (B_k + B_{k+1})/2 (t_k(mu_i) - t_{k+1}(mu_i))
 * for the layer between levels k and k+1 (t = exp(-tau/mu) from the top), and
 * at the last level integrated, kb (L-1, the cloud deck's level, or where the
 * optical-depth limit stops), C_kb = 2 pi sum_i w_i mu_i B_kb t_kb(mu_i);
 * C_k = 0 for k > kb.  sum_k C_k(nu) is the emission spectrum.
 *   grid, cfg, batch  as bart_forward_spectra_batch (cfg->geometry must be
 *            BART_EMISSION; n_angles 1, 2, 4, 8 or 16; 1-4 species)
 *   contrib  device [n][n_layers][nu.n_nu] or NULL: C_k at grid index j; only
 *            j inside the entry's span are written
 *   filters, bands  bands device [n][n_layers][filters->n_bands] or NULL: the
 *            band mean of each C_k (trapezoid weights over the entry's span,
 *            as bart_band_integrate); they add up over k to the band value of
 *            the spectrum.
 * At least one of contrib and bands.  Without contrib the rows go to context
 * scratch (n x n_layers x n_nu floats).  Errors: BART_EINVAL for the checks
 * of bart_forward_spectra_batch, transmission geometry, or nothing requested;
 * an entry with an invalid span makes bart_sync() return BART_ERANGE. */
bart_status bart_contribution_functions(bart_ctx* ctx, const bart_grid_desc* grid,
                                        const bart_fwd_cfg* cfg, const bart_batch* batch,
                                        float* contrib, const bart_filters* filters,
                                        float* bands);

/* -------------------------------------------------------- surrogate network */

/* Surrogate of the forward model used to screen sampler proposals.  The paper
 * has no learned component (surrogates appear only as related work, Sec. 1);
 * this network is the one the screened sampler uses: an MLP with GELU hidden
 * layers, FP32 master weights, BF16 weights in the forward pass (optional)
 * and FP32 accumulation, trained by Adam on mean squared error of
 * standardised targets.
 * Parameters are one flat FP32 vector: per layer W (row-major [out][in]) then
 * b ([out]).  Inputs are rescaled as (x - in_shift) * in_scale; targets are
 * standardised as (log10 t - out_shift) * out_scale if log_outputs, else
 * (t - out_shift) * out_scale; bart_mlp_forward returns physical values. */
typedef struct bart_mlp bart_mlp;

/* widths: host [n_widths] layer widths (input first), 2 <= n_widths <= 16,
 * each in [1, 4096]; max_batch: largest batch any call may use.
 * The network starts with zero parameters and unit scaling. */
bart_status bart_mlp_create(bart_ctx* ctx, const int32_t* widths, int n_widths, int bf16_weights,
                            int log_outputs, int max_batch, bart_mlp** out);
void bart_mlp_destroy(bart_mlp* net);
/* Number of parameters, or -1 for NULL. */
int64_t bart_mlp_num_params(const bart_mlp* net);
/* Host arrays [in], [in], [out], [out]. */
bart_status bart_mlp_set_scaling(bart_mlp* net, const float* in_shift, const float* in_scale,
                                 const float* out_shift, const float* out_scale);
/* params: device [num_params]; set also clears the Adam state. */
bart_status bart_mlp_set_params(bart_mlp* net, const float* params);
bart_status bart_mlp_get_params(bart_mlp* net, float* params);
/* x: device [B][in] -> y: device [B][out] (physical units), 1 <= B <= max_batch. */
bart_status bart_mlp_forward(bart_mlp* net, const float* x, int B, float* y);
/* Loss and its gradient for inputs x [B][in] and targets t [B][out] (physical
 * units, device).  grad: device [num_params] or NULL; loss: device [1] or NULL. */
bart_status bart_mlp_gradient(bart_mlp* net, const float* x, const float* t, int B, float* grad,
                              float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the batch; loss as above. */
bart_status bart_mlp_train_step(bart_mlp* net, const float* x, const float* t, int B, float lr,
                                float* loss);
/* n_steps Adam steps in one call, each on the batch of rows
 * batch_rows[k][0 .. B-1] (device int32, indices into the n_rows rows of x
 * [n_rows][in] and t [n_rows][out], device) with learning rate lr[k] (host
 * [n_steps]); the steps are those of bart_mlp_train_step on the gathered
 * rows.  loss: device [n_steps] or NULL.  An index outside [0, n_rows) is
 * replaced by row 0 and makes bart_sync() return BART_ERANGE. */
bart_status bart_mlp_train_steps(bart_mlp* net, const float* x, const float* t, int64_t n_rows,
                                 const int32_t* batch_rows, int B, int n_steps, const float* lr, float* loss);

/* ------------------------------------------------------------ sampler */

/* Differential-evolution MCMC (ter Braak 2006, the sampler of Sec. 3-4) over
 * n_params parameters with a uniform prior on [lo, hi] (host arrays), with
 * the chains split into two halves that update in alternate half-steps from
 * differences of the other half's chains:
 *   y_i = x_i + gamma (x_r1 - x_r2) + eps (hi - lo) N(0, 1),
 * gamma = 2.38 / sqrt(2 n_params) when the argument is 0, and gamma = 1 on
 * every jump_every-th generation (0 = never).  Random numbers come from a
 * counter-based generator keyed by (seed, half_step, chain, draw).
 * Screening is delayed acceptance: stage 1 keeps a proposal with probability
 * a1 = min(1, exp(ls_y - ls_x)) from the surrogate log-likelihood (tempered by
 * bart_demc_set_screen), stage 2 accepts a survivor with probability
 * min(1, exp(L_y - L_x) a1(y -> x) / a1(x -> y)) from the exact
 * log-likelihood, which keeps the exact posterior as the target.
 * 3 <= n_chains <= 65536 (DE-MC proposals need >= 6, DEMCzs >= 3),
 * 1 <= n_params <= 32. */
typedef struct bart_demc bart_demc;
bart_status bart_demc_create(bart_ctx* ctx, int n_chains, int n_params, const float* lo, const float* hi,
                             double gamma, int jump_every, double eps, uint64_t seed, bart_demc** out);
void bart_demc_destroy(bart_demc* s);
/* x: device [n_chains][n_params]; loglike, loglike_s: device [n_chains] FP64
 * (loglike_s may be NULL: surrogate values 0). */
bart_status bart_demc_set_state(bart_demc* s, const float* x, const double* loglike, const double* loglike_s);
bart_status bart_demc_get_state(bart_demc* s, float* x, double* loglike, double* loglike_s);
/* Proposals of half-step `half_step` (the half updated is half_step mod 2):
 * y device [n_chains][n_params]; inbox device [n_chains] = 1 for the updated
 * half's proposals inside the prior box, else 0 (other rows copy x). */
bart_status bart_demc_propose(bart_demc* s, int64_t half_step, float* y, int32_t* inbox);
/* Stage-1 acceptance of the screen, a1(x -> y) = min(1, exp(beta (ls_y - ls_x)
 * + margin)) (defaults beta = 1, margin = 0).  Stage 2 divides out a1 of the
 * forward and multiplies in a1 of the reverse move, so the exact posterior
 * stays the target for any beta >= 0 and margin; beta < 1 or margin > 0 make
 * the screen reject only clearly worse proposals. */
bart_status bart_demc_set_screen(bart_demc* s, double beta, double margin);
/* Stage 1: pass[i] = inbox[i] and the surrogate test (ls_y device [n_chains]
 * FP64, or NULL for no screening). */
bart_status bart_demc_screen(bart_demc* s, int64_t half_step, const int32_t* inbox, const double* ls_y,
                             int32_t* pass);
/* Stage 2 and state update: L_y device [n_chains] exact log-likelihood of the
 * proposals (read only where pass[i]); ls_y as in the screen or NULL;
 * accepted device [n_chains] or NULL. */
bart_status bart_demc_accept(bart_demc* s, int64_t half_step, const float* y, const int32_t* pass,
                             const double* L_y, const double* ls_y, int32_t* accepted);
/* Switches the sampler to DEMCzs (Sec. 4; ter Braak & Vrugt 2008): every
 * chain proposes from an archive Z of past states, so all chains move at each
 * half_step.  With probability p_snooker the move is a snooker update, z, z1,
 * z2 drawn from Z, y = x + g ((z1 - z2) . e) e with e the unit vector from z
 * to x and g uniform in [1.2, 2.2), accepted with the extra factor
 * (|y - z| / |x - z|)^(d - 1) (also inside the screen's two stages);
 * otherwise y = x + gamma (z1 - z2) + eps (hi - lo) N(0, 1).  Every `thin`
 * half_steps bart_demc_accept appends all chains' states to Z while it holds
 * fewer than `capacity` states (then it stops growing).
 *   z0  device [n0][n_params], the initial archive (copied), 3 <= n0 <= capacity
 * The archive (capacity x n_params x 4 bytes) is device memory owned by the
 * sampler.  Returns BART_EINVAL for bad sizes or p_snooker outside [0, 1],
 * BART_ENOMEM if the archive cannot be allocated. */
bart_status bart_demc_set_archive(bart_demc* s, const float* z0, int64_t n0, int64_t capacity, int thin,
                                  double p_snooker);
/* Number of states in the DEMCzs archive (0 for a DE-MC sampler); waits for
 * the stream. */
bart_status bart_demc_archive_size(bart_demc* s, int64_t* n);

/* Convergence and sample-size statistics of Sec. 5 and App. C on a chain
 * history chain[t][c][q] (device, n x n_chains x n_params FP32):
 *   speis  device [n_chains][n_params] or NULL: steps per effectively
 *          independent sample, 1 + 2 sum_k rho_k over lags k >= 1 until the
 *          autocorrelation rho_k first falls below `threshold` (lags < n/2);
 *          ESS = n n_chains / (largest over parameters of the mean over chains)
 *   gr     device [n_params] or NULL: Gelman-Rubin R, sqrt(V / W) with W the
 *          mean within-chain variance, B = n x the variance of the chain
 *          means, V = (n - 1)/n W + B/n (needs n_chains >= 2).
 * Returns BART_EINVAL for n < 4 or empty shapes. */
bart_status bart_chain_stats(bart_ctx* ctx, const float* chain, int n, int n_chains, int n_params,
                             double threshold, double* speis, double* gr);

/* Gaussian log-likelihood of band values (Sec. 3: model bands compared to
 * data): out[i] = -1/2 sum_b ((model[i][b] - data[b]) / sigma[b])^2 in FP64,
 * -inf where mask[i] == 0 (mask may be NULL).  model device [n][n_bands];
 * data, sigma device [n_bands]; out device [n]. */
bart_status bart_loglike_bands(bart_ctx* ctx, const float* model, int n, int n_bands, const float* data,
                               const float* sigma, const int32_t* mask, double* out);

/* ------------------------------------------------------------ retrieval */

typedef struct {
  int64_t proposals;        /* proposals inside the prior box */
  int64_t screened_out;     /* rejected by the surrogate stage */
  int64_t exact_evals;      /* proposals evaluated by the exact forward model */
  int64_t accepted;         /* accepted proposals */
  double surrogate_err_sum; /* sum over accepted samples of max_b |band_s/band_exact - 1| */
  double surrogate_err_max; /* largest such error */
} bart_retrieval_stats;

/* The retrieval loop of Sec. 3 (Fig. 1) on the GPU: n_generations DE-MC
 * generations (two half-steps each, starting at the even half-step index
 * first_half_step) of sampler `s` (state set beforehand with
 * bart_demc_set_state), each proposal's spectrum from the emission forward
 * model on `grid` integrated over `filters` and compared with `data` +-
 * `sigma` (device [n_bands]) by bart_loglike_bands.  With a surrogate, its
 * band values screen proposals first (delayed acceptance) and only survivors
 * reach the exact model; the exact model decides every acceptance and
 * the surrogate's band error on them is accumulated in `stats`.  The sampler
 * needs 5 + n_species parameters.  use_graph = 1 captures one generation in a
 * CUDA graph after an eager first generation and replays it (call this before
 * any outer stream capture).  chain: device [n_generations][n_chains][n_params]
 * states after each generation, or NULL.  stats: host, or NULL; filled after
 * the work completes (the call then waits for the stream). */
bart_status bart_retrieval_run(bart_ctx* ctx, bart_demc* s, bart_mlp* surrogate, const bart_grid_desc* grid,
                               const bart_fwd_cfg* cfg, const bart_filters* filters, const float* data,
                               const float* sigma, int64_t first_half_step, int n_generations, int use_graph,
                               float* chain, bart_retrieval_stats* stats);

/* ------------------------------------------------- allocation-free variant */

/* The emission path of bart_forward_spectra_batch for callers that cannot
 * allocate device memory: code that runs where cudaMalloc is not allowed or
 * would stall (inside another library's allocator hooks, a real-time loop with
 * a fixed memory budget, a process that reserves all device memory up front).
 * The paper has no counterpart; this entry point only changes where scratch
 * lives.  It takes no context and allocates nothing: its scratch (per-layer
 * brackets, abundance coefficients, per-tile band partial sums, constant
 * tables, a status word; about 8.5 MB) is a fixed array that every GPU loading
 * the library holds until the process exits.
 *   Limits: n <= 64 entries, n_layers <= 256, n_species <= 4, n_temps <= 64,
 *   n_nu <= 131072, n_bands <= 16, emission geometry only.  Larger requests
 *   return BART_ERANGE before any work; malformed ones BART_EINVAL (among
 *   them bands requested without filters, without weights or with
 *   n_bands < 1).
 *   Arguments and results are those of bart_forward_spectra_batch; the work is
 *   issued on cuda_stream (a cudaStream_t, NULL = default stream) of the
 *   current device.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, under a lock, so first calls from several host
 *   threads are safe); make that first call before any stream capture.  The
 *   call's constant tables reach the device as a kernel argument, so no host
 *   buffer has to outlive the call.
 *   All calls share the one array and reuse it without clearing it beyond
 *   what each call writes first: calls that overlap on the GPU (other streams,
 *   other host threads) race and must be serialised by the caller.
 *   Device-side range checks are not reported (there is no context): an
 *   entry whose nu_lo/nu_hi span is invalid keeps its spectrum untouched and
 *   gets band values 0. */
bart_status bart_forward_emission_noalloc(void* cuda_stream, const bart_grid_desc* grid, const bart_fwd_cfg* cfg,
                                          const bart_batch* batch, float* spectra, const bart_filters* filters,
                                          float* bands);

#ifdef __cplusplus
}
#endif

#endif /* BARTGPU_H */
