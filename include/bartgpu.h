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
 *      the transit ray geometry (Sec. 3, Sec. 5.1),
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

#define BART_ABI_VERSION 1

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

/* Line-by-line opacity at explicit (P, T) cells ("on the spot", Sec. 3):
 *   out[s][c][j] = sum_i S_i(T_c) V(nu_j - nu0_i; sigma_i(T_c), gamma_i(P_c, T_c))
 * in cm^2 molecule^-1, for species s < n_species, cell c < n_cells.
 * V is the Voigt profile of Sec. 5.1.1 (Eqs. 2-9), evaluated through the
 * Faddeeva function in FP32 with region-dependent approximations (relative
 * error <= 1e-5).  S(T): HITRAN convention, T_ref = 296 K, partition ratio
 * (T/T_ref)^1.5.  sigma = (nu0/c) sqrt(kT/m) (Gaussian standard deviation of
 * Eq. 2).  gamma = gamma_ref (P/1 bar) (296/T)^0.5.  A line contributes at
 * grid points with |nu_j - nu0| <= cutoff_cm, the difference taken in FP64 as
 * (nu_start + j*dnu) - nu0.  Lines are summed in FP32 with compensation
 * (per-block partial sums folded with TwoSum); the Doppler cores
 * (|z| < 24) are added through shared-memory atomics, so the last bit may
 * vary between runs.
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

/* Re w(x + i y) of the Faddeeva function (Sec. 5.1.1, Eqs. 4-9) as the
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

/* Forward-model constants (Sec. 3; Sec. 5.2 for the HD 189733 b-like values).
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
 *   x0            host [n_species] base volume mixing ratios X0_s */
typedef struct {
  int32_t geometry;
  int32_t n_angles;
  double g_cgs, mu_amu;
  double t_int_K, t_star_K, r_star_tp_cm, a_orbit_cm;
  double t_min_K, t_max_K;
  double p_ref_bar, p_top_bar, p_bot_bar;
  const double* x0;
} bart_fwd_cfg;

/* A batch of proposals (emission) or instances (transmission).
 *   n            number of entries, >= 1
 *   theta        device [n][5 + n_species]: log10 kappa, log10 gamma1,
 *                log10 gamma2, alpha, beta (the five T(P) parameters), then
 *                the log10 abundance scalings a_s (X_s = X0_s 10^a_s)
 *                (Sec. 7.1, nine free parameters)
 *   t_profile    device [n][n_layers] or NULL; if set, emission uses these
 *                layer temperatures instead of the T(P) profile of theta
 *   n_levels     transmission: device [n] level counts in [2, 192]
 *   nu_lo, nu_hi device [n] grid index span [lo, hi) of each entry, or NULL
 *                for the whole grid
 *   spec_offsets device [n+1] start of entry i's spectrum in the packed output
 *                (NULL: entry i starts at i * nu.n_nu)
 *   r_planet_cm, r_star_cm  transmission: device [n] radii */
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
 * with no weight on an entry's span yields 0. */
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

#ifdef __cplusplus
}
#endif

#endif /* BARTGPU_H */
