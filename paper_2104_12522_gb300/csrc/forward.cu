// Per-proposal forward model on the opacity grid (Sec. 3 second pass; Sec. 4
// items 3, 8 and 9) and the spectrum integrator (Sec. 3).
//
// Emission path, per batch: by default one persistent fused launch
// (forward_fused.cu, emission_fused.cuh); the three launches below remain
// as BART_LAUNCH_SPLIT, the path for grids too large for the fused kernel's
// 32-bit row offsets, and the kernels of the allocation-free entry point:
//   tp_kernel        one thread per (proposal, layer): T from the five-parameter
//                    profile (or the given profile), clamp, temperature bracket
//                    (m, w) on the grid axis; per proposal the mass-opacity
//                    coefficients X_s / (mu m_u).
//   emission_kernel  one thread per (proposal, wavenumber); layers top to
//                    bottom: opacity interpolated in T and summed over species
//                    (coalesced reads of grid rows) plus the Rayleigh term
//                    a nu^4 / (mu m_u), trapezoid optical depth, Planck
//                    source, and per Gauss-Legendre angle the log2 of the
//                    transmittance (a running sum of positive terms) with
//                    I += (B_k + B_{k+1})/2 (t_k - t_{k+1}).  A gray cloud
//                    deck ends the layer loop at its level (its blackbody is
//                    the bottom boundary).  Flux F = 2 pi sum_i w_i mu_i
//                    I(mu_i).  Band numerators and denominators are reduced
//                    per CTA (fused epilogue).
//   band_reduce      sums the per-CTA partials in a fixed order (FP64).
// Proposals run along blockIdx.x, so CTAs in flight share wavenumber tiles and
// the grid rows they read stay in L2.
#include <cmath>
#include <mutex>
#include <vector>

#include "bart_internal.cuh"
#include "emission.cuh"
#include "forward.cuh"

using namespace bartem;

namespace {

__global__ void tp_kernel(const float* __restrict__ theta, int n_theta, const float* __restrict__ t_profile,
                          int n, int L, int S, const float* __restrict__ p_cgs, const float* __restrict__ t_axis,
                          int M, int64_t N, float inv_g, float tint4, float tirr0, float t_min, float t_max,
                          const float* __restrict__ x0_over_mu, LayerTW* __restrict__ tw,
                          float* __restrict__ coef, const int32_t* __restrict__ act_mask,
                          int* __restrict__ status) {
  const int p = blockIdx.x;
  if (p >= n) return;
  if (act_mask && !act_mask[p]) return;      // skipped entry (its parameters may lie outside the prior)
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    float T;
    if (t_profile) {
      T = t_profile[(int64_t)p * L + k];
    } else {
      float th[5];
      for (int i = 0; i < 5; ++i) th[i] = theta[(int64_t)p * n_theta + i];
      T = bartf::tp_temperature(th, p_cgs[k], inv_g, tint4, tirr0);
    }
    tw[(int64_t)p * L + k] = layer_state(T, k, t_axis, M, N, t_min, t_max, status);
  }
  if (threadIdx.x < S) {
    float a = theta ? theta[(int64_t)p * n_theta + 5 + threadIdx.x] : 0.0f;
    coef[(int64_t)p * S + threadIdx.x] = x0_over_mu[threadIdx.x] * exp10f(a);
  }
}

// MODE bit 0: the FP64 Planck branch (c2 nu / T may exceed 20); bit 1: the
// optical-depth limit (an early exit from the layer loop; without it the loop
// has a fixed trip count the compiler can pipeline).
template <int S, int NA, int TW, int MODE>
__global__ void __launch_bounds__(TW)
emission_kernel(const float* __restrict__ grid, int L, int M, int64_t N, const LayerTW* __restrict__ tw,
                const float* __restrict__ coef, const float* __restrict__ dpg,
                const float* __restrict__ ang /* [2][NA]: -log2(e)/mu, 2 pi w mu / 2 */, double nu_start,
                double dnu, const int64_t* __restrict__ nu_lo, const int64_t* __restrict__ nu_hi,
                const int64_t* __restrict__ offs, float* __restrict__ spectra,
                const float* __restrict__ filt, int n_bands, float2* __restrict__ partial, int n_tiles,
                const int32_t* __restrict__ act_mask, int* __restrict__ status, EmExtra ex) {
  const int p = blockIdx.x;
  const int tile = blockIdx.y;
  const int tid = threadIdx.x;
  if (act_mask && !act_mask[p]) return;        // skipped entry: outputs untouched
  const int64_t lo = nu_lo ? nu_lo[p] : 0;
  const int64_t hi = nu_hi ? nu_hi[p] : N;
  if (lo < 0 || hi > N || lo >= hi) {
    // invalid span: report it, leave the spectrum untouched and give the
    // band reduction zero partials (band value 0, never a stale sum)
    if (tid == 0 && tile == 0) atomicOr(status, BART_DEV_RANGE);
    if (tid < n_bands) partial[((int64_t)p * n_tiles + tile) * n_bands + tid] = make_float2(0.f, 0.f);
    return;
  }
  const int64_t j = lo + (int64_t)tile * TW + tid;
  const bool active = j < hi;
  const int64_t jj = active ? j : lo;       // inactive lanes compute on a valid index

  __shared__ float s_coef[S];
  __shared__ float s_dpg[MAX_LAYERS];
  __shared__ float2 s_red[TW / 32][MAX_BANDS];
  if (tid < S) s_coef[tid] = coef[(int64_t)p * S + tid];
  for (int k = tid; k + 1 < L; k += TW) s_dpg[k] = dpg[k];
  __syncthreads();
  float xs[S];
#pragma unroll
  for (int s = 0; s < S; ++s) xs[s] = s_coef[s];

  const double nu = nu_start + (double)jj * dnu;
  const float nuf = (float)nu;
  const float c1nu3 = (float)(2.0 * bartc::H * bartc::C * bartc::C * nu * nu * nu);
  // Rayleigh mass opacity a nu^4 / (mu m_u), the same at every level
  const float chi_r = (float)(ex.ray * (nu * nu) * (nu * nu));

  // per angle: lt = log2 of the transmittance to the current level (a sum of
  // positive optical-depth terms times -log2(e)/mu), t = 2^lt, and the
  // intensity I accumulated over layers with positive terms only
  float nl2mu[NA], wmu[NA], lt[NA], t[NA], I[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    nl2mu[i] = ang[i];
    wmu[i] = ang[NA + i];
    lt[i] = 0.0f;
    t[i] = 1.0f;
    I[i] = 0.0f;
  }
  const LayerTW* twp = tw + (int64_t)p * L;
  const int64_t sstride = (int64_t)L * M * N;
  const int64_t dm = (M > 1) ? N : 0;          // offset of the upper temperature bracket
  const float* gj = grid + jj;

  auto chi_at = [&](const LayerTW& r) {
    const float* g0 = gj + r.row;
    float chi = chi_r;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const float a = __ldg(g0 + s * sstride);
      const float b = __ldg(g0 + s * sstride + dm);
      chi = fmaf(xs[s], fmaf(r.w, b - a, a), chi);
    }
    return chi;
  };

  LayerTW r = twp[0];
  float chi_prev = chi_at(r);
  constexpr bool WIDE_X = (MODE & 1) != 0, TAU_LIM = (MODE & 2) != 0;
  float B_prev = planck<WIDE_X>(c1nu3, nuf * r.c2_t);
  float tau_v = 0.0f;                            // vertical optical depth from the top
  // levels 0 .. L_run-1: a gray cloud deck on level L_run-1 ends the column
  for (int k = 1; k < ex.L_run; ++k) {
    r = twp[k];
    const float chi = chi_at(r);
    const float B = planck<WIDE_X>(c1nu3, nuf * r.c2_t);
    const float dtau = (chi_prev + chi) * s_dpg[k - 1];
    const float Bsum = B_prev + B;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      lt[i] = fmaf(dtau, nl2mu[i], lt[i]);
      const float te = bartf::ex2_approx(lt[i]);
      I[i] = fmaf(Bsum, t[i] - te, I[i]);
      t[i] = te;
    }
    chi_prev = chi;
    B_prev = B;
    if (TAU_LIM) {
      // Sec. 4 item 7: stop at the caller's optical-depth limit; the level
      // reached is then the bottom boundary (its blackbody below)
      tau_v += dtau;
      if (tau_v > ex.tau_cut) break;
    }
  }
  float F = 0.0f;
#pragma unroll
  for (int i = 0; i < NA; ++i) F = fmaf(wmu[i], fmaf(2.0f * B_prev, t[i], I[i]), F);
  // wmu = 2 pi w mu / 2: the 1/2 of the layer-mean source is folded in, so
  // the interior term carries 2 B.
  if (active && spectra) {
    const int64_t base = offs ? offs[p] : (int64_t)p * N;
    spectra[base + (j - lo)] = F;
  }
  if (n_bands > 0) {
    float dw = 0.0f;
    if (active) dw = (hi - lo == 1) ? 1.0f : ((j == lo || j == hi - 1) ? 0.5f : 1.0f);
    const int warp = tid >> 5, lane = tid & 31;
    for (int b = 0; b < n_bands; ++b) {
      const float W = active ? __ldg(filt + (int64_t)b * N + j) * dw : 0.0f;
      float num = W * F, den = W;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
      }
      if (lane == 0) s_red[warp][b] = make_float2(num, den);
    }
    __syncthreads();
    if (tid < n_bands) {
      float2 acc = make_float2(0.f, 0.f);
      for (int w = 0; w < TW / 32; ++w) {
        acc.x += s_red[w][tid].x;
        acc.y += s_red[w][tid].y;
      }
      partial[((int64_t)p * n_tiles + tile) * n_bands + tid] = acc;
    }
  }
}

__global__ void band_reduce_kernel(const float2* __restrict__ partial, int n, int n_tiles, int n_bands,
                                   const int32_t* __restrict__ active, float* __restrict__ bands) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n_bands) return;
  int p = (int)(idx / n_bands), b = (int)(idx % n_bands);
  if (active && !active[p]) return;
  double num = 0.0, den = 0.0;
  for (int t = 0; t < n_tiles; ++t) {
    float2 v = partial[((int64_t)p * n_tiles + t) * n_bands + b];
    num += v.x;
    den += v.y;
  }
  bands[idx] = den > 0.0 ? (float)(num / den) : 0.0f;
}

// Standalone spectrum integrator: one CTA per (spectrum, band).
__global__ void band_integrate_kernel(const float* __restrict__ spectra, const int64_t* __restrict__ offs,
                                      const int64_t* __restrict__ nu_lo, const int64_t* __restrict__ nu_hi,
                                      int64_t N, const float* __restrict__ filt, int n_bands,
                                      float* __restrict__ out, int* __restrict__ status) {
  const int i = blockIdx.x, b = blockIdx.y;
  const int64_t lo = nu_lo ? nu_lo[i] : 0, hi = nu_hi ? nu_hi[i] : N;
  if (lo < 0 || hi > N || lo >= hi) {
    if (threadIdx.x == 0) {
      atomicOr(status, BART_DEV_RANGE);
      out[(int64_t)i * n_bands + b] = 0.0f;
    }
    return;
  }
  const int64_t base = offs ? offs[i] : (int64_t)i * N;
  double num = 0.0, den = 0.0;
  for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    float dw = (hi - lo == 1) ? 1.0f : ((j == lo || j == hi - 1) ? 0.5f : 1.0f);
    float W = __ldg(filt + (int64_t)b * N + j) * dw;
    num += (double)(W * spectra[base + (j - lo)]);
    den += (double)W;
  }
  __shared__ double sn[32], sd[32];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sn[threadIdx.x >> 5] = num;
    sd[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, d = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += sn[w];
      d += sd[w];
    }
    out[(int64_t)i * n_bands + b] = d > 0.0 ? (float)(a / d) : 0.0f;
  }
}

// Contribution functions of the emission spectrum (post-processing of
// Sec. 3): the same layer loop as emission_kernel, one thread per (proposal,
// wavenumber), but each layer's term of the intensity sum is stored instead
// of accumulated: C_k = 2 pi sum_i w_i mu_i (B_k + B_{k+1})/2 (t_k - t_{k+1})
// for the layer between levels k and k+1, then at the last level integrated
// (kb: the deck, the optical-depth limit or L-1) its blackbody seen through
// the column, and zeros below.  sum_k C_k is the flux of emission_kernel.
// Species count and the Planck/limit options are runtime values here (a
// post-processing pass over a few spectra), only the angle count is a
// template parameter.
constexpr int CF_THREADS = 128;

template <int NA>
__global__ void __launch_bounds__(CF_THREADS)
contrib_kernel(const float* __restrict__ grid, int S, int L, int M, int64_t N, const LayerTW* __restrict__ tw,
               const float* __restrict__ coef, const float* __restrict__ dpg, const float* __restrict__ ang,
               double nu_start, double dnu, const int64_t* __restrict__ nu_lo, const int64_t* __restrict__ nu_hi,
               float* __restrict__ contrib, const int32_t* __restrict__ act_mask, int* __restrict__ status,
               EmExtra ex, int wide_x, int tau_lim) {
  const int p = blockIdx.x;
  const int tid = threadIdx.x;
  if (act_mask && !act_mask[p]) return;
  const int64_t lo = nu_lo ? nu_lo[p] : 0;
  const int64_t hi = nu_hi ? nu_hi[p] : N;
  if (lo < 0 || hi > N || lo >= hi) {
    if (tid == 0 && blockIdx.y == 0) atomicOr(status, BART_DEV_RANGE);
    return;
  }
  const int64_t j = lo + (int64_t)blockIdx.y * CF_THREADS + tid;
  if (j >= hi) return;                       // no block-level synchronisation below
  float xs[4];
  for (int s = 0; s < 4; ++s) xs[s] = s < S ? coef[(int64_t)p * S + s] : 0.0f;
  const double nu = nu_start + (double)j * dnu;
  const float nuf = (float)nu;
  const float c1nu3 = (float)(2.0 * bartc::H * bartc::C * bartc::C * nu * nu * nu);
  const float chi_r = (float)(ex.ray * (nu * nu) * (nu * nu));
  float nl2mu[NA], wmu[NA], lt[NA], t[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    nl2mu[i] = ang[i];
    wmu[i] = ang[NA + i];
    lt[i] = 0.0f;
    t[i] = 1.0f;
  }
  const LayerTW* twp = tw + (int64_t)p * L;
  const int64_t sstride = (int64_t)L * M * N;
  const int64_t dm = (M > 1) ? N : 0;
  const float* gj = grid + j;
  auto chi_at = [&](const LayerTW& r) {
    float chi = chi_r;
    for (int s = 0; s < S; ++s) {
      const float a = __ldg(gj + r.row + s * sstride);
      const float b = __ldg(gj + r.row + s * sstride + dm);
      chi = fmaf(xs[s], fmaf(r.w, b - a, a), chi);
    }
    return chi;
  };
  auto planck_x = [&](float x) { return wide_x ? planck<true>(c1nu3, x) : planck<false>(c1nu3, x); };
  float* out = contrib + (int64_t)p * L * N + j;
  LayerTW r = twp[0];
  float chi_prev = chi_at(r);
  float B_prev = planck_x(nuf * r.c2_t);
  float tau_v = 0.0f;
  int k = 1;
  for (; k < ex.L_run; ++k) {
    r = twp[k];
    const float chi = chi_at(r);
    const float B = planck_x(nuf * r.c2_t);
    const float dtau = (chi_prev + chi) * dpg[k - 1];
    const float Bsum = B_prev + B;
    float C = 0.0f;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      lt[i] = fmaf(dtau, nl2mu[i], lt[i]);
      const float te = bartf::ex2_approx(lt[i]);
      C = fmaf(wmu[i], Bsum * (t[i] - te), C);
      t[i] = te;
    }
    out[(int64_t)(k - 1) * N] = C;
    chi_prev = chi;
    B_prev = B;
    if (tau_lim) {
      tau_v += dtau;
      if (tau_v > ex.tau_cut) {
        ++k;
        break;
      }
    }
  }
  // k - 1 is now the last level integrated: its blackbody through the column
  float Cb = 0.0f;
#pragma unroll
  for (int i = 0; i < NA; ++i) Cb = fmaf(wmu[i], 2.0f * B_prev * t[i], Cb);
  out[(int64_t)(k - 1) * N] = Cb;
  for (int q = k; q < L; ++q) out[(int64_t)q * N] = 0.0f;
}

// Band means of contribution rows: one CTA per (row = proposal x level, band),
// trapezoid weights over the proposal's span, FP64 sums (as
// band_integrate_kernel).
__global__ void contrib_band_kernel(const float* __restrict__ contrib, int L, int64_t N,
                                    const int64_t* __restrict__ nu_lo, const int64_t* __restrict__ nu_hi,
                                    const float* __restrict__ filt, int n_bands, const int32_t* __restrict__ act_mask,
                                    float* __restrict__ out) {
  const int row = blockIdx.x, b = blockIdx.y;
  const int p = row / L;
  if (act_mask && !act_mask[p]) return;
  const int64_t lo = nu_lo ? nu_lo[p] : 0, hi = nu_hi ? nu_hi[p] : N;
  if (lo < 0 || hi > N || lo >= hi) return;   // reported by contrib_kernel
  const float* c = contrib + (int64_t)row * N;
  double num = 0.0, den = 0.0;
  for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    const float dw = (hi - lo == 1) ? 1.0f : ((j == lo || j == hi - 1) ? 0.5f : 1.0f);
    const float W = __ldg(filt + (int64_t)b * N + j) * dw;
    num += (double)W * (double)c[j];
    den += (double)W;
  }
  __shared__ double sn[32], sd[32];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sn[threadIdx.x >> 5] = num;
    sd[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, d = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += sn[w];
      d += sd[w];
    }
    out[(int64_t)row * n_bands + b] = d > 0.0 ? (float)(a / d) : 0.0f;
  }
}

using CfLauncher = void (*)(dim3, cudaStream_t, const float*, int, int, int, int64_t, const LayerTW*, const float*,
                            const float*, const float*, double, double, const int64_t*, const int64_t*, float*,
                            const int32_t*, int*, EmExtra, int, int);

template <int NA>
void launch_contrib(dim3 g, cudaStream_t st, const float* grid, int S, int L, int M, int64_t N, const LayerTW* tw,
                    const float* coef, const float* dpg, const float* ang, double nu_start, double dnu,
                    const int64_t* lo, const int64_t* hi, float* contrib, const int32_t* active, int* status,
                    EmExtra ex, int wide_x, int tau_lim) {
  contrib_kernel<NA><<<g, CF_THREADS, 0, st>>>(grid, S, L, M, N, tw, coef, dpg, ang, nu_start, dnu, lo, hi, contrib,
                                               active, status, ex, wide_x, tau_lim);
}

CfLauncher pick_contrib(int na) {
  switch (na) {
    case 1: return launch_contrib<1>;
    case 2: return launch_contrib<2>;
    case 4: return launch_contrib<4>;
    case 8: return launch_contrib<8>;
    case 16: return launch_contrib<16>;
    default: return nullptr;
  }
}

template <int S, int NA, int TW, int MODE>
void launch_emission(dim3 g, cudaStream_t st, const float* grid, int L, int M, int64_t N, const LayerTW* tw,
                     const float* coef, const float* dpg, const float* ang, double nu_start, double dnu,
                     const int64_t* lo, const int64_t* hi, const int64_t* offs, float* spectra,
                     const float* filt, int nb, float2* partial, int n_tiles, const int32_t* active, int* status,
                     EmExtra ex) {
  emission_kernel<S, NA, TW, MODE><<<g, TW, 0, st>>>(grid, L, M, N, tw, coef, dpg, ang, nu_start, dnu, lo, hi, offs,
                                               spectra, filt, nb, partial, n_tiles, active, status, ex);
}

using EmLauncher = void (*)(dim3, cudaStream_t, const float*, int, int, int64_t, const LayerTW*, const float*,
                            const float*, const float*, double, double, const int64_t*, const int64_t*,
                            const int64_t*, float*, const float*, int, float2*, int, const int32_t*, int*, EmExtra);


template <int S, int NA, int MODE>
EmLauncher pick_tile(int tw) {
  switch (tw) {
    case 64: return launch_emission<S, NA, 64, MODE>;
    case 128: return launch_emission<S, NA, 128, MODE>;
    case 256: return launch_emission<S, NA, 256, MODE>;
    default: return nullptr;
  }
}

template <int S, int MODE>
EmLauncher pick_na(int na, int tw) {
  switch (na) {
    case 1: return pick_tile<S, 1, MODE>(tw);
    case 2: return pick_tile<S, 2, MODE>(tw);
    case 4: return pick_tile<S, 4, MODE>(tw);
    case 8: return pick_tile<S, 8, MODE>(tw);
    case 16: return pick_tile<S, 16, MODE>(tw);
    default: return nullptr;
  }
}

template <int S>
EmLauncher pick_mode(int na, int tw, int mode) {
  switch (mode) {
    case 0: return pick_na<S, 0>(na, tw);
    case 1: return pick_na<S, 1>(na, tw);
    case 2: return pick_na<S, 2>(na, tw);
    default: return pick_na<S, 3>(na, tw);
  }
}

// The layer loop's optical-depth limit (cfg tau_max; <= 0: off).
float tau_cut_of(const bart_fwd_cfg* c) {
  return (c->tau_max > 0.0 && std::isfinite(c->tau_max)) ? (float)c->tau_max : 3.0e38f;
}

// Levels the emission integral keeps under a gray cloud deck at p_cloud_bar:
// the deck sits on the first grid level with P >= p_cloud (at least the
// second level); no such level, or p_cloud <= 0: all L levels.
int deck_levels_of(const bart_grid_desc* g, const bart_fwd_cfg* c) {
  const int L = g->n_layers;
  if (!(c->p_cloud_bar > 0.0)) return L;
  for (int k = 0; k < L; ++k)
    if (g->p_bar[k] >= c->p_cloud_bar) return std::max(k + 1, 2);
  return L;
}


// True where x = c2 nu / T can exceed 20 on the grid: T is clamped to
// [t_min, t_max] by tp_kernel, so x <= c2 nu_max / t_min.
bool planck_wide(const bart_nugrid& nu, double t_min) {
  if (!(t_min > 0)) return true;
  const double nu_max = nu.nu_start_cm + (double)(nu.n_nu - 1) * nu.dnu_cm;
  return bartc::C2 * nu_max / t_min > 19.9;
}

// mode: bit 0 the FP64 Planck branch, bit 1 the optical-depth limit
EmLauncher pick_emission(int S, int na, int tw = EM_THREADS, int mode = 1) {
  switch (S) {
    case 1: return pick_mode<1>(na, tw, mode);
    case 2: return pick_mode<2>(na, tw, mode);
    case 3: return pick_mode<3>(na, tw, mode);
    case 4: return pick_mode<4>(na, tw, mode);
    default: return nullptr;
  }
}


}  // namespace

// n-point Gauss-Legendre nodes/weights on [0, 1] (Newton on P_n).
void bartem::gauss_legendre01(int n, std::vector<double>& mu, std::vector<double>& w) {
  mu.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double x = std::cos(bartc::PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = x; p0 = 1.0; }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = (n == 1) ? 1.0 : n * (x * p1 - p0) / (x * x - 1.0);
    mu[i] = 0.5 * (x + 1.0);
    w[i] = 0.5 * 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

EmExtra bartem::emission_extra(const bart_grid_desc* g, const bart_fwd_cfg* c) {
  EmExtra ex;
  ex.L_run = deck_levels_of(g, c);
  ex.tau_cut = tau_cut_of(c);
  ex.ray = c->rayleigh_coef / (c->mu_amu * bartc::AMU);
  return ex;
}

int bartem::emission_mode(const bart_grid_desc* g, const bart_fwd_cfg* c) {
  return (planck_wide(g->nu, c->t_min_K) ? 1 : 0) | ((c->tau_max > 0.0 && std::isfinite(c->tau_max)) ? 2 : 0);
}

bart_status bart_transmission_batch(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c,
                                    const bart_batch* b, float* spectra, const bart_filters* f, float* bands);

namespace {

// Checks shared by the batched forward model and the contribution functions.
bart_status check_forward_request(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c,
                                  const bart_batch* b) {
  BART_REQUIRE(ctx, g && c && b, "NULL grid, cfg or batch");
  BART_REQUIRE(ctx, g->grid, "grid->grid is NULL");
  BART_REQUIRE(ctx, g->n_species >= 1 && g->n_layers >= 2 && g->n_layers <= MAX_LAYERS && g->n_temps >= 1,
               "grid shape out of range (S >= 1, 2 <= L <= %d, M >= 1)", MAX_LAYERS);
  BART_REQUIRE(ctx, g->p_bar && g->t_K, "grid axes are NULL");
  BART_REQUIRE(ctx, g->nu.n_nu >= 1 && g->nu.n_nu <= (int64_t)65535 * MIN_TILE && g->nu.dnu_cm > 0,
               "bad nu grid (1 <= n_nu <= %d, dnu > 0)", 65535 * MIN_TILE);
  for (int k = 0; k < g->n_layers; ++k)
    BART_REQUIRE(ctx, g->p_bar[k] > 0 && (k == 0 || g->p_bar[k] > g->p_bar[k - 1]),
                 "p_bar must be positive and strictly increasing");
  for (int m = 0; m < g->n_temps; ++m)
    BART_REQUIRE(ctx, g->t_K[m] > 0 && (m == 0 || g->t_K[m] > g->t_K[m - 1]),
                 "t_K must be positive and strictly increasing");
  BART_REQUIRE(ctx, c->g_cgs > 0 && c->mu_amu > 0 && c->x0, "cfg: g, mu must be > 0 and x0 set");
  BART_REQUIRE(ctx, c->rayleigh_coef >= 0 && std::isfinite(c->rayleigh_coef) && !std::isnan(c->p_cloud_bar),
               "cfg: rayleigh_coef must be finite and >= 0, p_cloud_bar not NaN");
  BART_REQUIRE(ctx, b->n >= 1, "batch.n must be >= 1");
  BART_REQUIRE(ctx, b->theta || b->t_profile, "batch needs theta or t_profile");
  BART_REQUIRE(ctx, (b->nu_lo == nullptr) == (b->nu_hi == nullptr), "nu_lo and nu_hi go together");
  return BART_OK;
}

// Constants, layer brackets and abundance coefficients of an emission batch:
// uploads the constant table and launches tp_kernel on the context's stream.
struct EmPrep {
  const float* dc;      // [p_cgs L][t_axis M][dpg L-1][ang 2NA][x0 S]
  size_t off_dpg, off_ang;
  LayerTW* tw;
  float* coef;
};

bart_status emission_prologue(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c, const bart_batch* b,
                              EmPrep* out) {
  const int S = g->n_species, L = g->n_layers, M = g->n_temps, n = b->n;
  const int64_t N = g->nu.n_nu;
  std::vector<double> mu, w;
  gauss_legendre01(c->n_angles, mu, w);
  const int NA = c->n_angles;
  std::vector<float> hconst;
  for (int k = 0; k < L; ++k) hconst.push_back((float)(g->p_bar[k] * bartc::BAR));
  for (int m = 0; m < M; ++m) hconst.push_back((float)g->t_K[m]);
  for (int k = 0; k + 1 < L; ++k)
    hconst.push_back((float)((g->p_bar[k + 1] - g->p_bar[k]) * bartc::BAR / (2.0 * c->g_cgs)));
  for (int i = 0; i < NA; ++i) hconst.push_back((float)(-1.4426950408889634 / mu[i]));
  for (int i = 0; i < NA; ++i) hconst.push_back((float)(2.0 * bartc::PI * w[i] * mu[i] * 0.5));
  for (int s = 0; s < S; ++s) hconst.push_back((float)(c->x0[s] / (c->mu_amu * bartc::AMU)));
  const size_t off_t = L, off_dpg = off_t + M, off_ang = off_dpg + (L - 1), off_x0 = off_ang + 2 * NA;
  void *p_const, *p_tw, *p_coef;
  bart_status st;
  if ((st = bart_upload_const(ctx, "fw_const", hconst.data(), hconst.size() * sizeof(float), &p_const)) != BART_OK)
    return st;
  if ((st = bart_scratch(ctx, "fw_tw", (size_t)n * L * sizeof(LayerTW), &p_tw)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "fw_coef", (size_t)n * S * sizeof(float), &p_coef)) != BART_OK) return st;
  const float* dc = (const float*)p_const;
  const double rs = c->r_star_tp_cm, a = c->a_orbit_cm;
  const float tirr0 = (rs > 0 && a > 0) ? (float)(std::sqrt(rs / (2.0 * a)) * c->t_star_K) : 0.0f;
  const float tint4 = (float)std::pow(c->t_int_K, 4.0);
  tp_kernel<<<n, 128, 0, ctx->stream>>>(b->theta, 5 + S, b->t_profile, n, L, S, dc, dc + off_t, M, N,
                                        (float)(1.0 / c->g_cgs), tint4, tirr0, (float)c->t_min_K,
                                        (float)std::min(c->t_max_K, 1e30), dc + off_x0, (LayerTW*)p_tw,
                                        (float*)p_coef, b->active, ctx->d_status);
  if ((st = bart_check_launch(ctx, "tp_kernel")) != BART_OK) return st;
  out->dc = dc;
  out->off_dpg = off_dpg;
  out->off_ang = off_ang;
  out->tw = (LayerTW*)p_tw;
  out->coef = (float*)p_coef;
  return BART_OK;
}

}  // namespace

extern "C" bart_status bart_forward_spectra_batch(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c,
                                                  const bart_batch* b, float* spectra, const bart_filters* f,
                                                  float* bands) {
  if (!ctx) return BART_EINVAL;
  bart_status st;
  if ((st = check_forward_request(ctx, g, c, b)) != BART_OK) return st;
  int nb = 0;
  if (bands) {
    BART_REQUIRE(ctx, f && f->weights, "bands requested without filters");
    nb = f->n_bands;
    BART_REQUIRE(ctx, nb >= 1 && nb <= MAX_BANDS, "n_bands must be in [1, %d]", MAX_BANDS);
  }
  if (c->geometry == BART_TRANSMISSION) return bart_transmission_batch(ctx, g, c, b, spectra, f, bands);
  BART_REQUIRE(ctx, c->geometry == BART_EMISSION, "unknown geometry %d", c->geometry);
  BART_REQUIRE(ctx, c->n_angles >= 1 && c->n_angles <= MAX_ANGLES, "n_angles must be in [1, %d]", MAX_ANGLES);
  const int S = g->n_species, L = g->n_layers, M = g->n_temps, n = b->n;
  const int64_t N = g->nu.n_nu;
  if (!pick_emission(S, c->n_angles))
    return bart_fail(ctx, BART_EUNSUPPORTED, "emission with %d species and %d angles is not instantiated "
                     "(species 1-4; angles 1, 2, 4, 8, 16)", S, c->n_angles);
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  if (ctx->em_launch != BART_LAUNCH_SPLIT && fused_offsets_fit(g))
    return fused_emission(ctx, g, c, b, spectra, f, bands, nb);

  const int NA = c->n_angles;
  EmPrep pr;
  if ((st = emission_prologue(ctx, g, c, b, &pr)) != BART_OK) return st;
  const int max_tiles = (int)((N + MIN_TILE - 1) / MIN_TILE);   // partials sized for the smallest tile
  void* p_part = nullptr;
  if (nb > 0 &&
      (st = bart_scratch(ctx, "fw_part", (size_t)n * max_tiles * nb * sizeof(float2), &p_part)) != BART_OK)
    return st;
  const int mode = emission_mode(g, c);
  const EmExtra ex = emission_extra(g, c);
  auto run = [&](int tw) {
    const int n_tiles = (int)((N + tw - 1) / tw);
    pick_emission(S, c->n_angles, tw, mode)(dim3((unsigned)n, (unsigned)n_tiles), ctx->stream, g->grid, L, M, N,
                                      pr.tw, pr.coef, pr.dc + pr.off_dpg, pr.dc + pr.off_ang,
                                      g->nu.nu_start_cm, g->nu.dnu_cm, b->nu_lo, b->nu_hi, b->spec_offsets, spectra,
                                      nb ? f->weights : nullptr, nb, (float2*)p_part, n_tiles, b->active,
                                      ctx->d_status, ex);
    return n_tiles;
  };
  // Tile width: cached per shape; measured once (each candidate timed with
  // CUDA events on the stream) unless the stream is being captured.
  char key[160];
  snprintf(key, sizeof(key), "em S%d A%d L%d/%d M%d N%lld n%d b%d span%d m%d", S, NA, L, ex.L_run, M, (long long)N,
           n, nb, b->nu_lo ? 1 : 0, mode);
  int tw = ctx->em_tile > 0 ? ctx->em_tile : EM_THREADS;
  auto it = ctx->tiles.find(key);
  if (ctx->em_tile > 0) {
    // fixed by the caller
  } else if (it != ctx->tiles.end()) {
    tw = it->second;
  } else if (ctx->autotune) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BART_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      cudaEvent_t e0, e1;
      BART_CUDA(ctx, cudaEventCreate(&e0));
      BART_CUDA(ctx, cudaEventCreate(&e1));
      float best = 1e30f;
      for (int cand : TILE_CHOICES) {
        BART_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        run(cand);
        BART_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
        BART_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        BART_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        if ((st = bart_check_launch(ctx, "emission_kernel (autotune)")) != BART_OK) return st;
        if (ms < best) {
          best = ms;
          tw = cand;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      ctx->tiles[key] = tw;
    }
  }
  const int n_tiles = run(tw);
  if ((st = bart_check_launch(ctx, "emission_kernel")) != BART_OK) return st;
  if (nb > 0) {
    int64_t tot = (int64_t)n * nb;
    band_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>((const float2*)p_part, n,
                                                                               n_tiles, nb, b->active, bands);
    if ((st = bart_check_launch(ctx, "band_reduce_kernel")) != BART_OK) return st;
  }
  return BART_OK;
}

extern "C" bart_status bart_band_integrate(bart_ctx* ctx, const float* spectra, const int64_t* spec_offsets,
                                           const int64_t* nu_lo, const int64_t* nu_hi, int n_spec,
                                           bart_nugrid nu, const bart_filters* f, float* out) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, spectra && f && f->weights && out, "NULL spectra, filters or out");
  BART_REQUIRE(ctx, n_spec >= 1 && n_spec <= 65535 * 1024, "n_spec out of range");
  BART_REQUIRE(ctx, f->n_bands >= 1 && f->n_bands <= 65535, "n_bands out of range");
  BART_REQUIRE(ctx, nu.n_nu >= 1, "n_nu must be >= 1");
  BART_REQUIRE(ctx, (nu_lo == nullptr) == (nu_hi == nullptr), "nu_lo and nu_hi go together");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  dim3 grid_dim((unsigned)n_spec, (unsigned)f->n_bands);
  band_integrate_kernel<<<grid_dim, 256, 0, ctx->stream>>>(spectra, spec_offsets, nu_lo, nu_hi, nu.n_nu,
                                                          f->weights, f->n_bands, out, ctx->d_status);
  return bart_check_launch(ctx, "band_integrate_kernel");
}

extern "C" bart_status bart_contribution_functions(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c,
                                                   const bart_batch* b, float* contrib, const bart_filters* f,
                                                   float* bands) {
  if (!ctx) return BART_EINVAL;
  bart_status st;
  if ((st = check_forward_request(ctx, g, c, b)) != BART_OK) return st;
  BART_REQUIRE(ctx, c->geometry == BART_EMISSION, "contribution functions are defined for emission only");
  BART_REQUIRE(ctx, contrib || bands, "nothing requested: contrib and bands are both NULL");
  int nb = 0;
  if (bands) {
    BART_REQUIRE(ctx, f && f->weights, "bands requested without filters");
    nb = f->n_bands;
    BART_REQUIRE(ctx, nb >= 1 && nb <= 65535, "n_bands must be in [1, 65535]");
  }
  CfLauncher launch = pick_contrib(c->n_angles);
  BART_REQUIRE(ctx, launch != nullptr, "n_angles must be 1, 2, 4, 8 or 16");
  BART_REQUIRE(ctx, g->n_species <= 4, "contribution functions support 1-4 species");
  const int S = g->n_species, L = g->n_layers, M = g->n_temps, n = b->n;
  const int64_t N = g->nu.n_nu;
  BART_REQUIRE(ctx, (int64_t)n * L <= 2147483647LL, "n x n_layers too large");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  EmPrep pr;
  if ((st = emission_prologue(ctx, g, c, b, &pr)) != BART_OK) return st;
  float* out = contrib;
  if (!out) {
    void* p = nullptr;
    if ((st = bart_scratch(ctx, "cf_rows", (size_t)n * L * N * sizeof(float), &p)) != BART_OK) return st;
    out = (float*)p;
  }
  const int mode = emission_mode(g, c);
  const int64_t n_tiles = (N + CF_THREADS - 1) / CF_THREADS;
  launch(dim3((unsigned)n, (unsigned)n_tiles), ctx->stream, g->grid, S, L, M, N, pr.tw, pr.coef,
         pr.dc + pr.off_dpg, pr.dc + pr.off_ang, g->nu.nu_start_cm, g->nu.dnu_cm, b->nu_lo, b->nu_hi, out, b->active,
         ctx->d_status, emission_extra(g, c), mode & 1, (mode >> 1) & 1);
  if ((st = bart_check_launch(ctx, "contrib_kernel")) != BART_OK) return st;
  if (nb > 0) {
    contrib_band_kernel<<<dim3((unsigned)(n * L), (unsigned)nb), 256, 0, ctx->stream>>>(
        out, L, N, b->nu_lo, b->nu_hi, f->weights, nb, b->active, bands);
    if ((st = bart_check_launch(ctx, "contrib_band_kernel")) != BART_OK) return st;
  }
  return BART_OK;
}

// ---------------------------------------------------------------------------
// Emission forward model that allocates nothing.
//
// For callers that cannot call cudaMalloc: code running where allocation is
// not allowed or would stall (inside another library's allocator hooks, a
// real-time loop with a fixed memory budget, a process whose device memory is
// fully reserved up front).  It runs the same kernels as the emission path of
// bart_forward_spectra_batch, but all of its scratch (layer temperature
// brackets, abundance coefficients, per-tile band partial sums, constant
// tables and a status word) lives in the fixed arrays below, which every GPU
// that loads this library holds until the process exits.  Host code must not
// pass an array's name to a kernel (on the host it is only a stand-in, not a
// device address); the device addresses are looked up once per device with
// cudaGetSymbolAddress on the first call.
namespace {

constexpr int NA_MAX_ENTRIES = 64;                   // proposals per call
constexpr int NA_MAX_LAYERS = 256;
constexpr int NA_MAX_SPECIES = 4;
constexpr int NA_MAX_BANDS = 16;
constexpr int64_t NA_MAX_NU = 131072;
constexpr int NA_MAX_TILES = (int)(NA_MAX_NU / EM_THREADS);
constexpr int NA_MAX_TEMPS = 64;
constexpr int NA_CONST = NA_MAX_LAYERS + NA_MAX_TEMPS + NA_MAX_LAYERS + 2 * MAX_ANGLES + NA_MAX_SPECIES;

static __device__ __align__(256) LayerTW na_tw[NA_MAX_ENTRIES * NA_MAX_LAYERS];
static __device__ __align__(256) float na_coef[NA_MAX_ENTRIES * NA_MAX_SPECIES];
static __device__ __align__(256) float2 na_part[(size_t)NA_MAX_ENTRIES * NA_MAX_TILES * NA_MAX_BANDS];
static __device__ __align__(256) float na_const[NA_CONST];
static __device__ __align__(256) int na_status[1];

struct NaAddrs {
  LayerTW* tw;
  float* coef;
  float2* part;
  float* cst;
  int* status;
};
constexpr int NA_MAX_DEVICES = 64;
NaAddrs g_na[NA_MAX_DEVICES];
bool g_na_ready[NA_MAX_DEVICES];
std::mutex g_na_mutex;             // guards the two tables above (first calls from several threads)

// The call's constant table, passed by value as a kernel argument (2.4 KB,
// inside the 4 KB parameter space), so no host buffer has to outlive the call.
struct NaConstArg {
  float v[NA_CONST];
  int n;
};

__global__ void na_fill_kernel(NaConstArg c, float* __restrict__ dst, int* __restrict__ status) {
  for (int i = threadIdx.x; i < c.n; i += blockDim.x) dst[i] = c.v[i];
  if (threadIdx.x == 0) *status = 0;
}

}  // namespace

extern "C" bart_status bart_forward_emission_noalloc(void* cuda_stream, const bart_grid_desc* g,
                                                     const bart_fwd_cfg* c, const bart_batch* b, float* spectra,
                                                     const bart_filters* f, float* bands) {
  if (!g || !c || !b || !g->grid || !g->p_bar || !g->t_K || !c->x0) return BART_EINVAL;
  const int S = g->n_species, L = g->n_layers, M = g->n_temps, n = b->n;
  const int64_t N = g->nu.n_nu;
  // bands need filters with at least one band and their weights
  const int nb = bands ? ((f && f->weights && f->n_bands >= 1) ? f->n_bands : -1) : 0;
  if (c->geometry != BART_EMISSION) return BART_EUNSUPPORTED;
  if (S < 1 || L < 2 || M < 1 || n < 1 || N < 1 || nb < 0 || !(g->nu.dnu_cm > 0) ||
      c->n_angles < 1 || !(c->g_cgs > 0) || !(c->mu_amu > 0) || (!b->theta && !b->t_profile) ||
      !(c->rayleigh_coef >= 0 && std::isfinite(c->rayleigh_coef)) || std::isnan(c->p_cloud_bar) ||
      ((b->nu_lo == nullptr) != (b->nu_hi == nullptr)))
    return BART_EINVAL;   // malformed request
  if (S > NA_MAX_SPECIES || L > NA_MAX_LAYERS || M > NA_MAX_TEMPS || n > NA_MAX_ENTRIES || N > NA_MAX_NU ||
      nb > NA_MAX_BANDS || c->n_angles > MAX_ANGLES)
    return BART_ERANGE;   // beyond the fixed scratch limits above
  for (int k = 0; k < L; ++k)
    if (!(g->p_bar[k] > 0) || (k > 0 && !(g->p_bar[k] > g->p_bar[k - 1]))) return BART_EINVAL;
  for (int m = 0; m < M; ++m)
    if (!(g->t_K[m] > 0) || (m > 0 && !(g->t_K[m] > g->t_K[m - 1]))) return BART_EINVAL;
  EmLauncher launch = pick_emission(S, c->n_angles, EM_THREADS, emission_mode(g, c));
  if (!launch) return BART_EUNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return BART_ECUDA;
  NaAddrs a{};
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ready[dev]) {   // set-up once per device, with that device current
      if (cudaGetSymbolAddress((void**)&a.tw, na_tw) != cudaSuccess ||
          cudaGetSymbolAddress((void**)&a.coef, na_coef) != cudaSuccess ||
          cudaGetSymbolAddress((void**)&a.part, na_part) != cudaSuccess ||
          cudaGetSymbolAddress((void**)&a.cst, na_const) != cudaSuccess ||
          cudaGetSymbolAddress((void**)&a.status, na_status) != cudaSuccess) {
        cudaGetLastError();
        return BART_ECUDA;
      }
      g_na[dev] = a;
      g_na_ready[dev] = true;
    }
    a = g_na[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  std::vector<double> mu, w;
  gauss_legendre01(c->n_angles, mu, w);
  const int NA = c->n_angles;
  NaConstArg carg;
  float* hconst = carg.v;
  int o = 0;
  for (int k = 0; k < L; ++k) hconst[o++] = (float)(g->p_bar[k] * bartc::BAR);
  const int off_t = o;
  for (int m = 0; m < M; ++m) hconst[o++] = (float)g->t_K[m];
  const int off_dpg = o;
  for (int k = 0; k + 1 < L; ++k) hconst[o++] = (float)((g->p_bar[k + 1] - g->p_bar[k]) * bartc::BAR / (2.0 * c->g_cgs));
  const int off_ang = o;
  for (int i = 0; i < NA; ++i) hconst[o++] = (float)(-1.4426950408889634 / mu[i]);
  for (int i = 0; i < NA; ++i) hconst[o++] = (float)(2.0 * bartc::PI * w[i] * mu[i] * 0.5);
  const int off_x0 = o;
  for (int s = 0; s < S; ++s) hconst[o++] = (float)(c->x0[s] / (c->mu_amu * bartc::AMU));
  // the table travels as a kernel argument; the same launch clears the status word
  carg.n = o;
  na_fill_kernel<<<1, 256, 0, st>>>(carg, a.cst, a.status);
  const double rs = c->r_star_tp_cm, ao = c->a_orbit_cm;
  const float tirr0 = (rs > 0 && ao > 0) ? (float)(std::sqrt(rs / (2.0 * ao)) * c->t_star_K) : 0.0f;
  const float tint4 = (float)std::pow(c->t_int_K, 4.0);
  tp_kernel<<<n, 128, 0, st>>>(b->theta, 5 + S, b->t_profile, n, L, S, a.cst, a.cst + off_t, M, N,
                               (float)(1.0 / c->g_cgs), tint4, tirr0, (float)c->t_min_K,
                               (float)std::min(c->t_max_K, 1e30), a.cst + off_x0, a.tw, a.coef, b->active,
                               a.status);
  const int n_tiles = (int)((N + EM_THREADS - 1) / EM_THREADS);
  launch(dim3((unsigned)n, (unsigned)n_tiles), st, g->grid, L, M, N, a.tw, a.coef, a.cst + off_dpg,
         a.cst + off_ang, g->nu.nu_start_cm, g->nu.dnu_cm, b->nu_lo, b->nu_hi, b->spec_offsets, spectra,
         nb ? f->weights : nullptr, nb, a.part, n_tiles, b->active, a.status, emission_extra(g, c));
  if (nb > 0) {
    const int64_t tot = (int64_t)n * nb;
    band_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a.part, n, n_tiles, nb, b->active, bands);
  }
  return cudaGetLastError() == cudaSuccess ? BART_OK : BART_ECUDA;
}
