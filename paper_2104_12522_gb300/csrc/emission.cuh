// Declarations shared by the emission forward-model translation units: the
// per-layer state of a proposal, the per-call options, the Planck function
// and the host-side helpers of bart_forward_spectra_batch (Sec. 3 forward
// model; Sec. 4 items 3 and 7).
#pragma once

#include <cstdint>
#include <vector>

#include "bart_internal.cuh"
#include "forward.cuh"

namespace bartem {

constexpr int EM_THREADS = 128;    // default wavenumber-tile width
constexpr int MIN_TILE = 64;       // smallest width the autotuner can choose
constexpr int TILE_CHOICES[3] = {64, 128, 256};   // widths the autotuner chooses from
constexpr int MAX_BANDS = 64;
constexpr int MAX_ANGLES = 16;
constexpr int MAX_LAYERS = 256;
constexpr float LOG2E = 1.4426950408889634f;

struct LayerTW {
  int64_t row;  // offset of grid row (layer k, lower temperature bracket m): (k M + m) n_nu
  float w;      // weight of the upper bracket
  float c2_t;   // c2 / T
};
static_assert(sizeof(LayerTW) == 16 && alignof(LayerTW) == 8, "LayerTW is loaded as one 16-byte word");

// Per-call options of the emission kernels (Sec. 3 cloud deck and Rayleigh
// scattering, Sec. 4 item 7 optical-depth limit).
struct EmExtra {
  int L_run;      // levels integrated: a gray cloud deck on level L_run-1 ends the column
  float tau_cut;  // vertical optical depth that ends the layer loop (MODE bit 1)
  double ray;     // Rayleigh a / (mu m_u): chi_R = ray nu^4, cm^2 g^-1
};

// State of one layer of a proposal from its temperature T: a NaN or
// non-positive T is reported (BART_DEV_RANGE) and replaced by t_min; T is
// clamped to [t_min, t_max]; the bracket on the temperature axis is
// m = max{m : t_axis[m] <= T} limited to [0, M-2] with the upper weight
// w = (T - T_m)/(T_{m+1} - T_m) limited to [0, 1] (linear in T, Sec. 4 item 3).
__device__ __forceinline__ LayerTW layer_state(float T, int k, const float* __restrict__ t_axis, int M, int64_t N,
                                               float t_min, float t_max, int* __restrict__ status) {
  if (!(T == T) || T <= 0.0f) {
    atomicOr(status, BART_DEV_RANGE);
    T = t_min > 0.0f ? t_min : 1.0f;
  }
  T = fminf(fmaxf(T, t_min), t_max);
  int m = 0;
  float w = 0.0f;
  if (M > 1) {
    int lo = 0, hi = M;               // first index with t_axis > T
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (t_axis[mid] <= T) lo = mid + 1; else hi = mid;
    }
    m = min(max(lo - 1, 0), M - 2);
    w = (T - t_axis[m]) / (t_axis[m + 1] - t_axis[m]);
    w = fminf(fmaxf(w, 0.0f), 1.0f);
  }
  LayerTW r;
  r.row = ((int64_t)k * M + m) * N;
  r.w = w;
  r.c2_t = (float)bartc::C2 / T;
  return r;
}

// Planck function per unit wavenumber, B = c1nu3 / (exp(x) - 1), x = c2 nu / T.
// For x <= 20 exp(x) = 2^(x log2 e) in FP32: the rounding of the product
// bounds the relative error of B by ~3e-6 for x >= 0.48 (the smallest
// c2 nu / T of a 1000 cm^-1, 3000 K grid); larger x, where 2^(x log2 e) would
// lose digits and eventually overflow, takes an FP64 exponential.
// WIDE_X: instantiated only where c2 nu / T can exceed 20 on this grid (the
// host bounds it by c2 nu_max / t_min), so the usual kernel has no branch.
template <bool WIDE_X>
__device__ __forceinline__ float planck(float c1nu3, float x) {
  if (WIDE_X && x > 20.0f) return (float)((double)c1nu3 / expm1((double)x));
  const float e = bartf::ex2_approx(x * LOG2E);
  return c1nu3 * bartf::rcp_approx(e - 1.0f);
}

// ---- host helpers (defined in forward.cu)

// n-point Gauss-Legendre nodes/weights on [0, 1] (Newton on P_n).
void gauss_legendre01(int n, std::vector<double>& mu, std::vector<double>& w);

// Options of one call: deck level count, optical-depth limit, Rayleigh term.
EmExtra emission_extra(const bart_grid_desc* g, const bart_fwd_cfg* c);

// Compile-time mode of a call: bit 0 the FP64 Planck branch (c2 nu / T can
// exceed 20 on the grid), bit 1 the optical-depth limit.
int emission_mode(const bart_grid_desc* g, const bart_fwd_cfg* c);

// The fused kernel addresses a layer's grid rows by 32-bit element offsets
// from the tile's column: it takes grids with S L M n_nu + n_nu < 2^32.
inline bool fused_offsets_fit(const bart_grid_desc* g) {
  return (int64_t)g->n_species * g->n_layers * g->n_temps * g->nu.n_nu + g->nu.n_nu <= (int64_t)UINT32_MAX;
}

// The persistent fused launch of an emission batch (forward_fused.cu).
bart_status fused_emission(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c, const bart_batch* b,
                           float* spectra, const bart_filters* f, float* bands, int nb);

}  // namespace bartem
