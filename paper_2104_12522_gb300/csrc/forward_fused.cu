// Host side of the persistent fused emission launch (the kernels are in
// emission_fused.cuh, instantiated per species count in fused_s1.cu ..
// fused_s4.cu so the translation units compile in parallel): constant tables,
// scratch (work counters, published layer states, band partials), the tile
// autotuner and the launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "emission_fused.cuh"

using namespace bartem;

namespace {

FusedLauncher pick_fused(int S, int na, bool tma, int tw, int mode) {
  switch (S) {
    case 1: return fused_launcher<1>(na, tma, tw, mode);
    case 2: return fused_launcher<2>(na, tma, tw, mode);
    case 3: return fused_launcher<3>(na, tma, tw, mode);
    case 4: return fused_launcher<4>(na, tma, tw, mode);
    default: return nullptr;
  }
}

}  // namespace

bart_status bartem::fused_emission(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c,
                                   const bart_batch* b, float* spectra, const bart_filters* f, float* bands, int nb) {
  const int S = g->n_species, L = g->n_layers, M = g->n_temps, n = b->n, NA = c->n_angles;
  const int64_t N = g->nu.n_nu;
  const int mode = emission_mode(g, c);
  // the bulk-copy variant on request, where its 16-byte row starts hold:
  // n_nu a multiple of 4 and an aligned grid
  const bool tma = ctx->em_launch == BART_LAUNCH_FUSED_TMA && (N % 4 == 0) &&
                   (reinterpret_cast<uintptr_t>(g->grid) % 16 == 0);
  if (S > FUSED_MAX_SPECIES || !pick_fused(S, NA, tma, FUSED_TILES[1], mode))
    return bart_fail(ctx, BART_EUNSUPPORTED, "emission with %d species and %d angles is not instantiated "
                     "(species 1-4; angles 1, 2, 4, 8, 16)", S, NA);
  bart_status st;
  // device table: level pressures, temperature axis, (P_{k+1} - P_k) / 2g
  std::vector<float> hconst;
  for (int k = 0; k < L; ++k) hconst.push_back((float)(g->p_bar[k] * bartc::BAR));
  for (int m = 0; m < M; ++m) hconst.push_back((float)g->t_K[m]);
  for (int k = 0; k + 1 < L; ++k)
    hconst.push_back((float)((g->p_bar[k + 1] - g->p_bar[k]) * bartc::BAR / (2.0 * c->g_cgs)));
  void *p_const, *p_work, *p_done = nullptr, *p_part = nullptr;
  if ((st = bart_upload_const(ctx, "ff_const", hconst.data(), hconst.size() * sizeof(float), &p_const)) != BART_OK)
    return st;
  void *p_twc, *p_flag;
  if ((st = bart_scratch(ctx, "ff_work", 3 * sizeof(unsigned long long), &p_work)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "ff_twc", (size_t)n * L * sizeof(LayerTW), &p_twc)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "ff_flag", (size_t)n * sizeof(unsigned int), &p_flag)) != BART_OK) return st;
  const int max_tiles = (int)((N + 3 + FUSED_TILES[0] - 1) / FUSED_TILES[0]);   // smallest tile, aligned start
  if (nb > 0) {
    if ((st = bart_scratch(ctx, "ff_done", (size_t)n * sizeof(unsigned int), &p_done)) != BART_OK) return st;
    if ((st = bart_scratch(ctx, "fw_part", (size_t)n * max_tiles * nb * sizeof(float2), &p_part)) != BART_OK)
      return st;
  }
  FusedArgs a{};
  a.grid = g->grid;
  a.L = L;
  a.M = M;
  a.N = N;
  a.theta = b->theta;
  a.n_theta = 5 + S;
  a.t_profile = b->t_profile;
  a.n = n;
  a.nu_lo = b->nu_lo;
  a.nu_hi = b->nu_hi;
  a.offs = b->spec_offsets;
  a.active = b->active;
  const float* dc = (const float*)p_const;
  a.p_cgs = dc;
  a.t_axis = dc + L;
  a.dpg = dc + L + M;
  for (int s = 0; s < S; ++s) a.x0mu[s] = (float)(c->x0[s] / (c->mu_amu * bartc::AMU));
  std::vector<double> mu, w;
  gauss_legendre01(NA, mu, w);
  float tw_top = 0.0f;
  for (int i = 0; i < NA; ++i) {
    a.ang[i] = (float)(-1.4426950408889634 / mu[i]);
    a.ang[NA + i] = (float)(2.0 * bartc::PI * w[i] * mu[i] * 0.5);   // the 1/2 of the layer-mean source
    tw_top += a.ang[NA + i];
  }
  a.tw_top = tw_top;
  a.inv_g = (float)(1.0 / c->g_cgs);
  a.tint4 = (float)std::pow(c->t_int_K, 4.0);
  const double rs = c->r_star_tp_cm, ao = c->a_orbit_cm;
  a.tirr0 = (rs > 0 && ao > 0) ? (float)(std::sqrt(rs / (2.0 * ao)) * c->t_star_K) : 0.0f;
  a.t_min = (float)c->t_min_K;
  a.t_max = (float)std::min(c->t_max_K, 1e30);
  a.nu_start = g->nu.nu_start_cm;
  a.dnu = g->nu.dnu_cm;
  a.spectra = spectra;
  a.filt = nb ? f->weights : nullptr;
  a.n_bands = nb;
  a.partial = (float2*)p_part;
  a.bands = bands;
  a.work = (unsigned long long*)p_work;
  a.p_done = (unsigned int*)p_done;
  a.tw_cache = (LayerTW*)p_twc;
  a.tw_flag = (unsigned int*)p_flag;
  a.status = ctx->d_status;
  a.ex = emission_extra(g, c);
  a.wide_x = (mode & 1) != 0;
  a.tau_lim = (mode & 2) != 0;

  // The CTAs in flight work on the same wavenumber span for neighbouring
  // proposals, which between them read the rows of every layer and
  // temperature bracket of that span: a unit spans at most as many
  // wavenumbers as keep those rows (S L M x span x 4 B) within half of L2.
  int l2_bytes = 0;
  if (cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    l2_bytes = 0;
  }
  const long long span_cap =
      (l2_bytes > 0 ? (long long)l2_bytes / 2 : (64LL << 20)) / ((long long)S * L * M * (long long)sizeof(float));
  auto run = [&](int tw) -> bart_status {
    // several consecutive tiles per unit amortise the unit's fixed work (layer
    // states, band partials and counts), as long as there are enough units to
    // balance the CTAs (about 8 per CTA of a full grid)
    const int n_tiles = (int)((N + 3 + tw - 1) / tw);                // tiles start on an aligned index
    const long long target = 8LL * ctx->sm_count * (2 * FUSED_OCC_THREADS / tw);
    const long long tpu_cap = std::max(1LL, std::min<long long>(MAX_TILES_PER_UNIT, span_cap / tw));
    a.tpu = (int)std::max(1LL, std::min<long long>(tpu_cap, (long long)n * n_tiles / target));
    a.n_groups = (n_tiles + a.tpu - 1) / a.tpu;
    a.n_units = (unsigned long long)a.n_groups * (unsigned long long)n;
    cudaError_t e = pick_fused(S, NA, tma, tw, mode)(a, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return bart_fail(ctx, BART_ECUDA, "launch of emission_fused_kernel failed: %s",
                                           cudaGetErrorString(e));
    return BART_OK;
  };
  // tile width: fixed by the caller, cached per shape, or measured once
  // (each candidate timed with CUDA events on the stream) outside a capture
  char key[160];
  snprintf(key, sizeof(key), "fused%s S%d A%d L%d/%d M%d N%lld n%d b%d span%d m%d", tma ? " tma" : "", S, NA, L,
           a.ex.L_run, M, (long long)N, n, nb, b->nu_lo ? 1 : 0, mode);
  // the caller's width is in threads of the one-wavenumber-per-thread
  // kernels; here a compute thread takes two
  int tw = ctx->em_tile > 0 ? 2 * ctx->em_tile : FUSED_TILES[1];
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
      for (int cand : FUSED_TILES) {
        BART_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        if ((st = run(cand)) != BART_OK) return st;
        BART_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
        BART_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        BART_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
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
  return run(tw);
}
