// Line-by-line opacity (Sec. 3 and Sec. 4 items 3-4): for every species and
// every (P, T) cell, the sum over lines of S(T) V(nu_j - nu0) on the output
// grid, each line cut off at |nu_j - nu0| <= cutoff and point-sampled at the
// grid wavenumbers (Sec. 4, text after the list of optimisations).
//
// Design (GB300, FP32 pipe bound):
//  * A prologue finds, per line and in FP64, the grid-index window of its
//    cutoff [jlo, jhi], the nearest grid index jc and the offset
//    delta = nu_jc - nu0 (all differences taken as (nu_start + j dnu) - nu0).
//  * The main kernel gives each CTA one (cell, 2048-point tile) of one
//    species.  Lines whose window meets the tile are staged through shared
//    memory in chunks of 256; per chunk every thread computes one line's
//    cell-dependent constants (strength, widths) once.
//  * Each thread owns 8 consecutive points and keeps their partial sums in
//    registers.  Line constants are shared-memory broadcasts.  The offset
//    x = (j - jc) dnu / (sigma sqrt 2) + delta / (sigma sqrt 2) is formed from
//    exact integer differences, so it stays relatively accurate near the core.
//  * Points outside a line's core (|z| >= 24) use the one-pole Faddeeva form:
//    six FP32 instructions and one MUFU reciprocal per line-point.  A warp
//    whose 256 points all lie inside the line's cutoff window and outside its
//    core runs without any per-point test; otherwise a predicate masks points.
//  * Core points (|z| < 24, a per-line integer window shared by both phases)
//    are evaluated afterwards by the accurate branch, one line per thread,
//    and added into a shared-memory accumulator with atomics.
//  * Partial sums are plain FP32 within a chunk and folded into a TwoSum
//    (hi, lo) pair per point after every chunk: compensated accumulation.
//  * All arithmetic runs at a 2^64 scale so far-wing terms of weak lines stay
//    normal FP32 numbers; the result is scaled back on the store.
#include <cmath>

#include "bart_internal.cuh"
#include "faddeeva.cuh"

namespace {

constexpr int OP_THREADS = 256;
constexpr int OP_R = 8;                          // points per thread
constexpr int OP_TILE = OP_THREADS * OP_R;       // points per CTA
constexpr int OP_CHUNK = OP_THREADS;             // lines per staged chunk
constexpr float CORE_S = 576.0f;                 // |z|^2 of the core boundary
constexpr float LN_2POW64 = 44.361419555836500f; // ln(2^64)
constexpr float INV_2POW64 = 5.421010862427522e-20f;
constexpr float LN10F = 2.302585092994046f;

struct LineWin {            // per line, from the FP64 prologue
  int jlo, jhi, jc;
  float delta;              // nu_jc - nu0 (cm^-1)
};

struct CellConst {
  float inv_t;              // 1 / T
  float ln_q;               // 1.5 ln(296 / T): partition-function ratio
  float gfac;               // P sqrt(296 / T)  (bar)
  float dfac;               // sqrt(2 k T / m) / c: sigma*sqrt2 = nu0 * dfac
  float c2_t;               // c2 / T
};

__device__ __forceinline__ double nu_minus(double nu_start, double dnu, int64_t j, double nu0) {
  // (nu_start + j*dnu) - nu0, each operation rounded separately (no FMA).
  return __dadd_rn(__dadd_rn(nu_start, __dmul_rn((double)j, dnu)), -nu0);
}

__global__ void line_window_kernel(const double* __restrict__ nu0, int64_t n_lines, double nu_start,
                                   double dnu, int64_t n_nu, double cutoff, int* __restrict__ jlo,
                                   int* __restrict__ jhi, LineWin* __restrict__ win) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_lines) return;
  double c = nu0[i];
  const double big = 1073741824.0;   // 2^30, keeps index arithmetic in int range
  double f = (c - nu_start) / dnu;
  f = fmin(fmax(f, -big), big);
  int64_t jc = llrint(f);
  // first j with (nu_j - nu0) >= -cutoff
  double flo = fmin(fmax(ceil((c - cutoff - nu_start) / dnu), -big), big);
  int64_t a = (int64_t)flo;
  for (int it = 0; it < 4 && nu_minus(nu_start, dnu, a - 1, c) >= -cutoff; ++it) --a;
  for (int it = 0; it < 4 && nu_minus(nu_start, dnu, a, c) < -cutoff; ++it) ++a;
  // last j with (nu_j - nu0) <= cutoff
  double fhi = fmin(fmax(floor((c + cutoff - nu_start) / dnu), -big), big);
  int64_t b = (int64_t)fhi;
  for (int it = 0; it < 4 && nu_minus(nu_start, dnu, b + 1, c) <= cutoff; ++it) ++b;
  for (int it = 0; it < 4 && nu_minus(nu_start, dnu, b, c) > cutoff; ++it) --b;
  if (a < 0) a = 0;
  if (a > n_nu) a = n_nu;
  if (b > n_nu - 1) b = n_nu - 1;
  if (b < -1) b = -1;
  jlo[i] = (int)a;
  jhi[i] = (int)b;
  LineWin w;
  w.jlo = (int)a;
  w.jhi = (int)b;
  w.jc = (int)jc;
  w.delta = (float)nu_minus(nu_start, dnu, jc, c);
  win[i] = w;
}

// First index in [lo, hi) with key[i] >= v (key nondecreasing).
__device__ int64_t lower_bound_i(const int* __restrict__ key, int64_t lo, int64_t hi, int v) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (key[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct ChunkSmem {
  float dx[OP_CHUNK], xc[OP_CHUNK], A[OP_CHUNK], qm[OP_CHUNK], q2[OP_CHUNK];
  float y[OP_CHUNK], B[OP_CHUNK];
  int jc[OP_CHUNK], jlo[OP_CHUNK], jhi[OP_CHUNK], klo[OP_CHUNK], khi[OP_CHUNK];
};

__global__ void __launch_bounds__(OP_THREADS)
opacity_kernel(const double* __restrict__ nu0, const float* __restrict__ log_s,
               const float* __restrict__ elow, const float* __restrict__ gref,
               const int* __restrict__ jlo_a, const int* __restrict__ jhi_a,
               const LineWin* __restrict__ win, int64_t n_lines,
               const CellConst* __restrict__ cells, double dnu, int64_t n_nu,
               float* __restrict__ out, const float2* __restrict__ wtab) {
  __shared__ ChunkSmem sm;
  __shared__ float core_acc[OP_TILE];
  __shared__ int64_t range[2];

  const int tid = threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.x * OP_TILE;
  const int64_t t1 = t0 + OP_TILE - 1;
  const int cell = blockIdx.y;
  const CellConst cc = cells[cell];

  for (int i = tid; i < OP_TILE; i += OP_THREADS) core_acc[i] = 0.0f;
  if (tid == 0) {
    // lines with jhi >= t0 and jlo <= t1
    range[0] = lower_bound_i(jhi_a, 0, n_lines, (int)t0);
    range[1] = lower_bound_i(jlo_a, range[0], n_lines, (int)(t1 + 1));
  }
  __syncthreads();
  const int64_t i_begin = range[0], i_end = range[1];

  const int j0 = (int)(t0 + tid * OP_R);             // first point of this thread
  const int lane = tid & 31;
  const int w0 = j0 - lane * OP_R;                    // warp span [w0, w1]
  const int w1 = w0 + 32 * OP_R - 1;

  float acc[OP_R], hi[OP_R], lo[OP_R];
#pragma unroll
  for (int r = 0; r < OP_R; ++r) { acc[r] = 0.f; hi[r] = 0.f; lo[r] = 0.f; }

  const float dnuf = (float)dnu;
  const float c2 = (float)bartc::C2;
  const float inv_tref = (float)(1.0 / bartc::TREF);

  for (int64_t base = i_begin; base < i_end; base += OP_CHUNK) {
    const int nl = (int)min((int64_t)OP_CHUNK, i_end - base);
    // ---- stage: cell-dependent constants of one line per thread
    if (tid < nl) {
      const int64_t i = base + tid;
      const LineWin w = win[i];
      const float nu0f = (float)nu0[i];
      const float sig2 = nu0f * cc.dfac;                 // sigma sqrt 2
      const float inv = 1.0f / sig2;
      const float y = gref[i] * cc.gfac * inv;
      const float q = y * y;
      const float stim = expm1f(-c2 * nu0f * cc.inv_t) / expm1f(-c2 * nu0f * inv_tref);
      const float ln_s = log_s[i] * LN10F + cc.ln_q - c2 * elow[i] * (cc.inv_t - inv_tref) + logf(stim);
      const float B = expf(ln_s + LN_2POW64) * inv * bartw::INV_SQRTPI;   // S/(sigma sqrt(2 pi)) scaled
      const float dx = dnuf * inv;
      const float xc = w.delta * inv;
      sm.dx[tid] = dx;
      sm.xc[tid] = xc;
      sm.A[tid] = B * y * bartw::INV_SQRTPI;
      sm.qm[tid] = q - 0.5f;
      sm.q2[tid] = 2.0f * q;
      sm.y[tid] = y;
      sm.B[tid] = B;
      sm.jc[tid] = w.jc;
      sm.jlo[tid] = w.jlo;
      sm.jhi[tid] = w.jhi;
      int klo = 0x7fffffff, khi = -0x7fffffff;   // empty core window
      if (q < CORE_S) {
        const float X = sqrtf(CORE_S - q);
        const float lo_f = fmaxf(floorf((-X - xc) / dx), -1073741824.0f);
        const float hi_f = fminf(ceilf((X - xc) / dx), 1073741824.0f);
        // int64 sums, clamped, so far-off-grid lines cannot overflow
        klo = (int)max((long long)w.jc + (long long)lo_f, -1073741824LL);
        khi = (int)min((long long)w.jc + (long long)hi_f, 1073741824LL);
      }
      sm.klo[tid] = klo;
      sm.khi[tid] = khi;
    }
    __syncthreads();

    // ---- far field: one-pole form, register-blocked over OP_R points
    for (int l = 0; l < nl; ++l) {
      const float dx = sm.dx[l], A = sm.A[l], qm = sm.qm[l], q2 = sm.q2[l];
      const int jc = sm.jc[l], jlo = sm.jlo[l], jhi = sm.jhi[l];
      const int klo = sm.klo[l], khi = sm.khi[l];
      const float x0 = fmaf((float)(j0 - jc), dx, sm.xc[l]);
      const bool fast = (jlo <= w0) && (jhi >= w1) && (khi < w0 || klo > w1);
      if (fast) {
#pragma unroll
        for (int r = 0; r < OP_R; ++r) {
          const float x = fmaf((float)r, dx, x0);
          const float u = fmaf(x, x, qm);
          const float num = fmaf(A, u, A);
          acc[r] = fmaf(num, bartw::rcp_approx(fmaf(u, u, q2)), acc[r]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < OP_R; ++r) {
          const int j = j0 + r;
          const bool in = (j >= jlo) && (j <= jhi) && (j < klo || j > khi);
          const float x = fmaf((float)r, dx, x0);
          const float u = fmaf(x, x, qm);
          const float num = fmaf(A, u, A);
          const float v = num * bartw::rcp_approx(fmaf(u, u, q2));
          acc[r] += in ? v : 0.0f;
        }
      }
    }
    // fold the chunk's partial sums into the compensated pair (TwoSum)
#pragma unroll
    for (int r = 0; r < OP_R; ++r) {
      const float s = hi[r] + acc[r];
      const float bp = s - hi[r];
      lo[r] += (hi[r] - (s - bp)) + (acc[r] - bp);
      hi[r] = s;
      acc[r] = 0.f;
    }

    // ---- core points of this chunk's lines: accurate branch, one line per thread
    if (tid < nl) {
      int a = max(max(sm.klo[tid], sm.jlo[tid]), (int)t0);
      int b = min(min(sm.khi[tid], sm.jhi[tid]), (int)min(t1, n_nu - 1));
      if (a <= b) {
        const float dx = sm.dx[tid], xc = sm.xc[tid], y = sm.y[tid], B = sm.B[tid];
        const int jc = sm.jc[tid];
        for (int j = a; j <= b; ++j) {
          const float x = fmaf((float)(j - jc), dx, xc);
          atomicAdd(&core_acc[j - t0], B * bartw::core_re(x, y, wtab));
        }
      }
    }
    __syncthreads();
  }

  // ---- store
#pragma unroll
  for (int r = 0; r < OP_R; ++r) {
    const int64_t j = (int64_t)j0 + r;
    if (j < n_nu) out[(int64_t)cell * n_nu + j] = ((hi[r] + lo[r]) + core_acc[j - t0]) * INV_2POW64;
  }
}

bart_status validate_lists(bart_ctx* ctx, const bart_linelist* species, int n_species) {
  BART_REQUIRE(ctx, species != nullptr, "species is NULL");
  BART_REQUIRE(ctx, n_species >= 1, "n_species must be >= 1");
  for (int s = 0; s < n_species; ++s) {
    const bart_linelist& L = species[s];
    BART_REQUIRE(ctx, L.n_lines >= 0 && L.n_lines < (int64_t(1) << 40), "species %d: bad n_lines", s);
    if (L.n_lines > 0)
      BART_REQUIRE(ctx, L.nu0_cm && L.log10_s296 && L.elow_cm && L.gamma_ref_cm,
                   "species %d: NULL line array", s);
    BART_REQUIRE(ctx, L.mass_amu > 0 && std::isfinite(L.mass_amu), "species %d: mass must be > 0", s);
  }
  return BART_OK;
}

bart_status validate_grid(bart_ctx* ctx, const bart_nugrid& nu, double cutoff) {
  BART_REQUIRE(ctx, nu.n_nu >= 1 && nu.n_nu < (int64_t(1) << 31) - OP_TILE, "n_nu out of range");
  BART_REQUIRE(ctx, nu.dnu_cm > 0 && std::isfinite(nu.dnu_cm) && std::isfinite(nu.nu_start_cm),
               "dnu must be > 0 and finite");
  BART_REQUIRE(ctx, cutoff > 0 && std::isfinite(cutoff), "cutoff must be > 0 and finite");
  return BART_OK;
}

// Shared driver for cells given as (P, T) pairs; `out` is [n_species][n_cells][n_nu].
bart_status run_cells(bart_ctx* ctx, const bart_linelist* species, int n_species,
                      const std::vector<double>& p, const std::vector<double>& t, bart_nugrid nu,
                      double cutoff, float* out) {
  const int n_cells = (int)p.size();
  BART_REQUIRE(ctx, n_cells >= 1 && n_cells <= 65535, "n_cells must be in [1, 65535]");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  bart_status st = bart_ensure_wtable(ctx);
  if (st != BART_OK) return st;

  int64_t max_lines = 0;
  for (int s = 0; s < n_species; ++s) max_lines = std::max(max_lines, species[s].n_lines);
  void *p_jlo, *p_jhi, *p_win, *p_cells;
  size_t nl = (size_t)std::max<int64_t>(max_lines, 1);
  if ((st = bart_scratch(ctx, "op_jlo", nl * sizeof(int), &p_jlo)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "op_jhi", nl * sizeof(int), &p_jhi)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "op_win", nl * sizeof(LineWin), &p_win)) != BART_OK) return st;

  std::vector<CellConst> hc((size_t)n_species * n_cells);
  for (int s = 0; s < n_species; ++s)
    for (int c = 0; c < n_cells; ++c) {
      const double T = t[c], P = p[c];
      CellConst k;
      k.inv_t = (float)(1.0 / T);
      k.ln_q = (float)(1.5 * std::log(bartc::TREF / T));
      k.gfac = (float)(P * std::sqrt(bartc::TREF / T));
      k.dfac = (float)(std::sqrt(2.0 * bartc::KB * T / (species[s].mass_amu * bartc::AMU)) / bartc::C);
      k.c2_t = (float)(bartc::C2 / T);
      hc[(size_t)s * n_cells + c] = k;
    }
  if ((st = bart_upload_const(ctx, "op_cells", hc.data(), hc.size() * sizeof(CellConst), &p_cells)) != BART_OK)
    return st;

  const int64_t n_tiles = (nu.n_nu + OP_TILE - 1) / OP_TILE;
  for (int s = 0; s < n_species; ++s) {
    const bart_linelist& L = species[s];
    float* o = out + (int64_t)s * n_cells * nu.n_nu;
    if (L.n_lines > 0) {
      line_window_kernel<<<(unsigned)((L.n_lines + 255) / 256), 256, 0, ctx->stream>>>(
          L.nu0_cm, L.n_lines, nu.nu_start_cm, nu.dnu_cm, nu.n_nu, cutoff, (int*)p_jlo, (int*)p_jhi,
          (LineWin*)p_win);
      if ((st = bart_check_launch(ctx, "line_window_kernel")) != BART_OK) return st;
    }
    dim3 grid((unsigned)n_tiles, (unsigned)n_cells);
    opacity_kernel<<<grid, OP_THREADS, 0, ctx->stream>>>(
        L.nu0_cm, L.log10_s296, L.elow_cm, L.gamma_ref_cm, (const int*)p_jlo, (const int*)p_jhi,
        (const LineWin*)p_win, L.n_lines, (const CellConst*)p_cells + (size_t)s * n_cells, nu.dnu_cm,
        nu.n_nu, o, ctx->d_wtable);
    if ((st = bart_check_launch(ctx, "opacity_kernel")) != BART_OK) return st;
  }
  return BART_OK;
}

}  // namespace

extern "C" bart_status bart_opacity_cells(bart_ctx* ctx, const bart_linelist* species, int n_species,
                                          const double* p_bar, const double* t_K, int n_cells,
                                          bart_nugrid nu, double cutoff_cm, float* out) {
  if (!ctx) return BART_EINVAL;
  bart_status st;
  if ((st = validate_lists(ctx, species, n_species)) != BART_OK) return st;
  if ((st = validate_grid(ctx, nu, cutoff_cm)) != BART_OK) return st;
  BART_REQUIRE(ctx, p_bar && t_K && out, "NULL p_bar, t_K or out");
  BART_REQUIRE(ctx, n_cells >= 1, "n_cells must be >= 1");
  std::vector<double> p(p_bar, p_bar + n_cells), t(t_K, t_K + n_cells);
  for (int c = 0; c < n_cells; ++c)
    BART_REQUIRE(ctx, p[c] > 0 && t[c] > 0 && std::isfinite(p[c]) && std::isfinite(t[c]),
                 "cell %d: P and T must be > 0 and finite", c);
  return run_cells(ctx, species, n_species, p, t, nu, cutoff_cm, out);
}

extern "C" bart_status bart_build_opacity_grid(bart_ctx* ctx, const bart_linelist* species, int n_species,
                                               const double* p_bar, int n_layers, const double* t_K,
                                               int n_temps, bart_nugrid nu, double cutoff_cm, float* grid) {
  if (!ctx) return BART_EINVAL;
  bart_status st;
  if ((st = validate_lists(ctx, species, n_species)) != BART_OK) return st;
  if ((st = validate_grid(ctx, nu, cutoff_cm)) != BART_OK) return st;
  BART_REQUIRE(ctx, p_bar && t_K && grid, "NULL p_bar, t_K or grid");
  BART_REQUIRE(ctx, n_layers >= 1 && n_temps >= 1, "n_layers and n_temps must be >= 1");
  for (int k = 0; k < n_layers; ++k) {
    BART_REQUIRE(ctx, p_bar[k] > 0 && std::isfinite(p_bar[k]), "p_bar[%d] must be > 0", k);
    BART_REQUIRE(ctx, k == 0 || p_bar[k] > p_bar[k - 1], "p_bar must be strictly increasing");
  }
  for (int m = 0; m < n_temps; ++m) {
    BART_REQUIRE(ctx, t_K[m] > 0 && std::isfinite(t_K[m]), "t_K[%d] must be > 0", m);
    BART_REQUIRE(ctx, m == 0 || t_K[m] > t_K[m - 1], "t_K must be strictly increasing");
  }
  std::vector<double> p, t;
  p.reserve((size_t)n_layers * n_temps);
  t.reserve((size_t)n_layers * n_temps);
  for (int k = 0; k < n_layers; ++k)
    for (int m = 0; m < n_temps; ++m) {
      p.push_back(p_bar[k]);
      t.push_back(t_K[m]);
    }
  return run_cells(ctx, species, n_species, p, t, nu, cutoff_cm, grid);
}
