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
//  * Blocks of 8 points holding a window edge or a line's core (|z| < 24) are
//    evaluated point by point in a fixup pass (lanes = points, accurate branch
//    inside the core) into a warp-private accumulator: deterministic.
//  * Partial sums are plain FP32 within a chunk and folded into a TwoSum
//    (hi, lo) pair per point after every chunk: compensated accumulation.
//  * All arithmetic runs at a 2^100 scale so far-wing terms of weak lines stay
//    normal FP32 numbers (and products of two denominators stay in range);
//    the result is scaled back on the store.
#include <cmath>
#include <cstddef>

#include "bart_internal.cuh"
#include "faddeeva.cuh"

namespace {

constexpr int OP_WARPS = 8;                      // independent warps per CTA
constexpr int OP_THREADS = 32 * OP_WARPS;
constexpr int OP_R = 8;                          // points per lane
constexpr int OP_SPAN = 32 * OP_R;               // points per warp
constexpr int OP_TILE = OP_WARPS * OP_SPAN;      // points per CTA
constexpr float CORE_S = 576.0f;                 // |z|^2 of the core boundary
constexpr float LN_SCALE = 69.314718055994531f;   // ln(2^100): internal scale of all terms
constexpr float INV_SCALE = 7.888609052210118e-31f; // 2^-100
constexpr float LOG2EF = 1.4426950408889634f;
constexpr float LN2F_ = 0.6931471805599453f;

__device__ __forceinline__ float ex2f_approx(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ float lg2f_approx(float a) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

struct LineWin {            // per line, from the FP64 prologue
  int jlo, jhi, jc;
  float delta;              // nu_jc - nu0 (cm^-1)
  float ln_s0;              // ln S_ref + c2 E''/T_ref - ln(1 - exp(-c2 nu0/T_ref)): the T-free part of ln S(T)
  float c2e;                // c2 E''
  float c2nu;               // c2 nu0
  float nu0f;               // nu0 in FP32
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

__global__ void line_window_kernel(const double* __restrict__ nu0, const float* __restrict__ log_s,
                                   const float* __restrict__ elow, int64_t n_lines, double nu_start,
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
  const double c2e = bartc::C2 * (double)elow[i], c2nu = bartc::C2 * c;
  w.ln_s0 = (float)((double)log_s[i] * 2.302585092994046 + c2e / bartc::TREF - log(-expm1(-c2nu / bartc::TREF)));
  w.c2e = (float)c2e;
  w.c2nu = (float)c2nu;
  w.nu0f = (float)c;
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

// Line ranges of one warp span [w0, w0 + OP_SPAN - 1] (independent of the
// cell): lines meeting the span, and the sub-range whose cutoff windows cover
// the whole span (no per-point cutoff test needed there).
struct SpanRange {
  int64_t i_lo, i_hi;     // lines with jhi >= w0 and jlo <= w1: [i_lo, i_hi)
  int64_t f_lo, f_hi;     // lines with jlo <= w0 and jhi >= w1: [f_lo, f_hi)
};

__global__ void span_range_kernel(const int* __restrict__ jlo, const int* __restrict__ jhi, int64_t n_lines,
                                  int n_spans, SpanRange* __restrict__ out) {
  const int sp = blockIdx.x * blockDim.x + threadIdx.x;
  if (sp >= n_spans) return;
  const int w0 = sp * OP_SPAN, w1 = w0 + OP_SPAN - 1;
  SpanRange r;
  r.i_lo = lower_bound_i(jhi, 0, n_lines, w0);
  r.i_hi = lower_bound_i(jlo, r.i_lo, n_lines, w1 + 1);
  r.f_lo = lower_bound_i(jhi, r.i_lo, r.i_hi, w1);
  r.f_hi = lower_bound_i(jlo, r.i_lo, r.i_hi, w0 + 1);
  out[sp] = r;
}

// Per-line constants of the current cell, staged per warp.  The far-field loop
// reads the first six fields (one 16-byte and one 8-byte shared load).
struct __align__(16) LineC {
  float dx, xc, A, qm;     // bytes  0-15: x = (j - jc) dx + xc; A = S y / (pi sqrt2 sigma) (scaled); qm = y^2 - 1/2
  float q2, jcf, y, B;     // bytes 16-31: 2 y^2; jc as float (exact below 2^24); y; B = S / (sigma sqrt(2 pi))
  int e0, e1, jlo, jhi;    // bytes 32-47: 8-point blocks [e0, e1] left to the fixup pass; cutoff window
  int jc, klo, khi, pad;   // bytes 48-63: centre index; integer superset of the core |z| < 24
};
static_assert(offsetof(LineC, q2) == 16 && offsetof(LineC, e0) == 32, "vector loads need these offsets");

// Each lane owns one 8-point block of the warp's 256-point span.  For a line,
// a block goes through the branch-free far-field loop if it lies entirely in
// the cutoff window and outside the line's core window; the remaining blocks
// with points in the window (the block holding a window edge, the blocks the
// core touches, and any blocks between them) form one interval [e0, e1] that
// the fixup pass evaluates point by point: the one-pole form where
// u = x^2 + y^2 - 1/2 >= 575.5, the accurate branch below.  Each (line, point)
// is therefore counted once.
constexpr float U_CORE = CORE_S - 0.5f;

__global__ void __launch_bounds__(OP_THREADS, 3)
opacity_kernel(const LineWin* __restrict__ win, const float* __restrict__ gref,
               const SpanRange* __restrict__ spans, const CellConst* __restrict__ cells, double dnu,
               int64_t n_nu, float* __restrict__ out, const float2* __restrict__ wtab) {
  __shared__ LineC s_line[OP_WARPS][32];
  __shared__ float s_core[OP_WARPS][OP_SPAN];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w0l = ((int64_t)blockIdx.x * OP_WARPS + warp) * OP_SPAN;
  if (w0l >= n_nu) return;                  // warps are independent: no CTA barrier below
  const int w0 = (int)w0l, w1 = w0 + OP_SPAN - 1;
  const int j0 = w0 + lane * OP_R;          // first point of this lane
  const float j0f = (float)j0;
  const int cell = blockIdx.y;
  const CellConst cc = cells[cell];
  const SpanRange rg = spans[blockIdx.x * OP_WARPS + warp];
  const int last = (int)min((int64_t)w1, n_nu - 1);

  float* fix = s_core[warp];
#pragma unroll
  for (int r = 0; r < OP_R; ++r) fix[lane * OP_R + r] = 0.0f;

  float acc[OP_R], hi[OP_R], lo[OP_R];
#pragma unroll
  for (int r = 0; r < OP_R; ++r) { acc[r] = 0.f; hi[r] = 0.f; lo[r] = 0.f; }

  const float dnuf = (float)dnu;
  LineC* sl = s_line[warp];
  int chunks = 0;

  for (int64_t base = rg.i_lo; base < rg.i_hi; base += 32) {
    const int nl = (int)min((int64_t)32, rg.i_hi - base);
    // ---- stage: one line's cell-dependent constants per lane, plus its class
    bool fast = false, needs_fix = false;
    if (lane < nl) {
      const int64_t i = base + lane;
      const LineWin w = win[i];
      const float inv = bartw::rcp_approx(w.nu0f * cc.dfac);   // 1 / (sigma sqrt 2)
      const float y = gref[i] * cc.gfac * inv;
      const float q = y * y;
      // ln S(T) = ln_s0 + 1.5 ln(T_ref/T) - c2 E''/T + ln(1 - exp(-c2 nu0/T))
      const float stim = 1.0f - ex2f_approx(-w.c2nu * cc.inv_t * LOG2EF);
      const float ln_s = w.ln_s0 + cc.ln_q - w.c2e * cc.inv_t + LN2F_ * lg2f_approx(stim);
      const float B = ex2f_approx((ln_s + LN_SCALE) * LOG2EF) * inv * bartw::INV_SQRTPI;
      LineC c;
      c.dx = dnuf * inv;
      c.xc = w.delta * inv;
      c.A = B * y * bartw::INV_SQRTPI;
      c.qm = q - 0.5f;
      c.q2 = 2.0f * q;
      c.jcf = (float)w.jc;
      c.y = y;
      c.B = B;
      c.jc = w.jc;
      c.jlo = w.jlo;
      c.jhi = w.jhi;
      int klo = 0x7fffffff, khi = -0x7fffffff;            // empty core window
      if (q < CORE_S) {
        const float X = sqrtf(CORE_S - q);
        const float rdx = bartw::rcp_approx(c.dx);
        // two extra points on each side: a generous superset of the core
        const float lo_f = fmaxf(floorf((-X - c.xc) * rdx) - 2.0f, -1073741824.0f);
        const float hi_f = fminf(ceilf((X - c.xc) * rdx) + 2.0f, 1073741824.0f);
        klo = (int)max((long long)w.jc + (long long)lo_f, -1073741824LL);
        khi = (int)min((long long)w.jc + (long long)hi_f, 1073741824LL);
      }
      c.klo = klo;
      c.khi = khi;
      c.pad = 0;
      // blocks for the fixup pass: window edges inside the span, core blocks
      const int a = max(c.jlo, w0), b = min(c.jhi, last);
      int e0 = 32, e1 = -1;
      if (a <= b) {
        if (a > w0 && ((a - w0) & (OP_R - 1))) { e0 = min(e0, (a - w0) >> 3); e1 = max(e1, (a - w0) >> 3); }
        if ((b < w1) && (((b - w0) & (OP_R - 1)) != OP_R - 1)) {
          e0 = min(e0, (b - w0) >> 3);
          e1 = max(e1, (b - w0) >> 3);
        }
        const int ca = max(klo, a), cb = min(khi, b);
        if (ca <= cb) { e0 = min(e0, (ca - w0) >> 3); e1 = max(e1, (cb - w0) >> 3); }
      }
      c.e0 = e0;
      c.e1 = e1;
      sl[lane] = c;
      needs_fix = e0 <= e1;
      fast = !needs_fix && (c.jlo <= w0) && (c.jhi >= w1);
    }
    const unsigned fast_mask = __ballot_sync(0xffffffffu, fast);
    const unsigned fix_mask = __ballot_sync(0xffffffffu, needs_fix);
    __syncwarp();

    // ---- far field: one-pole form over the lane's 8 points
    for (int l = 0; l < nl; ++l) {
      const float4 c4 = *reinterpret_cast<const float4*>(&sl[l].dx);
      const float2 c2 = *reinterpret_cast<const float2*>(&sl[l].q2);
      const float dx = c4.x, qm = c4.w, q2 = c2.x;
      const float x0 = fmaf(j0f - c2.y, dx, c4.y);
      if ((fast_mask >> l) & 1u) {
#pragma unroll
        for (int r = 0; r < OP_R; ++r) {
          const float x = fmaf((float)r, dx, x0);
          const float u = fmaf(x, x, qm);
          const float num = fmaf(c4.z, u, c4.z);
          acc[r] = fmaf(num, bartw::rcp_approx(fmaf(u, u, q2)), acc[r]);
        }
      } else {
        // this lane's block joins the far-field sum only if it is whole in the
        // window and outside the fixup interval; otherwise its weight is 0
        const int4 ew = *reinterpret_cast<const int4*>(&sl[l].e0);   // e0, e1, jlo, jhi
        const bool take = (lane < ew.x || lane > ew.y) && (ew.z <= j0) && (ew.w >= j0 + OP_R - 1);
        const float A = take ? c4.z : 0.0f;
#pragma unroll
        for (int r = 0; r < OP_R; ++r) {
          const float x = fmaf((float)r, dx, x0);
          const float u = fmaf(x, x, qm);
          const float num = fmaf(A, u, A);
          // the clamp keeps 0 * (1/d) finite where a skipped block holds a pole
          acc[r] = fmaf(num, bartw::rcp_approx(fmaxf(fmaf(u, u, q2), 1e-30f)), acc[r]);
        }
      }
    }

    // ---- fixup: the excluded blocks of each line, lanes take consecutive points
    unsigned m = fix_mask;
    while (m) {
      const int l = __ffs(m) - 1;
      m &= m - 1;
      const LineC c = sl[l];
      const int a = max(w0 + c.e0 * OP_R, c.jlo);
      const int b = min(min(w0 + c.e1 * OP_R + OP_R - 1, c.jhi), last);
      for (int p = a + lane; p <= b; p += 32) {
        const float x = fmaf((float)(p - c.jc), c.dx, c.xc);
        const float u = fmaf(x, x, c.qm);
        float v;
        if (u >= U_CORE) v = fmaf(c.A, u, c.A) * bartw::rcp_approx(fmaf(u, u, c.q2));
        else v = c.B * bartw::core_re(x, c.y, wtab);
        fix[p - w0] += v;
      }
      __syncwarp();          // the next line's lanes may touch the same points
    }
    __syncwarp();            // staged constants are reused by the next chunk

    // fold partial sums into the compensated pair every 4 chunks (TwoSum)
    if (++chunks == 4 || base + 32 >= rg.i_hi) {
      chunks = 0;
#pragma unroll
      for (int r = 0; r < OP_R; ++r) {
        const float s = hi[r] + acc[r];
        const float bp = s - hi[r];
        lo[r] += (hi[r] - (s - bp)) + (acc[r] - bp);
        hi[r] = s;
        acc[r] = 0.f;
      }
    }
  }
  __syncwarp();

  // ---- store
#pragma unroll
  for (int r = 0; r < OP_R; ++r) {
    const int64_t j = (int64_t)j0 + r;
    if (j < n_nu) out[(int64_t)cell * n_nu + j] = ((hi[r] + lo[r]) + fix[lane * OP_R + r]) * INV_SCALE;
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
  void *p_jlo, *p_jhi, *p_win, *p_cells, *p_spans;
  size_t nl = (size_t)std::max<int64_t>(max_lines, 1);
  const int64_t n_tiles = (nu.n_nu + OP_TILE - 1) / OP_TILE;
  const int n_spans = (int)(n_tiles * OP_WARPS);
  if ((st = bart_scratch(ctx, "op_jlo", nl * sizeof(int), &p_jlo)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "op_jhi", nl * sizeof(int), &p_jhi)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "op_win", nl * sizeof(LineWin), &p_win)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "op_spans", (size_t)n_spans * sizeof(SpanRange), &p_spans)) != BART_OK) return st;

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

  for (int s = 0; s < n_species; ++s) {
    const bart_linelist& L = species[s];
    float* o = out + (int64_t)s * n_cells * nu.n_nu;
    if (L.n_lines > 0) {
      line_window_kernel<<<(unsigned)((L.n_lines + 255) / 256), 256, 0, ctx->stream>>>(
          L.nu0_cm, L.log10_s296, L.elow_cm, L.n_lines, nu.nu_start_cm, nu.dnu_cm, nu.n_nu, cutoff, (int*)p_jlo,
          (int*)p_jhi, (LineWin*)p_win);
      if ((st = bart_check_launch(ctx, "line_window_kernel")) != BART_OK) return st;
    }
    span_range_kernel<<<(n_spans + 127) / 128, 128, 0, ctx->stream>>>((const int*)p_jlo, (const int*)p_jhi,
                                                                      L.n_lines, n_spans, (SpanRange*)p_spans);
    if ((st = bart_check_launch(ctx, "span_range_kernel")) != BART_OK) return st;
    dim3 grid((unsigned)n_tiles, (unsigned)n_cells);
    opacity_kernel<<<grid, OP_THREADS, 0, ctx->stream>>>(
        (const LineWin*)p_win, L.gamma_ref_cm, (const SpanRange*)p_spans,
        (const CellConst*)p_cells + (size_t)s * n_cells, nu.dnu_cm, nu.n_nu, o, ctx->d_wtable);
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
