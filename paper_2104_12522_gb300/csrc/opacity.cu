// Line-by-line opacity (Sec. 3 and Sec. 4 items 3-4): for every species and
// every (P, T) cell, the sum over lines of S(T) V(nu_j - nu0) on the output
// grid, each line cut off at |nu_j - nu0| <= cutoff and point-sampled at the
// grid wavenumbers (Sec. 4, text after the list of optimisations).
//
// Design (GB300, bound by FP32 instruction issue):
//  * A prologue finds, per line and in FP64, the grid-index window of its
//    cutoff [jlo, jhi], the nearest grid index jc and the offset
//    delta = nu_jc - nu0 (all differences taken as (nu_start + j dnu) - nu0),
//    and the temperature-free part of ln S.  A second prologue finds, per
//    512-point warp span, the range of lines whose windows meet it (binary
//    searches on the monotone windows).
//  * A CTA holds 8 independent warps, each one (cell, 512-point span).  A warp
//    walks its own line range 32 lines at a time: each lane computes one
//    line's cell-dependent constants (strength, widths, core window, lane
//    mask, class) and stores them, sorted by class, in warp-private shared
//    memory.  No CTA-wide barrier.
//  * Each lane owns 16 consecutive points and keeps their partial sums in
//    registers.  The offset x = (j - jc) dnu / (sigma sqrt 2) + delta /
//    (sigma sqrt 2) is formed from exact integer differences, so it stays
//    relatively accurate near the core.
//  * Far field: lines far from the whole span by a degree-5 expansion of
//    their shifted Lorentz term about each lane's block centre (coefficients
//    summed over lines, expanded once per chunk); otherwise, where x^2 + y^2
//    is large enough, the shifted Lorentz form with two lines per reciprocal;
//    elsewhere outside the core the one-pole form.  These loops work on two
//    points at a time with the packed FP32 instructions of sm_100+
//    (__ffma2_rn, __fmul2_rn, __fadd2_rn: two lanes of arithmetic per issue).
//    Lines covering the whole span run without any per-lane weight; the
//    others take a per-lane weight from a lane mask.
//  * Blocks of 16 points holding a window edge, a short stretch where the
//    far-field forms are not accurate enough, or a line's core (|z| < 24) go
//    to a fixup pass.  Lines with one-pole points only: lanes take the points
//    of their blocks and sum over the lines in registers (one add per point).
//    Lines with a core: point by point; where y <= 0.02 (Doppler-dominated
//    cells) one branch-free form over the line's whole range (the expansion
//    of Re w in y about the real axis), elsewhere core points gathered into
//    two per-warp lists (Taylor table, continued fraction) and evaluated 32
//    at a time, so lanes do not diverge across the branches.  All fixup sums go to
//    a warp-private accumulator in a fixed order: deterministic.
//  * Partial sums are plain FP32 over 4 chunks of 32 lines and folded into a
//    TwoSum (hi, lo) pair per point kept in shared memory: compensated
//    accumulation.
//  * All arithmetic runs at a 2^100 scale so far-wing terms of weak lines stay
//    normal FP32 numbers (and products of two denominators stay in range);
//    the result is scaled back on the store.
#include <algorithm>
#include <cmath>
#include <cstddef>

#include "bart_internal.cuh"
#include "faddeeva.cuh"

namespace {

constexpr int OP_WARPS = 8;                      // independent warps per CTA
constexpr int OP_THREADS = 32 * OP_WARPS;
constexpr int OP_R = 16;                         // points per lane
constexpr int OP_R_LOG = 4;
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

// ln S(T) = ln_s0 + 1.5 ln(T_ref/T) - c2 E''/T + ln(1 - exp(-c2 nu0/T)), in FP32
// (the staging of the opacity kernel and the threshold prologue share it).
__device__ __forceinline__ float line_ln_s(const LineWin& w, const CellConst& cc) {
  const float stim = 1.0f - ex2f_approx(-w.c2nu * cc.inv_t * LOG2EF);
  return w.ln_s0 + cc.ln_q - w.c2e * cc.inv_t + LN2F_ * lg2f_approx(stim);
}

// Order-preserving map of floats to ints (for atomicMax on floats).
__device__ __forceinline__ int ordered_int(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Largest ln S(T) of a species' lines at each temperature (Sec. 4 item 6:
// the line-strength bound is relative to the strongest line at each cell; S
// depends on T only).  smax[blockIdx.y] must start at a very negative
// ordered value.
__global__ void line_smax_kernel(const LineWin* __restrict__ win, int64_t n_lines,
                                 const CellConst* __restrict__ cells, int* __restrict__ smax) {
  const CellConst cc = cells[blockIdx.y];
  float m = -3.0e38f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_lines; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, line_ln_s(win[i], cc));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float s_m[32];
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? s_m[threadIdx.x] : -3.0e38f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(&smax[blockIdx.y], ordered_int(m));
  }
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

// Per-line constants of the current cell, staged per warp in four 16-byte
// groups (structure of arrays, so the staging stores are conflict free).
struct __align__(16) LineG0 {   // every far-field loop
  float dx;                     // dnu / (sigma sqrt 2)
  float xc;                     // (nu_jc - nu0) / (sigma sqrt 2)
  float A;                      // B y / sqrt(pi) (scaled)
  float jcr;                    // jc - w0 (exact below 2^24)
};
struct __align__(16) LineG1 {   // far-field denominators and the lane mask
  float qm;                     // y^2 - 1/2  (one-pole form)
  float q2;                     // 2 y^2      (one-pole form)
  float qL;                     // y^2 - 3/2  (shifted Lorentz form)
  unsigned take;                // lanes whose 16-point block joins the far-field sum
};
struct __align__(16) LineG2 {   // fixup range
  int pa, pb;                   // points [pa, pb] left to the fixup pass (blocks [e0, e1] in the window)
  int ka, kb;                   // their part inside the core window (lines with a core in the span)
};
struct __align__(8) LineG3 {    // accurate branch (expansion lines: -2 dx, dx^2)
  float y;
  float B;                      // S / (sigma sqrt(2 pi)) (scaled): V = B Re w
};

// Far-field classes of a (line, span) pair.  "L": every far-field point of
// the span (points too close to the line go to the fixup when there are at
// most LFIX_MAX of them) has x^2 + y^2 large enough for the shifted Lorentz form
//   Re w = (y/sqrt pi) / (x^2 + y^2 - 3/2)
// (the asymptotic series w ~ (i/sqrt pi)(1/z + 1/(2 z^3) + ...) to second
// order: relative error (2 y^2 + 3/2) / (x^2 + y^2)^2 to leading order, at most
// 0.6% more; the selection keeps it <= EPS_L with a 0.1% margin on x^2 + y^2);
// "P": the one-pole form.  "F": the window covers the whole span and no block
// is left to the fixup (no per-lane weight); "M": the lane weight is taken
// from the line's lane mask.
constexpr int CLS_FF = 4, CLS_LF = 0, CLS_LM = 1, CLS_PF = 2, CLS_PM = 3;
constexpr int CLS_F2 = 5, CLS_F4 = 6, CLS_F8 = 7;   // expansion about a block of G = 2, 4, 8 lanes
// "FF": every point of the span lies at |x| >= FF_RATIO dx from the line (and
// the shifted Lorentz form holds there): the line's contribution to a lane's
// 16 points is expanded to degree FF_DEG in the point offset t about the
// block centre, f(t) = (A/s) sum_n P_n t^n with s = xc^2 + y^2 - 3/2,
// alpha = 2 xc dx / s, beta = dx^2 / s, P_0 = 1, P_1 = -alpha,
// P_n = -alpha P_{n-1} - beta P_{n-2}; truncation error <= 2.6e-6 relative for
// |xc| >= 12 h (h = 7.5 dx, half a block), i.e. |x| >= 11 h on the block.
// The lane sums the coefficients over lines and expands them once per chunk.
// Lines farther away are expanded about the centre of a group of G = 2, 4 or
// 8 lanes (h = (16 G - 1) dx / 2, the same bound with |x| >= 11 h on the
// group's points) when their lane mask is uniform over each group: each lane
// of a group takes every G-th such line, the group adds its coefficients by
// shuffles, and each lane moves the polynomial to its own block centre
// (Taylor shift), so one line costs 1/G of a lane's work.
constexpr int FF_DEG = 5;
constexpr float FF_RATIO = 11.0f * 0.5f * (OP_R - 1);
__host__ __device__ constexpr float ff_ratio(int G) { return 11.0f * 0.5f * (G * OP_R - 1); }
constexpr float EPS_L = 2e-6f;
constexpr int LFIX_MAX = 64;              // longest stretch of one-pole points moved to the fixup
constexpr float FAR_X = 1.0e4f;           // x of lanes with weight 0 in the lane-mask Lorentz loop
constexpr int CORE_CAP = 352;             // deferred accurate points per warp before a flush
constexpr int ENT_SHIFT = 9;              // list entry: point in span (9 bits) | line slot << 9
static_assert(OP_SPAN <= (1 << ENT_SHIFT), "list entries hold a point of the span");

// Warp-private shared memory of the opacity kernel (dynamic: above the 48 KB
// static limit).  Line constants are structure-of-arrays so the staging
// stores are conflict free; the compensated pair is [point r][lane].
struct OpShared {
  float4 g0[OP_WARPS][32];
  float4 g1[OP_WARPS][32];
  int4 g2[OP_WARPS][32];
  float2 g3[OP_WARPS][32];
  float fix[OP_WARPS][OP_SPAN];
  float hi[OP_WARPS][OP_R][32];
  float lo[OP_WARPS][OP_R][32];
  unsigned list[OP_WARPS][CORE_CAP];
  int eidx[OP_WARPS][32];             // one-pole-only fixups: slot | first block << 5 | last block << 10
};

__device__ __forceinline__ unsigned lane_range_mask(int a, int b) {   // bits a..b, empty if a > b
  a = max(a, 0);
  b = min(b, 31);
  if (a > b) return 0u;
  const unsigned hi = (b == 31) ? 0xffffffffu : ((1u << (b + 1)) - 1u);
  return hi & ~((1u << a) - 1u);
}

// Expansion coefficients of lines [l0, l0 + n) about the centre of the lane's
// group of G lanes (16 G points); lane u of a group takes lines l0 + u,
// l0 + u + G, ...  Lines of this group size have a lane mask that is uniform
// over the group.
template <int G>
__device__ __forceinline__ void ff_lines(float (&C)[FF_DEG + 1], const float4* g0, const float4* g1,
                                         const float2* g3, int l0, int n, int lane) {
  const float tcg = (float)((lane & ~(G - 1)) * OP_R) + 0.5f * (G * OP_R - 1);
  for (int i = l0 + (lane & (G - 1)); i < l0 + n; i += G) {
    const float4 a = g0[i];
    const float4 b = g1[i];
    const float2 d = g3[i];                 // -2 dx, dx^2
    const float A = ((__float_as_uint(b.w) >> lane) & 1u) ? a.z : 0.0f;
    const float xc = fmaf(tcg - a.w, a.x, a.y);
    const float g = bartw::rcp_approx(fmaf(xc, xc, b.z));
    const float al = xc * g * d.x;          // -alpha
    const float be = d.y * g;               // beta
    const float Ag = A * g;
    float pm1 = 1.0f, pn = al;              // P_0, P_1
    C[0] += Ag;
    C[1] = fmaf(Ag, pn, C[1]);
#pragma unroll
    for (int k = 2; k <= FF_DEG; ++k) {
      const float pk = fmaf(al, pn, -be * pm1);
      pm1 = pn;
      pn = pk;
      C[k] = fmaf(Ag, pk, C[k]);
    }
  }
}

// Adds the partial sums over lane bit G/2 (the two halves of a group of G)
// and moves the polynomial from the group's centre to the centre of the
// lane's half: p(t) -> p(t + delta), delta = centre(G/2) - centre(G), by the
// Horner form of the Taylor shift.
template <int G>
__device__ __forceinline__ void ff_fold(float (&C)[FF_DEG + 1], int lane) {
#pragma unroll
  for (int k = 0; k <= FF_DEG; ++k) C[k] += __shfl_xor_sync(0xffffffffu, C[k], G / 2);
  const float c_g = (float)((lane & ~(G - 1)) * OP_R) + 0.5f * (G * OP_R - 1);
  const float c_h = (float)((lane & ~(G / 2 - 1)) * OP_R) + 0.5f * ((G / 2) * OP_R - 1);
  const float delta = c_h - c_g;
#pragma unroll
  for (int i = 0; i < FF_DEG; ++i) {
#pragma unroll
    for (int j = FF_DEG - 1; j >= i; --j) C[j] = fmaf(delta, C[j + 1], C[j]);
  }
}

// Far-field loops over the lane's 16 points, two points per packed FP32
// instruction (__ffma2_rn and friends: sm_100+).  x advances by 2 dx per
// pair (x_{r+2} = x_r + 2 dx): with |x| below 50 across a block the rounding
// this adds to s = x^2 + y^2 - 3/2 stays below 1e-6 relative where s >= 866.
// far != 0 moves the line to x = FAR_X (a lane that takes no weight).
__device__ __forceinline__ float2 pair_x0(float j0r, const float4& a, float far) {
  const float x0 = far != 0.0f ? FAR_X : fmaf(j0r - a.w, a.x, a.y);
  const float dx = far != 0.0f ? 0.0f : a.x;
  return make_float2(x0, x0 + dx);
}

// Two shifted-Lorentz lines per reciprocal: A1/s1 + A2/s2 = (A1 s2 + A2 s1) / (s1 s2).
__device__ __forceinline__ void lorentz_pair(float2 (&acc)[OP_R / 2], float j0r, const float4& a, const float4& a2,
                                             float A, float A2, float q, float q2, float far, float far2) {
  float2 X = pair_x0(j0r, a, far), X2 = pair_x0(j0r, a2, far2);
  const float2 D = make_float2(far != 0.0f ? 0.0f : 2.0f * a.x, far != 0.0f ? 0.0f : 2.0f * a.x);
  const float2 D2 = make_float2(far2 != 0.0f ? 0.0f : 2.0f * a2.x, far2 != 0.0f ? 0.0f : 2.0f * a2.x);
  const float2 Q = make_float2(q, q), Q2 = make_float2(q2, q2);
  const float2 AA = make_float2(A, A), AA2 = make_float2(A2, A2);
#pragma unroll
  for (int r = 0; r < OP_R / 2; ++r) {
    const float2 s1 = __ffma2_rn(X, X, Q), s2 = __ffma2_rn(X2, X2, Q2);
    const float2 num = __ffma2_rn(AA2, s1, __fmul2_rn(AA, s2));
    const float2 den = __fmul2_rn(s1, s2);
    const float2 inv = make_float2(bartw::rcp_approx(den.x), bartw::rcp_approx(den.y));
    acc[r] = __ffma2_rn(num, inv, acc[r]);
    X = __fadd2_rn(X, D);
    X2 = __fadd2_rn(X2, D2);
  }
}

__device__ __forceinline__ void lorentz_one(float2 (&acc)[OP_R / 2], float j0r, const float4& a, float A, float q,
                                            float far) {
  float2 X = pair_x0(j0r, a, far);
  const float2 D = make_float2(far != 0.0f ? 0.0f : 2.0f * a.x, far != 0.0f ? 0.0f : 2.0f * a.x);
  const float2 Q = make_float2(q, q), AA = make_float2(A, A);
#pragma unroll
  for (int r = 0; r < OP_R / 2; ++r) {
    const float2 s = __ffma2_rn(X, X, Q);
    const float2 inv = make_float2(bartw::rcp_approx(s.x), bartw::rcp_approx(s.y));
    acc[r] = __ffma2_rn(AA, inv, acc[r]);
    X = __fadd2_rn(X, D);
  }
}

// One-pole form A (u + 1) / (u^2 + 2 y^2), u = x^2 + y^2 - 1/2; CLAMP keeps
// the denominator >= 1e-30.
template <bool CLAMP>
__device__ __forceinline__ void one_pole(float2 (&acc)[OP_R / 2], float j0r, const float4& a, float A, float qm,
                                         float q2) {
  float2 X = pair_x0(j0r, a, 0.0f);
  const float2 D = make_float2(2.0f * a.x, 2.0f * a.x);
  const float2 QM = make_float2(qm, qm), Q2 = make_float2(q2, q2), AA = make_float2(A, A);
#pragma unroll
  for (int r = 0; r < OP_R / 2; ++r) {
    const float2 u = __ffma2_rn(X, X, QM);
    const float2 num = __ffma2_rn(AA, u, AA);
    const float2 den = __ffma2_rn(u, u, Q2);
    const float2 inv = CLAMP ? make_float2(bartw::rcp_approx(fmaxf(den.x, 1e-30f)), bartw::rcp_approx(fmaxf(den.y, 1e-30f)))
                             : make_float2(bartw::rcp_approx(den.x), bartw::rcp_approx(den.y));
    acc[r] = __ffma2_rn(num, inv, acc[r]);
    X = __fadd2_rn(X, D);
  }
}

// Each lane owns one 16-point block of the warp's 512-point span.  For a line,
// a block goes through a branch-free far-field loop if it lies entirely in
// the cutoff window and outside the line's fixup stretch; the remaining blocks
// with points in the window (the block holding a window edge, the blocks the
// stretch touches, and any blocks between them) form one interval [e0, e1]
// that the fixup pass evaluates point by point, lanes = points: the one-pole
// form outside the core window [klo, khi], the closed form of the continued
// fraction to depth 2 for |z| >= 14 inside it, and the rest deferred into two
// per-warp lists (Taylor table for |z| < 5, continued fraction to depth 6 for
// 5 <= |z| < 14) that are evaluated 32 points at a time.  Each (line, point)
// is counted once.
__global__ void __launch_bounds__(OP_THREADS, 3)
opacity_kernel(const LineWin* __restrict__ win, const float* __restrict__ gref,
               const SpanRange* __restrict__ spans, const CellConst* __restrict__ cells, double dnu,
               int64_t n_nu, float* __restrict__ out, const float2* __restrict__ wtab,
               const int* __restrict__ smax, const int* __restrict__ tmap, float ln_rel) {
  extern __shared__ __align__(16) unsigned char op_smem[];
  OpShared& sh = *reinterpret_cast<OpShared*>(op_smem);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w0l = ((int64_t)blockIdx.x * OP_WARPS + warp) * OP_SPAN;
  if (w0l >= n_nu) return;                  // warps are independent: no CTA barrier below
  const int w0 = (int)w0l, w1 = w0 + OP_SPAN - 1;
  const int j0 = w0 + lane * OP_R;          // first point of this lane
  const float j0r = (float)(lane * OP_R);   // its offset in the span
  const int cell = blockIdx.y;
  const CellConst cc = cells[cell];
  // line-strength bound: lines with ln S below this are left out
  const float ln_thr = smax ? ordered_float(smax[tmap[cell]]) + ln_rel : -3.0e38f;
  const SpanRange rg = spans[blockIdx.x * OP_WARPS + warp];
  const int last = (int)min((int64_t)w1, n_nu - 1);
  const unsigned lt_mask = (1u << lane) - 1u;

  float* fix = sh.fix[warp];
  unsigned* list = sh.list[warp];
  int* eidx = sh.eidx[warp];
  float4* g0 = sh.g0[warp];
  float4* g1 = sh.g1[warp];
  int4* g2 = sh.g2[warp];
  float2* g3 = sh.g3[warp];
#pragma unroll
  for (int r = 0; r < OP_R; ++r) fix[lane * OP_R + r] = 0.0f;

  float (*hi)[32] = sh.hi[warp];
  float (*lo)[32] = sh.lo[warp];
  // far-field sums of the lane's points, as pairs (r, r+1) for the packed
  // FP32 instructions of sm_100+ (two lanes of arithmetic per issue)
  float2 acc[OP_R / 2];
#pragma unroll
  for (int r = 0; r < OP_R; ++r) { hi[r][lane] = 0.f; lo[r][lane] = 0.f; }
#pragma unroll
  for (int r = 0; r < OP_R / 2; ++r) acc[r] = make_float2(0.f, 0.f);

  const float dnuf = (float)dnu;
  int chunks = 0;
  int nT = 0, nC = 0;                       // deferred Taylor / continued-fraction points

  // Evaluates the deferred accurate points and adds them to the fixup
  // accumulator.  Entries are in (line, point) order; one line never repeats
  // a point, so a group of 32 is added in rounds of equal line (ascending):
  // deterministic.
  auto flush = [&]() {
    __syncwarp();            // immediate fixup adds are visible to every lane
    for (int pass = 0; pass < 2; ++pass) {
      const int n = pass == 0 ? nT : nC;
      for (int g = 0; g < n; g += 32) {
        const int k = g + lane;
        const bool act = k < n;
        const unsigned e = act ? list[pass == 0 ? k : CORE_CAP - 1 - k] : 0u;
        const int l = (int)(e >> ENT_SHIFT), p = (int)(e & (OP_SPAN - 1));
        const float4 c0 = g0[l];
        const float2 c3 = g3[l];
        // idle lanes evaluate a harmless point (|z| = 6) and add nothing
        const float x = act ? fabsf(fmaf((float)p - c0.w, c0.x, c0.y)) : 6.0f;
        const float y = act ? c3.x : 0.0f;
        float v;
        if (pass == 0) {
          v = bartw::taylor_re<1>(x, y, wtab);
        } else {
          v = bartw::cf_gauss_re(x, y, 6);
        }
        v *= c3.y;
        const int lp = __shfl_up_sync(0xffffffffu, l, 1);
        unsigned seg = __ballot_sync(0xffffffffu, act && (lane == 0 || l != lp));
        while (seg) {
          const int s0 = __ffs(seg) - 1;
          seg &= seg - 1;
          const int s1 = seg ? __ffs(seg) - 1 : 32;
          if (act && lane >= s0 && lane < s1) fix[p] += v;
          __syncwarp();
        }
      }
    }
    nT = 0;
    nC = 0;
  };

  for (int64_t base = rg.i_lo; base < rg.i_hi; base += 32) {
    const int nl = (int)min((int64_t)32, rg.i_hi - base);
    // ---- stage: one line's cell-dependent constants per lane, its class,
    // and its slot (lines sorted by class)
    int cls = -1;
    bool needs_fix = false, has_core = false;
    int eb0 = 0, eb1 = 0;                   // blocks [eb0, eb1] of the line's fixup range
    float4 c0, c1;
    int4 c2;
    float2 c3;
    if (lane < nl) {
      const int64_t i = base + lane;
      const LineWin w = win[i];
      const float inv = bartw::rcp_approx(w.nu0f * cc.dfac);   // 1 / (sigma sqrt 2)
      const float y = gref[i] * cc.gfac * inv;
      const float q = y * y;
      const float ln_s = line_ln_s(w, cc);
      const bool keep = ln_s >= ln_thr;
      const float B = ex2f_approx((ln_s + LN_SCALE) * LOG2EF) * inv * bartw::INV_SQRTPI;
      const float dx = dnuf * inv, xc = w.delta * inv;
      const int jcr = w.jc - w0;
      // Integer supersets (two extra points on each side) of the points with
      // x^2 + y^2 < R2 on the grid, for R2 = 576 (the core) and for
      // R2 = S_L = sqrt((2 y^2 + 3/2) / EPS_L), where the shifted Lorentz form
      // is not accurate enough (S_L >= 866 > 576: it contains the core).
      const float rdx = bartw::rcp_approx(dx);
      auto window = [&](float R2, int& lo, int& hi) {
        lo = 0x7fffffff;
        hi = -0x7fffffff;
        if (q < R2) {
          const float X = sqrtf(R2 - q);
          const float lo_f = fmaxf(floorf((-X - xc) * rdx) - 2.0f, -1073741824.0f);
          const float hi_f = fminf(ceilf((X - xc) * rdx) + 2.0f, 1073741824.0f);
          lo = (int)max((long long)w.jc + (long long)lo_f, -1073741824LL);
          hi = (int)min((long long)w.jc + (long long)hi_f, 1073741824LL);
        }
      };
      const int a = max(w.jlo, w0), b = min(w.jhi, last);
      int klo, khi, ilo, ihi;
      window(CORE_S, klo, khi);
      has_core = max(klo, a) <= min(khi, b);
      window(sqrtf(fmaf(2.0f, q, 1.5f) * (1.0f / EPS_L)) * 1.001f, ilo, ihi);
      // A short stretch of such points in the span joins the fixup (one-pole
      // form there) and the rest of the span takes the shifted Lorentz form;
      // a long one makes the whole span one-pole, with only the core fixed up.
      const bool lor = min(ihi, b) - max(ilo, a) < LFIX_MAX;
      const int flo = lor ? ilo : klo, fhi = lor ? ihi : khi;
      // blocks for the fixup pass: window edges inside the span, the stretch above
      int e0 = 32, e1 = -1;
      if (a <= b) {
        if (a > w0 && ((a - w0) & (OP_R - 1))) { e0 = min(e0, (a - w0) >> OP_R_LOG); e1 = max(e1, (a - w0) >> OP_R_LOG); }
        if ((b < w1) && (((b - w0) & (OP_R - 1)) != OP_R - 1)) {
          e0 = min(e0, (b - w0) >> OP_R_LOG);
          e1 = max(e1, (b - w0) >> OP_R_LOG);
        }
        const int ca = max(flo, a), cb = min(fhi, b);
        if (ca <= cb) { e0 = min(e0, (ca - w0) >> OP_R_LOG); e1 = max(e1, (cb - w0) >> OP_R_LOG); }
      }
      needs_fix = e0 <= e1;
      has_core = has_core && needs_fix;
      eb0 = e0;
      eb1 = e1;
      // lanes whose block lies in the window: jlo <= w0 + 16k and w0 + 16k + 15 <= jhi
      unsigned take = lane_range_mask((w.jlo - w0 + OP_R - 1) >> OP_R_LOG, (w.jhi - w0 - (OP_R - 1)) >> OP_R_LOG);
      if (needs_fix) take &= ~lane_range_mask(e0, e1);
      const bool full = take == 0xffffffffu;
      // the whole span far from the line: expansion class (needs the shifted
      // Lorentz bound at the span's closest point as well)
      const float xa = fmaf((float)(w0 - w.jc), dx, xc), xb = fmaf((float)(w1 - w.jc), dx, xc);
      const float xm = xa > 0.0f ? xa : (xb < 0.0f ? -xb : 0.0f);
      const float smin = fmaf(xm, xm, q);
      const bool ff = !has_core && xm >= FF_RATIO * dx && smin * smin * (EPS_L * 0.999f) >= fmaf(2.0f, q, 1.5f);
      int ffc = CLS_FF;
      if (ff) {
        // largest group with a uniform lane mask within each group of G lanes
        const bool u2 = (((take >> 1) ^ take) & 0x55555555u) == 0u;
        const bool u4 = u2 && (((take >> 2) ^ take) & 0x33333333u) == 0u;
        const bool u8 = u4 && (((take >> 4) ^ take) & 0x0f0f0f0fu) == 0u;
        if (u8 && xm >= ff_ratio(8) * dx) ffc = CLS_F8;
        else if (u4 && xm >= ff_ratio(4) * dx) ffc = CLS_F4;
        else if (u2 && xm >= ff_ratio(2) * dx) ffc = CLS_F2;
      }
      cls = ff ? ffc : lor ? (full ? CLS_LF : CLS_LM) : (full ? CLS_PF : CLS_PM);
      if (!keep) {                          // below the line-strength bound: no slot
        cls = -1;
        needs_fix = false;
        has_core = false;
      }
      c0 = make_float4(dx, xc, B * y * bartw::INV_SQRTPI, (float)jcr);
      c1 = make_float4(q - 0.5f, 2.0f * q, q - 1.5f, __uint_as_float(take));
      {
        // the fixup ranges, once per line here rather than per line in the fixup
        const int pa = max(w0 + e0 * OP_R, w.jlo);
        const int pb = min(min(w0 + e1 * OP_R + OP_R - 1, w.jhi), last);
        c2 = make_int4(pa, pb, max(pa, klo), min(pb, khi));
      }
      // expansion lines have no core in the span: their slot of the
      // accurate-branch group holds -2 dx and dx^2 instead
      c3 = ff ? make_float2(-2.0f * dx, dx * dx) : make_float2(y, B);
    }
    const unsigned bF8 = __ballot_sync(0xffffffffu, cls == CLS_F8);
    const unsigned bF4 = __ballot_sync(0xffffffffu, cls == CLS_F4);
    const unsigned bF2 = __ballot_sync(0xffffffffu, cls == CLS_F2);
    const unsigned bF1 = __ballot_sync(0xffffffffu, cls == CLS_FF);
    const unsigned bLF = __ballot_sync(0xffffffffu, cls == CLS_LF);
    const unsigned bLM = __ballot_sync(0xffffffffu, cls == CLS_LM);
    const unsigned bPF = __ballot_sync(0xffffffffu, cls == CLS_PF);
    const unsigned bPM = __ballot_sync(0xffffffffu, cls == CLS_PM);
    const int n8 = __popc(bF8), n4 = __popc(bF4), n2 = __popc(bF2), n1 = __popc(bF1);
    const int nFF = n8 + n4 + n2 + n1;      // all expansion lines (slots [0, nFF))
    const int nLF = __popc(bLF), nLM = __popc(bLM), nPF = __popc(bPF), nPM = __popc(bPM);
    int slot = -1;
    if (cls == CLS_F8) slot = __popc(bF8 & lt_mask);
    else if (cls == CLS_F4) slot = n8 + __popc(bF4 & lt_mask);
    else if (cls == CLS_F2) slot = n8 + n4 + __popc(bF2 & lt_mask);
    else if (cls == CLS_FF) slot = n8 + n4 + n2 + __popc(bF1 & lt_mask);
    else if (cls == CLS_LF) slot = nFF + __popc(bLF & lt_mask);
    else if (cls == CLS_LM) slot = nFF + nLF + __popc(bLM & lt_mask);
    else if (cls == CLS_PF) slot = nFF + nLF + nLM + __popc(bPF & lt_mask);
    else if (cls == CLS_PM) slot = nFF + nLF + nLM + nPF + __popc(bPM & lt_mask);
    if (slot >= 0) {
      g0[slot] = c0;
      g1[slot] = c1;
      g2[slot] = c2;
      g3[slot] = c3;
    }
    const unsigned fix_slots = __reduce_or_sync(0xffffffffu, (slot >= 0 && needs_fix) ? (1u << slot) : 0u);
    const unsigned core_slots = __reduce_or_sync(0xffffffffu, (slot >= 0 && has_core) ? (1u << slot) : 0u);
    // lines whose fixup holds one-pole points only (window edges, short
    // stretches): their slots and fixup blocks, in line order, and the blocks
    // they touch
    const bool edge_only = slot >= 0 && needs_fix && !has_core;
    const unsigned b_edge = __ballot_sync(0xffffffffu, edge_only);
    const int n_edge = __popc(b_edge);
    if (edge_only) eidx[__popc(b_edge & lt_mask)] = slot | (eb0 << 5) | (eb1 << 10);
    const unsigned e_blocks = __reduce_or_sync(0xffffffffu, edge_only ? lane_range_mask(eb0, eb1) : 0u);
    __syncwarp();

    // ---- far field.  The shifted Lorentz classes take two lines per
    // reciprocal, A1/s1 + A2/s2 = (A1 s2 + A2 s1) / (s1 s2): the MUFU pipe
    // (a quarter of the issue rate) would otherwise bind at one reciprocal
    // in four instructions.  s >= 866 here, so s1 s2 stays far inside the
    // FP32 range at the 2^100 scale.
    int l = 0;
    if (nFF > 0) {                          // expansion class: coefficient sums
      float C[FF_DEG + 1];
#pragma unroll
      for (int k = 0; k <= FF_DEG; ++k) C[k] = 0.0f;
      // groups of 8, 4, 2 lanes, then single lanes: after a group size's lines,
      // the partial sums are added over the next lane bit and moved to the
      // centre of the next smaller group, so every group's sum is complete and
      // centred on the lane's own block at the end
      if (n8 > 0) ff_lines<8>(C, g0, g1, g3, 0, n8, lane);
      if (n8 > 0) ff_fold<8>(C, lane);
      if (n4 > 0) ff_lines<4>(C, g0, g1, g3, n8, n4, lane);
      if (n8 + n4 > 0) ff_fold<4>(C, lane);
      if (n2 > 0) ff_lines<2>(C, g0, g1, g3, n8 + n4, n2, lane);
      if (n8 + n4 + n2 > 0) ff_fold<2>(C, lane);
      ff_lines<1>(C, g0, g1, g3, n8 + n4 + n2, n1, lane);
      l = nFF;
#pragma unroll
      for (int r = 0; r < OP_R; r += 2) {   // expand at the lane's 16 points, two at a time
        const float2 t = make_float2((float)r - 0.5f * (OP_R - 1), (float)(r + 1) - 0.5f * (OP_R - 1));
        float2 v = make_float2(C[FF_DEG], C[FF_DEG]);
#pragma unroll
        for (int k = FF_DEG - 1; k >= 0; --k) v = __ffma2_rn(v, t, make_float2(C[k], C[k]));
        acc[r >> 1] = __fadd2_rn(acc[r >> 1], v);
      }
    }
    const int eLF = nFF + nLF;
    for (; l + 1 < eLF; l += 2) {           // shifted Lorentz, whole span
      const float4 a = g0[l], a2 = g0[l + 1];
      const float qL = g1[l].z, qL2 = g1[l + 1].z;
      lorentz_pair(acc, j0r, a, a2, a.z, a2.z, qL, qL2, 0.0f, 0.0f);
    }
    if (l < eLF) {                          // odd line out
      const float4 a = g0[l];
      const float qL = g1[l].z;
      lorentz_one(acc, j0r, a, a.z, qL, 0.0f);
      ++l;
    }
    const int eLM = eLF + nLM;
    for (; l + 1 < eLM; l += 2) {           // shifted Lorentz, lane weight
      const float4 a = g0[l], a2 = g0[l + 1];
      const float4 b = g1[l], b2 = g1[l + 1];
      const bool t1 = (__float_as_uint(b.w) >> lane) & 1u, t2 = (__float_as_uint(b2.w) >> lane) & 1u;
      const float A = t1 ? a.z : 0.0f, A2 = t2 ? a2.z : 0.0f;
      // a lane with weight 0 may hold points of the fixup stretch (small s):
      // it evaluates far-away points instead (x = FAR_X)
      lorentz_pair(acc, j0r, a, a2, A, A2, b.z, b2.z, t1 ? 0.0f : 1.0f, t2 ? 0.0f : 1.0f);
    }
    if (l < eLM) {
      const float4 a = g0[l];
      const float4 b = g1[l];
      const bool t1 = (__float_as_uint(b.w) >> lane) & 1u;
      const float A = t1 ? a.z : 0.0f;
      lorentz_one(acc, j0r, a, A, b.z, t1 ? 0.0f : 1.0f);
      ++l;
    }
    const int ePF = eLM + nPF;
#pragma unroll 2
    for (; l < ePF; ++l) {                  // one-pole, whole span
      const float4 a = g0[l];
      const float4 b = g1[l];
      one_pole<false>(acc, j0r, a, a.z, b.x, b.y);
    }
    const int ePM = ePF + nPM;
    for (; l < ePM; ++l) {                  // one-pole, lane weight
      const float4 a = g0[l];
      const float4 b = g1[l];
      const float A = ((__float_as_uint(b.w) >> lane) & 1u) ? a.z : 0.0f;
      // the clamp keeps 0 * (1/d) finite where a skipped block holds a pole
      one_pole<true>(acc, j0r, a, A, b.x, b.y);
    }

    // ---- fixup: the excluded blocks of each line.  One-pole-only lines:
    // lanes take the 16 points of two touched blocks (or of one block, the
    // halves taking alternate lines), loop over the lines touching them and
    // keep the sum in a register (points outside a line's range add 0); each
    // point is then added once: deterministic, no conflicting adds
    if (e_blocks) {
      const int ek = lane < n_edge ? eidx[lane] : -1;
      const int ke0 = ek < 0 ? 64 : (ek >> 5) & 31, ke1 = ek < 0 ? -1 : (ek >> 10) & 31;
      const int half = lane >> 4;
      unsigned bm = e_blocks;
      while (bm) {
        const int b0 = __ffs(bm) - 1;
        bm &= bm - 1;
        int b1 = -1;
        if (bm) {
          b1 = __ffs(bm) - 1;
          bm &= bm - 1;
        }
        const bool split = b1 < 0;
        unsigned lm = __ballot_sync(0xffffffffu, (ke0 <= b0 && b0 <= ke1) || (ke0 <= b1 && b1 <= ke1));
        const int pr = ((split || half == 0) ? b0 : b1) * OP_R + (lane & (OP_R - 1));   // point in span
        const float pf = (float)pr;
        float v = 0.0f;
        while (lm) {
          int k = __ffs(lm) - 1;
          lm &= lm - 1;
          if (split) {
            const int k2 = lm ? __ffs(lm) - 1 : -1;
            if (lm) lm &= lm - 1;
            if (half) k = k2;
          }
          if (k >= 0) {
            const int sl = eidx[k] & 31;
            const float4 a = g0[sl];
            const float4 b = g1[sl];
            const int4 e = g2[sl];
            const float x = fmaf(pf - a.w, a.x, a.y);
            const float u = fmaf(x, x, b.x);
            const float t = fmaf(a.z, u, a.z) * bartw::rcp_approx(fmaf(u, u, b.y));
            const int p = w0 + pr;
            v += (p >= e.x && p <= e.y) ? t : 0.0f;
          }
        }
        if (split) v += __shfl_down_sync(0xffffffffu, v, 16);
        if (!split || half == 0) fix[pr] += v;
        __syncwarp();
      }
    }
    // lines with a core in the span
    unsigned m = core_slots;
    while (m) {
      const int fl = __ffs(m) - 1;
      m &= m - 1;
      const float4 a = g0[fl];
      const float4 b = g1[fl];
      const int4 e = g2[fl];
      const int pa = e.x, pb = e.y;
      const float2 c = g3[fl];
      if (c.x <= bartw::SMALL_Y) {
        // small y (Doppler-dominated cells): one branch-free form, the
        // expansion of Re w in y about the real axis, over the whole range,
        // core and wings alike; no deferred points
        for (int p = pa + lane; p <= pb; p += 32) {
          const float x = fabsf(fmaf((float)(p - w0) - a.w, a.x, a.y));
          fix[p - w0] += c.y * bartw::small_y_re(x, c.x, wtab);
        }
        __syncwarp();          // the next line's lanes may touch the same points
        continue;
      }
      // one-pole points on both sides of the core window [klo, khi]
      const int ka = e.z, kb = e.w;
      const int n_left = max(ka - pa, 0), n_far = n_left + max(pb - kb, 0);
      for (int k = lane; k < n_far; k += 32) {
        const int p = k < n_left ? pa + k : kb + 1 + (k - n_left);
        const float x = fmaf((float)(p - w0) - a.w, a.x, a.y);
        const float u = fmaf(x, x, b.x);
        fix[p - w0] += fmaf(a.z, u, a.z) * bartw::rcp_approx(fmaf(u, u, b.y));
      }
      // the core window: |z| >= 14 at once (closed form of the continued
      // fraction to depth 2), |z| < 14 deferred to the lists
      for (int p0 = ka; p0 <= kb; p0 += 32) {
        if (nT + nC + 32 > CORE_CAP) flush();
        const int p = p0 + lane;
        const bool act = p <= kb;
        const float x = fmaf((float)(p - w0) - a.w, a.x, a.y);
        const float u = fmaf(x, x, b.x);
        const bool mid = act && u >= 195.5f;               // |z| >= 14
        if (mid) fix[p - w0] += c.y * bartw::cf2_re(fabsf(x), c.x);
        const bool tay = act && u < 24.5f;                 // |z| < 5
        const bool cfr = act && !mid && !tay;
        const unsigned bt = __ballot_sync(0xffffffffu, tay);
        const unsigned bc = __ballot_sync(0xffffffffu, cfr);
        const unsigned ent = (unsigned)(p - w0) | ((unsigned)fl << ENT_SHIFT);
        if (tay) list[nT + __popc(bt & lt_mask)] = ent;
        if (cfr) list[CORE_CAP - 1 - (nC + __popc(bc & lt_mask))] = ent;
        nT += __popc(bt);
        nC += __popc(bc);
      }
      __syncwarp();          // the next line's lanes may touch the same points
    }
    if (nT + nC) flush();
    __syncwarp();            // staged constants are reused by the next chunk

    // fold partial sums into the compensated pair every 4 chunks (TwoSum)
    if (++chunks == 4 || base + 32 >= rg.i_hi) {
      chunks = 0;
#pragma unroll
      for (int r = 0; r < OP_R; ++r) {
        const float ar = (r & 1) ? acc[r >> 1].y : acc[r >> 1].x;
        const float h = hi[r][lane];
        const float s = h + ar;
        const float bp = s - h;
        lo[r][lane] += (h - (s - bp)) + (ar - bp);
        hi[r][lane] = s;
      }
#pragma unroll
      for (int r = 0; r < OP_R / 2; ++r) acc[r] = make_float2(0.f, 0.f);
    }
  }
  __syncwarp();

  // ---- store
#pragma unroll
  for (int r = 0; r < OP_R; ++r) {
    const int64_t j = (int64_t)j0 + r;
    if (j < n_nu) out[(int64_t)cell * n_nu + j] = ((hi[r][lane] + lo[r][lane]) + fix[lane * OP_R + r]) * INV_SCALE;
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
  BART_CUDA(ctx, cudaFuncSetAttribute(opacity_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(OpShared)));

  // line-strength bound (Sec. 4 item 6): the strongest line per cell first.
  // S depends on T only, so it is found once per distinct temperature.
  const bool thr = ctx->line_rel > 0.0;
  void *p_smax = nullptr, *p_tmap = nullptr, *p_tcells = nullptr;
  std::vector<double> tu;                   // distinct temperatures
  std::vector<int> tmap(n_cells);           // cell -> index in tu
  if (thr) {
    std::vector<int> first;                 // first cell of each distinct temperature
    for (int c = 0; c < n_cells; ++c) {
      auto it = std::find(tu.begin(), tu.end(), t[c]);
      tmap[c] = (int)(it - tu.begin());
      if (it == tu.end()) {
        tu.push_back(t[c]);
        first.push_back(c);
      }
    }
    std::vector<CellConst> hu((size_t)n_species * tu.size());
    for (int s = 0; s < n_species; ++s)
      for (size_t u = 0; u < tu.size(); ++u) hu[(size_t)s * tu.size() + u] = hc[(size_t)s * n_cells + first[u]];
    if ((st = bart_scratch(ctx, "op_smax", tu.size() * sizeof(int), &p_smax)) != BART_OK) return st;
    if ((st = bart_upload_const(ctx, "op_tmap", tmap.data(), tmap.size() * sizeof(int), &p_tmap)) != BART_OK)
      return st;
    if ((st = bart_upload_const(ctx, "op_tcells", hu.data(), hu.size() * sizeof(CellConst), &p_tcells)) != BART_OK)
      return st;
  }
  const float ln_rel = thr ? (float)std::log(ctx->line_rel) : 0.0f;

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
    if (thr) {
      // 0x80 bytes: an ordered value below every finite ln S
      BART_CUDA(ctx, cudaMemsetAsync(p_smax, 0x80, tu.size() * sizeof(int), ctx->stream));
      if (L.n_lines > 0) {
        const unsigned gx = (unsigned)std::min<int64_t>((L.n_lines + 255) / 256, 1024);
        line_smax_kernel<<<dim3(gx, (unsigned)tu.size()), 256, 0, ctx->stream>>>(
            (const LineWin*)p_win, L.n_lines, (const CellConst*)p_tcells + (size_t)s * tu.size(), (int*)p_smax);
        if ((st = bart_check_launch(ctx, "line_smax_kernel")) != BART_OK) return st;
      }
    }
    dim3 grid((unsigned)n_tiles, (unsigned)n_cells);
    opacity_kernel<<<grid, OP_THREADS, sizeof(OpShared), ctx->stream>>>(
        (const LineWin*)p_win, L.gamma_ref_cm, (const SpanRange*)p_spans,
        (const CellConst*)p_cells + (size_t)s * n_cells, nu.dnu_cm, nu.n_nu, o, ctx->d_wtable,
        thr ? (const int*)p_smax : nullptr, (const int*)p_tmap, ln_rel);
    if ((st = bart_check_launch(ctx, "opacity_kernel")) != BART_OK) return st;
  }
  return BART_OK;
}

// ------------------------------------------------------------------------
// The paper's own scheme (Sec. 4 items 4-5, Sec. 6.1.1): a precomputed table
// of Voigt profiles on a grid of Doppler and Lorentz widths, each sampled
// `oversample` times per grid interval and aligned to the grid; a line takes
// the profile of the nearest widths (in ln sigma and ln gamma), with its
// centre rounded to the nearest fine sample, and reads it at the grid points
// inside the same cutoff window as the direct sum.
//
// Layout: data[is][ig][r][k], r = 0 .. O-1 the fine offset, k = 0 .. 2 KK the
// grid offset, value V(((k - KK) + r / O) dnu; sigma_is, gamma_ig).  A line
// whose quantised centre is s fine samples from nu_start (s = jc O - r,
// 0 <= r < O) reads data[is][ig][r][j - jc + KK] at grid point j: a warp's
// consecutive points are consecutive floats.

__global__ void table_fill_kernel(float* __restrict__ data, int n_sigma, double ln_slo, double sstep, int n_gamma,
                                  double ln_glo, double gstep, int O, int kk, double dnu,
                                  const float2* __restrict__ wtab) {
  const int nk = 2 * kk + 1;
  const int64_t total = (int64_t)n_sigma * n_gamma * O * nk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % nk);
    int64_t rest = e / nk;
    const int r = (int)(rest % O);
    rest /= O;
    const int ig = (int)(rest % n_gamma);
    const int is = (int)(rest / n_gamma);
    const double sigma = exp(ln_slo + is * sstep), gamma = exp(ln_glo + ig * gstep);
    const double d = ((double)(k - kk) + (double)r / O) * dnu;
    const double inv = 1.0 / (sigma * 1.4142135623730951);
    const float v = bartw::faddeeva_re((float)(d * inv), (float)(gamma * inv), wtab);
    data[e] = (float)(v * inv * 0.56418958354775628695);   // Re w / (sigma sqrt(2 pi))
  }
}

struct TabLine {            // per line, cell independent
  double ln_nu0, ln_gref;   // for the nearest-width choice (FP64)
  int jc, r;                // quantised centre s = jc O - r
};

__global__ void table_line_kernel(const double* __restrict__ nu0, const float* __restrict__ gref, int64_t n_lines,
                                  double nu_start, double dnu, int O, TabLine* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_lines) return;
  const double c = nu0[i];
  const double big = 1073741824.0;
  const double s = fmin(fmax(floor((c - nu_start) * O / dnu + 0.5), -big * O), big * O);
  const double jc = ceil(s / O);
  TabLine t;
  t.ln_nu0 = log(c);
  t.ln_gref = log((double)gref[i]);
  t.jc = (int)jc;
  t.r = (int)(jc * O - s);
  out[i] = t;
}

struct TabCell {            // per (species, cell), FP64
  double ln_sfac;           // ln(sigma / nu0) = ln(sqrt(k T / m) / c)
  double ln_gfac;           // ln(gamma / gamma_ref) = ln(P sqrt(296 / T))
};

struct TabSpec {
  int n_sigma, n_gamma, O, kk;
  double ln_slo, inv_sstep, ln_glo, inv_gstep;
};

__device__ __forceinline__ int nearest_index(double v, double lo, double inv_step, int n) {
  if (n == 1) return 0;
  const double k = floor((v - lo) * inv_step + 0.5);
  return (int)fmin(fmax(k, 0.0), (double)(n - 1));
}

// One warp per (cell, 512-point span), lane l owns points w0 + 32 q + l
// (q = 0 .. 15, coalesced table reads); partial sums over 4 chunks of 32
// lines folded into a TwoSum pair; terms at the 2^100 scale as in the direct
// kernel.
__global__ void __launch_bounds__(OP_THREADS)
table_opacity_kernel(const LineWin* __restrict__ win, const TabLine* __restrict__ tl,
                     const SpanRange* __restrict__ spans, const CellConst* __restrict__ cells,
                     const TabCell* __restrict__ tcells, TabSpec ts, const float* __restrict__ data, int64_t n_nu,
                     float* __restrict__ out) {
  __shared__ long long s_row[OP_WARPS][32];
  __shared__ float s_S[OP_WARPS][32];
  __shared__ int2 s_win[OP_WARPS][32];
  __shared__ int s_kofs[OP_WARPS][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w0l = ((int64_t)blockIdx.x * OP_WARPS + warp) * OP_SPAN;
  if (w0l >= n_nu) return;
  const int w0 = (int)w0l;
  const int cell = blockIdx.y;
  const CellConst cc = cells[cell];
  const TabCell tc = tcells[cell];
  const SpanRange rg = spans[blockIdx.x * OP_WARPS + warp];
  const int64_t nk = 2 * ts.kk + 1;
  float acc[OP_R], hi[OP_R], lo[OP_R];
#pragma unroll
  for (int q = 0; q < OP_R; ++q) { acc[q] = 0.f; hi[q] = 0.f; lo[q] = 0.f; }
  int chunks = 0;
  for (int64_t base = rg.i_lo; base < rg.i_hi; base += 32) {
    const int nl = (int)min((int64_t)32, rg.i_hi - base);
    if (lane < nl) {
      const int64_t i = base + lane;
      const LineWin w = win[i];
      const TabLine t = tl[i];
      const int is = nearest_index(t.ln_nu0 + tc.ln_sfac, ts.ln_slo, ts.inv_sstep, ts.n_sigma);
      const int ig = nearest_index(t.ln_gref + tc.ln_gfac, ts.ln_glo, ts.inv_gstep, ts.n_gamma);
      // element read at grid point j: row + (j - jc + kk), the grid offset
      // kept inside the profile row [0, 2 kk] (it is by construction)
      s_row[warp][lane] = (((long long)is * ts.n_gamma + ig) * ts.O + t.r) * nk;
      s_kofs[warp][lane] = ts.kk - t.jc;
      s_S[warp][lane] = ex2f_approx((line_ln_s(w, cc) + LN_SCALE) * LOG2EF);
      s_win[warp][lane] = make_int2(w.jlo, w.jhi);
    }
    __syncwarp();
    for (int l = 0; l < nl; ++l) {
      const long long row = s_row[warp][l];
      const float S = s_S[warp][l];
      const int2 wn = s_win[warp][l];
      const int kofs = s_kofs[warp][l];
#pragma unroll
      for (int q = 0; q < OP_R; ++q) {
        const int j = w0 + 32 * q + lane;
        const int k = min(max(j + kofs, 0), (int)nk - 1);
        if (j >= wn.x && j <= wn.y) acc[q] = fmaf(S, __ldg(data + (row + k)), acc[q]);
      }
    }
    __syncwarp();
    if (++chunks == 4 || base + 32 >= rg.i_hi) {
      chunks = 0;
#pragma unroll
      for (int q = 0; q < OP_R; ++q) {
        const float sum = hi[q] + acc[q];
        const float bp = sum - hi[q];
        lo[q] += (hi[q] - (sum - bp)) + (acc[q] - bp);
        hi[q] = sum;
        acc[q] = 0.f;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < OP_R; ++q) {
    const int64_t j = (int64_t)w0 + 32 * q + lane;
    if (j < n_nu) out[(int64_t)cell * n_nu + j] = (hi[q] + lo[q]) * INV_SCALE;
  }
}

}  // namespace

struct bart_voigt_table {
  int device = 0;
  int n_sigma = 0, n_gamma = 0, oversample = 0, kk = 0;
  double sigma_lo = 0, sigma_hi = 0, gamma_lo = 0, gamma_hi = 0, dnu = 0, cutoff = 0;
  float* data = nullptr;
  size_t bytes = 0;
};

namespace {

TabSpec table_spec(const bart_voigt_table* t) {
  TabSpec ts;
  ts.n_sigma = t->n_sigma;
  ts.n_gamma = t->n_gamma;
  ts.O = t->oversample;
  ts.kk = t->kk;
  ts.ln_slo = std::log(t->sigma_lo);
  ts.ln_glo = std::log(t->gamma_lo);
  ts.inv_sstep = t->n_sigma > 1 ? (t->n_sigma - 1) / (std::log(t->sigma_hi) - std::log(t->sigma_lo)) : 0.0;
  ts.inv_gstep = t->n_gamma > 1 ? (t->n_gamma - 1) / (std::log(t->gamma_hi) - std::log(t->gamma_lo)) : 0.0;
  return ts;
}

bart_status run_cells_table(bart_ctx* ctx, const bart_voigt_table* tab, const bart_linelist* species,
                            int n_species, const std::vector<double>& p, const std::vector<double>& t,
                            bart_nugrid nu, double cutoff, float* out) {
  const int n_cells = (int)p.size();
  BART_REQUIRE(ctx, n_cells >= 1 && n_cells <= 65535, "n_cells must be in [1, 65535]");
  BART_REQUIRE(ctx, tab->device == ctx->device, "the table lives on another device");
  BART_REQUIRE(ctx, std::fabs(tab->dnu - nu.dnu_cm) <= 1e-12 * nu.dnu_cm && tab->cutoff >= cutoff,
               "the table was built for another grid spacing or a smaller cutoff");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  int64_t max_lines = 0;
  for (int s = 0; s < n_species; ++s) max_lines = std::max(max_lines, species[s].n_lines);
  const size_t nl = (size_t)std::max<int64_t>(max_lines, 1);
  const int64_t n_tiles = (nu.n_nu + OP_TILE - 1) / OP_TILE;
  const int n_spans = (int)(n_tiles * OP_WARPS);
  void *p_jlo, *p_jhi, *p_win, *p_spans, *p_tl, *p_cells, *p_tcells;
  bart_status st;
  if ((st = bart_scratch(ctx, "op_jlo", nl * sizeof(int), &p_jlo)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "op_jhi", nl * sizeof(int), &p_jhi)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "op_win", nl * sizeof(LineWin), &p_win)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "op_spans", (size_t)n_spans * sizeof(SpanRange), &p_spans)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "tb_lines", nl * sizeof(TabLine), &p_tl)) != BART_OK) return st;
  std::vector<CellConst> hc((size_t)n_species * n_cells);
  std::vector<TabCell> ht((size_t)n_species * n_cells);
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
      TabCell q;
      q.ln_sfac = std::log(std::sqrt(bartc::KB * T / (species[s].mass_amu * bartc::AMU)) / bartc::C);
      q.ln_gfac = std::log(P * std::sqrt(bartc::TREF / T));
      ht[(size_t)s * n_cells + c] = q;
    }
  if ((st = bart_upload_const(ctx, "tb_cells", hc.data(), hc.size() * sizeof(CellConst), &p_cells)) != BART_OK)
    return st;
  if ((st = bart_upload_const(ctx, "tb_tcells", ht.data(), ht.size() * sizeof(TabCell), &p_tcells)) != BART_OK)
    return st;
  const TabSpec ts = table_spec(tab);
  for (int s = 0; s < n_species; ++s) {
    const bart_linelist& L = species[s];
    float* o = out + (int64_t)s * n_cells * nu.n_nu;
    if (L.n_lines > 0) {
      const unsigned gl = (unsigned)((L.n_lines + 255) / 256);
      line_window_kernel<<<gl, 256, 0, ctx->stream>>>(L.nu0_cm, L.log10_s296, L.elow_cm, L.n_lines, nu.nu_start_cm,
                                                      nu.dnu_cm, nu.n_nu, cutoff, (int*)p_jlo, (int*)p_jhi,
                                                      (LineWin*)p_win);
      if ((st = bart_check_launch(ctx, "line_window_kernel")) != BART_OK) return st;
      table_line_kernel<<<gl, 256, 0, ctx->stream>>>(L.nu0_cm, L.gamma_ref_cm, L.n_lines, nu.nu_start_cm,
                                                     nu.dnu_cm, tab->oversample, (TabLine*)p_tl);
      if ((st = bart_check_launch(ctx, "table_line_kernel")) != BART_OK) return st;
    }
    span_range_kernel<<<(n_spans + 127) / 128, 128, 0, ctx->stream>>>((const int*)p_jlo, (const int*)p_jhi,
                                                                      L.n_lines, n_spans, (SpanRange*)p_spans);
    if ((st = bart_check_launch(ctx, "span_range_kernel")) != BART_OK) return st;
    table_opacity_kernel<<<dim3((unsigned)n_tiles, (unsigned)n_cells), OP_THREADS, 0, ctx->stream>>>(
        (const LineWin*)p_win, (const TabLine*)p_tl, (const SpanRange*)p_spans,
        (const CellConst*)p_cells + (size_t)s * n_cells, (const TabCell*)p_tcells + (size_t)s * n_cells, ts,
        tab->data, nu.n_nu, o);
    if ((st = bart_check_launch(ctx, "table_opacity_kernel")) != BART_OK) return st;
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

extern "C" bart_status bart_voigt_table_create(bart_ctx* ctx, int n_sigma, double sigma_lo, double sigma_hi,
                                               int n_gamma, double gamma_lo, double gamma_hi, int oversample,
                                               double dnu_cm, double cutoff_cm, bart_voigt_table** out) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, out != nullptr, "out is NULL");
  *out = nullptr;
  BART_REQUIRE(ctx, n_sigma >= 1 && n_gamma >= 1 && oversample >= 1, "n_sigma, n_gamma, oversample must be >= 1");
  BART_REQUIRE(ctx, sigma_lo > 0 && sigma_hi >= sigma_lo && gamma_lo > 0 && gamma_hi >= gamma_lo &&
                        std::isfinite(sigma_hi) && std::isfinite(gamma_hi),
               "need 0 < sigma_lo <= sigma_hi and 0 < gamma_lo <= gamma_hi");
  BART_REQUIRE(ctx, dnu_cm > 0 && cutoff_cm > 0 && std::isfinite(dnu_cm) && std::isfinite(cutoff_cm),
               "dnu and cutoff must be > 0");
  const double kkd = std::ceil(cutoff_cm / dnu_cm) + 1.0;
  BART_REQUIRE(ctx, kkd < 1e8, "cutoff / dnu is too large");
  const int kk = (int)kkd;
  const double n_el = (double)n_sigma * n_gamma * oversample * (2.0 * kk + 1.0);
  BART_REQUIRE(ctx, n_el * 4.0 < 2.0e11, "the table would exceed 200 GB");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  bart_status st = bart_ensure_wtable(ctx);
  if (st != BART_OK) return st;
  auto* t = new bart_voigt_table;
  t->device = ctx->device;
  t->n_sigma = n_sigma;
  t->n_gamma = n_gamma;
  t->oversample = oversample;
  t->kk = kk;
  t->sigma_lo = sigma_lo;
  t->sigma_hi = sigma_hi;
  t->gamma_lo = gamma_lo;
  t->gamma_hi = gamma_hi;
  t->dnu = dnu_cm;
  t->cutoff = cutoff_cm;
  t->bytes = (size_t)n_el * sizeof(float);
  cudaError_t e = cudaMalloc(&t->data, t->bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete t;
    return bart_fail(ctx, BART_ENOMEM, "cudaMalloc of %zu bytes for the Voigt table failed", (size_t)n_el * 4);
  }
  const TabSpec ts = table_spec(t);
  table_fill_kernel<<<(unsigned)std::min<double>(std::ceil(n_el / 256.0), 152.0 * 64.0), 256, 0, ctx->stream>>>(
      t->data, n_sigma, ts.ln_slo, n_sigma > 1 ? 1.0 / ts.inv_sstep : 0.0, n_gamma, ts.ln_glo,
      n_gamma > 1 ? 1.0 / ts.inv_gstep : 0.0, oversample, kk, dnu_cm, ctx->d_wtable);
  if ((st = bart_check_launch(ctx, "table_fill_kernel")) != BART_OK) {
    cudaFree(t->data);
    delete t;
    return st;
  }
  *out = t;
  return BART_OK;
}

extern "C" void bart_voigt_table_destroy(bart_voigt_table* t) {
  if (!t) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(t->device);
  cudaFree(t->data);
  cudaSetDevice(cur);
  delete t;
}

extern "C" int64_t bart_voigt_table_bytes(const bart_voigt_table* t) { return t ? (int64_t)t->bytes : -1; }

extern "C" bart_status bart_opacity_cells_table(bart_ctx* ctx, const bart_voigt_table* table,
                                                const bart_linelist* species, int n_species, const double* p_bar,
                                                const double* t_K, int n_cells, bart_nugrid nu, double cutoff_cm,
                                                float* out) {
  if (!ctx) return BART_EINVAL;
  bart_status st;
  BART_REQUIRE(ctx, table != nullptr, "table is NULL");
  if ((st = validate_lists(ctx, species, n_species)) != BART_OK) return st;
  if ((st = validate_grid(ctx, nu, cutoff_cm)) != BART_OK) return st;
  BART_REQUIRE(ctx, p_bar && t_K && out, "NULL p_bar, t_K or out");
  BART_REQUIRE(ctx, n_cells >= 1, "n_cells must be >= 1");
  std::vector<double> p(p_bar, p_bar + n_cells), t(t_K, t_K + n_cells);
  for (int c = 0; c < n_cells; ++c)
    BART_REQUIRE(ctx, p[c] > 0 && t[c] > 0 && std::isfinite(p[c]) && std::isfinite(t[c]),
                 "cell %d: P and T must be > 0 and finite", c);
  for (int s = 0; s < n_species; ++s)
    BART_REQUIRE(ctx, species[s].gamma_ref_cm || species[s].n_lines == 0, "species %d: NULL widths", s);
  return run_cells_table(ctx, table, species, n_species, p, t, nu, cutoff_cm, out);
}

extern "C" bart_status bart_build_opacity_grid_table(bart_ctx* ctx, const bart_voigt_table* table,
                                                     const bart_linelist* species, int n_species,
                                                     const double* p_bar, int n_layers, const double* t_K,
                                                     int n_temps, bart_nugrid nu, double cutoff_cm, float* grid) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, p_bar && t_K && grid, "NULL p_bar, t_K or grid");
  BART_REQUIRE(ctx, n_layers >= 1 && n_temps >= 1, "n_layers and n_temps must be >= 1");
  for (int k = 0; k < n_layers; ++k)
    BART_REQUIRE(ctx, p_bar[k] > 0 && (k == 0 || p_bar[k] > p_bar[k - 1]), "p_bar must be > 0 and increasing");
  for (int m = 0; m < n_temps; ++m)
    BART_REQUIRE(ctx, t_K[m] > 0 && (m == 0 || t_K[m] > t_K[m - 1]), "t_K must be > 0 and increasing");
  std::vector<double> p, t;
  for (int k = 0; k < n_layers; ++k)
    for (int m = 0; m < n_temps; ++m) {
      p.push_back(p_bar[k]);
      t.push_back(t_K[m]);
    }
  return bart_opacity_cells_table(ctx, table, species, n_species, p.data(), t.data(), (int)p.size(), nu, cutoff_cm,
                                  grid);
}
