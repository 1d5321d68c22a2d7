// Transmission (transit) geometry of the forward model (Sec. 6.1, the transit
// case of test f01oneline: slant paths through the layers, optical depth and
// transmission along each ray, times 2 pi r, integrated over altitude).
//
//   trans_prologue  one CTA per instance: level pressures (log-spaced between
//                   p_top and p_bot), T(P), hydrostatic altitudes in FP64
//                   (g ~ r^-2, r = R_p at P_ref, trapezoid in ln P with P_ref as
//                   a node), number densities and the bilinear (log10 P, T)
//                   brackets on the grid; a gray cloud deck cuts the
//                   instance's level count at its level (opaque below).
//                   The same CTA then writes every chord of the instance,
//                   ds_ik = 2 (A - B) / (sqrt A + sqrt B) from altitude
//                   differences (no cancellation), block by block of 8 rays.
//   trans_kernel    persistent CTAs pulling (wavenumber tile, instance) units
//                   from an atomic counter; tile-major order keeps the grid
//                   slab of a tile in L2 while every instance covering it runs.
//                   Eight threads per pair of neighbouring wavenumbers of a
//                   128-point tile, the pair's arithmetic on packed FP32 and
//                   its grid values read as 8-byte pairs: each computes an
//                   eighth of the levels' extinction (lines plus Rayleigh
//                   a nu^4 per molecule) into the shared shell means, then an
//                   eighth of the ray blocks (a shallow and a deep block per
//                   group of 2 x 8, run in one pass over the shells) of
//                   tau_i = sum_{k<i} ds_ik (alpha_k + alpha_{k+1}) / 2,
//                   4 rays per register block with the chords read as
//                   broadcast loads, and its share of the trapezoid in impact
//                   parameter (each ray's weight (z_{i-1} - z_{i+1}) / 2); the
//                   shares are added and the band partials fused.
//   trans_band_reduce  per (instance, band): fixed-order FP64 sum of partials.
#include <cmath>
#include <vector>

#include "bart_internal.cuh"
#include "forward.cuh"

namespace {

constexpr int TR_COLS = 128;             // wavenumbers per unit
constexpr int TR_PAIRS = TR_COLS / 2;    // wavenumber pairs per unit
constexpr int TR_SPLIT = 8;              // threads per pair column
constexpr int TR_THREADS = TR_PAIRS * TR_SPLIT;
constexpr int TR_LMAX = 192;             // maximum levels per instance
constexpr int TR_RB = 4;                 // rays per register block
constexpr int TR_NBLK = (TR_LMAX - 1 + TR_RB - 1) / TR_RB;   // ray blocks of the deepest column
// chords of an instance, block by block: block b (rays 1 + TR_RB b ..) needs
// shells k < kmax_b <= TR_RB (b + 1), stored [k][TR_RB rays] from
// TR_RB^2 b (b + 1) / 2
__host__ __device__ constexpr int tr_block_offset(int b) { return TR_RB * TR_RB * b * (b + 1) / 2; }
constexpr int TR_DS_STRIDE = tr_block_offset(TR_NBLK);
constexpr int TR_MAX_BANDS = 64;
constexpr int TR_MAX_SPECIES = 8;

struct TrLevel {
  float z;        // altitude above r_planet, cm
  float ndens;    // number density P / (k T), cm^-3
  int a;          // lower grid layer of the log10 P bracket
  float u;        // weight of the upper layer
  int m;          // lower grid temperature of the T bracket
  float w;        // weight of the upper temperature
};

struct TrInst {
  int L;
  int ok;
  float r_planet, r_star;
  float x[TR_MAX_SPECIES];
};

__global__ void trans_prologue(const float* __restrict__ theta, int n_theta, int n, int S,
                               const int32_t* __restrict__ n_levels, const float* __restrict__ r_planet,
                               const float* __restrict__ r_star, const float* __restrict__ lp_axis, int Lg,
                               const float* __restrict__ t_axis, int M, double p_top, double p_bot,
                               double p_ref, double g, double mu_amu, float inv_g_f, float tint4, float tirr0,
                               float t_min, float t_max, const float* __restrict__ x0, TrLevel* __restrict__ lev,
                               TrInst* __restrict__ inst, const int32_t* __restrict__ act_mask,
                               int* __restrict__ status, double p_cloud, float* __restrict__ ds) {
  const int i = blockIdx.x;
  if (i >= n) return;
  if (act_mask && !act_mask[i]) return;      // skipped entry
  __shared__ double s_lnp[TR_LMAX], s_T[TR_LMAX], s_phi[TR_LMAX];
  __shared__ float s_z[TR_LMAX];
  __shared__ int s_bad, s_leff;
  const int L = n_levels[i];
  const float* th = theta + (int64_t)i * n_theta;
  if (threadIdx.x == 0) s_bad = (L < 2 || L > TR_LMAX || !(r_planet[i] > 0.f) || !(r_star[i] > 0.f));
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) {
      atomicOr(status, BART_DEV_RANGE);
      inst[i].ok = 0;
      inst[i].L = 0;
    }
    return;
  }
  const double lt = log10(p_top), lb = log10(p_bot);
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const double lp = lt + (lb - lt) * (double)k / (double)(L - 1);
    const double p = exp10(lp);
    float thv[5];
    for (int q = 0; q < 5; ++q) thv[q] = th[q];
    float T = bartf::tp_temperature(thv, (float)(p * bartc::BAR), inv_g_f, tint4, tirr0);
    if (!(T == T) || T <= 0.0f) {
      atomicOr(status, BART_DEV_RANGE);
      T = t_min;
    }
    T = fminf(fmaxf(T, t_min), t_max);
    s_lnp[k] = log(p);
    s_T[k] = T;
    TrLevel lv;
    lv.ndens = (float)(p * bartc::BAR / (bartc::KB * (double)T));
    // bracket in log10 P over the grid layers
    const float lpf = (float)lp;
    int a = 0;
    float u = 0.f;
    if (Lg > 1) {
      int lo = 0, hi = Lg;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (lp_axis[mid] <= lpf) lo = mid + 1; else hi = mid;
      }
      a = min(max(lo - 1, 0), Lg - 2);
      u = fminf(fmaxf((lpf - lp_axis[a]) / (lp_axis[a + 1] - lp_axis[a]), 0.f), 1.f);
    }
    int m = 0;
    float w = 0.f;
    if (M > 1) {
      int lo = 0, hi = M;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (t_axis[mid] <= T) lo = mid + 1; else hi = mid;
      }
      m = min(max(lo - 1, 0), M - 2);
      w = fminf(fmaxf((T - t_axis[m]) / (t_axis[m + 1] - t_axis[m]), 0.f), 1.f);
    }
    lv.a = a;
    lv.u = u;
    lv.m = m;
    lv.w = w;
    lv.z = 0.f;
    lev[(int64_t)i * TR_LMAX + k] = lv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // phi_k = integral_{ln P_ref}^{ln P_k} T dlnP, trapezoid with P_ref as a node
    const double lref = log(p_ref);
    double t_ref;
    if (lref <= s_lnp[0]) t_ref = s_T[0];
    else if (lref >= s_lnp[L - 1]) t_ref = s_T[L - 1];
    else {
      int k = 0;
      while (k + 1 < L && s_lnp[k + 1] < lref) ++k;
      const double f = (lref - s_lnp[k]) / (s_lnp[k + 1] - s_lnp[k]);
      t_ref = s_T[k] + f * (s_T[k + 1] - s_T[k]);
    }
    // cumulative integral from the top, then shift so that phi(P_ref) = 0
    double cum = 0.0, cum_ref = 0.0;
    bool ref_done = false;
    s_phi[0] = 0.0;
    if (lref <= s_lnp[0]) { cum_ref = -0.5 * (t_ref + s_T[0]) * (s_lnp[0] - lref); ref_done = true; }
    for (int k = 0; k + 1 < L; ++k) {
      if (!ref_done && lref < s_lnp[k + 1]) {
        cum_ref = cum + 0.5 * (s_T[k] + t_ref) * (lref - s_lnp[k]);
        ref_done = true;
      }
      cum += 0.5 * (s_T[k] + s_T[k + 1]) * (s_lnp[k + 1] - s_lnp[k]);
      s_phi[k + 1] = cum;
    }
    if (!ref_done) cum_ref = cum + 0.5 * (s_T[L - 1] + t_ref) * (lref - s_lnp[L - 1]);
    const double rp = (double)r_planet[i];
    const double C = bartc::KB / (mu_amu * bartc::AMU * g * rp * rp);
    for (int k = 0; k < L; ++k) {
      const double cphi = C * (s_phi[k] - cum_ref);
      // r = 1/(1/R_p + C phi): altitude r - R_p written without cancellation
      s_z[k] = (float)(-cphi * rp * rp / (1.0 + cphi * rp));
      lev[(int64_t)i * TR_LMAX + k].z = s_z[k];
    }
    // gray cloud deck: the column ends on the first level with P >= p_cloud
    // (at least two levels); altitudes above stay those of the whole column
    int L_eff = L;
    if (p_cloud > 0.0) {
      for (int k = 0; k < L; ++k) {
        const double lp = lt + (lb - lt) * (double)k / (double)(L - 1);
        if (exp10(lp) >= p_cloud) {
          L_eff = max(k + 1, 2);
          break;
        }
      }
    }
    TrInst in;
    in.L = L_eff;
    in.ok = 1;
    in.r_planet = r_planet[i];
    in.r_star = r_star[i];
    for (int s = 0; s < TR_MAX_SPECIES; ++s)
      in.x[s] = s < S ? x0[s] * exp10f(theta[(int64_t)i * n_theta + 5 + s]) : 0.f;
    inst[i] = in;
    s_leff = L_eff;
  }
  __syncthreads();
  // chords of every ray through the shells above it, block by block of TR_RB
  // rays: ds_ik = 2 (sqrt(r_k^2 - b^2) - sqrt(r_{k+1}^2 - b^2)), b = r_i,
  // written as 2 (A - B) / (sqrt A + sqrt B) with A = r_k^2 - b^2 and
  // B = r_{k+1}^2 - b^2 formed from altitude differences (no cancellation)
  const int Le = s_leff;
  const float rp = r_planet[i];
  float* dsi = ds + (int64_t)i * TR_DS_STRIDE;
  const int nblk = (Le - 1 + TR_RB - 1) / TR_RB;
  for (int b = 0; b < nblk; ++b) {
    const int i0 = 1 + b * TR_RB, nr = min(TR_RB, Le - i0), kmax = i0 + nr - 1;
    float* db = dsi + tr_block_offset(b);
    for (int e = threadIdx.x; e < kmax * TR_RB; e += blockDim.x) {
      const int k = e / TR_RB, r = e % TR_RB, ir = i0 + r;
      float d = 0.f;
      if (r < nr && k < ir) {
        const float zb = s_z[ir], zk = s_z[k], zk1 = s_z[k + 1];
        const float A = (zk - zb) * (2.f * rp + zk + zb);
        const float B = (k + 1 < ir) ? (zk1 - zb) * (2.f * rp + zk1 + zb) : 0.f;
        const float AmB = (zk - zk1) * (2.f * rp + zk + zk1);
        d = 2.f * AmB / (sqrtf(A) + sqrtf(B));
      }
      db[e] = d;
    }
  }
}

// 1 - exp(-tau) with relative accuracy for small tau.
__device__ __forceinline__ float one_minus_exp(float tau) {
  if (tau < 0.125f) {
    // tau (1 - tau/2 (1 - tau/3 (1 - tau/4 (1 - tau/5 (1 - tau/6)))))
    float s = 1.0f - tau * (1.0f / 6.0f);
    s = 1.0f - tau * 0.2f * s;
    s = 1.0f - tau * 0.25f * s;
    s = 1.0f - tau * (1.0f / 3.0f) * s;
    s = 1.0f - tau * 0.5f * s;
    return tau * s;
  }
  return 1.0f - bartf::ex2_approx(-tau * 1.4426950408889634f);
}

__device__ __forceinline__ float2 tr_f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 tr_fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int S>
__global__ void __launch_bounds__(TR_THREADS, 2)
trans_kernel(const float* __restrict__ grid, int Lg, int M, int64_t N, const TrLevel* __restrict__ lev,
             const TrInst* __restrict__ inst, const float* __restrict__ ds, int n,
             const int64_t* __restrict__ nu_lo, const int64_t* __restrict__ nu_hi, const int64_t* __restrict__ offs,
             float* __restrict__ spectra, const float* __restrict__ filt, int n_bands, float2* __restrict__ partial,
             int n_gtiles, unsigned long long n_units, unsigned long long* __restrict__ counter,
             const int32_t* __restrict__ active, int* __restrict__ status, double nu_start, double dnu,
             double ray) {
  extern __shared__ float2 smem2[];
  float2* s_alpha = smem2;                                // [TR_LMAX - 1][TR_PAIRS] shell extinction pairs
  __shared__ TrLevel s_lev[TR_LMAX];
  __shared__ TrInst s_in;
  __shared__ unsigned long long s_unit;
  __shared__ float2 s_part[TR_SPLIT - 1][TR_PAIRS];
  __shared__ float2 s_red[TR_PAIRS / 32][TR_MAX_BANDS];
  const int tid = threadIdx.x;
  const int c = tid % TR_PAIRS, h = tid / TR_PAIRS;         // pair column, part
  const int64_t sstride = (int64_t)Lg * M * N;
  // float2 grid reads need an even row length and an 8-byte aligned grid
  const bool pair_loads = ((N & 1) == 0) && ((reinterpret_cast<uintptr_t>(grid) & 7) == 0);

  for (;;) {
    if (tid == 0) s_unit = atomicAdd(counter, 1ULL);
    __syncthreads();
    const unsigned long long u = s_unit;
    if (u >= n_units) break;
    const int g = (int)(u / (unsigned long long)n);
    const int i = (int)(u % (unsigned long long)n);
    if (active && !active[i]) {                   // skipped entry: outputs untouched
      __syncthreads();
      continue;
    }
    const int64_t lo = nu_lo ? nu_lo[i] : 0, hi = nu_hi ? nu_hi[i] : N;
    const int64_t g0 = (int64_t)g * TR_COLS;
    if (lo < 0 || hi > N || lo >= hi) {
      if (tid == 0 && g == 0) atomicOr(status, BART_DEV_RANGE);
      __syncthreads();
      continue;
    }
    if (g0 + TR_COLS <= lo || g0 >= hi) {         // this tile is outside the instance's span
      __syncthreads();
      continue;
    }
    if (tid == 0) s_in = inst[i];
    __syncthreads();
    if (!s_in.ok) {
      __syncthreads();
      continue;
    }
    const int L = s_in.L;
    for (int k = tid; k < L; k += TR_THREADS) s_lev[k] = lev[(int64_t)i * TR_LMAX + k];
    __syncthreads();

    // the pair (ja, ja + 1); idle lanes compute on a valid pair
    const int64_t ja = g0 + 2 * c, jb = ja + 1;
    const bool act_a = (ja >= lo) && (ja < hi), act_b = (jb >= lo) && (jb < hi);
    const int64_t lo2 = lo & ~(int64_t)1;
    const int64_t ka = (ja < N) ? ja : lo2;       // even; with an even N, ka + 1 < N
    const int64_t kb = (ka + 1 < N) ? ka + 1 : ka;
    // Rayleigh cross-section per molecule a nu^4, the same at every level
    float2 sig_r = tr_f2(0.f);
    if (ray != 0.0) {
      const double nua = nu_start + (double)ka * dnu, nub = nu_start + (double)kb * dnu;
      sig_r = make_float2((float)(ray * (nua * nua) * (nua * nua)), (float)(ray * (nub * nub) * (nub * nub)));
    }
    // extinction at levels k0 .. k1 of this part (the boundary level is
    // evaluated by both neighbours), shell means k0 .. k1-1 into shared memory
    {
      const int k0 = (L - 1) * h / TR_SPLIT, k1 = (L - 1) * (h + 1) / TR_SPLIT;
      const int64_t dl = (Lg > 1) ? (int64_t)M * N : 0;
      const int64_t dm = (M > 1) ? N : 0;
      const int64_t dkb = kb - ka;
      float2 a_prev = tr_f2(0.f);
#pragma unroll 2
      for (int k = k0; k <= k1; ++k) {
        const TrLevel lv = s_lev[k];
        const float* base = grid + ((int64_t)lv.a * M + lv.m) * N + ka;
        float2 sig = sig_r;
#pragma unroll
        for (int q = 0; q < S; ++q) {
          const float* b = base + q * sstride;
          float2 v00, v01, v10, v11;
          if (pair_loads) {
            v00 = __ldg(reinterpret_cast<const float2*>(b));
            v01 = __ldg(reinterpret_cast<const float2*>(b + dm));
            v10 = __ldg(reinterpret_cast<const float2*>(b + dl));
            v11 = __ldg(reinterpret_cast<const float2*>(b + dl + dm));
          } else {
            v00 = make_float2(__ldg(b), __ldg(b + dkb));
            v01 = make_float2(__ldg(b + dm), __ldg(b + dm + dkb));
            v10 = make_float2(__ldg(b + dl), __ldg(b + dl + dkb));
            v11 = make_float2(__ldg(b + dl + dm), __ldg(b + dl + dm + dkb));
          }
          const float2 lo_l = tr_fma2(tr_f2(lv.w), __fadd2_rn(v01, __fmul2_rn(v00, tr_f2(-1.f))), v00);
          const float2 hi_l = tr_fma2(tr_f2(lv.w), __fadd2_rn(v11, __fmul2_rn(v10, tr_f2(-1.f))), v10);
          const float2 pl = tr_fma2(tr_f2(lv.u), __fadd2_rn(hi_l, __fmul2_rn(lo_l, tr_f2(-1.f))), lo_l);
          sig = tr_fma2(tr_f2(s_in.x[q]), pl, sig);
        }
        const float2 a = __fmul2_rn(sig, tr_f2(lv.ndens));
        if (k > k0) s_alpha[(k - 1) * TR_PAIRS + c] = __fmul2_rn(tr_f2(0.5f), __fadd2_rn(a_prev, a));
        a_prev = a;
      }
    }
    __syncthreads();
    // rays b_i = r_i, i = 1 .. L-1 (ray 0 grazes the top level: tau = 0) in
    // blocks of TR_RB; this thread's share of the trapezoid in impact parameter,
    // integral (1 - e^-tau) b db = sum_i f_i b_i (z_{i-1} - z_{i+1}) / 2
    // (altitude differences keep full precision; the deepest ray's weight
    // is (z_{L-2} - z_{L-1}) / 2)
    const float rp = s_in.r_planet;
    const float* dsi = ds + (int64_t)i * TR_DS_STRIDE;
    const int nblk = (L - 1 + TR_RB - 1) / TR_RB;
    float2 integ = tr_f2(0.f);
    // this thread's share of the trapezoid from a block's path sums
    auto add_rays = [&](int i0, int nr, const float2* tau) {
#pragma unroll
      for (int r = 0; r < TR_RB; ++r) {
        if (r < nr) {
          const int ir = i0 + r;
          const float zb = s_lev[ir].z;
          const float wgt = 0.5f * (s_lev[ir - 1].z - (ir + 1 < L ? s_lev[ir + 1].z : zb));
          const float2 f = make_float2(one_minus_exp(tau[r].x), one_minus_exp(tau[r].y));
          integ = tr_fma2(f, tr_f2((rp + zb) * wgt), integ);
        }
      }
    };
    // the snake order gives this thread the blocks 2 TR_SPLIT g + h (shallow)
    // and 2 TR_SPLIT g + 2 TR_SPLIT - 1 - h (deep) of each group g: both run
    // in one pass over the shells (each shell's extinction read once for
    // both, eight independent sums)
    for (int g = 0; 2 * TR_SPLIT * g + h < nblk; ++g) {
      const int ba = 2 * TR_SPLIT * g + h, bb = 2 * TR_SPLIT * g + 2 * TR_SPLIT - 1 - h;
      const int i0a = 1 + ba * TR_RB, nra = min(TR_RB, L - i0a), kma = i0a + nra - 1;
      const float* da = dsi + tr_block_offset(ba);
      float2 ta[TR_RB], tb[TR_RB];
#pragma unroll
      for (int r = 0; r < TR_RB; ++r) ta[r] = tb[r] = tr_f2(0.f);
      if (bb < nblk) {
        const int i0b = 1 + bb * TR_RB, nrb = min(TR_RB, L - i0b), kmb = i0b + nrb - 1;   // kmb > kma
        const float* dbp = dsi + tr_block_offset(bb);
        int k = 0;
#pragma unroll 2
        for (; k < kma; ++k) {
          const float2 a = s_alpha[k * TR_PAIRS + c];
          const float4 d = __ldg(reinterpret_cast<const float4*>(da + k * TR_RB));
          const float4 e = __ldg(reinterpret_cast<const float4*>(dbp + k * TR_RB));
          ta[0] = tr_fma2(tr_f2(d.x), a, ta[0]);
          ta[1] = tr_fma2(tr_f2(d.y), a, ta[1]);
          ta[2] = tr_fma2(tr_f2(d.z), a, ta[2]);
          ta[3] = tr_fma2(tr_f2(d.w), a, ta[3]);
          tb[0] = tr_fma2(tr_f2(e.x), a, tb[0]);
          tb[1] = tr_fma2(tr_f2(e.y), a, tb[1]);
          tb[2] = tr_fma2(tr_f2(e.z), a, tb[2]);
          tb[3] = tr_fma2(tr_f2(e.w), a, tb[3]);
        }
#pragma unroll 4
        for (; k < kmb; ++k) {
          const float2 a = s_alpha[k * TR_PAIRS + c];
          const float4 e = __ldg(reinterpret_cast<const float4*>(dbp + k * TR_RB));
          tb[0] = tr_fma2(tr_f2(e.x), a, tb[0]);
          tb[1] = tr_fma2(tr_f2(e.y), a, tb[1]);
          tb[2] = tr_fma2(tr_f2(e.z), a, tb[2]);
          tb[3] = tr_fma2(tr_f2(e.w), a, tb[3]);
        }
        add_rays(i0b, nrb, tb);
      } else {
#pragma unroll 4
        for (int k = 0; k < kma; ++k) {
          const float2 a = s_alpha[k * TR_PAIRS + c];
          const float4 d = __ldg(reinterpret_cast<const float4*>(da + k * TR_RB));
          ta[0] = tr_fma2(tr_f2(d.x), a, ta[0]);
          ta[1] = tr_fma2(tr_f2(d.y), a, ta[1]);
          ta[2] = tr_fma2(tr_f2(d.z), a, ta[2]);
          ta[3] = tr_fma2(tr_f2(d.w), a, ta[3]);
        }
      }
      add_rays(i0a, nra, ta);
    }
    if (h > 0) s_part[h - 1][c] = integ;
    __syncthreads();
    if (h == 0) {
#pragma unroll
      for (int q = 0; q < TR_SPLIT - 1; ++q) integ = __fadd2_rn(integ, s_part[q][c]);
      const float rbot = rp + s_lev[L - 1].z;
      const float rs = s_in.r_star;
      const float d0 = (rbot / rs) * (rbot / rs);
      const float2 delta = make_float2(d0 + 2.f * integ.x / (rs * rs), d0 + 2.f * integ.y / (rs * rs));
      if (spectra) {
        const int64_t o = (offs ? offs[i] : (int64_t)i * N) - lo;
        if (act_a) spectra[o + ja] = delta.x;
        if (act_b) spectra[o + jb] = delta.y;
      }
      s_part[0][c] = delta;                       // the column's depths for every part's bands
    }
    if (n_bands > 0) {
      __syncthreads();
      // band sums of the tile: part h takes bands h, h + TR_SPLIT, ..., four
      // at a time with their filter weights loaded together
      const float2 delta = s_part[0][c];
      const float dwa = act_a ? ((hi - lo == 1) ? 1.f : ((ja == lo || ja == hi - 1) ? 0.5f : 1.f)) : 0.f;
      const float dwb = act_b ? ((hi - lo == 1) ? 1.f : ((jb == lo || jb == hi - 1) ? 0.5f : 1.f)) : 0.f;
      const int wp = (tid & (TR_PAIRS - 1)) >> 5, lane = tid & 31;   // warp within the part
      for (int b0 = h; b0 < n_bands; b0 += 4 * TR_SPLIT) {
        float Wa[4], Wb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int b = b0 + q * TR_SPLIT;
          Wa[q] = (act_a && b < n_bands) ? __ldg(filt + (int64_t)b * N + ja) * dwa : 0.f;
          Wb[q] = (act_b && b < n_bands) ? __ldg(filt + (int64_t)b * N + jb) * dwb : 0.f;
        }
        float num[4], den[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          num[q] = fmaf(Wa[q], delta.x, Wb[q] * delta.y);
          den[q] = Wa[q] + Wb[q];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            num[q] += __shfl_xor_sync(0xffffffffu, num[q], o);
            den[q] += __shfl_xor_sync(0xffffffffu, den[q], o);
          }
        }
        if (lane == 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (b0 + q * TR_SPLIT < n_bands) s_red[wp][b0 + q * TR_SPLIT] = make_float2(num[q], den[q]);
        }
      }
      __syncthreads();
      if (tid < n_bands) {
        float2 acc = make_float2(0.f, 0.f);
        for (int w = 0; w < TR_PAIRS / 32; ++w) {
          acc.x += s_red[w][tid].x;
          acc.y += s_red[w][tid].y;
        }
        partial[((int64_t)i * n_gtiles + g) * n_bands + tid] = acc;
      }
    }
    __syncthreads();
  }
}

__global__ void trans_band_reduce(const float2* __restrict__ partial, const int64_t* __restrict__ nu_lo,
                                  const int64_t* __restrict__ nu_hi, int64_t N, int n, int n_gtiles, int nb,
                                  const int32_t* __restrict__ active, float* __restrict__ bands) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * nb) return;
  const int i = (int)(idx / nb), b = (int)(idx % nb);
  if (active && !active[i]) return;
  const int64_t lo = nu_lo ? nu_lo[i] : 0, hi = nu_hi ? nu_hi[i] : N;
  if (lo < 0 || hi > N || lo >= hi) {
    bands[idx] = 0.f;
    return;
  }
  double num = 0.0, den = 0.0;
  for (int64_t g = lo / TR_COLS; g <= (hi - 1) / TR_COLS; ++g) {
    const float2 v = partial[((int64_t)i * n_gtiles + g) * nb + b];
    num += v.x;
    den += v.y;
  }
  bands[idx] = den > 0.0 ? (float)(num / den) : 0.f;
}

using TrLauncher = void (*)(int, size_t, cudaStream_t, const float*, int, int, int64_t, const TrLevel*,
                            const TrInst*, const float*, int, const int64_t*, const int64_t*, const int64_t*,
                            float*, const float*, int, float2*, int, unsigned long long, unsigned long long*,
                            const int32_t*, int*, double, double, double);

template <int S>
void launch_trans(int grid_dim, size_t smem, cudaStream_t st, const float* grid, int Lg, int M, int64_t N,
                  const TrLevel* lev, const TrInst* inst, const float* ds, int n, const int64_t* lo,
                  const int64_t* hi, const int64_t* offs, float* spectra, const float* filt, int nb, float2* partial,
                  int ngt, unsigned long long nu, unsigned long long* counter, const int32_t* active, int* status,
                  double nu_start, double dnu, double ray) {
  trans_kernel<S><<<grid_dim, TR_THREADS, smem, st>>>(grid, Lg, M, N, lev, inst, ds, n, lo, hi, offs, spectra,
                                                      filt, nb, partial, ngt, nu, counter, active, status,
                                                      nu_start, dnu, ray);
}

template <int S>
cudaError_t set_smem(size_t smem, int* per_sm) {
  // opt in to the dynamic shared memory, then ask how many CTAs of this
  // instantiation fit on an SM with it (the persistent grid size)
  cudaError_t e = cudaFuncSetAttribute(trans_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, trans_kernel<S>, TR_THREADS, smem);
}

}  // namespace

bart_status bart_transmission_batch(bart_ctx* ctx, const bart_grid_desc* g, const bart_fwd_cfg* c,
                                    const bart_batch* b, float* spectra, const bart_filters* f, float* bands) {
  const int S = g->n_species, Lg = g->n_layers, M = g->n_temps, n = b->n;
  const int64_t N = g->nu.n_nu;
  BART_REQUIRE(ctx, b->theta, "transmission needs theta");
  BART_REQUIRE(ctx, b->n_levels && b->r_planet_cm && b->r_star_cm,
               "transmission needs n_levels, r_planet_cm and r_star_cm");
  BART_REQUIRE(ctx, c->p_top_bar > 0 && c->p_bot_bar > c->p_top_bar && c->p_ref_bar > 0,
               "need 0 < p_top < p_bot and p_ref > 0");
  BART_REQUIRE(ctx, S >= 1 && S <= 4, "transmission supports 1-4 species");
  const int nb = bands ? f->n_bands : 0;
  BART_CUDA(ctx, cudaSetDevice(ctx->device));

  TrLauncher launch = nullptr;
  cudaError_t ce = cudaSuccess;
  int per_sm = 0;
  const size_t smem = (size_t)(TR_LMAX - 1) * TR_PAIRS * sizeof(float2);
  switch (S) {
    case 1: launch = launch_trans<1>; ce = set_smem<1>(smem, &per_sm); break;
    case 2: launch = launch_trans<2>; ce = set_smem<2>(smem, &per_sm); break;
    case 3: launch = launch_trans<3>; ce = set_smem<3>(smem, &per_sm); break;
    case 4: launch = launch_trans<4>; ce = set_smem<4>(smem, &per_sm); break;
  }
  if (ce != cudaSuccess) return bart_fail(ctx, BART_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(ce));

  std::vector<float> hconst;      // [log10 p grid Lg][t axis M][x0 S]
  for (int k = 0; k < Lg; ++k) hconst.push_back((float)std::log10(g->p_bar[k]));
  for (int m = 0; m < M; ++m) hconst.push_back((float)g->t_K[m]);
  for (int s = 0; s < S; ++s) hconst.push_back((float)c->x0[s]);
  const int n_gtiles = (int)((N + TR_COLS - 1) / TR_COLS);
  void *p_const, *p_lev, *p_inst, *p_part = nullptr, *p_counter, *p_ds;
  bart_status st;
  if ((st = bart_upload_const(ctx, "tr_const", hconst.data(), hconst.size() * sizeof(float), &p_const)) != BART_OK)
    return st;
  if ((st = bart_scratch(ctx, "tr_lev", (size_t)n * TR_LMAX * sizeof(TrLevel), &p_lev)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "tr_inst", (size_t)n * sizeof(TrInst), &p_inst)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "tr_ds", (size_t)n * TR_DS_STRIDE * sizeof(float), &p_ds)) != BART_OK) return st;
  if ((st = bart_scratch(ctx, "tr_counter", sizeof(unsigned long long), &p_counter)) != BART_OK) return st;
  if (nb > 0 &&
      (st = bart_scratch(ctx, "tr_part", (size_t)n * n_gtiles * nb * sizeof(float2), &p_part)) != BART_OK)
    return st;
  BART_CUDA(ctx, cudaMemsetAsync(p_counter, 0, sizeof(unsigned long long), ctx->stream));
  const float* dc = (const float*)p_const;
  const double rs = c->r_star_tp_cm, a = c->a_orbit_cm;
  const float tirr0 = (rs > 0 && a > 0) ? (float)(std::sqrt(rs / (2.0 * a)) * c->t_star_K) : 0.0f;
  trans_prologue<<<n, 128, 0, ctx->stream>>>(
      b->theta, 5 + S, n, S, b->n_levels, b->r_planet_cm, b->r_star_cm, dc, Lg, dc + Lg, M, c->p_top_bar,
      c->p_bot_bar, c->p_ref_bar, c->g_cgs, c->mu_amu, (float)(1.0 / c->g_cgs), (float)std::pow(c->t_int_K, 4.0),
      tirr0, (float)c->t_min_K, (float)std::min(c->t_max_K, 1e30), dc + Lg + M, (TrLevel*)p_lev,
      (TrInst*)p_inst, b->active, ctx->d_status, c->p_cloud_bar, (float*)p_ds);
  if ((st = bart_check_launch(ctx, "trans_prologue")) != BART_OK) return st;
  const unsigned long long n_units = (unsigned long long)n_gtiles * (unsigned long long)n;
  if (per_sm < 1) per_sm = 1;
  int grid_dim = ctx->sm_count * per_sm;
  if ((unsigned long long)grid_dim > n_units) grid_dim = (int)n_units;
  launch(grid_dim, smem, ctx->stream, g->grid, Lg, M, N, (const TrLevel*)p_lev, (const TrInst*)p_inst,
         (const float*)p_ds, n,
         b->nu_lo, b->nu_hi, b->spec_offsets, spectra, nb ? f->weights : nullptr, nb, (float2*)p_part, n_gtiles,
         n_units, (unsigned long long*)p_counter, b->active, ctx->d_status, g->nu.nu_start_cm, g->nu.dnu_cm,
         c->rayleigh_coef);
  if ((st = bart_check_launch(ctx, "trans_kernel")) != BART_OK) return st;
  if (nb > 0) {
    const int64_t tot = (int64_t)n * nb;
    trans_band_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(
        (const float2*)p_part, b->nu_lo, b->nu_hi, N, n, n_gtiles, nb, b->active, bands);
    if ((st = bart_check_launch(ctx, "trans_band_reduce")) != BART_OK) return st;
  }
  return BART_OK;
}
