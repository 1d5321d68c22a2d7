// Kernels of the persistent fused launch per emission batch: a whole sampler generation
// of proposals (Sec. 3 forward model -- profile generator, transit and the
// spectrum integrator -- for every proposal; Sec. 4 items 3 and 7; Sec. 7
// nine-parameter model) in a single kernel.
//
// CTAs (as many as fit on the SMs) take units (wavenumber tile, proposal)
// from a device counter in tile-major order: the CTAs in flight work on the
// same tile for neighbouring proposals, so the grid rows they read (the same
// rows for proposals whose layer temperatures fall in the same bracket) are
// shared through L2.  For its unit a CTA
//   1. evaluates the proposal's five-parameter T(P) profile at every layer
//      (one thread per layer) and keeps, per layer, the grid row offsets of
//      its temperature bracket, the interpolation weights times the
//      abundance coefficients X_s / (mu m_u) = X0_s 10^{a_s} / (mu m_u) and
//      the Planck terms in a shared-memory record;
//   2. runs one thread per pair of neighbouring wavenumbers down the column,
//      the pair's arithmetic on packed FP32: opacity interpolated in T and
//      summed over species (8-byte grid-row reads, the next layer's rows
//      requested before the current layer is computed), the trapezoid
//      optical depth, the Planck source, the transmittance at each
//      Gauss-Legendre angle from the running vertical optical depth, and the
//      flux as a sum over layers of the layer-mean source times the drop of
//      the quadrature-weighted transmittance (the angle sum taken inside the
//      layer sum, so no per-angle state is kept);
//   3. writes the spectrum and the tile's band partial sums; the CTA that
//      finishes a proposal's last tile sums its partials in a fixed order
//      (FP64) into the band values.
// Nothing waits on another CTA: the last-tile test is an atomic count, a
// proposal's layer states are published by its first unit with an epoch mark
// (a unit that does not see the mark computes them itself), and the last CTA
// to leave resets the counters and advances the epoch, so the launch can be
// replayed from a CUDA graph unchanged.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "bart_internal.cuh"
#include "emission.cuh"
#include "forward.cuh"

namespace bartem {


constexpr int FUSED_MAX_SPECIES = 4;
constexpr int MAX_TILES_PER_UNIT = 8;

// GPU-scope acquire load and release store of a 32-bit flag, and an
// acquire-release add (PTX memory model): the release makes the writes that
// the CTA ordered before it by a barrier visible to a thread that acquires
// the flag, without a full fence in every writing thread.
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// ---- mbarrier and bulk-copy (TMA) helpers, CTA scope
constexpr unsigned int MBAR_SPIN_LIMIT = 1u << 22;   // try_wait rounds before a wait is given up

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity to complete: gives up after
// MBAR_SPIN_LIMIT rounds, or once another thread of the CTA has given up
// (*abort), and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int parity, volatile int* abort) {
  for (unsigned int it = 0; it < MBAR_SPIN_LIMIT; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort) return false;
  }
  return false;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned int bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

struct FusedArgs {
  const float* grid;                 // [S][L][M][N]
  int L, M;
  int64_t N;
  const float* theta;                // [n][n_theta] or NULL
  int n_theta;
  const float* t_profile;            // [n][L] or NULL
  int n;
  const int64_t* nu_lo;
  const int64_t* nu_hi;
  const int64_t* offs;
  const int32_t* active;
  const float* p_cgs;                // [L] level pressures, dyn cm^-2
  const float* t_axis;               // [M]
  const float* dpg;                  // [L-1] (P_{k+1} - P_k) / (2 g)
  float x0mu[FUSED_MAX_SPECIES];     // X0_s / (mu m_u)
  float ang[2 * MAX_ANGLES];         // -log2(e) / mu_i, then 2 pi w_i mu_i / 2
  float tw_top;                      // sum_i 2 pi w_i mu_i / 2 (all transmittances 1)
  float inv_g, tint4, tirr0, t_min, t_max;
  double nu_start, dnu;
  float* spectra;
  const float* filt;
  int n_bands;
  float2* partial;                   // [n][n_groups][n_bands]
  float* bands;
  int tpu;                           // tiles per unit (consecutive tiles of one proposal)
  int n_groups;                      // units per proposal over the whole grid: ceil(n_tiles / tpu)
  unsigned long long n_units;        // n_groups x n
  unsigned long long* work;          // [0] next unit, [1] CTAs finished, [2] launch epoch
  unsigned int* p_done;              // [n] tiles finished per proposal
  LayerTW* tw_cache;                 // [n][L] layer states published by the first unit of a proposal
  unsigned int* tw_flag;             // [n] epoch + 1 once tw_cache[p] holds this launch's states
  int* status;
  EmExtra ex;
  bool wide_x;                       // c2 nu / T can exceed 20: FP64 Planck branch
  bool tau_lim;                      // the optical-depth limit is on
};

// Resident threads per SM the register allocation is sized for (768: six
// CTAs of 128 threads, at most 80 registers a thread; measured faster than
// 512 threads at 112 registers).
#ifndef FUSED_OCC_THREADS
#define FUSED_OCC_THREADS 768
#endif

// Two wavenumbers per thread, their arithmetic on packed FP32 pairs
// (FFMA2/FADD2/FMUL2 of sm_100+: one issue slot for both); the MUFU
// exponentials and reciprocals stay per wavenumber.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }   // exact
__device__ __forceinline__ float2 ex2_2(float2 y) {
  return make_float2(bartf::ex2_approx(y.x), bartf::ex2_approx(y.y));
}

// Planck function from y = (c2 nu / T) log2(e): B = c1nu3 / (2^y - 1); where
// c2 nu / T can exceed 20 (WIDE_X), larger arguments take an FP64 expm1.
template <bool WIDE_X>
__device__ __forceinline__ float2 planck2(float2 c1nu3, float2 y) {
  const float2 e = add2(ex2_2(y), f2(-1.0f));
  float2 B = mul2(c1nu3, make_float2(bartf::rcp_approx(e.x), bartf::rcp_approx(e.y)));
  if (WIDE_X) {
    constexpr float Y20 = 20.0f * LOG2E;
    if (y.x > Y20) B.x = (float)((double)c1nu3.x / expm1((double)y.x * 0.6931471805599453));
    if (y.y > Y20) B.y = (float)((double)c1nu3.y / expm1((double)y.y * 0.6931471805599453));
  }
  return B;
}

// The same with the FP64 branch chosen at run time (wide: c2 nu / T can
// exceed 20 on this grid).
template <bool ALLOW_WIDE>
__device__ __forceinline__ float2 planck2(float2 c1nu3, float2 y, bool wide) {
  return (ALLOW_WIDE && wide) ? planck2<true>(c1nu3, y) : planck2<false>(c1nu3, y);
}

// Per layer of the unit's proposal, in shared memory: the 32-bit element
// offsets of the 2 S grid rows the layer reads (species s: the lower
// temperature bracket at (k M + m) n_nu + s L M n_nu, the upper n_nu further;
// the host takes this kernel only where S L M n_nu + n_nu < 2^32), the
// interpolation weights times the abundance coefficients
// (chi = sum_s X_s (1 - w) sigma_lo + X_s w sigma_hi), and the Planck terms:
// y = (c2 / T) log2(e), (P_k - P_{k-1}) / 2g and r = 2^(y dnu), the ratio of
// exp(c2 nu / T) between neighbouring wavenumbers.
template <int S>
struct __align__(16) LayerRec {
  static constexpr int NCF = (2 * S + 3) / 4;
  uint4 off[NCF];    // lower, upper bracket of species 0, of species 1, ...
  float4 cf[NCF];    // X_s (1 - w), X_s w, s = 0 .. S-1
  float4 pl;         // y, (P_k - P_{k-1}) / 2g, r, unused
};

// Planck function of a pair of neighbouring wavenumbers (nu, nu + dnu) at
// one temperature from 2^(nu y) and r = 2^(dnu y): one exponential and one
// reciprocal for both, B_a = c1nu3_a (e_b - 1) / ((e_a - 1)(e_b - 1)) and
// B_b = c1nu3_b (e_a - 1) / (...).  Used where c2 nu / T <= 20, so the
// product stays below 2.4e17.
__device__ __forceinline__ float2 planck_pair(float2 c1nu3, float nu_a, float y, float r) {
  const float ea = bartf::ex2_approx(nu_a * y);
  const float eb = ea * r;
  const float2 em1 = add2(make_float2(eb, ea), f2(-1.0f));   // (e_b - 1, e_a - 1)
  const float R = bartf::rcp_approx(em1.x * em1.y);
  return mul2(mul2(c1nu3, f2(R)), em1);
}

// TW wavenumbers per tile, TW / 2 threads per CTA.
template <int S, int NA, int TW, int MODE>
__global__ void __launch_bounds__(TW / 2, FUSED_OCC_THREADS / (TW / 2))
emission_fused_kernel(const __grid_constant__ FusedArgs a) {
  constexpr int NT = TW / 2;
  constexpr int NCF = LayerRec<S>::NCF;
  __shared__ LayerRec<S> s_rec[MAX_LAYERS];
  __shared__ float s_xs[S];
  __shared__ float2 s_red[NT / 32 > 0 ? NT / 32 : 1][MAX_BANDS];
  __shared__ unsigned long long s_unit;
  __shared__ int s_last, s_ready;
  constexpr bool WIDE_X = (MODE & 1) != 0, TAU_LIM = (MODE & 2) != 0;
  const int tid = threadIdx.x;
  const int L = a.L, nb = a.n_bands;
  const int64_t sstride = (int64_t)L * a.M * a.N;
  const unsigned int dm = (a.M > 1) ? (unsigned int)a.N : 0u;   // offset of the upper temperature bracket
  const float dnu_f = (float)a.dnu;
  // float2 grid reads need an even row length and an 8-byte aligned grid
  const bool pair_loads = ((a.N & 1) == 0) && ((reinterpret_cast<uintptr_t>(a.grid) & 7) == 0);
  // the epoch only changes when the last CTA of a launch leaves, so every CTA
  // of this launch reads the same value
  const unsigned int ready_mark = (unsigned int)*(volatile unsigned long long*)(a.work + 2) + 1u;
  unsigned long long next_unit = 0;
  if (tid == 0) next_unit = atomicAdd(a.work, 1ULL);

  for (;;) {
    if (tid == 0) {
      s_unit = next_unit;
      next_unit = atomicAdd(a.work, 1ULL);       // the following unit, fetched while this one runs
    }
    __syncthreads();
    const unsigned long long u = s_unit;
    if (u >= a.n_units) break;
    const int p = (int)(u % (unsigned long long)a.n);
    const int grp = (int)(u / (unsigned long long)a.n);
    // every value below is uniform over the CTA
    bool skip = a.active && !a.active[p];
    int64_t lo = 0, hi = a.N;
    if (!skip) {
      lo = a.nu_lo ? a.nu_lo[p] : 0;
      hi = a.nu_hi ? a.nu_hi[p] : a.N;
      if (lo < 0 || hi > a.N || lo >= hi) {
        // invalid span: report it once, band values 0, spectrum untouched
        if (grp == 0) {
          if (tid == 0) atomicOr(a.status, BART_DEV_RANGE);
          if (a.bands && tid < nb) a.bands[(int64_t)p * nb + tid] = 0.0f;
        }
        skip = true;
      }
    }
    const int64_t lo2 = lo & ~(int64_t)1;          // tiles start on even indices (pairs)
    const int n_tiles_p = skip ? 0 : (int)((hi - lo2 + TW - 1) / TW);
    const int n_groups_p = (n_tiles_p + a.tpu - 1) / a.tpu;
    if (!skip && grp < n_groups_p) {
      // 1. the proposal's layers: T(P) (or the given profile), bracket, c2/T,
      // computed by the first unit of the proposal and published for the
      // others (a unit that finds them unpublished computes them itself),
      // and from them the layer records
      if (tid == 0) s_ready = (ld_acquire(a.tw_flag + p) == ready_mark);
      if (tid < S) {
        const float ab = a.theta ? a.theta[(int64_t)p * a.n_theta + 5 + tid] : 0.0f;
        s_xs[tid] = a.x0mu[tid] * exp10f(ab);
      }
      __syncthreads();
      const bool ready = s_ready;
      for (int k = tid; k < L; k += NT) {
        LayerTW r;
        if (ready) {
          // one 16-byte L2 load per layer state: row (two words), w, c2/T
          const int4 v = __ldcg(reinterpret_cast<const int4*>(a.tw_cache + (int64_t)p * L + k));
          r.row = (int64_t)(((unsigned long long)(unsigned int)v.y << 32) | (unsigned int)v.x);
          r.w = __int_as_float(v.z);
          r.c2_t = __int_as_float(v.w);
        } else {
          float T;
          if (a.t_profile) {
            T = a.t_profile[(int64_t)p * L + k];
          } else {
            float th[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) th[i] = a.theta[(int64_t)p * a.n_theta + i];
            T = bartf::tp_temperature(th, a.p_cgs[k], a.inv_g, a.tint4, a.tirr0);
          }
          r = layer_state(T, k, a.t_axis, a.M, a.N, a.t_min, a.t_max, a.status);
          a.tw_cache[(int64_t)p * L + k] = r;
        }
        unsigned int of[4 * NCF] = {};
        float cf[4 * NCF] = {};
#pragma unroll
        for (int q = 0; q < S; ++q) {
          of[2 * q] = (unsigned int)(r.row + q * sstride);
          of[2 * q + 1] = of[2 * q] + dm;
          cf[2 * q] = s_xs[q] * (1.0f - r.w);
          cf[2 * q + 1] = s_xs[q] * r.w;
        }
#pragma unroll
        for (int q = 0; q < NCF; ++q) {
          s_rec[k].off[q] = make_uint4(of[4 * q], of[4 * q + 1], of[4 * q + 2], of[4 * q + 3]);
          s_rec[k].cf[q] = make_float4(cf[4 * q], cf[4 * q + 1], cf[4 * q + 2], cf[4 * q + 3]);
        }
        const float y = r.c2_t * LOG2E;
        s_rec[k].pl = make_float4(y, k > 0 ? __ldg(a.dpg + k - 1) : 0.0f, exp2f(y * dnu_f), 0.0f);
      }
      __syncthreads();
      if (!ready && tid == 0) st_release(a.tw_flag + p, ready_mark);   // publishes the CTA's stores above
      float2 band_acc = make_float2(0.f, 0.f);      // thread b < nb: band b over the unit's tiles
      const int t_end = min((grp + 1) * a.tpu, n_tiles_p);

      // 2. the columns of wavenumbers ja and ja + 1 of one tile; PAIR: both
      // read by one 8-byte load per row
      auto column = [&](auto pair_c, int tile) {
        constexpr bool PAIR = decltype(pair_c)::value;
        const int64_t ja = lo2 + (int64_t)tile * TW + 2 * tid, jb = ja + 1;
        const bool act_a = ja >= lo && ja < hi, act_b = jb < hi;
        // idle lanes compute on valid indices
        const int64_t ka = (ja < hi) ? ja : lo2, kb = (jb < hi) ? jb : ka;
        // the wavenumbers from their FP64 positions, the rest in FP32
        const float2 nuf = make_float2((float)(a.nu_start + (double)ka * a.dnu), (float)(a.nu_start + (double)kb * a.dnu));
        constexpr float C1 = (float)(2.0 * bartc::H * bartc::C * bartc::C);
        const float2 c1nu3 = mul2(mul2(f2(C1), nuf), mul2(nuf, nuf));
        // Rayleigh a nu^4 / (mu m_u) (in FP64: a / (mu m_u) may be below the FP32 range)
        float2 chi_r = f2(0.0f);
        if (a.ex.ray != 0.0) {
          const double nua = a.nu_start + (double)ka * a.dnu, nub = a.nu_start + (double)kb * a.dnu;
          chi_r = make_float2((float)(a.ex.ray * (nua * nua) * (nua * nua)), (float)(a.ex.ray * (nub * nub) * (nub * nub)));
        }
        const float* ga = a.grid + ka;
        const unsigned int dkb = (unsigned int)(kb - ka);
        // the flux needs the per-angle transmittances t_i = 2^(tau ang_i)
        // (tau the vertical optical depth from the top, ang_i = -log2(e)/mu_i)
        // only through their quadrature sum Tw = sum_i 2 pi w_i mu_i / 2 t_i,
        // so F = sum_k (B_{k-1} + B_k) (Tw_{k-1} - Tw_k) + 2 B_bottom Tw_bottom
        float2 tau = f2(0.0f), Tw_prev = f2(a.tw_top), F = f2(0.0f);
        const int L_run = a.ex.L_run;
        // grid values of a layer for both wavenumbers: lower (x) and upper (y)
        // temperature bracket per species
        auto fetch = [&](int k, float2* x, float2* y) {
          unsigned int of[4 * NCF];
#pragma unroll
          for (int q = 0; q < NCF; ++q) {
            const uint4 v = s_rec[k].off[q];
            of[4 * q] = v.x;
            of[4 * q + 1] = v.y;
            of[4 * q + 2] = v.z;
            of[4 * q + 3] = v.w;
          }
#pragma unroll
          for (int q = 0; q < S; ++q) {
            if (PAIR) {                            // ka is even and ka + 1 < N here
              x[q] = __ldg(reinterpret_cast<const float2*>(ga + of[2 * q]));
              y[q] = __ldg(reinterpret_cast<const float2*>(ga + of[2 * q + 1]));
            } else {
              x[q] = make_float2(__ldg(ga + of[2 * q]), __ldg(ga + (of[2 * q] + dkb)));
              y[q] = make_float2(__ldg(ga + of[2 * q + 1]), __ldg(ga + (of[2 * q + 1] + dkb)));
            }
          }
        };
        auto chi_of = [&](int k, const float2* x, const float2* y) {
          float cf[4 * NCF];
#pragma unroll
          for (int q = 0; q < NCF; ++q) {
            const float4 v = s_rec[k].cf[q];
            cf[4 * q] = v.x;
            cf[4 * q + 1] = v.y;
            cf[4 * q + 2] = v.z;
            cf[4 * q + 3] = v.w;
          }
          float2 chi = chi_r;
#pragma unroll
          for (int q = 0; q < S; ++q) {
            chi = fma2(f2(cf[2 * q]), x[q], chi);
            chi = fma2(f2(cf[2 * q + 1]), y[q], chi);
          }
          return chi;
        };
        auto planck_k = [&](const float4& pl) {
          if (WIDE_X) return planck2<true>(c1nu3, mul2(nuf, f2(pl.x)));
          return planck_pair(c1nu3, nuf.x, pl.x, pl.z);
        };
        float2 cx[S], cy[S], nx[S], ny[S];
        fetch(0, cx, cy);
        fetch(min(1, L_run - 1), nx, ny);
        float2 chi_prev = chi_of(0, cx, cy);
        float2 B_prev = planck_k(s_rec[0].pl);
        bool done_a = false, done_b = false;       // lane reached the optical-depth limit
#pragma unroll 2
        for (int k = 1; k < L_run; ++k) {
#pragma unroll
          for (int q = 0; q < S; ++q) {
            cx[q] = nx[q];
            cy[q] = ny[q];
          }
          fetch(min(k + 1, L_run - 1), nx, ny);    // the next layer's rows are in flight meanwhile
          const float2 chi = chi_of(k, cx, cy);
          const float4 pl = s_rec[k].pl;
          const float2 B = planck_k(pl);
          const float2 dtau = mul2(add2(chi_prev, chi), f2(pl.y));
          const float2 Bsum = add2(B_prev, B);
          tau = add2(tau, dtau);
          float2 Tw0 = f2(0.0f), Tw1 = f2(0.0f);    // two partial sums: a shorter dependence chain
#pragma unroll
          for (int i = 0; i < NA; ++i) {
            const float2 t = ex2_2(mul2(tau, f2(a.ang[i])));
            if (i & 1) Tw1 = fma2(f2(a.ang[NA + i]), t, Tw1);
            else Tw0 = fma2(f2(a.ang[NA + i]), t, Tw0);
          }
          const float2 Tw = add2(Tw0, Tw1);
          const float2 Fn = fma2(Bsum, sub2(Tw_prev, Tw), F);
          chi_prev = chi;
          if (!TAU_LIM) {
            F = Fn;
            Tw_prev = Tw;
            B_prev = B;
          } else {
            // Sec. 4 item 7: stop at the caller's optical-depth limit; the level
            // reached is the bottom boundary (its blackbody below).  Each
            // wavenumber of the pair keeps its state from the level where it
            // stopped while the other goes on.
            if (!done_a) {
              F.x = Fn.x;
              Tw_prev.x = Tw.x;
              B_prev.x = B.x;
            }
            if (!done_b) {
              F.y = Fn.y;
              Tw_prev.y = Tw.y;
              B_prev.y = B.y;
            }
            done_a = done_a || tau.x > a.ex.tau_cut;
            done_b = done_b || tau.y > a.ex.tau_cut;
            if (done_a && done_b) break;
          }
        }
        F = fma2(mul2(f2(2.0f), B_prev), Tw_prev, F);   // the bottom level's blackbody through the column
        if (a.spectra) {
          const int64_t base = (a.offs ? a.offs[p] : (int64_t)p * a.N) - lo;
          if (act_a) a.spectra[base + ja] = F.x;
          if (act_b) a.spectra[base + jb] = F.y;
        }

        // 3. band sums of the tile, added to the unit's
        if (nb > 0) {
          const float dwa = act_a ? ((hi - lo == 1) ? 1.0f : ((ja == lo || ja == hi - 1) ? 0.5f : 1.0f)) : 0.0f;
          const float dwb = act_b ? ((hi - lo == 1) ? 1.0f : ((jb == lo || jb == hi - 1) ? 0.5f : 1.0f)) : 0.0f;
          const int warp = tid >> 5, lane = tid & 31;
          for (int b = 0; b < nb; ++b) {
            const float Wa = act_a ? __ldg(a.filt + (int64_t)b * a.N + ja) * dwa : 0.0f;
            const float Wb = act_b ? __ldg(a.filt + (int64_t)b * a.N + jb) * dwb : 0.0f;
            float num = fmaf(Wa, F.x, Wb * F.y), den = Wa + Wb;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              num += __shfl_xor_sync(0xffffffffu, num, o);
              den += __shfl_xor_sync(0xffffffffu, den, o);
            }
            if (lane == 0) s_red[warp][b] = make_float2(num, den);
          }
          __syncthreads();
          if (tid < nb) {
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) {
              band_acc.x += s_red[w][tid].x;
              band_acc.y += s_red[w][tid].y;
            }
          }
          __syncthreads();                         // s_red is rewritten by the next tile
        }
      };
      for (int tile = grp * a.tpu; tile < t_end; ++tile) {
        if (pair_loads) column(std::true_type{}, tile);
        else column(std::false_type{}, tile);
      }

      // the unit's band partials; the proposal's last unit reduces them
      if (nb > 0) {
        if (tid < nb) a.partial[((int64_t)p * a.n_groups + grp) * nb + tid] = band_acc;
        __syncthreads();
        if (tid == 0) s_last = (add_acq_rel(a.p_done + p, 1u) + 1u == (unsigned)n_groups_p);
        __syncthreads();
        if (s_last) {
          if (tid < nb) {
            double num = 0.0, den = 0.0;
            for (int q = 0; q < n_groups_p; ++q) {
              const float2 v = __ldcg(a.partial + ((int64_t)p * a.n_groups + q) * nb + tid);
              num += v.x;
              den += v.y;
            }
            a.bands[(int64_t)p * nb + tid] = den > 0.0 ? (float)(num / den) : 0.0f;
          }
          if (tid == 0) a.p_done[p] = 0u;           // ready for the next launch
        }
      }
    }
    __syncthreads();                               // shared state is reused by the next unit
  }
  // the last CTA to leave resets the counters for the next launch
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.work + 1, 1ULL) + 1ULL == (unsigned long long)gridDim.x) {
      a.work[0] = 0ULL;
      a.work[1] = 0ULL;
      a.work[2] += 1ULL;                          // new epoch: published layer states expire
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// The same generation with the grid rows staged in shared memory by bulk
// copies (TMA, cp.async.bulk): a producer warp streams, for each layer of the
// tile, the 2 S rows (species x lower/upper temperature bracket) of TW
// wavenumbers into a ring of TMA_STAGES buffers, each completing on a "full"
// mbarrier; the compute warps read their pairs of wavenumbers from shared
// memory and release the buffer on an "empty" mbarrier.  The compute threads
// issue no global loads and no address arithmetic for the grid, and the rows
// of the next layers are in flight while a layer is computed.  Needs rows
// that start on 16-byte boundaries (n_nu a multiple of 4, 16-byte aligned
// grid); tiles start on a multiple of 4.
constexpr int TMA_STAGES = 4;                  // a power of two: stage and phase by masks
#ifndef TMA_OCC_THREADS
#define TMA_OCC_THREADS 768
#endif

template <int S, int NA, int TW>
__global__ void __launch_bounds__(TW / 2 + 32, TMA_OCC_THREADS / (TW / 2 + 32))
emission_tma_kernel(const __grid_constant__ FusedArgs a) {
  constexpr int NT = TW / 2;                      // compute threads, two wavenumbers each
  constexpr int ROWS = 2 * S;                     // rows per layer: species x (lower, upper bracket)
  extern __shared__ __align__(128) float s_stage[];   // [TMA_STAGES][ROWS][TW]
  __shared__ unsigned long long s_full[TMA_STAGES], s_empty[TMA_STAGES];
  __shared__ LayerTW s_tw[MAX_LAYERS];
  __shared__ float4 s_cf[MAX_LAYERS][(2 * S + 3) / 4];   // per layer: X_s (1 - w), X_s w
  __shared__ float s_y[MAX_LAYERS];                       // (c2 / T) log2(e)
  __shared__ float s_dpg[MAX_LAYERS];
  __shared__ float s_xs[S];
  __shared__ float2 s_red[NT / 32][MAX_BANDS];
  __shared__ unsigned long long s_unit;
  __shared__ int s_last, s_ready;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr int NTH = NT + 32;
  const bool producer = tid >= NT;                // the last warp issues the copies
  const int L = a.L, nb = a.n_bands;
  if (tid == 0) {
    for (int q = 0; q < TMA_STAGES; ++q) {
      mbar_init(&s_full[q], 1);
      mbar_init(&s_empty[q], NT / 32);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int k = tid; k + 1 < L; k += NTH) s_dpg[k] = a.dpg[k];
  const int64_t sstride = (int64_t)L * a.M * a.N;
  const int64_t dm = (a.M > 1) ? a.N : 0;          // offset of the upper temperature bracket
  const unsigned int ready_mark = (unsigned int)*(volatile unsigned long long*)(a.work + 2) + 1u;
  unsigned long long next_unit = 0;
  if (tid == 0) next_unit = atomicAdd(a.work, 1ULL);
  unsigned int q_layer = 0;                        // layers streamed so far (all roles agree)
  unsigned int q_issued = 0;                       // producer: layers whose copies were issued

  for (;;) {
    if (tid == 0) {
      s_unit = next_unit;
      next_unit = atomicAdd(a.work, 1ULL);
    }
    __syncthreads();
    const unsigned long long u = s_unit;
    if (u >= a.n_units || s_abort) break;
    const int p = (int)(u % (unsigned long long)a.n);
    const int grp = (int)(u / (unsigned long long)a.n);
    bool skip = a.active && !a.active[p];
    int64_t lo = 0, hi = a.N;
    if (!skip) {
      lo = a.nu_lo ? a.nu_lo[p] : 0;
      hi = a.nu_hi ? a.nu_hi[p] : a.N;
      if (lo < 0 || hi > a.N || lo >= hi) {
        if (grp == 0) {
          if (tid == 0) atomicOr(a.status, BART_DEV_RANGE);
          if (a.bands && tid < nb) a.bands[(int64_t)p * nb + tid] = 0.0f;
        }
        skip = true;
      }
    }
    const int64_t lo4 = lo & ~(int64_t)3;          // tiles start on a multiple of 4 (16-byte rows)
    const int n_tiles_p = skip ? 0 : (int)((hi - lo4 + TW - 1) / TW);
    const int n_groups_p = (n_tiles_p + a.tpu - 1) / a.tpu;
    if (!skip && grp < n_groups_p) {
      // 1. layer states of the proposal (published once per proposal, as in
      // emission_fused_kernel), then per layer the interpolation-abundance
      // coefficients and the Planck exponent
      if (tid == 0) s_ready = (ld_acquire(a.tw_flag + p) == ready_mark);
      if (tid < S) {
        const float ab = a.theta ? a.theta[(int64_t)p * a.n_theta + 5 + tid] : 0.0f;
        s_xs[tid] = a.x0mu[tid] * exp10f(ab);
      }
      __syncthreads();
      if (s_ready) {
        for (int k = tid; k < L; k += NTH) {
          const int4 v = __ldcg(reinterpret_cast<const int4*>(a.tw_cache + (int64_t)p * L + k));
          LayerTW r;
          r.row = (int64_t)(((unsigned long long)(unsigned int)v.y << 32) | (unsigned int)v.x);
          r.w = __int_as_float(v.z);
          r.c2_t = __int_as_float(v.w);
          s_tw[k] = r;
        }
      } else {
        for (int k = tid; k < L; k += NTH) {
          float T;
          if (a.t_profile) {
            T = a.t_profile[(int64_t)p * L + k];
          } else {
            float th[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) th[i] = a.theta[(int64_t)p * a.n_theta + i];
            T = bartf::tp_temperature(th, a.p_cgs[k], a.inv_g, a.tint4, a.tirr0);
          }
          const LayerTW r = layer_state(T, k, a.t_axis, a.M, a.N, a.t_min, a.t_max, a.status);
          s_tw[k] = r;
          a.tw_cache[(int64_t)p * L + k] = r;
        }
        __syncthreads();
        if (tid == 0) st_release(a.tw_flag + p, ready_mark);
      }
      __syncthreads();
      for (int k = tid; k < L; k += NTH) {
        const float w = s_tw[k].w;
        float cf[4 * ((2 * S + 3) / 4)] = {};
#pragma unroll
        for (int q = 0; q < S; ++q) {
          cf[2 * q] = s_xs[q] * (1.0f - w);
          cf[2 * q + 1] = s_xs[q] * w;
        }
#pragma unroll
        for (int q = 0; q < (2 * S + 3) / 4; ++q)
          s_cf[k][q] = make_float4(cf[4 * q], cf[4 * q + 1], cf[4 * q + 2], cf[4 * q + 3]);
        s_y[k] = s_tw[k].c2_t * LOG2E;
      }
      __syncthreads();
      float2 band_acc = make_float2(0.f, 0.f);
      const int t_end = min((grp + 1) * a.tpu, n_tiles_p);
      const int L_run = a.ex.L_run;

      for (int tile = grp * a.tpu; tile < t_end; ++tile) {
        const int64_t t0 = lo4 + (int64_t)tile * TW;
        if (producer) {
          // 2a. stream the tile's rows layer by layer (one lane)
          if (lane == 0) {
            const unsigned int bytes = (unsigned int)(min((int64_t)TW, a.N - t0) * (int64_t)sizeof(float));
            for (int k = 0; k < L_run; ++k) {
              const unsigned int q = q_layer + k, st = q & (TMA_STAGES - 1), ph = (q / TMA_STAGES) & 1u;
              if (!mbar_wait(&s_empty[st], ph ^ 1u, &s_abort)) {
                s_abort = 1;
                atomicOr(a.status, BART_DEV_TIMEOUT);
                break;
              }
              mbar_arrive_expect_tx(&s_full[st], bytes * ROWS);
              const float* src = a.grid + s_tw[k].row + t0;
              float* dst = s_stage + (size_t)st * ROWS * TW;
#pragma unroll
              for (int sp = 0; sp < S; ++sp) {
                bulk_load(dst + (2 * sp) * TW, src + sp * sstride, bytes, &s_full[st]);
                bulk_load(dst + (2 * sp + 1) * TW, src + sp * sstride + dm, bytes, &s_full[st]);
              }
              q_issued = q + 1;
            }
          }
        } else {
          // 2b. the columns of wavenumbers ja and ja + 1 from the staged rows
          const int64_t ja = t0 + 2 * tid, jb = ja + 1;
          const bool act_a = ja >= lo && ja < hi, act_b = jb >= lo && jb < hi;
          const int64_t ka = (ja < hi) ? ja : lo, kb = (jb < hi) ? jb : lo;
          const double nua = a.nu_start + (double)ka * a.dnu, nub = a.nu_start + (double)kb * a.dnu;
          const float2 c1nu3 = make_float2((float)(2.0 * bartc::H * bartc::C * bartc::C * nua * nua * nua),
                                           (float)(2.0 * bartc::H * bartc::C * bartc::C * nub * nub * nub));
          const float2 nuf = make_float2((float)nua, (float)nub);
          const float2 chi_r = make_float2((float)(a.ex.ray * (nua * nua) * (nua * nua)),
                                           (float)(a.ex.ray * (nub * nub) * (nub * nub)));
          float2 lt[NA];
#pragma unroll
          for (int i = 0; i < NA; ++i) lt[i] = f2(0.0f);
          float2 Tw_prev = f2(a.tw_top), F = f2(0.0f), chi_prev, B_prev;
          float2 tau_v = f2(0.0f);
          bool done_a = false, done_b = false;
          unsigned int st = q_layer & (TMA_STAGES - 1), ph = (q_layer / TMA_STAGES) & 1u;
          const float* my_stage = s_stage + 2 * tid;
          // layer k's rows from the ring: opacity of both wavenumbers; false
          // when the wait for the rows was given up
          auto take = [&](int k, float2& chi) -> bool {
            if (!mbar_wait(&s_full[st], ph, &s_abort)) {
              s_abort = 1;
              atomicOr(a.status, BART_DEV_TIMEOUT);
              return false;
            }
            const float* buf = my_stage + st * (ROWS * TW);
            float2 x[S], y[S];
#pragma unroll
            for (int sp = 0; sp < S; ++sp) {
              x[sp] = *reinterpret_cast<const float2*>(buf + (2 * sp) * TW);
              y[sp] = *reinterpret_cast<const float2*>(buf + (2 * sp + 1) * TW);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_empty[st]);      // the buffer may be refilled
            st = (st + 1) & (TMA_STAGES - 1);
            ph ^= (st == 0) ? 1u : 0u;
            float cf[4 * ((2 * S + 3) / 4)];
#pragma unroll
            for (int q4 = 0; q4 < (2 * S + 3) / 4; ++q4) {
              const float4 v = s_cf[k][q4];
              cf[4 * q4] = v.x;
              cf[4 * q4 + 1] = v.y;
              cf[4 * q4 + 2] = v.z;
              cf[4 * q4 + 3] = v.w;
            }
            chi = chi_r;
#pragma unroll
            for (int sp = 0; sp < S; ++sp) {
              chi = fma2(f2(cf[2 * sp]), x[sp], chi);
              chi = fma2(f2(cf[2 * sp + 1]), y[sp], chi);
            }
            return true;
          };
          bool ok = take(0, chi_prev);
          B_prev = planck2<true>(c1nu3, mul2(nuf, f2(s_y[0])), a.wide_x);
          for (int k = 1; ok && k < L_run; ++k) {
            float2 chi;
            if (!take(k, chi)) break;
            const float2 B = planck2<true>(c1nu3, mul2(nuf, f2(s_y[k])), a.wide_x);
            const float2 dtau = mul2(add2(chi_prev, chi), f2(s_dpg[k - 1]));
            const float2 Bsum = add2(B_prev, B);
            float2 Tw0 = f2(0.0f), Tw1 = f2(0.0f);
#pragma unroll
            for (int i = 0; i < NA; ++i) {
              lt[i] = fma2(dtau, f2(a.ang[i]), lt[i]);
              if (i & 1) Tw1 = fma2(f2(a.ang[NA + i]), ex2_2(lt[i]), Tw1);
              else Tw0 = fma2(f2(a.ang[NA + i]), ex2_2(lt[i]), Tw0);
            }
            const float2 Tw = add2(Tw0, Tw1);
            const float2 Fn = fma2(Bsum, sub2(Tw_prev, Tw), F);
            chi_prev = chi;
            if (!a.tau_lim) {
              F = Fn;
              Tw_prev = Tw;
              B_prev = B;
            } else {
              // Sec. 4 item 7: each wavenumber keeps its state from the level
              // where its vertical optical depth first exceeds the limit
              if (!done_a) {
                F.x = Fn.x;
                Tw_prev.x = Tw.x;
                B_prev.x = B.x;
              }
              if (!done_b) {
                F.y = Fn.y;
                Tw_prev.y = Tw.y;
                B_prev.y = B.y;
              }
              tau_v = add2(tau_v, dtau);
              done_a = done_a || tau_v.x > a.ex.tau_cut;
              done_b = done_b || tau_v.y > a.ex.tau_cut;
            }
          }
          F = fma2(mul2(f2(2.0f), B_prev), Tw_prev, F);
          if (a.spectra) {
            const int64_t base = (a.offs ? a.offs[p] : (int64_t)p * a.N) - lo;
            if (act_a) a.spectra[base + ja] = F.x;
            if (act_b) a.spectra[base + jb] = F.y;
          }
          if (nb > 0) {
            const float dwa = act_a ? ((hi - lo == 1) ? 1.0f : ((ja == lo || ja == hi - 1) ? 0.5f : 1.0f)) : 0.0f;
            const float dwb = act_b ? ((hi - lo == 1) ? 1.0f : ((jb == lo || jb == hi - 1) ? 0.5f : 1.0f)) : 0.0f;
            const int warp = tid >> 5;
            for (int b = 0; b < nb; ++b) {
              const float Wa = act_a ? __ldg(a.filt + (int64_t)b * a.N + ja) * dwa : 0.0f;
              const float Wb = act_b ? __ldg(a.filt + (int64_t)b * a.N + jb) * dwb : 0.0f;
              // idle lanes add exact zeros (their F may be computed on stale rows)
              float num = (act_a ? Wa * F.x : 0.0f) + (act_b ? Wb * F.y : 0.0f), den = Wa + Wb;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                num += __shfl_xor_sync(0xffffffffu, num, o);
                den += __shfl_xor_sync(0xffffffffu, den, o);
              }
              if (lane == 0) s_red[warp][b] = make_float2(num, den);
            }
          }
        }
        q_layer += L_run;
        if (nb > 0) {
          __syncthreads();
          if (tid < nb) {
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) {
              band_acc.x += s_red[w][tid].x;
              band_acc.y += s_red[w][tid].y;
            }
          }
        }
        __syncthreads();                           // s_red and the ring are reused by the next tile
        if (s_abort) break;
      }

      if (nb > 0 && !s_abort) {
        if (tid < nb) a.partial[((int64_t)p * a.n_groups + grp) * nb + tid] = band_acc;
        __syncthreads();
        if (tid == 0) s_last = (add_acq_rel(a.p_done + p, 1u) + 1u == (unsigned)n_groups_p);
        __syncthreads();
        if (s_last) {
          if (tid < nb) {
            double num = 0.0, den = 0.0;
            for (int q = 0; q < n_groups_p; ++q) {
              const float2 v = __ldcg(a.partial + ((int64_t)p * a.n_groups + q) * nb + tid);
              num += v.x;
              den += v.y;
            }
            a.bands[(int64_t)p * nb + tid] = den > 0.0 ? (float)(num / den) : 0.0f;
          }
          if (tid == 0) a.p_done[p] = 0u;
        }
      }
    }
    __syncthreads();
  }
  // after a timeout the producer waits (bounded) for the copies it issued
  // that may still be in flight, so none lands after the CTA has left
  if (s_abort && producer && lane == 0) {
    const unsigned int first = q_issued > (unsigned)TMA_STAGES ? q_issued - TMA_STAGES : 0u;
    for (unsigned int q = first; q < q_issued; ++q) {
      volatile int no_abort = 0;
      mbar_wait(&s_full[q & (TMA_STAGES - 1)], (q / TMA_STAGES) & 1u, &no_abort);
    }
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.work + 1, 1ULL) + 1ULL == (unsigned long long)gridDim.x) {
      a.work[0] = 0ULL;
      a.work[1] = 0ULL;
      a.work[2] += 1ULL;
      __threadfence();
    }
  }
}

using FusedLauncher = cudaError_t (*)(const FusedArgs&, int, cudaStream_t);

// Wavenumbers per tile the autotuner chooses from (two per compute thread;
// at least 128, so a CTA has a thread for each of up to 64 bands).
constexpr int FUSED_TILES[3] = {128, 256, 512};

template <int S, int NA, int TW, int MODE>
cudaError_t launch_pair(const FusedArgs& a, int sm_count, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, emission_fused_kernel<S, NA, TW, MODE>, TW / 2, 0);
  if (e != cudaSuccess) return e;
  unsigned long long grid = (unsigned long long)(per_sm < 1 ? 1 : per_sm) * (unsigned long long)sm_count;
  if (grid > a.n_units) grid = a.n_units;
  emission_fused_kernel<S, NA, TW, MODE><<<(unsigned)grid, TW / 2, 0, st>>>(a);
  return cudaGetLastError();
}

template <int S, int NA, int TW>
cudaError_t launch_tma(const FusedArgs& a, int sm_count, cudaStream_t st) {
  const size_t smem = (size_t)TMA_STAGES * 2 * S * TW * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(emission_tma_kernel<S, NA, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, emission_tma_kernel<S, NA, TW>, TW / 2 + 32, smem);
  if (e != cudaSuccess) return e;
  unsigned long long grid = (unsigned long long)(per_sm < 1 ? 1 : per_sm) * (unsigned long long)sm_count;
  if (grid > a.n_units) grid = a.n_units;
  emission_tma_kernel<S, NA, TW><<<(unsigned)grid, TW / 2 + 32, smem, st>>>(a);
  return cudaGetLastError();
}

// Launcher of the fused generation for S species and na angles at tile tw:
// the bulk-copy kernel (tma; its options are run-time flags), else the
// global-load kernel with the compile-time mode (bit 0 FP64 Planck branch,
// bit 1 optical-depth limit).  Instantiated once per species count, each in
// its own translation unit.
template <int S>
FusedLauncher fused_launcher(int na, bool tma, int tw, int mode);

extern template FusedLauncher fused_launcher<1>(int, bool, int, int);
extern template FusedLauncher fused_launcher<2>(int, bool, int, int);
extern template FusedLauncher fused_launcher<3>(int, bool, int, int);
extern template FusedLauncher fused_launcher<4>(int, bool, int, int);

template <int S, int NA, int TW>
FusedLauncher pick_mode(bool tma, int mode) {
  if (tma) return launch_tma<S, NA, TW>;
  switch (mode) {
    case 0: return launch_pair<S, NA, TW, 0>;
    case 1: return launch_pair<S, NA, TW, 1>;
    case 2: return launch_pair<S, NA, TW, 2>;
    default: return launch_pair<S, NA, TW, 3>;
  }
}

template <int S, int NA>
FusedLauncher pick_tile(bool tma, int tw, int mode) {
  switch (tw) {
    case 128: return pick_mode<S, NA, 128>(tma, mode);
    case 256: return pick_mode<S, NA, 256>(tma, mode);
    case 512: return pick_mode<S, NA, 512>(tma, mode);
    default: return nullptr;
  }
}

template <int S>
FusedLauncher fused_launcher(int na, bool tma, int tw, int mode) {
  switch (na) {
    case 1: return pick_tile<S, 1>(tma, tw, mode);
    case 2: return pick_tile<S, 2>(tma, tw, mode);
    case 4: return pick_tile<S, 4>(tma, tw, mode);
    case 8: return pick_tile<S, 8>(tma, tw, mode);
    case 16: return pick_tile<S, 16>(tma, tw, mode);
    default: return nullptr;
  }
}

}  // namespace bartem
