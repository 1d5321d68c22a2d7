// Differential-evolution MCMC with surrogate screening (Sec. 3: the sampler
// proposes parameter sets and compares the band-integrated spectra to data;
// Sec. 4 item 10 and Sec. 5, ter Braak 2006 DE-MC).
//
// Chains are split into two halves; a half-step updates the chains of one
// half with differences of chains drawn from the other half, so every update
// is a Metropolis-Hastings step conditional on the other half and the
// population keeps the target as its stationary distribution.
//   proposal  y_i = x_i + gamma (x_r1 - x_r2) + e_i,  r1 != r2 from the other
//             half, e_i ~ N(0, (eps * box width)^2) per parameter;
//             gamma = 2.38 / sqrt(2 d) except every `jump_every`-th
//             generation, where gamma = 1 lets chains jump between modes.
//   prior     uniform on the box [lo, hi]; a proposal outside is rejected.
//   screen    delayed acceptance (two-stage Metropolis-Hastings): stage 1
//             passes with probability min(1, exp(ls_y - ls_x)) from the
//             surrogate log-likelihood; stage 2 accepts a survivor with
//             probability min(1, exp((L_y - L_x) - (ls_y - ls_x))) from the
//             exact model.  Rejected proposals never reach the exact model;
//             every accepted sample has its exact log-likelihood.
// DEMCzs (Sec. 4; ter Braak & Vrugt 2008), set by bart_demc_set_archive:
// every chain proposes from an archive Z of past states, so all chains move
// in one step.  With probability p_snooker a snooker move: z, z1, z2 from Z,
// y = x + g_s ((z1 - z2) . e) e, e the unit vector from z to x, g_s in
// [1.2, 2.2), and the factor q = (|y - z| / |x - z|)^(d - 1) in the
// Metropolis ratio; otherwise y = x + gamma (z1 - z2) + noise (q = 1).  The
// screen's stage 1 is min(1, exp(beta (ls_y - ls_x) + margin) q) and stage 2
// min(1, exp(L_y - L_x) q a1(y -> x) / a1(x -> y)).  Every `thin` steps the
// chains' states are appended to Z while it has room; the count lives on the
// device so a replayed graph keeps appending.
// Random numbers come from a counter-based generator (SplitMix64 finaliser
// of seed, generation, chain and draw index), so a generation's draws do not
// depend on launch order and the loop can be captured in a CUDA graph.
#include <cmath>
#include <vector>

#include "bart_internal.cuh"

struct bart_demc {
  bart_ctx* ctx = nullptr;
  int C = 0, d = 0;
  double gamma = 0.0;
  int jump_every = 0;
  double eps = 0.0;
  uint64_t seed = 0;
  float* lo = nullptr;      // device [d]
  float* hi = nullptr;      // device [d]
  float* x = nullptr;       // device [C][d] current states
  double* L = nullptr;      // device [C] exact log-likelihood
  double* Ls = nullptr;     // device [C] surrogate log-likelihood
  const int64_t* hs_dev = nullptr;   // if set, kernels read the half-step index here
  double beta = 1.0;        // stage-1 temperature of the surrogate log-likelihood
  double margin = 0.0;      // stage-1 margin
  // DEMCzs archive (zs mode)
  bool zs = false;
  float* Z = nullptr;       // device [cap][d]
  int64_t cap = 0;
  long long* zc = nullptr;  // device: states in Z
  int thin = 10;
  double p_snooker = 0.1;
  double* logq = nullptr;   // device [C] log proposal factor of the last proposal
};

namespace {

constexpr int DEMC_MAX_PARAMS = 32;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Uniform (0, 1) double from the counter (seed, gen, chain, k).
__device__ __forceinline__ double uniform(uint64_t seed, int64_t gen, int chain, int k) {
  uint64_t h = mix64(seed ^ mix64((uint64_t)gen * 0x100000001B3ULL ^ mix64(((uint64_t)chain << 32) | (uint32_t)k)));
  return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double normal(uint64_t seed, int64_t gen, int chain, int k) {
  // Box-Muller on two uniforms of this counter
  double u1 = uniform(seed, gen, chain, 2 * k), u2 = uniform(seed, gen, chain, 2 * k + 1);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Chains of half h: [h*C/2, (h+1)*C/2) with C/2 rounded down for h = 0.
__device__ __forceinline__ void half_range(int C, int h, int& b, int& e) {
  const int c0 = C / 2;
  b = h ? c0 : 0;
  e = h ? C : c0;
}

__global__ void propose_kernel(int C, int d, const float* __restrict__ x, const float* __restrict__ lo,
                               const float* __restrict__ hi, int64_t gen_arg, const int64_t* __restrict__ gen_dev,
                               uint64_t seed, double gamma, int jump_every, double eps, float* __restrict__ y,
                               int32_t* __restrict__ inbox) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int64_t gen = gen_dev ? *gen_dev : gen_arg;
  const int h = (int)(gen & 1);               // half updated this half-step
  int b, e, ob, oe;
  half_range(C, h, b, e);
  half_range(C, 1 - h, ob, oe);
  if (i < b || i >= e) {                      // not updated: copy, mark inactive
    for (int q = 0; q < d; ++q) y[(int64_t)i * d + q] = x[(int64_t)i * d + q];
    inbox[i] = 0;
    return;
  }
  const int no = oe - ob;
  const int r1 = ob + min((int)(uniform(seed, gen, i, 0) * no), no - 1);
  int r2 = ob + min((int)(uniform(seed, gen, i, 1) * (no - 1)), no - 2);
  if (r2 >= r1) ++r2;
  const int64_t g2 = gen >> 1;                // generation index (two half-steps each)
  const double gm = (jump_every > 0 && (g2 % jump_every) == jump_every - 1) ? 1.0 : gamma;
  int ok = 1;
  for (int q = 0; q < d; ++q) {
    const double w = (double)hi[q] - (double)lo[q];
    const double v = (double)x[(int64_t)i * d + q] +
                     gm * ((double)x[(int64_t)r1 * d + q] - (double)x[(int64_t)r2 * d + q]) +
                     eps * w * normal(seed, gen, i, 8 + q);
    const float vf = (float)v;
    y[(int64_t)i * d + q] = vf;
    ok &= (vf >= lo[q]) && (vf <= hi[q]);
  }
  inbox[i] = ok;
}

// DEMCzs proposals: all chains, from the archive.
__global__ void propose_zs_kernel(int C, int d, const float* __restrict__ x, const float* __restrict__ lo,
                                  const float* __restrict__ hi, int64_t gen_arg, const int64_t* __restrict__ gen_dev,
                                  uint64_t seed, double gamma, int jump_every, double eps, const float* __restrict__ Z,
                                  const long long* __restrict__ zc, double p_snooker, float* __restrict__ y,
                                  int32_t* __restrict__ inbox, double* __restrict__ logq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int64_t gen = gen_dev ? *gen_dev : gen_arg;
  const int m = (int)*zc;
  const int a = min((int)(uniform(seed, gen, i, 51) * m), m - 1);
  int b = min((int)(uniform(seed, gen, i, 52) * (m - 1)), m - 2);
  if (b >= a) ++b;
  const float* xi = x + (int64_t)i * d;
  const float* za = Z + (int64_t)a * d;
  const float* zb = Z + (int64_t)b * d;
  double lq = 0.0;
  int ok = 1;
  if (uniform(seed, gen, i, 50) < p_snooker) {
    const int c = min((int)(uniform(seed, gen, i, 53) * m), m - 1);
    const float* zz = Z + (int64_t)c * d;
    double nn = 0.0, proj = 0.0;
    for (int q = 0; q < d; ++q) {
      const double e = (double)xi[q] - zz[q];
      nn += e * e;
      proj += ((double)za[q] - zb[q]) * e;
    }
    if (nn == 0.0) {                          // x on an archive state: no move
      ok = 0;
      for (int q = 0; q < d; ++q) y[(int64_t)i * d + q] = xi[q];
    } else {
      const double gs = 1.2 + uniform(seed, gen, i, 54);
      const double f = gs * proj / nn;
      double ny = 0.0;
      for (int q = 0; q < d; ++q) {
        const double e = (double)xi[q] - zz[q];
        const float vf = (float)((double)xi[q] + f * e);
        y[(int64_t)i * d + q] = vf;
        ok &= (vf >= lo[q]) && (vf <= hi[q]);
        const double dy = (double)vf - zz[q];
        ny += dy * dy;
      }
      lq = (d - 1) * 0.5 * (log(ny) - log(nn));
    }
  } else {
    const double gm = (jump_every > 0 && (gen % jump_every) == jump_every - 1) ? 1.0 : gamma;
    for (int q = 0; q < d; ++q) {
      const double w = (double)hi[q] - (double)lo[q];
      const float vf = (float)((double)xi[q] + gm * ((double)za[q] - zb[q]) + eps * w * normal(seed, gen, i, 8 + q));
      y[(int64_t)i * d + q] = vf;
      ok &= (vf >= lo[q]) && (vf <= hi[q]);
    }
  }
  inbox[i] = ok;
  logq[i] = lq;
}

// Appends the chains' states to the archive every `thin` steps while it has room.
__global__ void archive_kernel(int C, int d, const float* __restrict__ x, int64_t gen_arg,
                               const int64_t* __restrict__ gen_dev, int thin, float* __restrict__ Z, int64_t cap,
                               long long* __restrict__ zc) {
  const int64_t gen = gen_dev ? *gen_dev : gen_arg;
  const long long m = *zc;
  if ((gen + 1) % thin != 0 || m + C > cap) return;
  for (int64_t e = threadIdx.x; e < (int64_t)C * d; e += blockDim.x) Z[m * d + e] = x[e];
  __syncthreads();
  if (threadIdx.x == 0) *zc = m + C;
}

// log of the stage-1 acceptance a1(x -> y) = min(1, exp(beta (ls_y - ls_x) + margin) q)
__device__ __forceinline__ double log_a1(double d, double beta, double margin, double lq = 0.0) {
  return fmin(0.0, beta * d + margin + lq);
}

__global__ void screen_kernel(int C, const int32_t* __restrict__ inbox, const double* __restrict__ ls_y,
                              const double* __restrict__ ls_x, int64_t gen_arg, const int64_t* __restrict__ gen_dev,
                              uint64_t seed, double beta, double margin, const double* __restrict__ logq,
                              int32_t* __restrict__ pass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int64_t gen = gen_dev ? *gen_dev : gen_arg;
  int p = inbox[i];
  if (p && ls_y) {
    const double lu = log(uniform(seed, gen, i, 100));
    p = lu < log_a1(ls_y[i] - ls_x[i], beta, margin, logq ? logq[i] : 0.0);
  }
  pass[i] = p;
}

__global__ void accept_kernel(int C, int d, float* __restrict__ x, double* __restrict__ L, double* __restrict__ Ls,
                              const float* __restrict__ y, const int32_t* __restrict__ pass,
                              const double* __restrict__ L_y, const double* __restrict__ ls_y, int64_t gen_arg,
                              const int64_t* __restrict__ gen_dev, uint64_t seed, double beta, double margin,
                              const double* __restrict__ logq, int32_t* __restrict__ accepted) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int64_t gen = gen_dev ? *gen_dev : gen_arg;
  int a = 0;
  if (pass[i]) {
    const double lq = logq ? logq[i] : 0.0;   // proposal factor (DEMCzs snooker moves)
    double r = L_y[i] - L[i] + lq;
    if (ls_y) {
      // delayed acceptance: the stage-1 probabilities of the reverse and the
      // forward move enter the stage-2 ratio (for beta = 1, margin = 0 and a
      // symmetric proposal this is -(ls_y - ls_x))
      const double d = ls_y[i] - Ls[i];
      r += log_a1(-d, beta, margin, -lq) - log_a1(d, beta, margin, lq);
    }
    const double lu = log(uniform(seed, gen, i, 101));
    a = (r >= 0.0) || (lu < r);
    if (!(L_y[i] == L_y[i])) a = 0;           // a NaN likelihood is never accepted
  }
  if (a) {
    for (int q = 0; q < d; ++q) x[(int64_t)i * d + q] = y[(int64_t)i * d + q];
    L[i] = L_y[i];
    if (ls_y) Ls[i] = ls_y[i];
  }
  if (accepted) accepted[i] = a;
}

// out[i] = -1/2 sum_b ((m_ib - d_b) / s_b)^2 in FP64; -inf where mask[i] == 0.
__global__ void loglike_kernel(const float* __restrict__ m, int n, int nb, const float* __restrict__ data,
                               const float* __restrict__ sigma, const int32_t* __restrict__ mask,
                               double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mask && !mask[i]) {
    out[i] = -INFINITY;
    return;
  }
  double s = 0.0;
  for (int b = 0; b < nb; ++b) {
    const double r = ((double)m[(int64_t)i * nb + b] - (double)data[b]) / (double)sigma[b];
    s += r * r;
  }
  out[i] = -0.5 * s;
}

unsigned nblk(int n) { return (unsigned)((n + 127) / 128); }

}  // namespace

extern "C" bart_status bart_demc_create(bart_ctx* ctx, int n_chains, int n_params, const float* lo, const float* hi,
                                        double gamma, int jump_every, double eps, uint64_t seed, bart_demc** out) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, out && lo && hi, "NULL out, lo or hi");
  *out = nullptr;
  BART_REQUIRE(ctx, n_chains >= 3 && n_chains <= 65536, "n_chains must be in [3, 65536]");
  BART_REQUIRE(ctx, n_params >= 1 && n_params <= DEMC_MAX_PARAMS, "n_params must be in [1, %d]", DEMC_MAX_PARAMS);
  for (int q = 0; q < n_params; ++q)
    BART_REQUIRE(ctx, std::isfinite(lo[q]) && std::isfinite(hi[q]) && hi[q] > lo[q], "bad prior box");
  BART_REQUIRE(ctx, gamma >= 0 && std::isfinite(gamma) && eps >= 0 && std::isfinite(eps) && jump_every >= 0,
               "bad gamma, eps or jump_every");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  bart_demc* s = new bart_demc();
  s->ctx = ctx;
  s->C = n_chains;
  s->d = n_params;
  s->gamma = gamma > 0 ? gamma : 2.38 / std::sqrt(2.0 * n_params);
  s->jump_every = jump_every;
  s->eps = eps;
  s->seed = seed;
  bool ok = cudaMalloc(&s->lo, n_params * 4) == cudaSuccess && cudaMalloc(&s->hi, n_params * 4) == cudaSuccess &&
            cudaMalloc(&s->x, (size_t)n_chains * n_params * 4) == cudaSuccess &&
            cudaMalloc(&s->L, (size_t)n_chains * 8) == cudaSuccess &&
            cudaMalloc(&s->Ls, (size_t)n_chains * 8) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    bart_demc_destroy(s);
    return bart_fail(ctx, BART_ENOMEM, "DE-MC allocation failed");
  }
  BART_CUDA(ctx, cudaMemcpy(s->lo, lo, n_params * 4, cudaMemcpyHostToDevice));
  BART_CUDA(ctx, cudaMemcpy(s->hi, hi, n_params * 4, cudaMemcpyHostToDevice));
  BART_CUDA(ctx, cudaMemset(s->Ls, 0, (size_t)n_chains * 8));
  *out = s;
  return BART_OK;
}

extern "C" void bart_demc_destroy(bart_demc* s) {
  if (!s) return;
  cudaSetDevice(s->ctx->device);
  cudaStreamSynchronize(s->ctx->stream);
  for (void* p : {(void*)s->lo, (void*)s->hi, (void*)s->x, (void*)s->L, (void*)s->Ls, (void*)s->Z, (void*)s->zc,
                  (void*)s->logq})
    if (p) cudaFree(p);
  delete s;
}

extern "C" bart_status bart_demc_set_state(bart_demc* s, const float* x, const double* loglike,
                                           const double* loglike_s) {
  if (!s) return BART_EINVAL;
  BART_REQUIRE(s->ctx, x && loglike, "NULL x or loglike");
  cudaStream_t st = s->ctx->stream;
  BART_CUDA(s->ctx, cudaMemcpyAsync(s->x, x, (size_t)s->C * s->d * 4, cudaMemcpyDeviceToDevice, st));
  BART_CUDA(s->ctx, cudaMemcpyAsync(s->L, loglike, (size_t)s->C * 8, cudaMemcpyDeviceToDevice, st));
  if (loglike_s)
    BART_CUDA(s->ctx, cudaMemcpyAsync(s->Ls, loglike_s, (size_t)s->C * 8, cudaMemcpyDeviceToDevice, st));
  else
    BART_CUDA(s->ctx, cudaMemsetAsync(s->Ls, 0, (size_t)s->C * 8, st));
  return BART_OK;
}

extern "C" bart_status bart_demc_get_state(bart_demc* s, float* x, double* loglike, double* loglike_s) {
  if (!s) return BART_EINVAL;
  cudaStream_t st = s->ctx->stream;
  if (x) BART_CUDA(s->ctx, cudaMemcpyAsync(x, s->x, (size_t)s->C * s->d * 4, cudaMemcpyDeviceToDevice, st));
  if (loglike) BART_CUDA(s->ctx, cudaMemcpyAsync(loglike, s->L, (size_t)s->C * 8, cudaMemcpyDeviceToDevice, st));
  if (loglike_s)
    BART_CUDA(s->ctx, cudaMemcpyAsync(loglike_s, s->Ls, (size_t)s->C * 8, cudaMemcpyDeviceToDevice, st));
  return BART_OK;
}

extern "C" bart_status bart_demc_propose(bart_demc* s, int64_t half_step, float* y, int32_t* inbox) {
  if (!s) return BART_EINVAL;
  BART_REQUIRE(s->ctx, y && inbox, "NULL y or inbox");
  BART_REQUIRE(s->ctx, half_step >= 0, "half_step must be >= 0");
  if (s->zs) {
    propose_zs_kernel<<<nblk(s->C), 128, 0, s->ctx->stream>>>(s->C, s->d, s->x, s->lo, s->hi, half_step, s->hs_dev,
                                                              s->seed, s->gamma, s->jump_every, s->eps, s->Z, s->zc,
                                                              s->p_snooker, y, inbox, s->logq);
    return bart_check_launch(s->ctx, "propose_zs_kernel");
  }
  BART_REQUIRE(s->ctx, s->C >= 6, "DE-MC needs at least 6 chains (3 per half); DEMCzs needs 3");
  propose_kernel<<<nblk(s->C), 128, 0, s->ctx->stream>>>(s->C, s->d, s->x, s->lo, s->hi, half_step, s->hs_dev,
                                                         s->seed, s->gamma, s->jump_every, s->eps, y, inbox);
  return bart_check_launch(s->ctx, "propose_kernel");
}

extern "C" bart_status bart_demc_screen(bart_demc* s, int64_t half_step, const int32_t* inbox, const double* ls_y,
                                        int32_t* pass) {
  if (!s) return BART_EINVAL;
  BART_REQUIRE(s->ctx, inbox && pass, "NULL inbox or pass");
  screen_kernel<<<nblk(s->C), 128, 0, s->ctx->stream>>>(s->C, inbox, ls_y, s->Ls, half_step, s->hs_dev, s->seed,
                                                        s->beta, s->margin, s->zs ? s->logq : nullptr, pass);
  return bart_check_launch(s->ctx, "screen_kernel");
}

extern "C" bart_status bart_demc_accept(bart_demc* s, int64_t half_step, const float* y, const int32_t* pass,
                                        const double* L_y, const double* ls_y, int32_t* accepted) {
  if (!s) return BART_EINVAL;
  BART_REQUIRE(s->ctx, y && pass && L_y, "NULL y, pass or L_y");
  accept_kernel<<<nblk(s->C), 128, 0, s->ctx->stream>>>(s->C, s->d, s->x, s->L, s->Ls, y, pass, L_y, ls_y,
                                                        half_step, s->hs_dev, s->seed, s->beta, s->margin,
                                                        s->zs ? s->logq : nullptr, accepted);
  bart_status st = bart_check_launch(s->ctx, "accept_kernel");
  if (st != BART_OK || !s->zs) return st;
  archive_kernel<<<1, 256, 0, s->ctx->stream>>>(s->C, s->d, s->x, half_step, s->hs_dev, s->thin, s->Z, s->cap,
                                                s->zc);
  return bart_check_launch(s->ctx, "archive_kernel");
}

extern "C" bart_status bart_loglike_bands(bart_ctx* ctx, const float* model, int n, int n_bands, const float* data,
                                          const float* sigma, const int32_t* mask, double* out) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, model && data && sigma && out, "NULL array");
  BART_REQUIRE(ctx, n >= 1 && n_bands >= 1, "n and n_bands must be >= 1");
  loglike_kernel<<<nblk(n), 128, 0, ctx->stream>>>(model, n, n_bands, data, sigma, mask, out);
  return bart_check_launch(ctx, "loglike_kernel");
}

extern "C" bart_status bart_demc_set_screen(bart_demc* s, double beta, double margin) {
  if (!s) return BART_EINVAL;
  BART_REQUIRE(s->ctx, beta >= 0 && std::isfinite(beta) && std::isfinite(margin), "bad beta or margin");
  s->beta = beta;
  s->margin = margin;
  return BART_OK;
}

// Internal hooks of the retrieval driver.
void bart_demc_use_counter(bart_demc* s, const int64_t* hs_dev) { s->hs_dev = hs_dev; }
int bart_demc_chains(const bart_demc* s) { return s->C; }
int bart_demc_params(const bart_demc* s) { return s->d; }
const float* bart_demc_states(const bart_demc* s) { return s->x; }

extern "C" bart_status bart_demc_set_archive(bart_demc* s, const float* z0, int64_t n0, int64_t capacity, int thin,
                                             double p_snooker) {
  if (!s) return BART_EINVAL;
  bart_ctx* ctx = s->ctx;
  BART_REQUIRE(ctx, z0 != nullptr, "z0 is NULL");
  BART_REQUIRE(ctx, n0 >= 3 && capacity >= n0 && capacity <= ((int64_t)1 << 31), "need 3 <= n0 <= capacity <= 2^31");
  BART_REQUIRE(ctx, thin >= 1, "thin must be >= 1");
  BART_REQUIRE(ctx, p_snooker >= 0 && p_snooker <= 1, "p_snooker must be in [0, 1]");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  if (s->Z) cudaFree(s->Z);
  s->Z = nullptr;
  if (!s->zc && cudaMalloc(&s->zc, sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    return bart_fail(ctx, BART_ENOMEM, "DEMCzs counter allocation failed");
  }
  if (!s->logq && cudaMalloc(&s->logq, (size_t)s->C * 8) != cudaSuccess) {
    cudaGetLastError();
    return bart_fail(ctx, BART_ENOMEM, "DEMCzs buffer allocation failed");
  }
  if (cudaMalloc(&s->Z, (size_t)capacity * s->d * 4) != cudaSuccess) {
    cudaGetLastError();
    s->Z = nullptr;
    return bart_fail(ctx, BART_ENOMEM, "DEMCzs archive of %lld states failed", (long long)capacity);
  }
  const long long n0ll = n0;
  BART_CUDA(ctx, cudaMemcpyAsync(s->Z, z0, (size_t)n0 * s->d * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  BART_CUDA(ctx, cudaMemcpy(s->zc, &n0ll, sizeof(long long), cudaMemcpyHostToDevice));
  BART_CUDA(ctx, cudaMemsetAsync(s->logq, 0, (size_t)s->C * 8, ctx->stream));
  s->cap = capacity;
  s->thin = thin;
  s->p_snooker = p_snooker;
  s->zs = true;
  return BART_OK;
}

extern "C" bart_status bart_demc_archive_size(bart_demc* s, int64_t* n) {
  if (!s) return BART_EINVAL;
  BART_REQUIRE(s->ctx, n != nullptr, "n is NULL");
  long long v = 0;
  if (s->zs) {
    BART_CUDA(s->ctx, cudaMemcpyAsync(&v, s->zc, sizeof(long long), cudaMemcpyDeviceToHost, s->ctx->stream));
    BART_CUDA(s->ctx, cudaStreamSynchronize(s->ctx->stream));
  }
  *n = v;
  return BART_OK;
}

// ---------------------------------------------------------------- chain statistics

namespace {

__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();                           // sh is reused by consecutive calls
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

// SPEIS of one (chain, parameter) series per block: 1 + 2 sum of the
// autocorrelation from lag 1 until it first falls below `threshold` (Sec. 5).
__global__ void speis_kernel(const float* __restrict__ chain, int n, int C, int d, double threshold,
                             double* __restrict__ out) {
  __shared__ double sh[32];
  const int c = blockIdx.x / d, q = blockIdx.x % d;
  auto at = [&](int t) { return (double)chain[((int64_t)t * C + c) * d + q]; };
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += at(t);
  const double mean = block_sum(s, sh) / n;
  double v = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) v += (at(t) - mean) * (at(t) - mean);
  const double var = block_sum(v, sh) / n;
  double speis = 1.0;
  if (var > 0.0) {
    for (int k = 1; k < n / 2; ++k) {
      double a = 0.0;
      for (int t = threadIdx.x; t + k < n; t += blockDim.x) a += (at(t) - mean) * (at(t + k) - mean);
      const double rho = block_sum(a, sh) / (n * var);
      if (rho < threshold) break;            // the same value in every thread
      speis += 2.0 * rho;
    }
  }
  if (threadIdx.x == 0) out[(int64_t)c * d + q] = speis;
}

// Gelman-Rubin R of one parameter per block over C chains of length n.
__global__ void gr_kernel(const float* __restrict__ chain, int n, int C, int d, double* __restrict__ out) {
  __shared__ double sh[32];
  const int q = blockIdx.x;
  double sw = 0.0, sm = 0.0, sm2 = 0.0;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double m = 0.0;
    for (int t = 0; t < n; ++t) m += chain[((int64_t)t * C + c) * d + q];
    m /= n;
    double v = 0.0;
    for (int t = 0; t < n; ++t) {
      const double e = chain[((int64_t)t * C + c) * d + q] - m;
      v += e * e;
    }
    sw += v / (n - 1);
    sm += m;
    sm2 += m * m;
  }
  const double W = block_sum(sw, sh) / C;
  const double M = block_sum(sm, sh) / C;
  const double M2 = block_sum(sm2, sh);
  const double B = n * (M2 - C * M * M) / (C - 1);
  const double V = (n - 1.0) / n * W + B / n;
  if (threadIdx.x == 0) out[q] = W > 0.0 ? sqrt(V / W) : 1.0;
}

}  // namespace

extern "C" bart_status bart_chain_stats(bart_ctx* ctx, const float* chain, int n, int n_chains, int n_params,
                                        double threshold, double* speis, double* gr) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, chain != nullptr, "chain is NULL");
  BART_REQUIRE(ctx, n >= 4 && n_chains >= 1 && n_params >= 1, "need n >= 4, n_chains >= 1, n_params >= 1");
  BART_REQUIRE(ctx, (int64_t)n_chains * n_params <= 0x7fffffff, "too many series");
  BART_REQUIRE(ctx, !gr || n_chains >= 2, "the Gelman-Rubin statistic needs at least 2 chains");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  if (speis) {
    speis_kernel<<<n_chains * n_params, 256, 0, ctx->stream>>>(chain, n, n_chains, n_params, threshold, speis);
    bart_status st = bart_check_launch(ctx, "speis_kernel");
    if (st != BART_OK) return st;
  }
  if (gr) {
    gr_kernel<<<n_params, 256, 0, ctx->stream>>>(chain, n, n_chains, n_params, gr);
    return bart_check_launch(ctx, "gr_kernel");
  }
  return BART_OK;
}
