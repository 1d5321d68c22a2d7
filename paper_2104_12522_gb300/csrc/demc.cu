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

// log of the stage-1 acceptance a1(x -> y) = min(1, exp(beta (ls_y - ls_x) + margin))
__device__ __forceinline__ double log_a1(double d, double beta, double margin) {
  return fmin(0.0, beta * d + margin);
}

__global__ void screen_kernel(int C, const int32_t* __restrict__ inbox, const double* __restrict__ ls_y,
                              const double* __restrict__ ls_x, int64_t gen_arg, const int64_t* __restrict__ gen_dev,
                              uint64_t seed, double beta, double margin, int32_t* __restrict__ pass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int64_t gen = gen_dev ? *gen_dev : gen_arg;
  int p = inbox[i];
  if (p && ls_y) {
    const double lu = log(uniform(seed, gen, i, 100));
    p = lu < log_a1(ls_y[i] - ls_x[i], beta, margin);
  }
  pass[i] = p;
}

__global__ void accept_kernel(int C, int d, float* __restrict__ x, double* __restrict__ L, double* __restrict__ Ls,
                              const float* __restrict__ y, const int32_t* __restrict__ pass,
                              const double* __restrict__ L_y, const double* __restrict__ ls_y, int64_t gen_arg,
                              const int64_t* __restrict__ gen_dev, uint64_t seed, double beta, double margin,
                              int32_t* __restrict__ accepted) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int64_t gen = gen_dev ? *gen_dev : gen_arg;
  int a = 0;
  if (pass[i]) {
    double r = L_y[i] - L[i];
    if (ls_y) {
      // delayed acceptance: the stage-1 probabilities of the reverse and the
      // forward move enter the stage-2 ratio (for beta = 1, margin = 0 this is
      // -(ls_y - ls_x))
      const double d = ls_y[i] - Ls[i];
      r += log_a1(-d, beta, margin) - log_a1(d, beta, margin);
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
  BART_REQUIRE(ctx, n_chains >= 6 && n_chains <= 65536, "n_chains must be in [6, 65536]");
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
  for (void* p : {(void*)s->lo, (void*)s->hi, (void*)s->x, (void*)s->L, (void*)s->Ls})
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
  propose_kernel<<<nblk(s->C), 128, 0, s->ctx->stream>>>(s->C, s->d, s->x, s->lo, s->hi, half_step, s->hs_dev,
                                                         s->seed, s->gamma, s->jump_every, s->eps, y, inbox);
  return bart_check_launch(s->ctx, "propose_kernel");
}

extern "C" bart_status bart_demc_screen(bart_demc* s, int64_t half_step, const int32_t* inbox, const double* ls_y,
                                        int32_t* pass) {
  if (!s) return BART_EINVAL;
  BART_REQUIRE(s->ctx, inbox && pass, "NULL inbox or pass");
  screen_kernel<<<nblk(s->C), 128, 0, s->ctx->stream>>>(s->C, inbox, ls_y, s->Ls, half_step, s->hs_dev, s->seed,
                                                        s->beta, s->margin, pass);
  return bart_check_launch(s->ctx, "screen_kernel");
}

extern "C" bart_status bart_demc_accept(bart_demc* s, int64_t half_step, const float* y, const int32_t* pass,
                                        const double* L_y, const double* ls_y, int32_t* accepted) {
  if (!s) return BART_EINVAL;
  BART_REQUIRE(s->ctx, y && pass && L_y, "NULL y, pass or L_y");
  accept_kernel<<<nblk(s->C), 128, 0, s->ctx->stream>>>(s->C, s->d, s->x, s->L, s->Ls, y, pass, L_y, ls_y,
                                                        half_step, s->hs_dev, s->seed, s->beta, s->margin,
                                                        accepted);
  return bart_check_launch(s->ctx, "accept_kernel");
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
