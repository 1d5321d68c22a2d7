// Retrieval driver: the sampler loop of the paper (Sec. 3, Fig. 1: the
// sampler proposes parameters, the profile generator and transit produce a
// spectrum, the spectrum integrator gives band values compared with the data)
// run natively, one generation per CUDA-graph launch.
//
// A generation is two half-steps.  Each half-step is, on the context's stream:
//   propose -> [surrogate forward -> surrogate log-likelihood] -> screen ->
//   exact forward model of the survivors only (inactive proposals' CTAs exit
//   at once) -> exact log-likelihood -> accept -> statistics,
// followed by an increment of the device half-step counter that the sampler
// kernels read, so the captured graph replays every generation unchanged.
// The first generation runs eagerly: it sizes the scratch buffers and uploads
// the constant tables, after which the captured calls launch kernels only.
#include <cmath>
#include <cstring>
#include <vector>

#include "bart_internal.cuh"

void bart_demc_use_counter(bart_demc* s, const int64_t* hs_dev);
int bart_demc_chains(const bart_demc* s);
int bart_demc_params(const bart_demc* s);
const float* bart_demc_states(const bart_demc* s);

namespace {

struct DevStats {
  unsigned long long proposals, screened_out, exact_evals, accepted;
  double err_sum;
  unsigned int err_max_bits;    // non-negative float, ordered as its bit pattern
};

__global__ void stats_kernel(int C, int nb, const int32_t* __restrict__ inbox, const int32_t* __restrict__ pass,
                             const int32_t* __restrict__ acc, const float* __restrict__ bs,
                             const float* __restrict__ be, DevStats* __restrict__ st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  if (inbox[i]) atomicAdd(&st->proposals, 1ULL);
  if (inbox[i] && !pass[i]) atomicAdd(&st->screened_out, 1ULL);
  if (pass[i]) atomicAdd(&st->exact_evals, 1ULL);
  if (acc[i]) {
    atomicAdd(&st->accepted, 1ULL);
    if (bs) {
      float e = 0.f;
      for (int b = 0; b < nb; ++b) {
        const float ref = be[(int64_t)i * nb + b];
        e = fmaxf(e, fabsf(bs[(int64_t)i * nb + b] - ref) / fabsf(ref));
      }
      atomicAdd(&st->err_sum, (double)e);
      atomicMax(&st->err_max_bits, __float_as_uint(e));
    }
  }
}

__global__ void advance_kernel(int64_t* hs) { *hs += 1; }

__global__ void record_kernel(const float* __restrict__ x, int n, const int64_t* __restrict__ hs, int64_t first,
                              float* __restrict__ chain) {
  const int64_t gen = (*hs - first) / 2 - 1;    // generation just completed
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    chain[gen * n + i] = x[i];
}

}  // namespace

extern "C" bart_status bart_retrieval_run(bart_ctx* ctx, bart_demc* s, bart_mlp* surrogate,
                                          const bart_grid_desc* grid, const bart_fwd_cfg* cfg,
                                          const bart_filters* filters, const float* data, const float* sigma,
                                          int64_t first_half_step, int n_generations, int use_graph,
                                          float* chain, bart_retrieval_stats* stats) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, s && grid && cfg && filters && filters->weights && data && sigma,
               "NULL sampler, grid, cfg, filters, data or sigma");
  BART_REQUIRE(ctx, n_generations >= 1 && first_half_step >= 0 && (first_half_step % 2) == 0,
               "n_generations >= 1 and an even first_half_step are required");
  BART_REQUIRE(ctx, cfg->geometry == BART_EMISSION || cfg->geometry == BART_TRANSMISSION, "bad geometry");
  const int C = bart_demc_chains(s), d = bart_demc_params(s), nb = filters->n_bands;
  BART_REQUIRE(ctx, d == 5 + grid->n_species, "the sampler needs 5 + n_species parameters");
  BART_REQUIRE(ctx, cfg->geometry == BART_EMISSION, "the retrieval loop runs the emission geometry");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  bart_status r;
  void *p_y, *p_inbox, *p_pass, *p_acc, *p_ly, *p_lsy, *p_be, *p_bs, *p_hs, *p_stats;
  if ((r = bart_scratch(ctx, "rt_y", (size_t)C * d * 4, &p_y)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_inbox", (size_t)C * 4, &p_inbox)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_pass", (size_t)C * 4, &p_pass)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_acc", (size_t)C * 4, &p_acc)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_ly", (size_t)C * 8, &p_ly)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_lsy", (size_t)C * 8, &p_lsy)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_be", (size_t)C * nb * 4, &p_be)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_bs", (size_t)C * nb * 4, &p_bs)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_hs", sizeof(int64_t), &p_hs)) != BART_OK) return r;
  if ((r = bart_scratch(ctx, "rt_stats", sizeof(DevStats), &p_stats)) != BART_OK) return r;
  int64_t* hs = (int64_t*)p_hs;
  float* y = (float*)p_y;
  int32_t *inbox = (int32_t*)p_inbox, *pass = (int32_t*)p_pass, *acc = (int32_t*)p_acc;
  double *ly = (double*)p_ly, *lsy = (double*)p_lsy;
  float *be = (float*)p_be, *bs = (float*)p_bs;
  // host staging copies live in the context's constant cache so the async
  // uploads read memory that outlives this call
  void* dummy;
  if ((r = bart_upload_const(ctx, "rt_hs_init", &first_half_step, sizeof(int64_t), &dummy)) != BART_OK) return r;
  BART_CUDA(ctx, cudaMemcpyAsync(hs, dummy, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  BART_CUDA(ctx, cudaMemsetAsync(p_stats, 0, sizeof(DevStats), st));
  bart_demc_use_counter(s, hs);

  bart_batch batch{};
  batch.n = C;
  batch.theta = y;
  batch.active = pass;

  auto half_step = [&]() -> bart_status {
    bart_status q;
    if ((q = bart_demc_propose(s, 0, y, inbox)) != BART_OK) return q;
    if (surrogate) {
      if ((q = bart_mlp_forward(surrogate, y, C, bs)) != BART_OK) return q;
      if ((q = bart_loglike_bands(ctx, bs, C, nb, data, sigma, inbox, lsy)) != BART_OK) return q;
    }
    if ((q = bart_demc_screen(s, 0, inbox, surrogate ? lsy : nullptr, pass)) != BART_OK) return q;
    if ((q = bart_forward_spectra_batch(ctx, grid, cfg, &batch, nullptr, filters, be)) != BART_OK) return q;
    if ((q = bart_loglike_bands(ctx, be, C, nb, data, sigma, pass, ly)) != BART_OK) return q;
    if ((q = bart_demc_accept(s, 0, y, pass, ly, surrogate ? lsy : nullptr, acc)) != BART_OK) return q;
    // ctx->stream, not st: during capture it is the capture stream
    stats_kernel<<<(C + 127) / 128, 128, 0, ctx->stream>>>(C, nb, inbox, pass, acc, surrogate ? bs : nullptr, be,
                                                           (DevStats*)p_stats);
    advance_kernel<<<1, 1, 0, ctx->stream>>>(hs);
    return bart_check_launch(ctx, "retrieval half-step");
  };
  auto generation = [&]() -> bart_status {
    bart_status q;
    if ((q = half_step()) != BART_OK) return q;
    if ((q = half_step()) != BART_OK) return q;
    if (chain) {
      record_kernel<<<(C * d + 255) / 256, 256, 0, ctx->stream>>>(bart_demc_states(s), C * d, hs, first_half_step,
                                                                  chain);
      if ((q = bart_check_launch(ctx, "record_kernel")) != BART_OK) return q;
    }
    return BART_OK;
  };

  r = generation();           // eager: sizes scratch, uploads constants
  if (r == BART_OK && n_generations > 1) {
    if (use_graph) {
      // Capture on a private non-blocking stream ordered after the caller's
      // (the legacy default stream cannot be captured), replay on the caller's.
      cudaStream_t cap = nullptr;
      cudaEvent_t ev = nullptr;
      BART_CUDA(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(ev, st) != cudaSuccess || cudaStreamWaitEvent(cap, ev, 0) != cudaSuccess) {
        cudaGetLastError();
        if (ev) cudaEventDestroy(ev);
        cudaStreamDestroy(cap);
        bart_demc_use_counter(s, nullptr);
        return bart_fail(ctx, BART_ECUDA, "could not order the capture stream");
      }
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      bart_status rc = BART_OK;
      if (ce == cudaSuccess) {
        ctx->stream = cap;
        rc = generation();
        ctx->stream = st;
        ce = cudaStreamEndCapture(cap, &graph);   // always ends the capture
      }
      cudaEventDestroy(ev);
      cudaStreamDestroy(cap);
      if (rc != BART_OK || ce != cudaSuccess) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        bart_demc_use_counter(s, nullptr);
        return rc != BART_OK ? rc : bart_fail(ctx, BART_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
      }
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        bart_demc_use_counter(s, nullptr);
        return bart_fail(ctx, BART_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
      }
      for (int gidx = 1; gidx < n_generations && ce == cudaSuccess; ++gidx) ce = cudaGraphLaunch(exec, st);
      cudaGraphExecDestroy(exec);
      if (ce != cudaSuccess) {
        bart_demc_use_counter(s, nullptr);
        return bart_fail(ctx, BART_ECUDA, "graph launch failed: %s", cudaGetErrorString(ce));
      }
    } else {
      for (int gidx = 1; gidx < n_generations && r == BART_OK; ++gidx) r = generation();
    }
  }
  bart_demc_use_counter(s, nullptr);
  if (r != BART_OK) return r;
  if (stats) {
    DevStats h{};
    BART_CUDA(ctx, cudaMemcpyAsync(&h, p_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, st));
    BART_CUDA(ctx, cudaStreamSynchronize(st));
    stats->proposals = (int64_t)h.proposals;
    stats->screened_out = (int64_t)h.screened_out;
    stats->exact_evals = (int64_t)h.exact_evals;
    stats->accepted = (int64_t)h.accepted;
    stats->surrogate_err_sum = h.err_sum;
    float m;
    std::memcpy(&m, &h.err_max_bits, 4);
    stats->surrogate_err_max = m;
  }
  return BART_OK;
}
