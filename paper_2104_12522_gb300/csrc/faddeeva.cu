// Host-side construction of the Faddeeva Taylor table and the bart_faddeeva_re
// entry point.
//
// Table nodes z0 = ix/8 + i iy/8 (0 <= ix, iy <= 40).  w(z0) is found in FP64:
// the Laplace continued fraction to depth 200 gives w at x0 + 8i, where it has
// converged to round-off, and w is then carried down the vertical line through
// every node of the column by fourth-order Runge-Kutta on
// w' = -2 z w + 2i/sqrt(pi) (dw/dy = i w').  Downward integration damps the exp(-z^2) mode of the
// equation, so the error stays at the level of the step error.  On the real
// axis the real part is set to exp(-x0^2), its exact value.  The Taylor
// coefficients then follow from c_0 = w, c_1 = w', and
// c_{n+1} = (-2 z0 c_n - 2 c_{n-1}) / (n + 1).
#include <complex>
#include <cmath>

#include "bart_internal.cuh"
#include "faddeeva.cuh"

namespace {

using cd = std::complex<double>;
const double SQRTPI = 1.772453850905516027298167483341;

cd cf_w(cd z, int depth) {
  cd t = z;
  for (int k = depth; k >= 1; --k) t = z - (0.5 * k) / t;
  return cd(0.0, 1.0 / SQRTPI) / t;
}

// w along the vertical line x = x0 at every table node y0 = iy H, integrated
// downward from y = 8 (where the continued fraction has converged) with RK4
// steps that land on the nodes.
void w_column(double x0, std::vector<cd>& out) {
  const double H = wtab::H;
  const int sub = 64;                       // steps per node spacing
  const int n_steps = (int)std::lround(8.0 / H) * sub;
  const double dy = -H / sub;
  auto f = [&](double y, cd w) {
    cd z(x0, y);
    cd wp = -2.0 * z * w + cd(0.0, 2.0 / SQRTPI);
    return cd(0.0, 1.0) * wp;
  };
  out.assign(wtab::NY, cd(0.0, 0.0));
  double y = 8.0;
  cd w = cf_w(cd(x0, y), 200);
  for (int step = 0; step <= n_steps; ++step) {
    if (step % sub == 0) {
      const int iy = (n_steps - step) / sub;
      if (iy < wtab::NY) out[iy] = w;
    }
    if (step == n_steps) break;
    cd k1 = f(y, w);
    cd k2 = f(y + 0.5 * dy, w + 0.5 * dy * k1);
    cd k3 = f(y + 0.5 * dy, w + 0.5 * dy * k2);
    cd k4 = f(y + dy, w + dy * k3);
    w += dy / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    y = 8.0 + (step + 1) * dy;
  }
  out[0] = cd(std::exp(-x0 * x0), out[0].imag());   // exact real part on the real axis
}

void build_table(std::vector<float2>& out) {
  out.resize((size_t)wtab::NX * wtab::NY * wtab::NT);
  std::vector<cd> col;
  for (int ix = 0; ix < wtab::NX; ++ix) {
    const double x0 = ix * (double)wtab::H;
    w_column(x0, col);
    for (int iy = 0; iy < wtab::NY; ++iy) {
      const double y0 = iy * (double)wtab::H;
      cd z0(x0, y0);
      cd c[wtab::NT];
      c[0] = col[iy];
      c[1] = -2.0 * z0 * c[0] + cd(0.0, 2.0 / SQRTPI);
      for (int n = 1; n + 1 < wtab::NT; ++n) c[n + 1] = (-2.0 * z0 * c[n] - 2.0 * c[n - 1]) / double(n + 1);
      float2* dst = &out[((size_t)iy * wtab::NX + ix) * wtab::NT];
      for (int n = 0; n < wtab::NT; ++n) dst[n] = make_float2((float)c[n].real(), (float)c[n].imag());
    }
  }
}

__global__ void faddeeva_kernel(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
                                float* __restrict__ out, const float2* __restrict__ tab) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = bartw::faddeeva_re(x[i], y[i], tab);
}

}  // namespace

bart_status bart_ensure_wtable(bart_ctx* ctx) {
  if (ctx->wtable_ready) return BART_OK;
  // Same for every context; built once (thread-safe static initialisation).
  static const std::vector<float2> host = [] {
    std::vector<float2> v;
    build_table(v);
    return v;
  }();
  size_t bytes = host.size() * sizeof(float2);
  if (!ctx->d_wtable) BART_CUDA(ctx, cudaMalloc(&ctx->d_wtable, bytes));
  BART_CUDA(ctx, cudaMemcpy(ctx->d_wtable, host.data(), bytes, cudaMemcpyHostToDevice));
  ctx->wtable_ready = true;
  return BART_OK;
}

extern "C" bart_status bart_faddeeva_re(bart_ctx* ctx, const float* x, const float* y, int64_t n, float* out) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, n >= 0, "n must be >= 0");
  if (n == 0) return BART_OK;
  BART_REQUIRE(ctx, x && y && out, "NULL array");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  bart_status st = bart_ensure_wtable(ctx);
  if (st != BART_OK) return st;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)ctx->sm_count * 32) blocks = (int64_t)ctx->sm_count * 32;
  faddeeva_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(x, y, n, out, ctx->d_wtable);
  return bart_check_launch(ctx, "faddeeva_kernel");
}
