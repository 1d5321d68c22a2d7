// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <map>

#include "../../include/bartgpu.h"

// Device status word bits (set by kernels, read and cleared by bart_sync).
enum : int {
  BART_DEV_TIMEOUT = 1,
  BART_DEV_RANGE = 2,
};

struct bart_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  std::string err;
  // Growable scratch: one buffer per purpose so calls can keep it resident.
  std::map<std::string, std::pair<void*, size_t>> scratch;
  std::map<std::string, std::vector<unsigned char>> uploaded;   // host copy of each constant buffer
  std::map<std::string, int> tiles;  // autotuned tile width per launch shape
  int autotune = 1;
  double line_rel = 0.0;            // line-strength lower bound (<= 0: off)
  int em_tile = 0;                  // emission tile width fixed by the caller (0: autotuner)
  int em_launch = BART_LAUNCH_FUSED; // emission launch structure (bart_set_emission_launch)
  cudaStream_t user_stream = nullptr;  // the caller's stream while a capture is open
  bool capturing = false;           // between bart_capture_begin and bart_capture_end
  int* d_status = nullptr;          // device status word
  float2* d_wtable = nullptr;       // Faddeeva Taylor-coefficient table
  bool wtable_ready = false;
};

// Record an error message on the context and return the status.
bart_status bart_fail(bart_ctx* ctx, bart_status st, const char* fmt, ...);

// Check a CUDA call; on failure record it and return BART_ECUDA.
#define BART_CUDA(ctx, call)                                                          \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return bart_fail((ctx), BART_ECUDA, "%s failed: %s (%s:%d)", #call,             \
                       cudaGetErrorString(e_), __FILE__, __LINE__);                   \
  } while (0)

#define BART_REQUIRE(ctx, cond, ...)                                                  \
  do {                                                                                \
    if (!(cond)) return bart_fail((ctx), BART_EINVAL, __VA_ARGS__);                   \
  } while (0)

// Scratch buffer of at least `bytes` bytes named `name`, kept for later calls.
bart_status bart_scratch(bart_ctx* ctx, const char* name, size_t bytes, void** out);

// Device copy of a small host constant buffer, kept in scratch `name`.  The
// copy is issued only when the bytes differ from the last upload, so a call
// repeated with the same arguments launches kernels only (and can be captured
// in a CUDA graph).
bart_status bart_upload_const(bart_ctx* ctx, const char* name, const void* data, size_t bytes, void** dev);

// Launch-error check after a kernel launch.
bart_status bart_check_launch(bart_ctx* ctx, const char* what);

// Make sure the Faddeeva Taylor table is on the device.
bart_status bart_ensure_wtable(bart_ctx* ctx);

// Physical constants (cgs, CODATA 2018 exact SI values converted).
namespace bartc {
constexpr double H = 6.62607015e-27;
constexpr double C = 2.99792458e10;
constexpr double KB = 1.380649e-16;
constexpr double AMU = 1.66053906660e-24;
constexpr double C2 = H * C / KB;  // cm K
constexpr double TREF = 296.0;
constexpr double BAR = 1e6;
constexpr double PI = 3.141592653589793238462643383279502884;
}  // namespace bartc

// Faddeeva Taylor table geometry: nodes z0 = ix*H + i*iy*H, |x|,y in [0, 5].
namespace wtab {
constexpr int NX = 41, NY = 41, NT = 8;
constexpr float H = 0.125f;
}  // namespace wtab
