// Context management of the C ABI: creation, streams, errors, status word and
// scratch memory.
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "bart_internal.cuh"

extern "C" int bart_abi_version(void) { return BART_ABI_VERSION; }

bart_status bart_fail(bart_ctx* ctx, bart_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

bart_status bart_check_launch(bart_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return bart_fail(ctx, BART_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return BART_OK;
}

// True while work issued on the context's stream is being captured.
static bool stream_capturing(bart_ctx* ctx) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

bart_status bart_scratch(bart_ctx* ctx, const char* name, size_t bytes, void** out) {
  auto it = ctx->scratch.find(name);
  if (it != ctx->scratch.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return BART_OK;
  }
  if (stream_capturing(ctx))
    return bart_fail(ctx, BART_EINVAL, "scratch '%s' (%zu bytes) must be sized by an eager call of the same "
                     "shape before a stream capture", name, bytes);
  if (it != ctx->scratch.end()) {
    // The old buffer may still be in use by queued work on this stream.
    BART_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(it->second.first);
    ctx->scratch.erase(it);
  }
  void* p = nullptr;
  size_t sz = bytes < 256 ? 256 : bytes;
  if (cudaMalloc(&p, sz) != cudaSuccess) {
    cudaGetLastError();
    return bart_fail(ctx, BART_ENOMEM, "scratch '%s': cudaMalloc of %zu bytes failed", name, sz);
  }
  // zeroed once, so counters kept in scratch start at 0
  if (cudaMemsetAsync(p, 0, sz, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p);
    return bart_fail(ctx, BART_ECUDA, "scratch '%s': clearing %zu bytes failed", name, sz);
  }
  ctx->scratch[name] = {p, sz};
  *out = p;
  return BART_OK;
}

bart_status bart_upload_const(bart_ctx* ctx, const char* name, const void* data, size_t bytes, void** dev) {
  void* before = nullptr;
  auto it0 = ctx->scratch.find(name);
  if (it0 != ctx->scratch.end()) before = it0->second.first;
  bart_status st = bart_scratch(ctx, name, bytes, dev);
  if (st != BART_OK) return st;
  auto& host = ctx->uploaded[name];
  const unsigned char* src = static_cast<const unsigned char*>(data);
  if (*dev == before && host.size() == bytes && std::memcmp(host.data(), src, bytes) == 0) return BART_OK;
  if (stream_capturing(ctx))
    return bart_fail(ctx, BART_EINVAL, "constant table '%s' changed inside a stream capture: make an eager "
                     "call with the same arguments first", name);
  host.assign(src, src + bytes);
  // from the retained host copy, which outlives the asynchronous copy
  BART_CUDA(ctx, cudaMemcpyAsync(*dev, host.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
  return BART_OK;
}

extern "C" bart_status bart_create(bart_ctx** out, int device, void* cuda_stream) {
  if (!out) return BART_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return BART_EINVAL;
  }
  bart_ctx* ctx = new bart_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return BART_ECUDA;
  }
  *out = ctx;
  return BART_OK;
}

extern "C" void bart_destroy(bart_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->scratch) cudaFree(kv.second.first);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_wtable) cudaFree(ctx->d_wtable);
  delete ctx;
}

extern "C" bart_status bart_set_stream(bart_ctx* ctx, void* cuda_stream) {
  if (!ctx) return BART_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return BART_OK;
}

extern "C" const char* bart_last_error(const bart_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "NULL context";
}

extern "C" bart_status bart_sync(bart_ctx* ctx) {
  if (!ctx) return BART_EINVAL;
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  BART_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int st = 0;
  BART_CUDA(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    BART_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (st & BART_DEV_TIMEOUT) return bart_fail(ctx, BART_ETIMEOUT, "device watchdog expired (status %d)", st);
    return bart_fail(ctx, BART_ERANGE, "device range check failed (status %d)", st);
  }
  return BART_OK;
}

extern "C" bart_status bart_set_autotune(bart_ctx* ctx, int enable) {
  if (!ctx) return BART_EINVAL;
  ctx->autotune = enable ? 1 : 0;
  if (!enable) ctx->tiles.clear();
  return BART_OK;
}

extern "C" bart_status bart_set_emission_tile(bart_ctx* ctx, int tile) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, tile == 0 || tile == 64 || tile == 128 || tile == 256,
               "emission tile must be 0 (autotuner), 64, 128 or 256, got %d", tile);
  ctx->em_tile = tile;
  return BART_OK;
}

extern "C" bart_status bart_set_emission_launch(bart_ctx* ctx, int mode) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, mode == BART_LAUNCH_FUSED || mode == BART_LAUNCH_SPLIT || mode == BART_LAUNCH_FUSED_TMA,
               "unknown emission launch mode %d", mode);
  ctx->em_launch = mode;
  return BART_OK;
}

struct bart_graph {
  cudaGraphExec_t exec = nullptr;
};

extern "C" bart_status bart_capture_begin(bart_ctx* ctx) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, !ctx->capturing, "a capture is already open on this context");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  // capture on a private non-blocking stream ordered after the caller's (the
  // legacy default stream cannot be captured); the graph replays on the caller's
  cudaStream_t cap = nullptr;
  cudaEvent_t ev = nullptr;
  BART_CUDA(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev, 0);
  if (ev) cudaEventDestroy(ev);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(cap);
    return bart_fail(ctx, BART_ECUDA, "could not begin the capture: %s", cudaGetErrorString(e));
  }
  ctx->user_stream = ctx->stream;
  ctx->stream = cap;
  ctx->capturing = true;
  return BART_OK;
}

extern "C" bart_status bart_capture_end(bart_ctx* ctx, bart_graph** out) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, ctx->capturing, "no capture is open on this context");
  if (out) *out = nullptr;
  cudaStream_t cap = ctx->stream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap, &graph);    // always ends the capture
  ctx->stream = ctx->user_stream;
  ctx->user_stream = nullptr;
  ctx->capturing = false;
  cudaStreamDestroy(cap);
  if (e != cudaSuccess || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return bart_fail(ctx, BART_ECUDA, "graph capture failed: %s (a library call inside it may have failed: "
                     "see its status)", cudaGetErrorString(e));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bart_fail(ctx, BART_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  BART_REQUIRE(ctx, out != nullptr, "out is NULL");
  bart_graph* g = new bart_graph();
  g->exec = exec;
  *out = g;
  return BART_OK;
}

extern "C" bart_status bart_graph_launch(bart_ctx* ctx, const bart_graph* graph) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, graph && graph->exec, "NULL graph");
  BART_REQUIRE(ctx, !ctx->capturing, "close the open capture first");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  BART_CUDA(ctx, cudaGraphLaunch(graph->exec, ctx->stream));
  return BART_OK;
}

extern "C" void bart_graph_destroy(bart_graph* graph) {
  if (!graph) return;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  delete graph;
}

extern "C" bart_status bart_set_line_threshold(bart_ctx* ctx, double rel) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, std::isfinite(rel), "line threshold must be finite");
  ctx->line_rel = rel;
  return BART_OK;
}

extern "C" int bart_autotune_report(const bart_ctx* ctx, char* buf, int len) {
  if (!ctx) return -1;
  std::string out;
  for (auto& kv : ctx->tiles) out += kv.first + " -> " + std::to_string(kv.second) + "\n";
  if (buf && len > 0) {
    std::strncpy(buf, out.c_str(), (size_t)len - 1);
    buf[len - 1] = 0;
  }
  return (int)out.size();
}
