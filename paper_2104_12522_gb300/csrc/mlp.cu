// Surrogate network of the screened sampler: hand-written forward, backward
// and Adam kernels (the paper has no learned component; the network is the
// task's: theta -> 256 -> 256 -> 256 -> band values, GELU, BF16 weights with
// FP32 accumulation).
//
// Layout: flat FP32 master parameters, per layer W_l row-major [out][in] then
// b_l [out].  The forward pass reads either BF16 copies of the weights (made
// after every update, round to nearest even) or the FP32 master (test mode).
//
// With BF16 weights every GEMM of the forward and backward passes runs on the
// 5th-generation tensor cores (tcgen05.mma kind::f16, BF16 operands staged in
// shared memory, FP32 accumulators in tensor memory) with a fused epilogue
// (bias, GELU, GELU').  FP32 operands
// (activations, output gradients) are carried as a pair of BF16 numbers,
// x = hi + lo with hi = bf16(x) and lo = bf16(x - hi), and multiplied term by
// term (hi*hi + lo*hi + hi*lo), which keeps about 16 bits of the FP32 operand:
// the products are those of BF16 weights with FP32 activations to ~1e-5.  The
// FP32-weight test mode keeps a SIMT FP32 GEMM (64 x 64 tiles, 4 x 4 outputs
// per thread), the reference precision of the gradient tests.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "bart_internal.cuh"

struct bart_mlp {
  bart_ctx* ctx = nullptr;
  std::vector<int> widths;
  int n_layers = 0;
  int64_t n_params = 0;
  int bf16 = 1;
  int log_outputs = 0;
  int max_batch = 0;
  int64_t step = 0;
  std::vector<int64_t> w_off, b_off;   // offsets into the flat vector
  float* p = nullptr;                  // master FP32 params
  float* m = nullptr;                  // Adam moments
  float* v = nullptr;
  float* g = nullptr;                  // gradient
  __nv_bfloat16* wb = nullptr;         // BF16 weights (same offsets as p)
  float* act = nullptr;                // activations: per layer z and h, [max_batch][width]
  std::vector<int64_t> z_off, h_off;
  float* scale = nullptr;              // in_shift[in], in_scale[in], out_shift[out], out_scale[out]
  float* loss = nullptr;
  float* part = nullptr;               // K-slice partial sums of the tensor-core GEMMs
  int64_t part_elems = 0;
  float* xg = nullptr;                 // gathered batch inputs [max_batch][in] (bart_mlp_train_steps)
  float* tg = nullptr;                 // gathered batch targets [max_batch][out]
};

namespace {

constexpr int TM = 64, TN = 64, TK = 16;   // CTA tile and K step
constexpr int MLP_THREADS = 256;           // 16 x 16 threads, 4 x 4 outputs each

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * expf(-0.5f * x * x);
}

template <typename T>
__device__ __forceinline__ float ld(const T* p) { return (float)p[0]; }

// C[M][N] = sum_k A(m, k) B(k, n), with A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].
// Epilogue modes:
//   0  C = acc                                  (plain)
//   1  z = acc + bias[n]; C = z; H = GELU(z)    (hidden layer forward)
//   2  C = acc + bias[n]                        (output layer forward)
//   3  C = acc * GELU'(Z[m][n])                 (backward through a hidden layer)
template <typename TA, typename TB>
__global__ void __launch_bounds__(MLP_THREADS)
gemm_kernel(int M, int N, int K, const TA* __restrict__ A, int64_t sam, int64_t sak, const TB* __restrict__ B,
            int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t ldc, int mode, const float* __restrict__ bias,
            float* __restrict__ H, const float* __restrict__ Z) {
  __shared__ float sA[TK][TM + 4];
  __shared__ float sB[TK][TN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += MLP_THREADS) {
      const int mm = e / TK, kk = e % TK;
      const int gm = m0 + mm, gk = k0 + kk;
      sA[kk][mm] = (gm < M && gk < K) ? ld(A + gm * sam + gk * sak) : 0.f;
    }
    for (int e = threadIdx.x; e < TN * TK; e += MLP_THREADS) {
      const int nn = e % TN, kk = e / TN;
      const int gn = n0 + nn, gk = k0 + kk;
      sB[kk][nn] = (gn < N && gk < K) ? ld(B + gk * sbk + gn * sbn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = acc[i][j];
      const int64_t o = (int64_t)gm * ldc + gn;
      if (mode == 1) {
        v += bias[gn];
        C[o] = v;
        H[o] = gelu(v);
      } else if (mode == 2) {
        C[o] = v + bias[gn];
      } else if (mode == 3) {
        C[o] = v * gelu_grad(Z[o]);
      } else {
        C[o] = v;
      }
    }
  }
}

// ---- BF16 splitting of the tensor-core operands
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}
__device__ __forceinline__ void split_bf16(__nv_bfloat16 v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = v;
  lo = __float2bfloat16_rn(0.0f);
}

// Sum of the K slices in a fixed order, then the epilogue of umma_gemm_kernel.
__global__ void split_k_reduce(int M, int N, int n_split, const float* __restrict__ P, float* __restrict__ C,
                               int64_t ldc, int mode, const float* __restrict__ bias, float* __restrict__ H,
                               const float* __restrict__ Z) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * N) return;
  const int gm = (int)(e / N), gn = (int)(e % N);
  float v = 0.0f;
  for (int z = 0; z < n_split; ++z) v += P[(int64_t)z * M * N + e];
  const int64_t o = (int64_t)gm * ldc + gn;
  if (mode == 1) {
    v += bias[gn];
    C[o] = v;
    H[o] = gelu(v);
  } else if (mode == 2) {
    C[o] = v + bias[gn];
  } else if (mode == 3) {
    C[o] = v * gelu_grad(Z[o]);
  } else {
    C[o] = v;
  }
}

// ---- tensor-core GEMM on the 5th-generation tensor cores (tcgen05, TMEM)
//
// C[M][N] = sum_k A(m, k) B(k, n), with A(m, k) = A[m sam + k sak] and
// B(k, n) = B[k sbk + n sbn] (so transposed operands need no copy), on
// tcgen05.mma: a CTA of 4 warps owns a 128 x BN output tile whose FP32
// accumulator lives in tensor memory (BN columns of the CTA's 128 TMEM
// lanes).  Per 64-wide K block the threads convert their share of the
// operands to BF16 (an FP32 operand as hi and lo parts) and store them in
// shared memory in the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, K-adjacent core matrices 128 bytes apart
// (leading-dimension offset), 8-row groups UM_BK / 8 * 128 bytes apart
// (stride offset); two stages, so block kb + 1 is staged while the MMAs of
// block kb run.  One thread issues the MMAs (M = 128, N = BN, K = 16 each;
// hi*hi, lo_A*hi_B and hi_A*lo_B) and commits them to the stage's mbarrier;
// the CTA waits on it (bounded, BART_DEV_TIMEOUT when it runs out) before it
// overwrites the stage.  The epilogue reads the accumulator back with
// tcgen05.ld (warp w: TMEM lanes 32 w .. 32 w + 31, i.e. output rows) and
// applies the mode: 1 z = acc + bias and h = GELU(z), 2 acc + bias, 3 acc
// GELU'(Z), 0 acc; with split K the raw sums go to P[z][M][N] instead.
constexpr int UM_BM = 128, UM_BK = 64;
constexpr int UM_THREADS = 128;
constexpr unsigned int UM_SPIN_LIMIT = 1u << 24;   // try_wait rounds before a wait is given up

__device__ __forceinline__ unsigned int um_smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05: start address, leading- and
// stride-dimension byte offsets (all >> 4), the fixed version bits 46..48 =
// 0b001, no swizzle.
__device__ __forceinline__ unsigned long long um_desc(unsigned int addr, unsigned int lbo, unsigned int sbo) {
  return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
         ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N >> 3 at bits 17..22, M >> 4 at bits 24..28.
__host__ __device__ constexpr unsigned int um_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned int)(n >> 3) << 17) | ((unsigned int)(m >> 4) << 24);
}

__device__ __forceinline__ bool um_wait(unsigned long long* bar, unsigned int parity) {
  const unsigned int a = um_smem_u32(bar);
  for (unsigned int it = 0; it < UM_SPIN_LIMIT; ++it) {
    unsigned int ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// D (+)= A B^T for one 128 x N x 16 step: A and B from their descriptors, D
// in tensor memory; acc = 0 overwrites D
__device__ __forceinline__ void um_mma(unsigned int tmem, unsigned long long a, unsigned long long b,
                                       unsigned int idesc, unsigned int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// byte offset of element (r, k) of a [rows][UM_BK] operand tile
__device__ __forceinline__ unsigned int um_off(int r, int k) {
  return (unsigned int)((((r >> 3) * (UM_BK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Stages rows [r0, r0 + R) x k in [k0, k0 + UM_BK) of the operand X(r, k) =
// X[r * s_r + k * s_k] (zero outside [0, n_r) x [k0, k_end)) as BF16 hi and lo
// tiles; each thread converts 8 consecutive k (one 16-byte core-matrix row).
template <typename T, bool LO, int R>
__device__ __forceinline__ void um_stage(const T* __restrict__ X, int64_t s_r, int64_t s_k, int r0, int n_r, int k0,
                                         int k_end, unsigned char* hi_tile, unsigned char* lo_tile) {
  for (int e = threadIdx.x; e < R * (UM_BK / 8); e += UM_THREADS) {
    const int r = e % R, k8 = e / R;            // consecutive threads: consecutive rows
    const int gr = r0 + r;
    uint32_t h[4], l[4];
    const T* src = X + gr * s_r + (int64_t)(k0 + k8 * 8) * s_k;
    if (s_k == 1 && gr < n_r && k0 + k8 * 8 + 8 <= k_end && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
      // eight contiguous elements: 16-byte loads
      if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(src));
        h[0] = q.x; h[1] = q.y; h[2] = q.z; h[3] = q.w;
        l[0] = l[1] = l[2] = l[3] = 0u;
      } else {
        const float4 q0 = __ldg(reinterpret_cast<const float4*>(src));
        const float4 q1 = __ldg(reinterpret_cast<const float4*>(src) + 1);
        const float f[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          __nv_bfloat16 h0, l0, h1, l1;
          split_bf16(f[j], h0, l0);
          split_bf16(f[j + 1], h1, l1);
          h[j >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
          l[j >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
      }
      const unsigned int o = um_off(r, k8 * 8);
      *reinterpret_cast<uint4*>(hi_tile + o) = make_uint4(h[0], h[1], h[2], h[3]);
      if (LO) *reinterpret_cast<uint4*>(lo_tile + o) = make_uint4(l[0], l[1], l[2], l[3]);
      continue;
    }
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const int gk = k0 + k8 * 8 + j;
      __nv_bfloat16 h0, l0, h1, l1;
      if (gr < n_r && gk < k_end) split_bf16(X[gr * s_r + gk * s_k], h0, l0);
      else h0 = l0 = __float2bfloat16_rn(0.0f);
      if (gr < n_r && gk + 1 < k_end) split_bf16(X[gr * s_r + (gk + 1) * s_k], h1, l1);
      else h1 = l1 = __float2bfloat16_rn(0.0f);
      h[j >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      l[j >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    const unsigned int o = um_off(r, k8 * 8);
    *reinterpret_cast<uint4*>(hi_tile + o) = make_uint4(h[0], h[1], h[2], h[3]);
    if (LO) *reinterpret_cast<uint4*>(lo_tile + o) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

template <typename TA, typename TB, int BN>
__global__ void __launch_bounds__(UM_THREADS)
umma_gemm_kernel(int M, int N, int K, int k_per, const TA* __restrict__ A, int64_t sam, int64_t sak,
                 const TB* __restrict__ B, int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t ldc, int mode,
                 const float* __restrict__ bias, float* __restrict__ H, const float* __restrict__ Z,
                 float* __restrict__ P, int* __restrict__ status) {
  static_assert(BN == 32 || BN == 64 || BN == 128 || BN == 256, "TMEM columns: a power of two >= 32");
  constexpr bool A_LO = !std::is_same<TA, __nv_bfloat16>::value;
  constexpr bool B_LO = !std::is_same<TB, __nv_bfloat16>::value;
  constexpr unsigned int A_BYTES = UM_BM * UM_BK * 2, B_BYTES = BN * UM_BK * 2;
  constexpr unsigned int STAGE = A_BYTES * (A_LO ? 2 : 1) + B_BYTES * (B_LO ? 2 : 1);
  // two stages of operand tiles: block kb + 1 is staged while the MMAs of
  // block kb run
  extern __shared__ __align__(1024) unsigned char um_smem[];
  __shared__ __align__(8) unsigned long long s_bar[2];
  __shared__ unsigned int s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * UM_BM, n0 = blockIdx.x * BN;
  const int k_begin = blockIdx.z * k_per, k_end = min(K, k_begin + k_per);

  if (warp == 0) {   // the accumulator: BN TMEM columns, address written to s_tmem
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(um_smem_u32(&s_tmem)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(um_smem_u32(&s_bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(um_smem_u32(&s_bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned int tmem = s_tmem;
  constexpr unsigned int IDESC = um_idesc(UM_BM, BN);
  constexpr unsigned int LBO = 128, SBO = (UM_BK / 8) * 128;

  const int nk = k_end > k_begin ? (k_end - k_begin + UM_BK - 1) / UM_BK : 0;
  for (int kb = 0; kb < nk; ++kb) {
    const int st = kb & 1;
    unsigned char* sAh = um_smem + st * STAGE;
    unsigned char* sAl = sAh + A_BYTES;
    unsigned char* sBh = sAl + (A_LO ? A_BYTES : 0);
    unsigned char* sBl = sBh + B_BYTES;
    if (kb >= 2) {
      // the MMAs of block kb - 2 read this stage: their commit must have
      // arrived (a wait that runs out is reported and ends the loop)
      if (!um_wait(&s_bar[st], (unsigned int)((kb - 2) >> 1) & 1u)) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
    }
    const int k0 = k_begin + kb * UM_BK;
    um_stage<TA, A_LO, UM_BM>(A, sam, sak, m0, M, k0, k_end, sAh, sAl);
    um_stage<TB, B_LO, BN>(B, sbn, sbk, n0, N, k0, k_end, sBh, sBl);
    // the operands written through the generic proxy are read by the tensor
    // cores through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int s = 0; s < UM_BK / 16; ++s) {
        const unsigned int ko = (unsigned int)s * 256;   // two core matrices per 16-wide step
        const unsigned long long ah = um_desc(um_smem_u32(sAh) + ko, LBO, SBO);
        const unsigned long long bh = um_desc(um_smem_u32(sBh) + ko, LBO, SBO);
        um_mma(tmem, ah, bh, IDESC, (kb == 0 && s == 0) ? 0u : 1u);
        if (A_LO) um_mma(tmem, um_desc(um_smem_u32(sAl) + ko, LBO, SBO), bh, IDESC, 1u);
        if (B_LO) um_mma(tmem, ah, um_desc(um_smem_u32(sBl) + ko, LBO, SBO), IDESC, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       um_smem_u32(&s_bar[st]))
                   : "memory");
    }
  }
  // the last block's commit arrives after every earlier MMA has completed
  if (nk > 0 && !s_fail && !um_wait(&s_bar[(nk - 1) & 1], (unsigned int)((nk - 1) >> 1) & 1u)) s_fail = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_fail) {
    if (tid == 0) atomicOr(status, BART_DEV_TIMEOUT);
  } else {
    // epilogue: warp w reads output rows m0 + 32 w + lane, 32 columns at a time
    // (an empty K slice contributes zeros)
    const bool empty = k_begin >= k_end;
    const int gm = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t v[32] = {};
      const unsigned int ta = tmem + ((unsigned int)(warp * 32) << 16) + (unsigned int)c0;
      if (!empty) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(ta)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      }
      if (gm < M) {
        const int nb = n0 + c0;
        float x[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = empty ? 0.0f : __uint_as_float(v[j]);
        if (P) {
          float* dst = P + ((int64_t)blockIdx.z * M + gm) * N + nb;
          if (nb + 32 <= N && (N & 3) == 0) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(dst + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (nb + j < N) dst[j] = x[j];
          }
        } else {
          const int64_t o = (int64_t)gm * ldc + nb;
          const bool vec = nb + 32 <= N && (ldc & 3) == 0;
          if (mode == 1 || mode == 2) {
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] += (nb + j < N) ? bias[nb + j] : 0.0f;
          } else if (mode == 3) {
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] *= (nb + j < N) ? gelu_grad(Z[o + j]) : 0.0f;
          }
          if (vec) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              *reinterpret_cast<float4*>(C + o + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
              if (mode == 1)
                *reinterpret_cast<float4*>(H + o + j) =
                    make_float4(gelu(x[j]), gelu(x[j + 1]), gelu(x[j + 2]), gelu(x[j + 3]));
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (nb + j < N) {
                C[o + j] = x[j];
                if (mode == 1) H[o + j] = gelu(x[j]);
              }
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// x_scaled[b][i] = (x[b][i] - shift[i]) * scale[i]
__global__ void scale_inputs(const float* __restrict__ x, int B, int n, const float* __restrict__ shift,
                             const float* __restrict__ scale, float* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * n) return;
  int i = (int)(e % n);
  out[e] = (x[e] - shift[i]) * scale[i];
}

// Physical outputs from the standardised prediction.
__global__ void unscale_outputs(const float* __restrict__ y, int B, int n, const float* __restrict__ shift,
                                const float* __restrict__ scale, int log_outputs, float* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * n) return;
  int i = (int)(e % n);
  float v = y[e] / scale[i] + shift[i];
  out[e] = log_outputs ? exp10f(v) : v;
}

// dY = 2 (y - t_std) / (B n); loss = mean (y - t_std)^2 (one CTA, fixed order).
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, int B, int n,
                           const float* __restrict__ shift, const float* __restrict__ scale, int log_outputs,
                           float* __restrict__ dy, float* __restrict__ loss) {
  __shared__ double red[1024];
  double acc = 0.0;
  const float inv = 2.0f / (float)((int64_t)B * n);
  for (int64_t e = threadIdx.x; e < (int64_t)B * n; e += blockDim.x) {
    int i = (int)(e % n);
    float tv = log_outputs ? log10f(t[e]) : t[e];
    float r = y[e] - (tv - shift[i]) * scale[i];
    dy[e] = inv * r;
    acc += (double)r * r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = (float)(red[0] / ((double)B * n));
}

// db[n] = sum_b dz[b][n]: a CTA per 32 columns, 8 rows of threads each summing
// every 8th row of its column (coalesced), then the 8 partial sums in order.
__global__ void bias_grad(const float* __restrict__ dz, int B, int n, float* __restrict__ db) {
  __shared__ float part[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + tx;
  float s = 0.f;
  if (j < n)
    for (int b = ty; b < B; b += 8) s += dz[(int64_t)b * n + j];
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && j < n) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][tx];
    db[j] = t;
  }
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(p[i]);
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// dst[b][c] = src[idx[b]][c]; an index outside [0, n_rows) is reported and
// row 0 is taken instead.
__global__ void gather_rows(const float* __restrict__ src, int64_t n_rows, int n_cols,
                            const int32_t* __restrict__ idx, int B, float* __restrict__ dst,
                            int* __restrict__ status) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * n_cols) return;
  const int b = (int)(e / n_cols), c = (int)(e % n_cols);
  int64_t r = idx[b];
  if (r < 0 || r >= n_rows) {
    atomicOr(status, BART_DEV_RANGE);
    r = 0;
  }
  dst[e] = src[r * n_cols + c];
}

// SIMT FP32 GEMM (the FP32-weight mode)
template <typename TA, typename TB>
void gemm(cudaStream_t st, int M, int N, int K, const TA* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk,
          int64_t sbn, float* C, int64_t ldc, int mode, const float* bias = nullptr, float* H = nullptr,
          const float* Z = nullptr) {
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_kernel<TA, TB><<<grid, MLP_THREADS, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, mode, bias, H, Z);
}

// tensor-core GEMM (the BF16-weight mode) on tcgen05, split over K when the
// tile grid alone would leave SMs idle (the partial sums go to net->part)
template <typename TA, typename TB, int BN>
void umma_launch(bart_mlp* net, int M, int N, int K, const TA* A, int64_t sam, int64_t sak, const TB* B,
                 int64_t sbk, int64_t sbn, float* C, int64_t ldc, int mode, const float* bias, float* H,
                 const float* Z) {
  cudaStream_t st = net->ctx->stream;
  constexpr bool A_LO = !std::is_same<TA, __nv_bfloat16>::value;
  constexpr bool B_LO = !std::is_same<TB, __nv_bfloat16>::value;
  const size_t smem = 2 * ((size_t)UM_BM * UM_BK * 2 * (A_LO ? 2 : 1) + (size_t)BN * UM_BK * 2 * (B_LO ? 2 : 1));
  cudaFuncSetAttribute(umma_gemm_kernel<TA, TB, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int gx = (N + BN - 1) / BN, gy = (M + UM_BM - 1) / UM_BM;
  int z = 1;
  while (z * 2 <= K / UM_BK && gx * gy * z * 2 <= 2 * net->ctx->sm_count) z *= 2;
  while (z > 1 && (int64_t)z * M * N > net->part_elems) z /= 2;
  const int k_per = ((K + z - 1) / z + UM_BK - 1) / UM_BK * UM_BK;
  z = (K + k_per - 1) / k_per;
  dim3 grid(gx, gy, z);
  float* P = z > 1 ? net->part : nullptr;
  umma_gemm_kernel<TA, TB, BN><<<grid, UM_THREADS, smem, st>>>(M, N, K, k_per, A, sam, sak, B, sbk, sbn, C, ldc,
                                                              mode, bias, H, Z, P, net->ctx->d_status);
  if (P) {
    const int64_t tot = (int64_t)M * N;
    split_k_reduce<<<blocks_for(tot, 256), 256, 0, st>>>(M, N, z, P, C, ldc, mode, bias, H, Z);
  }
}

template <typename TA, typename TB>
void tc_gemm(bart_mlp* net, int M, int N, int K, const TA* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk,
             int64_t sbn, float* C, int64_t ldc, int mode, const float* bias = nullptr, float* H = nullptr,
             const float* Z = nullptr) {
  // 128 x 32 output tiles: the surrogate's GEMMs are small, so more CTAs (and
  // a shorter epilogue per thread) beat wider tiles (measured per training
  // step at batch 1,024: 0.248 ms at 32 columns, 0.267 at 64, 0.309 at 128)
  umma_launch<TA, TB, 32>(net, M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, mode, bias, H, Z);
}

// Forward pass of B rows already scaled into act layer 0; fills z/h of every layer.
void run_forward(bart_mlp* net, int B) {
  cudaStream_t st = net->ctx->stream;
  for (int l = 0; l < net->n_layers; ++l) {
    const int n_in = net->widths[l], n_out = net->widths[l + 1];
    const float* h_prev = net->act + net->h_off[l];
    float* z = net->act + net->z_off[l + 1];
    float* h = net->act + net->h_off[l + 1];
    const int mode = (l + 1 < net->n_layers) ? 1 : 2;
    const float* bias = net->p + net->b_off[l];
    // z[b][o] = sum_i h_prev[b][i] W[o][i]
    if (net->bf16)
      tc_gemm<float, __nv_bfloat16>(net, B, n_out, n_in, h_prev, n_in, 1, net->wb + net->w_off[l], 1, n_in, z,
                                    n_out, mode, bias, h);
    else
      gemm<float, float>(st, B, n_out, n_in, h_prev, n_in, 1, net->p + net->w_off[l], 1, n_in, z, n_out, mode,
                         bias, h);
  }
}

bart_status check_batch(bart_mlp* net, int B) {
  if (B < 1 || B > net->max_batch)
    return bart_fail(net->ctx, BART_EINVAL, "batch %d outside [1, %d]", B, net->max_batch);
  return BART_OK;
}

bart_status backward(bart_mlp* net, const float* x, const float* t, int B, float* loss_out) {
  cudaStream_t st = net->ctx->stream;
  const int n_in = net->widths[0], n_out = net->widths[net->n_layers];
  scale_inputs<<<blocks_for((int64_t)B * n_in, 256), 256, 0, st>>>(x, B, n_in, net->scale, net->scale + n_in,
                                                                  net->act + net->h_off[0]);
  run_forward(net, B);
  // gradient of the standardised output: reuse the last layer's h slot as dY
  const float* osh = net->scale + 2 * n_in;
  const float* osc = osh + n_out;
  float* dy = net->act + net->h_off[net->n_layers];
  mse_kernel<<<1, 1024, 0, st>>>(net->act + net->z_off[net->n_layers], t, B, n_out, osh, osc, net->log_outputs, dy,
                                 loss_out ? loss_out : net->loss);
  // dz of the current layer lives in its h slot (h is dead once z is kept)
  for (int l = net->n_layers - 1; l >= 0; --l) {
    const int ni = net->widths[l], no = net->widths[l + 1];
    float* dz = net->act + net->h_off[l + 1];
    // h_prev: layer 0 input, else GELU(z_prev) recomputed below into a temp?  The
    // hidden h of layer l is still intact: only slots above l were reused.
    const float* h_prev = net->act + net->h_off[l];
    // dW[o][i] = sum_b dz[b][o] h_prev[b][i]
    if (net->bf16)
      tc_gemm<float, float>(net, no, ni, B, dz, 1, no, h_prev, ni, 1, net->g + net->w_off[l], ni, 0);
    else
      gemm<float, float>(st, no, ni, B, dz, 1, no, h_prev, ni, 1, net->g + net->w_off[l], ni, 0);
    bias_grad<<<blocks_for(no, 32), 256, 0, st>>>(dz, B, no, net->g + net->b_off[l]);
    if (l > 0) {
      // dh_prev[b][i] = sum_o dz[b][o] W[o][i]; then dz_prev = dh_prev * GELU'(z_prev)
      float* dz_prev = net->act + net->h_off[l];
      const float* z_prev = net->act + net->z_off[l];
      // h_prev (this slot) was consumed by the dW GEMM above, which runs first on the stream.
      if (net->bf16)
        tc_gemm<float, __nv_bfloat16>(net, B, ni, no, dz, no, 1, net->wb + net->w_off[l], ni, 1, dz_prev, ni, 3,
                                      nullptr, nullptr, z_prev);
      else
        gemm<float, float>(st, B, ni, no, dz, no, 1, net->p + net->w_off[l], ni, 1, dz_prev, ni, 3, nullptr,
                           nullptr, z_prev);
    }
  }
  return bart_check_launch(net->ctx, "mlp backward");
}

}  // namespace

extern "C" bart_status bart_mlp_create(bart_ctx* ctx, const int32_t* widths, int n_widths, int bf16_weights,
                                       int log_outputs, int max_batch, bart_mlp** out) {
  if (!ctx) return BART_EINVAL;
  BART_REQUIRE(ctx, out && widths, "NULL out or widths");
  *out = nullptr;
  BART_REQUIRE(ctx, n_widths >= 2 && n_widths <= 16, "n_widths must be in [2, 16]");
  for (int i = 0; i < n_widths; ++i) BART_REQUIRE(ctx, widths[i] >= 1 && widths[i] <= 4096, "width out of range");
  BART_REQUIRE(ctx, max_batch >= 1 && max_batch <= (1 << 20), "max_batch out of range");
  BART_CUDA(ctx, cudaSetDevice(ctx->device));
  bart_mlp* net = new bart_mlp();
  net->ctx = ctx;
  net->widths.assign(widths, widths + n_widths);
  net->n_layers = n_widths - 1;
  net->bf16 = bf16_weights ? 1 : 0;
  net->log_outputs = log_outputs ? 1 : 0;
  net->max_batch = max_batch;
  int64_t o = 0;
  for (int l = 0; l < net->n_layers; ++l) {
    net->w_off.push_back(o);
    o += (int64_t)widths[l + 1] * widths[l];
    net->b_off.push_back(o);
    o += widths[l + 1];
  }
  net->n_params = o;
  int64_t a = 0;
  for (int l = 0; l <= net->n_layers; ++l) {
    net->z_off.push_back(a);
    a += (int64_t)max_batch * widths[l];
    net->h_off.push_back(a);
    a += (int64_t)max_batch * widths[l];
  }
  const int n_scale = 2 * widths[0] + 2 * widths[n_widths - 1];
  // K-slice partials: up to 16 slices of a weight-gradient GEMM [out][in], or
  // of an activation GEMM [max_batch][width]
  int64_t wmax = 0, amax = 0;
  for (int l = 0; l < net->n_layers; ++l) {
    wmax = std::max<int64_t>(wmax, (int64_t)widths[l] * widths[l + 1]);
    amax = std::max<int64_t>(amax, (int64_t)max_batch * std::max(widths[l], widths[l + 1]));
  }
  net->part_elems = std::max(16 * wmax, 16 * amax);
  bool ok = cudaMalloc(&net->p, o * 4) == cudaSuccess && cudaMalloc(&net->m, o * 4) == cudaSuccess &&
            cudaMalloc(&net->v, o * 4) == cudaSuccess && cudaMalloc(&net->g, o * 4) == cudaSuccess &&
            cudaMalloc(&net->wb, o * 2) == cudaSuccess && cudaMalloc(&net->act, a * 4) == cudaSuccess &&
            cudaMalloc(&net->scale, n_scale * 4) == cudaSuccess && cudaMalloc(&net->loss, 4) == cudaSuccess &&
            cudaMalloc(&net->part, (size_t)net->part_elems * 4) == cudaSuccess &&
            cudaMalloc(&net->xg, (size_t)max_batch * widths[0] * 4) == cudaSuccess &&
            cudaMalloc(&net->tg, (size_t)max_batch * widths[n_widths - 1] * 4) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    bart_mlp_destroy(net);
    return bart_fail(ctx, BART_ENOMEM, "MLP allocation failed");
  }
  std::vector<float> sc(n_scale, 0.f);
  for (int i = 0; i < widths[0]; ++i) sc[widths[0] + i] = 1.f;
  for (int i = 0; i < widths[n_widths - 1]; ++i) sc[2 * widths[0] + widths[n_widths - 1] + i] = 1.f;
  BART_CUDA(ctx, cudaMemcpy(net->scale, sc.data(), n_scale * 4, cudaMemcpyHostToDevice));
  BART_CUDA(ctx, cudaMemset(net->p, 0, o * 4));
  BART_CUDA(ctx, cudaMemset(net->m, 0, o * 4));
  BART_CUDA(ctx, cudaMemset(net->v, 0, o * 4));
  BART_CUDA(ctx, cudaMemset(net->wb, 0, o * 2));
  *out = net;
  return BART_OK;
}

extern "C" void bart_mlp_destroy(bart_mlp* net) {
  if (!net) return;
  cudaSetDevice(net->ctx->device);
  cudaStreamSynchronize(net->ctx->stream);
  for (void* q : {(void*)net->p, (void*)net->m, (void*)net->v, (void*)net->g, (void*)net->wb, (void*)net->act,
                  (void*)net->scale, (void*)net->loss, (void*)net->part, (void*)net->xg, (void*)net->tg})
    if (q) cudaFree(q);
  delete net;
}

extern "C" int64_t bart_mlp_num_params(const bart_mlp* net) { return net ? net->n_params : -1; }

extern "C" bart_status bart_mlp_set_scaling(bart_mlp* net, const float* in_shift, const float* in_scale,
                                            const float* out_shift, const float* out_scale) {
  if (!net) return BART_EINVAL;
  BART_REQUIRE(net->ctx, in_shift && in_scale && out_shift && out_scale, "NULL scaling array");
  const int ni = net->widths[0], no = net->widths[net->n_layers];
  std::vector<float> sc;
  sc.insert(sc.end(), in_shift, in_shift + ni);
  sc.insert(sc.end(), in_scale, in_scale + ni);
  sc.insert(sc.end(), out_shift, out_shift + no);
  sc.insert(sc.end(), out_scale, out_scale + no);
  for (float v : sc) BART_REQUIRE(net->ctx, std::isfinite(v), "non-finite scaling");
  BART_CUDA(net->ctx, cudaMemcpyAsync(net->scale, sc.data(), sc.size() * 4, cudaMemcpyHostToDevice,
                                      net->ctx->stream));
  BART_CUDA(net->ctx, cudaStreamSynchronize(net->ctx->stream));
  return BART_OK;
}

extern "C" bart_status bart_mlp_set_params(bart_mlp* net, const float* params) {
  if (!net) return BART_EINVAL;
  BART_REQUIRE(net->ctx, params, "NULL params");
  cudaStream_t st = net->ctx->stream;
  BART_CUDA(net->ctx, cudaMemcpyAsync(net->p, params, net->n_params * 4, cudaMemcpyDeviceToDevice, st));
  BART_CUDA(net->ctx, cudaMemsetAsync(net->m, 0, net->n_params * 4, st));
  BART_CUDA(net->ctx, cudaMemsetAsync(net->v, 0, net->n_params * 4, st));
  to_bf16<<<blocks_for(net->n_params, 256), 256, 0, st>>>(net->p, net->wb, net->n_params);
  net->step = 0;
  return bart_check_launch(net->ctx, "to_bf16");
}

extern "C" bart_status bart_mlp_get_params(bart_mlp* net, float* params) {
  if (!net) return BART_EINVAL;
  BART_REQUIRE(net->ctx, params, "NULL params");
  BART_CUDA(net->ctx, cudaMemcpyAsync(params, net->p, net->n_params * 4, cudaMemcpyDeviceToDevice,
                                      net->ctx->stream));
  return BART_OK;
}

extern "C" bart_status bart_mlp_forward(bart_mlp* net, const float* x, int B, float* y) {
  if (!net) return BART_EINVAL;
  BART_REQUIRE(net->ctx, x && y, "NULL x or y");
  bart_status st = check_batch(net, B);
  if (st != BART_OK) return st;
  const int ni = net->widths[0], no = net->widths[net->n_layers];
  cudaStream_t s = net->ctx->stream;
  scale_inputs<<<blocks_for((int64_t)B * ni, 256), 256, 0, s>>>(x, B, ni, net->scale, net->scale + ni,
                                                               net->act + net->h_off[0]);
  run_forward(net, B);
  unscale_outputs<<<blocks_for((int64_t)B * no, 256), 256, 0, s>>>(net->act + net->z_off[net->n_layers], B, no,
                                                                  net->scale + 2 * ni, net->scale + 2 * ni + no,
                                                                  net->log_outputs, y);
  return bart_check_launch(net->ctx, "mlp forward");
}

extern "C" bart_status bart_mlp_gradient(bart_mlp* net, const float* x, const float* t, int B, float* grad,
                                         float* loss) {
  if (!net) return BART_EINVAL;
  BART_REQUIRE(net->ctx, x && t, "NULL x or t");
  bart_status st = check_batch(net, B);
  if (st != BART_OK) return st;
  if ((st = backward(net, x, t, B, loss)) != BART_OK) return st;
  if (grad)
    BART_CUDA(net->ctx, cudaMemcpyAsync(grad, net->g, net->n_params * 4, cudaMemcpyDeviceToDevice,
                                        net->ctx->stream));
  return BART_OK;
}

namespace {

// One Adam step on the batch (x, t): gradient, moments, BF16 copy.
bart_status adam_step(bart_mlp* net, const float* x, const float* t, int B, float lr, float* loss) {
  bart_status st;
  if ((st = backward(net, x, t, B, loss)) != BART_OK) return st;
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)net->step));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)net->step));
  cudaStream_t s = net->ctx->stream;
  adam_kernel<<<blocks_for(net->n_params, 256), 256, 0, s>>>(net->p, net->m, net->v, net->g, net->n_params, lr, b1,
                                                            b2, 1e-8f, c1, c2);
  to_bf16<<<blocks_for(net->n_params, 256), 256, 0, s>>>(net->p, net->wb, net->n_params);
  return bart_check_launch(net->ctx, "adam");
}

}  // namespace

extern "C" bart_status bart_mlp_train_step(bart_mlp* net, const float* x, const float* t, int B, float lr,
                                           float* loss) {
  if (!net) return BART_EINVAL;
  BART_REQUIRE(net->ctx, x && t, "NULL x or t");
  BART_REQUIRE(net->ctx, lr > 0 && std::isfinite(lr), "lr must be > 0");
  bart_status st = check_batch(net, B);
  if (st != BART_OK) return st;
  return adam_step(net, x, t, B, lr, loss);
}

extern "C" bart_status bart_mlp_train_steps(bart_mlp* net, const float* x, const float* t, int64_t n_rows,
                                            const int32_t* batch_rows, int B, int n_steps, const float* lr,
                                            float* loss) {
  if (!net) return BART_EINVAL;
  BART_REQUIRE(net->ctx, x && t && batch_rows && lr, "NULL x, t, batch_rows or lr");
  BART_REQUIRE(net->ctx, n_rows >= 1 && n_steps >= 0, "n_rows must be >= 1 and n_steps >= 0");
  bart_status st = check_batch(net, B);
  if (st != BART_OK) return st;
  for (int k = 0; k < n_steps; ++k)
    BART_REQUIRE(net->ctx, lr[k] > 0 && std::isfinite(lr[k]), "lr[%d] must be > 0", k);
  const int ni = net->widths[0], no = net->widths[net->n_layers];
  cudaStream_t s = net->ctx->stream;
  for (int k = 0; k < n_steps; ++k) {
    const int32_t* rows = batch_rows + (int64_t)k * B;
    gather_rows<<<blocks_for((int64_t)B * ni, 256), 256, 0, s>>>(x, n_rows, ni, rows, B, net->xg,
                                                                 net->ctx->d_status);
    gather_rows<<<blocks_for((int64_t)B * no, 256), 256, 0, s>>>(t, n_rows, no, rows, B, net->tg,
                                                                 net->ctx->d_status);
    if ((st = adam_step(net, net->xg, net->tg, B, lr[k], loss ? loss + k : nullptr)) != BART_OK) return st;
  }
  return bart_check_launch(net->ctx, "mlp train steps");
}
