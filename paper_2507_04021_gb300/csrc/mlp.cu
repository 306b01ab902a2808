// Learned launch proposal: a 96 -> 128 -> 128 -> 128 -> 1 ReLU network that
// scores launch directions, trained on the tracer's own per-ray labels, and
// a Gumbel-top-k draw over its logits.  The paper traces a fixed Fibonacci
// launch (Sec. II-B); this proposal is an addition on top of it.
//
// Tensor-core path (sm_103a): every contraction -- the forward layers, the
// input-gradient products and the weight-gradient products of training --
// runs through one tcgen05 kernel, D[M x N] (+)= A[M x K] B[N x K]^T with BF16
// operands in K-major rows and an FP32 accumulator in tensor memory:
//   * operands staged in shared memory in the canonical no-swizzle K-major
//     layout (8-row x 16-byte core matrices),
//   * one elected thread issues tcgen05.mma (kind::f16, M = 128, N <= 256,
//     K = 16 per instruction) and commits to an mbarrier,
//   * the accumulator is read back with tcgen05.ld (32x32b) by the four
//     warps, one TMEM lane (= one output row) per thread.
// Every mbarrier wait is bounded: on timeout the kernel records an error
// flag, waits (bounded) for its own MMAs, frees its tensor memory and
// returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "nrt_internal.h"

using bf16 = __nv_bfloat16;

namespace {

using namespace nrt;

constexpr int kIn = 96;       // 6 coordinates x 8 octaves x (sin, cos)
constexpr int kH = 128;       // hidden width
constexpr int kOct = 8;
constexpr int64_t kNParams = (int64_t)kH * kIn + kH + 2 * ((int64_t)kH * kH + kH) + kH + 1;
// packed parameter offsets: W1[h][in], b1, W2[h][h], b2, W3[h][h], b3, w4[h], b4
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH,
                  kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH,
                  kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH;
static_assert(kOffB4 + 1 == kNParams, "parameter packing");

constexpr uint32_t kErrMmaTimeout = 1u;

// grid-stride launches of 256 threads
inline unsigned blocks_for_n(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192));
}

// ---------------------------------------------------------------- tcgen05 GEMM
constexpr int kGemmThreads = 128;
constexpr int kKChunk = 64;          // K elements staged per round
constexpr int kMaxN = 256;
// default spin limit of a bounded mbarrier wait (nrt_set_wait_limit replaces
// it for the waits on the MMAs; the drain after a timeout always uses it)
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// byte offset (between core matrices adjacent in K), stride-dimension byte
// offset (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait; false on timeout.  polls = 0: the default watchdog,
// kSpinLimit potentially blocking try_waits; polls > 0 (set by the host
// through nrt_set_wait_limit): that many non-blocking test_waits.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long polls = 0) {
  if (polls > 0) {
    for (long long i = 0; i < polls; ++i)
      if (mbar_test_wait(bar, phase)) return true;
    return false;
  }
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Stage rows [r0, r0 + rows) x K [k0, k0 + 64) of a K-major BF16 matrix into
// the core-matrix layout: core (row group g, k group c) at (g * 8 + c) * 128 B,
// row r of a core at r * 16 B.  Out-of-range rows and K are zero.
__device__ __forceinline__ void stage_tile(uint8_t* dst, const bf16* __restrict__ src, int64_t ld,
                                           int64_t r0, int rows, int64_t n_rows, int64_t k0,
                                           int64_t n_k) {
  const int vecs = rows * (kKChunk / 8);
  for (int v = threadIdx.x; v < vecs; v += blockDim.x) {
    const int r = v >> 3, c = v & 7;
    const int64_t gr = r0 + r, gk = k0 + 8 * c;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (gr < n_rows && gk < n_k) val = *reinterpret_cast<const uint4*>(src + gr * ld + gk);
    *reinterpret_cast<uint4*>(dst + ((r >> 3) * 8 + c) * 128 + (r & 7) * 16) = val;
  }
}

// D tile rows [m0, m0 + 128) x all N columns, K range [k_begin, k_end).
// kAtomic: add into C (split-K partials); otherwise store.
template <bool kAtomic>
__global__ void __launch_bounds__(kGemmThreads)
    gemm_bf16_tc_kernel(const bf16* __restrict__ A, int64_t lda, const bf16* __restrict__ B,
                        int64_t ldb, float* __restrict__ Cm, int64_t ldc, int64_t M, int N,
                        int64_t K, int64_t k_split, uint32_t* __restrict__ err, long long spin) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                                 // 128 x 64 bf16 = 16 KB
  uint8_t* sB = smem + 128 * kKChunk * 2;             // N x 64 bf16 <= 32 KB
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + kMaxN * kKChunk * 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int warp = threadIdx.x >> 5;
  const int64_t m0 = (int64_t)blockIdx.x * 128;
  const int64_t k_begin = (int64_t)blockIdx.y * k_split;
  const int64_t k_end = min(K, k_begin + k_split);
  // fp32 accumulator columns: a power of two >= max(32, N)
  const uint32_t tmem_cols = N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : 256u;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) mbar_init(smem_u32(bar), 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_bf16(128, N);
  uint32_t phase = 0;
  bool ok = true;
  bool issued = false;
  for (int64_t k0 = k_begin; k0 < k_end; k0 += kKChunk) {
    stage_tile(sA, A, lda, m0, 128, M, k0, k_end);
    stage_tile(sB, B, ldb, 0, N, N, k0, k_end);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < kKChunk / 16; ++kk) {
        // K = 16 per instruction = two core matrices along K (256 B)
        const uint64_t ad = smem_desc(a0 + kk * 256, 128, 1024);
        const uint64_t bd = smem_desc(b0 + kk * 256, 128, 1024);
        tc_mma(tmem, ad, bd, idesc, (k0 > k_begin || kk > 0) ? 1u : 0u);
      }
      tc_commit(smem_u32(bar));
    }
    issued = true;
    const bool got = mbar_wait(smem_u32(bar), phase, spin);
    // block-wide: every thread leaves the loop together; the staged tiles
    // may be overwritten once all have seen the MMAs complete
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    phase ^= 1u;
    tc_fence_after();
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(err, kErrMmaTimeout);
    if (issued) mbar_wait(smem_u32(bar), phase);  // bounded: let our MMAs drain
  } else if (issued) {
    const int64_t row = m0 + warp * 32 + (threadIdx.x & 31);
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < M) {
        float* dst = Cm + row * ldc + c0;
        if (kAtomic) {
#pragma unroll
          for (int i = 0; i < 16; ++i) atomicAdd(dst + i, v[i]);
        } else {
#pragma unroll
          for (int i = 0; i < 16; i += 4)
            *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

constexpr size_t kGemmSmem = 128 * kKChunk * 2 + kMaxN * kKChunk * 2 + 16;

}  // namespace

namespace nrt {

long long wait_limit(const nrt_ctx* ctx) { return ctx->wait_limit > 0 ? (long long)ctx->wait_limit : 0; }

// C (+)= A B^T.  Requirements checked here: N a multiple of 16 in [16, 256],
// K, lda, ldb multiples of 8 (16-byte rows), ldc a multiple of 4, 16-byte
// aligned base pointers.  k_split > 0 splits K across CTAs (atomic adds).
nrt_status gemm_bf16(nrt_ctx* ctx, const bf16* A, int64_t lda, const bf16* B, int64_t ldb,
                     float* C, int64_t ldc, int64_t M, int N, int64_t K, bool accumulate,
                     int64_t k_split, uint32_t* err) {
  if (M <= 0 || N < 16 || N > kMaxN || (N & 15) || K <= 0 || (K & 7) || (lda & 7) || (ldb & 7) ||
      (ldc & 3) || (((uintptr_t)A | (uintptr_t)B) & 15) || ((uintptr_t)C & 15)) {
    ctx->last_error = "gemm_bf16: unsupported shape, stride or alignment";
    return NRT_ERR_ARG;
  }
  static bool attr_set[2] = {false, false};
  const bool atomic = accumulate || (k_split > 0 && k_split < K);
  if (!attr_set[atomic]) {
    cudaError_t e = atomic ? cudaFuncSetAttribute(gemm_bf16_tc_kernel<true>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)kGemmSmem)
                           : cudaFuncSetAttribute(gemm_bf16_tc_kernel<false>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)kGemmSmem);
    if (e != cudaSuccess) {
      ctx->last_error = std::string("gemm_bf16 attribute: ") + cudaGetErrorString(e);
      return NRT_ERR_CUDA;
    }
    attr_set[atomic] = true;
  }
  int64_t ks = (k_split > 0 && k_split < K) ? ((k_split + kKChunk - 1) / kKChunk) * kKChunk : K;
  const dim3 grid((unsigned)((M + 127) / 128), (unsigned)((K + ks - 1) / ks));
  if (atomic)
    gemm_bf16_tc_kernel<true><<<grid, kGemmThreads, kGemmSmem, ctx->stream>>>(A, lda, B, ldb, C, ldc, M,
                                                                             N, K, ks, err,
                                                                             wait_limit(ctx));
  else
    gemm_bf16_tc_kernel<false><<<grid, kGemmThreads, kGemmSmem, ctx->stream>>>(A, lda, B, ldb, C, ldc,
                                                                              M, N, K, ks, err,
                                                                              wait_limit(ctx));
  count_launch();
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  return NRT_OK;
}

}  // namespace nrt

namespace {

// ---------------------------------------------------------------- features
// Column (c * 8 + k) * 2 + {0: sin, 1: cos} of pi 2^k v_c, v = (direction,
// (tx - center) / half); rounded to BF16.
__device__ __forceinline__ void write_features(float v[6], bf16* __restrict__ X, int64_t b,
                                               bf16* __restrict__ XT, int64_t ldt) {
  for (int c = 0; c < 6; ++c)
    for (int k = 0; k < kOct; ++k) {
      float s, co;
      sincospif(ldexpf(v[c], k), &s, &co);
      const int f = (c * kOct + k) * 2;
      const bf16 bs = __float2bfloat16_rn(s), bc = __float2bfloat16_rn(co);
      X[b * kIn + f] = bs;
      X[b * kIn + f + 1] = bc;
      if (XT) {
        XT[(int64_t)f * ldt + b] = bs;
        XT[(int64_t)(f + 1) * ldt + b] = bc;
      }
    }
}

struct SampleSrc {
  const float* tx_table;    // [n_tx][3] (training) or nullptr
  const int32_t* tx_index;  // [n] or nullptr
  float tx0[3];             // single TX (scoring)
  const uint32_t* ray_id;   // [n] or nullptr: sample index is the ray id
  const uint32_t* order;    // [n] permutation or nullptr
  int64_t n;                // samples available
  int64_t start;            // first position in the order
  float cen[3], inv_half_num[3];
};

__global__ void features_kernel(SampleSrc S, int64_t B, int64_t n_rays, bf16* __restrict__ X,
                                bf16* __restrict__ XT, int64_t ldt, uint32_t* __restrict__ idx_out) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = (S.start + b) % S.n;
    const uint32_t s = S.order ? S.order[pos] : (uint32_t)pos;
    if (idx_out) idx_out[b] = s;
    const uint32_t ray = S.ray_id ? S.ray_id[s] : s;
    float t[3] = {S.tx0[0], S.tx0[1], S.tx0[2]};
    if (S.tx_index) {
      const int32_t ti = S.tx_index[s];
      t[0] = S.tx_table[3 * ti];
      t[1] = S.tx_table[3 * ti + 1];
      t[2] = S.tx_table[3 * ti + 2];
    }
    const float3 d = fib_dir(ray, n_rays);
    float v[6] = {d.x, d.y, d.z, 0.f, 0.f, 0.f};
    for (int c = 0; c < 3; ++c) v[3 + c] = __fdiv_rn(__fsub_rn(t[c], S.cen[c]), S.inv_half_num[c]);
    write_features(v, X, b, XT, ldt);
  }
}

// launch directions of the N-ray Fibonacci launch, as fib_dir gives them
// (scoring reads them instead of recomputing them per row); networks whose
// launch is larger than kDirTableMax directions compute them per row
constexpr int64_t kDirTableMax = 1ll << 26;
__global__ void dir_table_kernel(int64_t n_rays, float4* __restrict__ dirs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float3 d = fib_dir((uint32_t)i, n_rays);
    dirs[i] = make_float4(d.x, d.y, d.z, 0.0f);
  }
}

// ---------------------------------------------------------------- fused scoring
// One persistent CTA per SM scores 128-row tiles end to end on the tensor
// cores: a tile's Fourier features are written straight into the MMA operand
// layout in shared memory, the three hidden layers run as chained tcgen05.mma
// into a tensor-memory accumulator (bias, ReLU and the BF16 rounding applied
// by the epilogue, which writes the next layer's operand back to shared
// memory), and the output layer is folded into the last epilogue: each thread
// owns one row, so the logit is a per-thread dot product.  W1, W2, W3 stay in
// shared memory for the whole launch.
//
// The launch directions come from a table computed once per network (the
// same float values fib_dir gives, without its FP64 arithmetic per row), and
// the TX half of the features, equal for every row of a launch, is computed
// once per CTA.
//
// The CTA runs kScoreGroups independent groups of 128 threads, each with its
// own tiles, activation tile, 128 accumulator columns, mbarrier and named
// barrier; the first thread of a group issues that group's MMAs and commits
// them to the group's mbarrier (a commit tracks the MMAs its own thread
// issued).  One tile's feature and epilogue work on the CUDA cores thus
// overlaps the other groups' MMAs on the tensor core.
constexpr int kScoreGroups = 4;
constexpr int kScoreThreads = 128 * kScoreGroups;
constexpr int kSW1 = 0;                          // W1: 128 x 96 bf16
constexpr int kSW2 = kSW1 + kH * kIn * 2;        // W2: 128 x 128 bf16
constexpr int kSW3 = kSW2 + kH * kH * 2;         // W3
constexpr int kSAct = kSW3 + kH * kH * 2;        // activations: one 128 x 128 bf16 tile per group
constexpr int kSActBytes = 128 * kH * 2;
constexpr int kSVec = kSAct + kScoreGroups * kSActBytes;  // b1, b2, b3, w4 (fp32)
constexpr int kSTx = kSVec + 4 * kH * 4;         // the TX's 48 features (24 packed BF16 pairs)
constexpr int kSBar = kSTx + 24 * 4;             // one mbarrier per group, then the TMEM address
constexpr size_t kScoreSmem = (size_t)kSBar + 8 * kScoreGroups + 8;
constexpr uint32_t kScoreTmemCols = 128 * kScoreGroups;  // a power of two in [32, 512]
static_assert(kScoreSmem <= 227 * 1024, "fused scoring shared memory");
static_assert(kScoreTmemCols == 128 || kScoreTmemCols == 256 || kScoreTmemCols == 512,
              "tensor-memory allocation");

// byte offset of element (r, k) in the no-swizzle K-major core-matrix layout
// of a tile with kdim columns: core (r / 8, k / 8) at ((r/8)(kdim/8) + k/8) 128 B
__device__ __forceinline__ uint32_t cm_off(int r, int k, int kdim) {
  return (uint32_t)((((r >> 3) * (kdim >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void stage_weights(uint8_t* dst, const bf16* __restrict__ src, int kdim) {
  const int per_row = kdim / 8;
  for (int v = threadIdx.x; v < kH * per_row; v += blockDim.x) {
    const int r = v / per_row, c = v - r * per_row;
    *reinterpret_cast<uint4*>(dst + cm_off(r, 8 * c, kdim)) =
        *reinterpret_cast<const uint4*>(src + (int64_t)r * kdim + 8 * c);
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// barrier of one 128-thread group (named barrier `id`, 1 + group)
__device__ __forceinline__ void group_sync(uint32_t id) {
  asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}

// the group's threads agree on v (AND) at named barrier `id`
__device__ __forceinline__ bool group_and(bool v, uint32_t id) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)v), "r"(id)
      : "memory");
  return out != 0;
}

// bounded wait for the group's MMAs, agreed by the whole group
__device__ __forceinline__ bool group_wait(uint32_t bar, uint32_t phase, long long spin, uint32_t id) {
  const bool got = mbar_wait(bar, phase, spin);
  return group_and(got, id);
}

__device__ __forceinline__ void issue_layer(bool leader, uint32_t tmem, uint32_t a0, uint32_t b0,
                                            int kdim, uint32_t bar) {
  if (leader) {
    tc_fence_after();
    const uint32_t sbo = (uint32_t)(kdim / 8) * 128u;
    for (int kk = 0; kk < kdim / 16; ++kk)
      tc_mma(tmem, smem_desc(a0 + kk * 256, 128, sbo), smem_desc(b0 + kk * 256, 128, sbo),
             idesc_bf16(128, kH), kk > 0 ? 1u : 0u);
    tc_commit(bar);
  }
}

// hidden-layer epilogue: row r of the group's accumulator (tensor-memory
// lanes of warp quarter q = r / 32) + bias, ReLU, BF16, into the activation
// tile (K = 128 layout)
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem, int r, const float* bias, uint8_t* act) {
  const int q = r >> 5;
  for (int c0 = 0; c0 < kH; c0 += 16) {
    float v[16];
    tc_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      w[i] = pack_bf16x2(fmaxf(v[2 * i] + bias[c0 + 2 * i], 0.0f),
                         fmaxf(v[2 * i + 1] + bias[c0 + 2 * i + 1], 0.0f));
    *reinterpret_cast<uint4*>(act + cm_off(r, c0, kH)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(act + cm_off(r, c0 + 8, kH)) = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

__global__ void __launch_bounds__(kScoreThreads, 1)
    mlp_score_fused_kernel(SampleSrc S, int64_t n, int64_t n_rays, const float4* __restrict__ dirs,
                           const bf16* __restrict__ W1, const bf16* __restrict__ W2,
                           const bf16* __restrict__ W3, const float* __restrict__ theta,
                           float* __restrict__ logits, uint32_t* __restrict__ err, long long spin) {
  extern __shared__ __align__(1024) uint8_t smem[];
  float* vec = reinterpret_cast<float*>(smem + kSVec);
  uint32_t* txw = reinterpret_cast<uint32_t*>(smem + kSTx);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kSBar + 8 * kScoreGroups);
  const int warp = threadIdx.x >> 5;
  const int g = threadIdx.x >> 7;        // group
  const int r = threadIdx.x & 127;       // the group's row of a tile
  const uint32_t gbar_id = 1u + (uint32_t)g;
  const bool leader = r == 0;
  stage_weights(smem + kSW1, W1, kIn);
  stage_weights(smem + kSW2, W2, kH);
  stage_weights(smem + kSW3, W3, kH);
  for (int f = threadIdx.x; f < kH; f += blockDim.x) {
    vec[f] = theta[kOffB1 + f];
    vec[kH + f] = theta[kOffB2 + f];
    vec[2 * kH + f] = theta[kOffB3 + f];
    vec[3 * kH + f] = __bfloat162float(__float2bfloat16_rn(theta[kOffW4 + f]));
  }
  if (threadIdx.x < 24) {  // feature (3 + c, octave k) of the TX
    const int c = threadIdx.x >> 3, k = threadIdx.x & 7;
    const float vt = __fdiv_rn(__fsub_rn(S.tx0[c], S.cen[c]), S.inv_half_num[c]);
    float sn, cs;
    sincospif(ldexpf(vt, k), &sn, &cs);
    txw[threadIdx.x] = pack_bf16x2(sn, cs);
  }
  const float b4 = theta[kOffB4];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kScoreTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (leader) mbar_init(smem_u32(smem + kSBar + 8 * g), 1);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot + 128u * (uint32_t)g;  // the group's accumulator columns
  uint8_t* act = smem + kSAct + g * kSActBytes;
  const uint32_t sact = smem_u32(act), bar_a = smem_u32(smem + kSBar + 8 * g);
  uint32_t phase = 0;
  bool ok = true, issued = false;
  const int64_t n_tiles = (n + 127) / 128;
  const int64_t stride = (int64_t)gridDim.x * kScoreGroups;
  for (int64_t tile = (int64_t)blockIdx.x * kScoreGroups + g; tile < n_tiles && ok; tile += stride) {
    // features of row r, eight columns per 16-byte store (K = 96 layout)
    const int64_t row = tile * 128 + r;
    float v[3] = {0.f, 0.f, 0.f};
    if (row < n) {
      const uint32_t ray = S.ray_id ? S.ray_id[row] : (uint32_t)row;
      if (dirs && (int64_t)ray < n_rays) {  // (an id past the launch: computed below)
        const float4 d = __ldg(dirs + ray);
        v[0] = d.x;
        v[1] = d.y;
        v[2] = d.z;
      } else {
        const float3 d = fib_dir(ray, n_rays);
        v[0] = d.x;
        v[1] = d.y;
        v[2] = d.z;
      }
    }
    for (int c = 0; c < 6; ++c) {
      uint32_t w[8];
#pragma unroll
      for (int k = 0; k < kOct; ++k) {
        if (c < 3) {
          float sn, cs;
          sincospif(ldexpf(v[c], k), &sn, &cs);
          w[k] = row < n ? pack_bf16x2(sn, cs) : 0u;
        } else {
          w[k] = row < n ? txw[(c - 3) * 8 + k] : 0u;
        }
      }
      // columns (c * 8 + k) * 2 + {0, 1}: 16 columns per coordinate
      *reinterpret_cast<uint4*>(act + cm_off(r, 16 * c, kIn)) = make_uint4(w[0], w[1], w[2], w[3]);
      *reinterpret_cast<uint4*>(act + cm_off(r, 16 * c + 8, kIn)) = make_uint4(w[4], w[5], w[6], w[7]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    group_sync(gbar_id);
    // layer 1 (K = 96)
    issue_layer(leader, tmem, sact, smem_u32(smem + kSW1), kIn, bar_a);
    issued = true;
    if (!(ok = group_wait(bar_a, phase, spin, gbar_id))) break;
    phase ^= 1u;
    tc_fence_after();
    hidden_epilogue(tmem, r, vec, act);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    group_sync(gbar_id);
    // layer 2
    issue_layer(leader, tmem, sact, smem_u32(smem + kSW2), kH, bar_a);
    if (!(ok = group_wait(bar_a, phase, spin, gbar_id))) break;
    phase ^= 1u;
    tc_fence_after();
    hidden_epilogue(tmem, r, vec + kH, act);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    group_sync(gbar_id);
    // layer 3 and the output layer
    issue_layer(leader, tmem, sact, smem_u32(smem + kSW3), kH, bar_a);
    if (!(ok = group_wait(bar_a, phase, spin, gbar_id))) break;
    phase ^= 1u;
    tc_fence_after();
    float z = 0.0f;
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float a[16];
      tc_ld16(tmem + ((uint32_t)((r >> 5) * 32) << 16) + (uint32_t)c0, a);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float h = __bfloat162float(__float2bfloat16_rn(fmaxf(a[i] + vec[2 * kH + c0 + i], 0.0f)));
        z = fmaf(h, vec[3 * kH + c0 + i], z);
      }
    }
    if (row < n) logits[row] = z + b4;
    tc_fence_before();
    group_sync(gbar_id);
  }
  if (!ok) {
    if (r == 0) atomicOr(err, kErrMmaTimeout);
    if (issued) mbar_wait(bar_a, phase);  // bounded: let the group's MMAs drain
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot),
                 "r"(kScoreTmemCols));
}

// H = bf16(relu(Z + bias)) [B x 128], optionally also transposed [128 x ldt].
// Block: 128 threads = the 128 features, 64 samples per block.
__global__ void act_kernel(const float* __restrict__ Z, const float* __restrict__ bias, int64_t B,
                           bf16* __restrict__ H, bf16* __restrict__ HT, int64_t ldt) {
  const int f = threadIdx.x;
  const float bf = bias[f];
  const int64_t b0 = (int64_t)blockIdx.x * 64;
  for (int64_t b = b0; b < min(B, b0 + 64); ++b) {
    const bf16 h = __float2bfloat16_rn(fmaxf(Z[b * kH + f] + bf, 0.0f));
    H[b * kH + f] = h;
    if (HT) HT[(int64_t)f * ldt + b] = h;
  }
}

// Output layer, loss and its gradient.  Per sample: z = H3 . w4 + b4,
// loss = -[w_p y log s(z) + (1 - y) log(1 - s(z))], dz = (s (w_p y + 1 - y)
// - w_p y) / B; dZ3 = bf16(dz w4 * [H3 > 0]).  Accumulates g(w4), g(b4),
// g(b3) and the mean loss.  Scoring (label == nullptr): writes z only.
__global__ void head_kernel(const bf16* __restrict__ H3, const bf16* __restrict__ w4b,
                            const float* __restrict__ b4, int64_t B, const float* __restrict__ label,
                            const uint32_t* __restrict__ idx, float pos_weight, float inv_batch,
                            float* __restrict__ z_out, bf16* __restrict__ dZ, bf16* __restrict__ dZT,
                            int64_t ldt, float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float red[4];
  __shared__ float zsh;
  const int f = threadIdx.x;
  const int lane = f & 31, w = f >> 5;
  const float wf = __bfloat162float(w4b[f]);
  float gw4 = 0.f, gb3 = 0.f, gb4 = 0.f, ls = 0.f;
  const int64_t b0 = (int64_t)blockIdx.x * 64;
  for (int64_t b = b0; b < min(B, b0 + 64); ++b) {
    const float h = __bfloat162float(H3[b * kH + f]);
    float p = h * wf;
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xFFFFFFFFu, p, o);
    if (lane == 0) red[w] = p;
    __syncthreads();
    if (f == 0) zsh = ((red[0] + red[1]) + (red[2] + red[3])) + b4[0];
    __syncthreads();
    const float z = zsh;
    __syncthreads();
    if (!label) {
      if (f == 0) z_out[b] = z;
      continue;
    }
    const float y = label[idx[b]];
    const float s = 1.0f / (1.0f + expf(-z));
    const float dz = (s * (pos_weight * y + 1.0f - y) - pos_weight * y) * inv_batch;
    if (f == 0) {
      // softplus(-z) = -log s(z), softplus(z) = -log(1 - s(z))
      const float sp_neg = fmaxf(-z, 0.f) + log1pf(expf(-fabsf(z)));
      const float sp_pos = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
      ls += (pos_weight * y * sp_neg + (1.0f - y) * sp_pos) * inv_batch;
      gb4 += dz;
      if (z_out) z_out[b] = z;
    }
    gw4 += dz * h;
    const bf16 g = __float2bfloat16_rn(h > 0.f ? dz * wf : 0.f);
    dZ[b * kH + f] = g;
    dZT[(int64_t)f * ldt + b] = g;
    gb3 += __bfloat162float(g);
  }
  if (!label) return;
  atomicAdd(grad + kOffW4 + f, gw4);
  atomicAdd(grad + kOffB3 + f, gb3);
  if (f == 0) {
    atomicAdd(grad + kOffB4, gb4);
    atomicAdd(loss, ls);
  }
}

// dZ = bf16(dH * [H > 0]) [B x 128] and transposed; g(bias) += column sums.
__global__ void backact_kernel(const float* __restrict__ dH, const bf16* __restrict__ H, int64_t B,
                               bf16* __restrict__ dZ, bf16* __restrict__ dZT, int64_t ldt,
                               float* __restrict__ gbias) {
  const int f = threadIdx.x;
  float acc = 0.f;
  const int64_t b0 = (int64_t)blockIdx.x * 64;
  for (int64_t b = b0; b < min(B, b0 + 64); ++b) {
    const float h = __bfloat162float(H[b * kH + f]);
    const bf16 g = __float2bfloat16_rn(h > 0.f ? dH[b * kH + f] : 0.f);
    dZ[b * kH + f] = g;
    dZT[(int64_t)f * ldt + b] = g;
    acc += __bfloat162float(g);
  }
  atomicAdd(gbias + f, acc);
}

// Adam with bias correction c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// BF16 copies of the weights for the contractions: W1, W2, W3 (row = output),
// w4, and W2^T, W3^T (row = input) for the input-gradient products.
__global__ void cast_weights_kernel(const float* __restrict__ theta, bf16* __restrict__ W1,
                                    bf16* __restrict__ W2, bf16* __restrict__ W3,
                                    bf16* __restrict__ w4, bf16* __restrict__ W2T,
                                    bf16* __restrict__ W3T) {
  const int64_t total = (int64_t)kH * kIn + 2 * kH * kH + kH;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < kH * kIn) {
      W1[i] = __float2bfloat16_rn(theta[kOffW1 + i]);
    } else if (i < kH * kIn + kH * kH) {
      const int64_t j = i - kH * kIn;
      const bf16 w = __float2bfloat16_rn(theta[kOffW2 + j]);
      W2[j] = w;
      W2T[(j % kH) * kH + j / kH] = w;
    } else if (i < kH * kIn + 2 * kH * kH) {
      const int64_t j = i - kH * kIn - kH * kH;
      const bf16 w = __float2bfloat16_rn(theta[kOffW3 + j]);
      W3[j] = w;
      W3T[(j % kH) * kH + j / kH] = w;
    } else {
      const int64_t j = i - kH * kIn - 2 * kH * kH;
      w4[j] = __float2bfloat16_rn(theta[kOffW4 + j]);
    }
  }
}

// ---------------------------------------------------------------- selection
// SplitMix64 (Steele, Lea and Flood 2014) as a counter-based generator:
// u_i = ((mix(seed + (i + 1) gamma) >> 11) + 0.5) 2^-53.
__device__ __forceinline__ double counter_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return ((double)(z >> 11) + 0.5) * 1.1102230246251565e-16;
}

// Sort keys: descending fl32(logit + fl32(gumbel)), ascending index.
__global__ void gumbel_keys_kernel(const float* __restrict__ logits, int64_t n, uint64_t seed,
                                   uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double g = -log(-log(counter_uniform(seed, (uint64_t)i)));
    const float k = __fadd_rn(logits[i], (float)g);
    const uint32_t b = __float_as_uint(k);
    const uint32_t ord = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // ascending with k
    key[i] = ((uint64_t)(~ord) << 32) | (uint64_t)(uint32_t)i;
    val[i] = (uint32_t)i;
  }
}

__global__ void mark_top_kernel(const uint32_t* __restrict__ sorted, int64_t k,
                                uint32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[sorted[i]] = 1u;
}

// one uniform index per stratum [s n / k_u, (s + 1) n / k_u), counters n + s
__global__ void mark_strata_kernel(int64_t n, int64_t k_u, uint64_t seed, uint32_t* __restrict__ flag) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k_u;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = s * n / k_u, hi = (s + 1) * n / k_u;
    if (hi <= lo) continue;
    const double u = counter_uniform(seed, (uint64_t)(n + s));
    const int64_t pick = lo + (int64_t)floor(u * (double)(hi - lo));
    flag[min(pick, hi - 1)] = 1u;
  }
}

__global__ void compact_kernel(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ off,
                               int64_t n, uint32_t* __restrict__ ids, unsigned long long* count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (flag[i]) ids[off[i]] = (uint32_t)i;
    if (i == n - 1) *count = (unsigned long long)off[i] + flag[i];
  }
}

}  // namespace

// ---------------------------------------------------------------- the network object
struct nrt_mlp {
  nrt_ctx* ctx = nullptr;
  int64_t n_rays = 0;
  float cen[3], half[3];
  float* theta = nullptr;  // fp32 master parameters (packed)
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  bf16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *w4 = nullptr, *W2T = nullptr, *W3T = nullptr;
  int64_t t = 0;           // Adam steps taken
  // training workspace for `cap` samples per step
  int64_t cap = 0;
  bf16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *H2T = nullptr,
       *H3 = nullptr, *dZ = nullptr, *dZT = nullptr;
  float* Z = nullptr;
  float* loss = nullptr;   // [steps] device
  int64_t loss_cap = 0;
  uint32_t* idx = nullptr;
  uint32_t* err = nullptr;
  float4* dirs = nullptr;  // launch directions [n_rays] for scoring (built at the first score)
  bool holds_ctx = false;
};

namespace {

void free_ws(nrt_mlp* m) {
  void* p[] = {m->X, m->XT, m->H1, m->H1T, m->H2, m->H2T, m->H3, m->dZ, m->dZT, m->Z, m->idx};
  for (void* q : p)
    if (q) cudaFree(q);
  m->X = m->XT = m->H1 = m->H1T = m->H2 = m->H2T = m->H3 = m->dZ = m->dZT = nullptr;
  m->Z = nullptr;
  m->idx = nullptr;
  m->cap = 0;
}

nrt_status ensure_ws(nrt_mlp* m, int64_t B) {
  nrt_ctx* ctx = m->ctx;
  if (B <= m->cap) return NRT_OK;
  free_ws(m);
  const size_t a = (size_t)B * kH * sizeof(bf16);
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->X, (size_t)B * kIn * sizeof(bf16)));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->XT, (size_t)B * kIn * sizeof(bf16)));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->H1, a));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->H1T, a));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->H2, a));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->H2T, a));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->H3, a));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->dZ, a));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->dZT, a));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->Z, (size_t)B * kH * sizeof(float)));
  NRT_CUDA_TRY(ctx, cudaMalloc(&m->idx, (size_t)B * sizeof(uint32_t)));
  m->cap = B;
  return NRT_OK;
}

nrt_status cast_weights(nrt_mlp* m) {
  cast_weights_kernel<<<64, 256, 0, m->ctx->stream>>>(m->theta, m->W1, m->W2, m->W3, m->w4, m->W2T,
                                                      m->W3T);
  count_launch();
  NRT_CUDA_TRY(m->ctx, cudaGetLastError());
  return NRT_OK;
}

nrt_status check_err(nrt_mlp* m) {
  uint32_t e = 0;
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(&e, m->err, 4, cudaMemcpyDeviceToHost, m->ctx->stream));
  NRT_CUDA_TRY(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  if (e) {
    m->ctx->last_error = "tensor-core wait timed out";
    return NRT_ERR_TIMEOUT;
  }
  return NRT_OK;
}

#define MTRY(expr)                        \
  do {                                    \
    nrt_status _s = (expr);               \
    if (_s != NRT_OK) return _s;          \
  } while (0)

// Forward pass over B samples whose features are in m->X (and XT);
// activations H1, H2 (with transposes when training) and H3.
nrt_status forward_layers(nrt_mlp* m, int64_t B, bool train) {
  nrt_ctx* ctx = m->ctx;
  cudaStream_t st = ctx->stream;
  const unsigned blocks = (unsigned)((B + 63) / 64);
  MTRY(gemm_bf16(ctx, m->X, kIn, m->W1, kIn, m->Z, kH, B, kH, kIn, false, 0, m->err));
  act_kernel<<<blocks, kH, 0, st>>>(m->Z, m->theta + kOffB1, B, m->H1, train ? m->H1T : nullptr, B);
  count_launch();
  MTRY(gemm_bf16(ctx, m->H1, kH, m->W2, kH, m->Z, kH, B, kH, kH, false, 0, m->err));
  act_kernel<<<blocks, kH, 0, st>>>(m->Z, m->theta + kOffB2, B, m->H2, train ? m->H2T : nullptr, B);
  count_launch();
  MTRY(gemm_bf16(ctx, m->H2, kH, m->W3, kH, m->Z, kH, B, kH, kH, false, 0, m->err));
  act_kernel<<<blocks, kH, 0, st>>>(m->Z, m->theta + kOffB3, B, m->H3, nullptr, B);
  count_launch();
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  return NRT_OK;
}

SampleSrc norm_src(const nrt_mlp* m) {
  SampleSrc S{};
  for (int c = 0; c < 3; ++c) {
    S.cen[c] = m->cen[c];
    S.inv_half_num[c] = m->half[c];
  }
  return S;
}

}  // namespace

extern "C" {

nrt_status nrt_mlp_create(nrt_ctx* ctx, const float* params, int64_t n_params, const float* box_min,
                          const float* box_max, int64_t n_rays, nrt_mlp** out) {
  if (!ctx || !params || !box_min || !box_max || !out || n_rays <= 0 || n_rays > 0xFFFFFFFFll)
    return NRT_ERR_ARG;
  if (n_params != kNParams) {
    ctx->last_error = "nrt_mlp_create: expected " + std::to_string(kNParams) + " parameters";
    return NRT_ERR_ARG;
  }
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  nrt_mlp* m = new nrt_mlp();
  m->ctx = ctx;
  m->n_rays = n_rays;
  for (int c = 0; c < 3; ++c) {
    m->cen[c] = 0.5f * (box_min[c] + box_max[c]);
    m->half[c] = 0.5f * (box_max[c] - box_min[c]);
    if (!(m->half[c] > 0.0f)) {
      delete m;
      ctx->last_error = "nrt_mlp_create: empty scene box";
      return NRT_ERR_ARG;
    }
  }
  auto fail = [&](cudaError_t e) {
    ctx->last_error = std::string("nrt_mlp_create: ") + cudaGetErrorString(e);
    nrt_mlp_free(m);
    return e == cudaErrorMemoryAllocation ? NRT_ERR_OOM : NRT_ERR_CUDA;
  };
  const size_t pb = (size_t)kNParams * sizeof(float);
  cudaError_t e;
  if ((e = cudaMalloc(&m->theta, pb)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->grad, pb)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->m, pb)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->v, pb)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->W1, (size_t)kH * kIn * sizeof(bf16))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->W2, (size_t)kH * kH * sizeof(bf16))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->W3, (size_t)kH * kH * sizeof(bf16))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->W2T, (size_t)kH * kH * sizeof(bf16))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->W3T, (size_t)kH * kH * sizeof(bf16))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->w4, (size_t)kH * sizeof(bf16))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&m->err, 4)) != cudaSuccess) return fail(e);
  cudaStream_t st = ctx->stream;
  if ((e = cudaMemcpyAsync(m->theta, params, pb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(m->grad, 0, pb, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(m->m, 0, pb, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(m->v, 0, pb, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(m->err, 0, 4, st)) != cudaSuccess) return fail(e);
  nrt_status s = cast_weights(m);
  if (s != NRT_OK) {
    nrt_mlp_free(m);
    return s;
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
  ctx->refs++;  // the network keeps its context alive
  m->holds_ctx = true;
  *out = m;
  return NRT_OK;
}

void nrt_mlp_free(nrt_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->ctx->stream);
  free_ws(m);
  void* p[] = {m->theta, m->grad, m->m, m->v, m->W1, m->W2, m->W3, m->W2T, m->W3T, m->w4, m->err,
               m->loss, m->dirs};
  for (void* q : p)
    if (q) cudaFree(q);
  nrt_ctx* ctx = m->ctx;
  const bool held = m->holds_ctx;
  delete m;
  if (held) ctx_release(ctx);
}

nrt_status nrt_mlp_params_read(const nrt_mlp* m, float* params) {
  if (!m || !params) return NRT_ERR_ARG;
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(params, m->theta, (size_t)kNParams * 4, cudaMemcpyDeviceToHost,
                                       m->ctx->stream));
  NRT_CUDA_TRY(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  return NRT_OK;
}

nrt_status nrt_mlp_state_read(const nrt_mlp* m, float* params, float* adam_m, float* adam_v,
                              int64_t* step) {
  if (!m || !params || !adam_m || !adam_v || !step) return NRT_ERR_ARG;
  cudaStream_t st = m->ctx->stream;
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(params, m->theta, (size_t)kNParams * 4, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(adam_m, m->m, (size_t)kNParams * 4, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(adam_v, m->v, (size_t)kNParams * 4, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(m->ctx, cudaStreamSynchronize(st));
  *step = m->t;
  return NRT_OK;
}

nrt_status nrt_mlp_state_write(nrt_mlp* m, const float* params, const float* adam_m,
                               const float* adam_v, int64_t step) {
  if (!m || !params || !adam_m || !adam_v || step < 0) return NRT_ERR_ARG;
  for (int64_t i = 0; i < kNParams; ++i)
    if (!std::isfinite(params[i]) || !std::isfinite(adam_m[i]) || !(adam_v[i] >= 0.0f) ||
        !std::isfinite(adam_v[i])) {
      m->ctx->last_error = "nrt_mlp_state_write: non-finite value or negative second moment";
      return NRT_ERR_ARG;
    }
  NRT_CUDA_TRY(m->ctx, cudaSetDevice(m->ctx->device));
  cudaStream_t st = m->ctx->stream;
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(m->theta, params, (size_t)kNParams * 4, cudaMemcpyHostToDevice, st));
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(m->m, adam_m, (size_t)kNParams * 4, cudaMemcpyHostToDevice, st));
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(m->v, adam_v, (size_t)kNParams * 4, cudaMemcpyHostToDevice, st));
  MTRY(cast_weights(m));  // BF16 copies of the restored master weights
  NRT_CUDA_TRY(m->ctx, cudaStreamSynchronize(st));
  m->t = step;
  return NRT_OK;
}

nrt_status nrt_mlp_grads_read(const nrt_mlp* m, float* grads) {
  if (!m || !grads) return NRT_ERR_ARG;
  NRT_CUDA_TRY(m->ctx, cudaMemcpyAsync(grads, m->grad, (size_t)kNParams * 4, cudaMemcpyDeviceToHost,
                                       m->ctx->stream));
  NRT_CUDA_TRY(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  return NRT_OK;
}

nrt_status nrt_mlp_features(nrt_mlp* m, const float* tx, const uint32_t* ray_ids, int64_t n,
                            uint16_t* out) {
  if (!m || !tx || !out || n <= 0) return NRT_ERR_ARG;
  SampleSrc S = norm_src(m);
  for (int c = 0; c < 3; ++c) S.tx0[c] = tx[c];
  S.ray_id = ray_ids;
  S.n = n;
  features_kernel<<<blocks_for_n(n), 256, 0, m->ctx->stream>>>(S, n, m->n_rays, (bf16*)out, nullptr,
                                                               0, nullptr);
  count_launch();
  NRT_CUDA_TRY(m->ctx, cudaGetLastError());
  return NRT_OK;
}

nrt_status nrt_mlp_score(nrt_mlp* m, const float* tx, const uint32_t* ray_ids, int64_t n,
                         float* logits) {
  if (!m || !tx || !logits || n <= 0) return NRT_ERR_ARG;
  nrt_ctx* ctx = m->ctx;
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  launch_counter() = 0;
  SampleSrc S = norm_src(m);
  for (int c = 0; c < 3; ++c) S.tx0[c] = tx[c];
  S.ray_id = ray_ids;
  S.n = n;
  cudaStream_t st = ctx->stream;
  NRT_CUDA_TRY(ctx, cudaFuncSetAttribute(mlp_score_fused_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kScoreSmem));
  if (!m->dirs && m->n_rays <= kDirTableMax) {
    NRT_CUDA_TRY(ctx, cudaMalloc(&m->dirs, (size_t)m->n_rays * sizeof(float4)));
    dir_table_kernel<<<blocks_for_n(m->n_rays), 256, 0, st>>>(m->n_rays, m->dirs);
    count_launch();
  }
  const int64_t tiles = (n + 127) / 128;
  const unsigned grid = (unsigned)std::min<int64_t>((tiles + kScoreGroups - 1) / kScoreGroups,
                                                    ctx->sm_count);
  mlp_score_fused_kernel<<<grid, kScoreThreads, kScoreSmem, st>>>(S, n, m->n_rays, m->dirs, m->W1,
                                                                 m->W2, m->W3, m->theta, logits,
                                                                 m->err, wait_limit(ctx));
  count_launch();
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  return NRT_OK;
}

nrt_status nrt_mlp_train(nrt_mlp* m, const float* tx_table, int32_t n_tx, const int32_t* tx_index,
                         const uint32_t* ray_id, const float* label, int64_t n,
                         const uint32_t* order, int64_t start, int32_t n_steps,
                         const nrt_mlp_train_opts* o, float* loss_host) {
  if (!m || !tx_table || n_tx <= 0 || !tx_index || !ray_id || !label || n <= 0 || !o ||
      n_steps <= 0)
    return NRT_ERR_ARG;
  nrt_ctx* ctx = m->ctx;
  const int64_t B = o->batch;
  if (B < 128 || (B % 128) || B > (1 << 24)) {
    ctx->last_error = "nrt_mlp_train: batch must be a positive multiple of 128";
    return NRT_ERR_ARG;
  }
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  launch_counter() = 0;
  MTRY(ensure_ws(m, B));
  cudaStream_t st = ctx->stream;
  if (m->loss_cap < n_steps) {
    if (m->loss) cudaFree(m->loss);
    NRT_CUDA_TRY(ctx, cudaMalloc(&m->loss, (size_t)n_steps * sizeof(float)));
    m->loss_cap = n_steps;
  }
  NRT_CUDA_TRY(ctx, cudaMemsetAsync(m->loss, 0, (size_t)n_steps * sizeof(float), st));
  NRT_CUDA_TRY(ctx, cudaMemsetAsync(m->err, 0, 4, st));
  SampleSrc S = norm_src(m);
  S.tx_table = tx_table;
  S.tx_index = tx_index;
  S.ray_id = ray_id;
  S.order = order;
  S.n = n;
  const unsigned blocks = (unsigned)((B + 63) / 64);
  const float inv_b = 1.0f / (float)B;
  const int64_t ks = 1024;  // split-K chunk of the weight-gradient products
  for (int32_t step = 0; step < n_steps; ++step) {
    S.start = (start + (int64_t)step * B) % n;
    NRT_CUDA_TRY(ctx, cudaMemsetAsync(m->grad, 0, (size_t)kNParams * sizeof(float), st));
    features_kernel<<<blocks_for_n(B), 256, 0, st>>>(S, B, m->n_rays, m->X, m->XT, B, m->idx);
    count_launch();
    MTRY(forward_layers(m, B, true));
    head_kernel<<<blocks, kH, 0, st>>>(m->H3, m->w4, m->theta + kOffB4, B, label, m->idx,
                                       o->pos_weight, inv_b, nullptr, m->dZ, m->dZT, B, m->grad,
                                       m->loss + step);
    count_launch();
    // layer 3: g(W3) = dZ3^T H2, dH2 = dZ3 W3
    MTRY(gemm_bf16(ctx, m->dZT, B, m->H2T, B, m->grad + kOffW3, kH, kH, kH, B, true, ks, m->err));
    MTRY(gemm_bf16(ctx, m->dZ, kH, m->W3T, kH, m->Z, kH, B, kH, kH, false, 0, m->err));
    backact_kernel<<<blocks, kH, 0, st>>>(m->Z, m->H2, B, m->dZ, m->dZT, B, m->grad + kOffB2);
    count_launch();
    // layer 2
    MTRY(gemm_bf16(ctx, m->dZT, B, m->H1T, B, m->grad + kOffW2, kH, kH, kH, B, true, ks, m->err));
    MTRY(gemm_bf16(ctx, m->dZ, kH, m->W2T, kH, m->Z, kH, B, kH, kH, false, 0, m->err));
    backact_kernel<<<blocks, kH, 0, st>>>(m->Z, m->H1, B, m->dZ, m->dZT, B, m->grad + kOffB1);
    count_launch();
    // layer 1: g(W1) = dZ1^T X
    MTRY(gemm_bf16(ctx, m->dZT, B, m->XT, B, m->grad + kOffW1, kIn, kH, kIn, B, true, ks, m->err));
    ++m->t;
    const double c1 = 1.0 / (1.0 - std::pow((double)o->beta1, (double)m->t));
    const double c2 = 1.0 / (1.0 - std::pow((double)o->beta2, (double)m->t));
    adam_kernel<<<64, 256, 0, st>>>(m->theta, m->grad, m->m, m->v, kNParams, o->lr, o->beta1,
                                    o->beta2, o->eps, (float)c1, (float)c2);
    count_launch();
    MTRY(cast_weights(m));
  }
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  if (loss_host)
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(loss_host, m->loss, (size_t)n_steps * sizeof(float),
                                      cudaMemcpyDeviceToHost, st));
  return check_err(m);
}

nrt_status nrt_propose(nrt_ctx* ctx, const float* logits, int64_t n, int64_t k_top,
                       int64_t k_uniform, uint64_t seed, uint32_t* ids, int64_t* n_ids) {
  if (!ctx || !logits || !ids || !n_ids || n <= 0 || n > 0xFFFFFFFFll || k_top < 0 ||
      k_uniform < 0)
    return NRT_ERR_ARG;
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  k_top = std::min(k_top, n);
  uint64_t *key = nullptr, *tk = nullptr;
  uint32_t *val = nullptr, *tv = nullptr, *flag = nullptr, *off = nullptr;
  unsigned long long* cnt = nullptr;
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&key, n * 8, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&tk, n * 8, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&val, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&tv, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&flag, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&off, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&cnt, 8, st));
  NRT_CUDA_TRY(ctx, cudaMemsetAsync(flag, 0, n * 4, st));
  const unsigned g = blocks_for_n(n);
  gumbel_keys_kernel<<<g, 256, 0, st>>>(logits, n, seed, key, val);
  count_launch();
  if (k_top > 0) {
    radix_sort_pairs(key, val, tk, tv, n, 64, st);
    mark_top_kernel<<<blocks_for_n(k_top), 256, 0, st>>>(val, k_top, flag);
    count_launch();
  }
  if (k_uniform > 0) {
    mark_strata_kernel<<<blocks_for_n(k_uniform), 256, 0, st>>>(n, k_uniform, seed, flag);
    count_launch();
  }
  scan_exclusive(flag, off, n, st);
  compact_kernel<<<g, 256, 0, st>>>(flag, off, n, ids, cnt);
  count_launch();
  unsigned long long hc = 0;
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(&hc, cnt, 8, cudaMemcpyDeviceToHost, st));
  void* p[] = {key, tk, val, tv, flag, off, cnt};
  for (void* q : p) cudaFreeAsync(q, st);
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  *n_ids = (int64_t)hc;
  return NRT_OK;
}

nrt_status nrt_gemm_bf16(nrt_ctx* ctx, const uint16_t* A, int64_t lda, const uint16_t* B,
                         int64_t ldb, float* C, int64_t ldc, int64_t M, int32_t N, int64_t K,
                         int32_t accumulate, int64_t k_split) {
  if (!ctx || !A || !B || !C) return NRT_ERR_ARG;
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  uint32_t* err = nullptr;
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&err, 4, ctx->stream));
  NRT_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 4, ctx->stream));
  nrt_status s = gemm_bf16(ctx, (const bf16*)A, lda, (const bf16*)B, ldb, C, ldc, M, N, K,
                           accumulate != 0, k_split, err);
  uint32_t he = 0;
  if (s == NRT_OK) {
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(&he, err, 4, cudaMemcpyDeviceToHost, ctx->stream));
  }
  cudaFreeAsync(err, ctx->stream);
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (s != NRT_OK) return s;
  if (he) {
    ctx->last_error = "tensor-core wait timed out";
    return NRT_ERR_TIMEOUT;
  }
  return NRT_OK;
}

}  // extern "C"
