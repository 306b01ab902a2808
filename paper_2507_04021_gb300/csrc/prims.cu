// Device primitives: exclusive scan and a stable LSD radix sort of
// (uint64 key, uint32 value) pairs.  Used by the scene build (Morton order of
// the points) and to put paths in a deterministic order.
#include <cstdio>

#include "nrt_internal.h"

namespace nrt {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// exclusive scan of one tile per block; writes the tile total to sums[block]
__global__ void scan_tile_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                 int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t sh[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t acc = 0;
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    acc += v[i];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    uint32_t t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0u;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  uint32_t run = sh[threadIdx.x] - acc;  // exclusive prefix of this thread
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == kScanThreads - 1 && sums) sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void scan_add_kernel(uint32_t* __restrict__ out, int64_t n,
                                const uint32_t* __restrict__ offs) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const uint32_t add = offs[blockIdx.x];
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
    if (base + i < n) out[base + i] += add;
}

}  // namespace

int64_t& launch_counter() {
  static thread_local int64_t c = 0;
  return c;
}

#ifdef NRT_CHECK_BOUNDS
thread_local bool g_dbg_capturing = false;
void debug_capture(bool on) { g_dbg_capturing = on; }

void debug_launch_check(const char* file, int line) {
  static bool reported = false;
  if (g_dbg_capturing) return;  // no synchronisation inside a stream capture
  const cudaError_t e = cudaDeviceSynchronize();
  const cudaError_t l = cudaPeekAtLastError();
  if (!reported && (e != cudaSuccess || l != cudaSuccess)) {
    reported = true;
    fprintf(stderr, "[nrt debug] launch at %s:%d (launch #%lld): %s / %s\n", file, line,
            (long long)launch_counter(), cudaGetErrorString(e), cudaGetErrorString(l));
  }
}
#endif

void scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t blocks = (n + kScanTile - 1) / kScanTile;
  if (blocks == 1) {
    scan_tile_kernel<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
    count_launch();
    return;
  }
  uint32_t *sums = nullptr, *offs = nullptr;
  cudaMallocAsync(&sums, blocks * sizeof(uint32_t), st);
  cudaMallocAsync(&offs, blocks * sizeof(uint32_t), st);
  scan_tile_kernel<<<(unsigned)blocks, kScanThreads, 0, st>>>(in, out, n, sums);
  scan_exclusive(sums, offs, blocks, st);
  scan_add_kernel<<<(unsigned)blocks, kScanThreads, 0, st>>>(out, n, offs);
  count_launch(2);
  cudaFreeAsync(sums, st);
  cudaFreeAsync(offs, st);
}

// ---------------------------------------------------------------- radix sort
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kWarps = kSortThreads / 32;

// n_dev (optional): the live element count on the device; entries past it
// are neither counted nor moved
__device__ __forceinline__ int64_t live_count(int64_t cap, const unsigned long long* n_dev) {
  return n_dev ? min((int64_t)*n_dev, cap) : cap;
}

__global__ void radix_hist_kernel(const uint64_t* __restrict__ keys, int64_t cap,
                                  const unsigned long long* __restrict__ n_dev, int shift,
                                  uint32_t* __restrict__ counts, int n_blocks) {
  __shared__ uint32_t h[256];
  const int64_t n = live_count(cap, n_dev);
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * n_blocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: elements of a tile are ranked in input order, round by
// round; within a round a warp ranks with match_any and warps are ordered by
// per-warp digit counts in shared memory.
__global__ void radix_scatter_kernel(const uint64_t* __restrict__ kin,
                                     const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
                                     uint32_t* __restrict__ vout, int64_t cap,
                                     const unsigned long long* __restrict__ n_dev, int shift,
                                     const uint32_t* __restrict__ offsets, int n_blocks) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[kWarps][256];
  const int64_t n = live_count(cap, n_dev);
  if ((int64_t)blockIdx.x * kSortTile >= n) return;  // a tile past the live count moves nothing
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offsets[(int64_t)tid * n_blocks + blockIdx.x];
  for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + tid;
    const bool valid = i < n;
    uint64_t k = 0;
    uint32_t v = 0, dg = 0, rank_w = 0;
    if (valid) {
      k = kin[i];
      if (vin) v = vin[i];
      dg = (uint32_t)(k >> shift) & 0xFF;
    }
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
    if (valid) {
      const unsigned peers = __match_any_sync(vm, dg);
      rank_w = __popc(peers & ((1u << lane) - 1u));
      if (rank_w == 0) wcnt[warp][dg] = __popc(peers);
    }
    __syncthreads();
    if (valid) {
      uint32_t before = 0;
      for (int w = 0; w < warp; ++w) before += wcnt[w][dg];
      const uint32_t pos = run[dg] + before + rank_w;
      kout[pos] = k;
      if (vout) vout[pos] = v;
    }
    __syncthreads();
    uint32_t tot = 0;
    for (int w = 0; w < kWarps; ++w) {
      tot += wcnt[w][tid];
      wcnt[w][tid] = 0;
    }
    run[tid] += tot;
    __syncthreads();
  }
}

}  // namespace

// Sort (keys, vals) stably by key bits [lo_bit, bits) (lower bits keep their
// input order).  The result ends in keys/vals; tk/tv are scratch of n
// entries; vals (and tv) may be null for a keys-only sort.
void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, int64_t n,
                      int bits, cudaStream_t st, int lo_bit, const unsigned long long* n_dev) {
  if (n <= 1) return;
  const int n_blocks = (int)((n + kSortTile - 1) / kSortTile);
  uint32_t *counts = nullptr, *offs = nullptr;
  cudaMallocAsync(&counts, (size_t)256 * n_blocks * sizeof(uint32_t), st);
  cudaMallocAsync(&offs, (size_t)256 * n_blocks * sizeof(uint32_t), st);
  uint64_t *ka = keys, *kb = tk;
  uint32_t *va = vals, *vb = tv;
  int passes = 0;
  for (int shift = lo_bit; shift < bits; shift += 8, ++passes) {
    radix_hist_kernel<<<n_blocks, kSortThreads, 0, st>>>(ka, n, n_dev, shift, counts, n_blocks);
    scan_exclusive(counts, offs, (int64_t)256 * n_blocks, st);
    radix_scatter_kernel<<<n_blocks, kSortThreads, 0, st>>>(ka, va, kb, vb, n, n_dev, shift,
                                                            offs, n_blocks);
    count_launch(2);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (passes & 1) {
    cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    if (vals) cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
  }
  cudaFreeAsync(counts, st);
  cudaFreeAsync(offs, st);
}

// ---------------------------------------------------------------- L2 probe
// Read bandwidth of the L2 cache, for the L2 roofline of the traversal
// kernels: a buffer well under the L2 size (129 MB on GB300) is read once to
// warm it, then `reps` times by a grid of resident blocks with 16-byte loads
// that bypass L1 (ld.global.cg), each block sweeping a fixed slice.
namespace {

__global__ void __launch_bounds__(512)
    l2_read_kernel(const float4* __restrict__ buf, int64_t n4, int reps, float* __restrict__ sink) {
  float acc = 0.0f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc += v.x + v.y + v.z + v.w;
    }
  }
  if (acc == 1.2345678e-30f) sink[0] = acc;  // keeps the loads; never true for the zero fill
}

}  // namespace

}  // namespace nrt

extern "C" nrt_status nrt_measure_l2(nrt_ctx* ctx, int64_t bytes, int32_t reps, float* gbs) {
  using namespace nrt;
  if (!ctx || !gbs || bytes < (1 << 20) || bytes > ((int64_t)1 << 30) || reps < 1 || reps > 1000)
    return NRT_ERR_ARG;
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int64_t n4 = bytes / 16;
  float4* buf = nullptr;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&buf, n4 * 16, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&sink, 4, st));
  NRT_CUDA_TRY(ctx, cudaMemsetAsync(buf, 0, n4 * 16, st));
  NRT_CUDA_TRY(ctx, cudaEventCreate(&e0));
  NRT_CUDA_TRY(ctx, cudaEventCreate(&e1));
  const unsigned grid = (unsigned)ctx->sm_count * 4;
  l2_read_kernel<<<grid, 512, 0, st>>>(buf, n4, 1, sink);  // warm: the buffer into L2
  count_launch();
  NRT_CUDA_TRY(ctx, cudaEventRecord(e0, st));
  l2_read_kernel<<<grid, 512, 0, st>>>(buf, n4, reps, sink);
  count_launch();
  NRT_CUDA_TRY(ctx, cudaEventRecord(e1, st));
  NRT_CUDA_TRY(ctx, cudaEventSynchronize(e1));
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, st);
  cudaFreeAsync(sink, st);
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  *gbs = (float)((double)n4 * 16.0 * reps / (ms * 1e-3) / 1e9);
  return NRT_OK;
}

