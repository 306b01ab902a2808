// Ray-range shards of one simulation (Sec. II-B: rays are independent until
// duplicates are removed, Sec. II-B-4): each rank traces a contiguous range
// of the launch and exports its paths (key, representative, |a|^2); after an
// all-gather the entries of every shard are merged on the device.  Per key
// the shards are visited in ray-range order and the first one whose valid
// candidate fits the remaining try budget represents the key -- with no cap
// (the paper's rule) simply the lowest shard holding a valid path, which is
// the key's lowest valid ray id, so the merge reproduces the single run.
#include <algorithm>

#include "nrt_internal.h"

namespace nrt {
namespace {

__global__ void export_paths_kernel(const PathRec* __restrict__ P, const float2* __restrict__ a,
                                    const unsigned long long* __restrict__ n_p, int64_t cap,
                                    const uint32_t* __restrict__ ray_of_row, uint64_t* __restrict__ hi,
                                    uint64_t* __restrict__ lo, uint32_t* __restrict__ rep,
                                    double* __restrict__ power) {
  const int64_t n = min((int64_t)*n_p, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const PathRec& p = P[i];
    if (hi) hi[i] = p.hi;
    if (lo) lo[i] = p.lo;
    if (rep) {  // LOS and diffracted paths have no ray: 0 (the same on every shard)
      const bool ray = p.rep != kNone && !((p.jtk >> 12) & 1);
      rep[i] = ray ? (ray_of_row ? ray_of_row[p.rep] : p.rep) : 0u;
    }
    if (power) {
      const float2 v = a[i];
      power[i] = (double)v.x * v.x + (double)v.y * v.y;
    }
  }
}

__global__ void iota_kernel(uint32_t* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

template <class T>
__global__ void gather64_kernel(const T* __restrict__ src, const uint32_t* __restrict__ perm,
                                int64_t n, uint64_t* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (uint64_t)src[perm[i]];
}

// one thread per group start in the sorted order: walk the key's entries in
// shard order with the try budget
__global__ void merge_pick_kernel(const uint32_t* __restrict__ perm, int64_t n,
                                  const uint64_t* __restrict__ hi, const uint64_t* __restrict__ lo,
                                  const uint32_t* __restrict__ tried, const uint32_t* __restrict__ rep,
                                  int32_t rep_tries, const double* __restrict__ power, int n_rx,
                                  uint8_t* __restrict__ win, double* __restrict__ power_out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = perm[i];
    const uint64_t h = hi[e], l = lo[e];
    if (i > 0) {
      const uint32_t p = perm[i - 1];
      if (hi[p] == h && lo[p] == l) continue;  // not the first entry of its key
    }
    int64_t budget = rep_tries > 0 ? (int64_t)rep_tries : INT64_MAX;
    for (int64_t g = i; g < n; ++g) {
      const uint32_t f = perm[g];
      if (hi[f] != h || lo[f] != l) break;
      const int64_t t = tried ? (int64_t)tried[f] : 1;
      if (rep[f] != kNone && t <= budget) {
        win[f] = 1;
        const int j = (int)(h >> 56);
        if (power && power_out && j < n_rx) atomicAdd(power_out + j, power[f]);
        break;
      }
      budget -= t;
      if (budget <= 0) break;
    }
  }
}

inline unsigned grid_of(int64_t n, int sm) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm * 16));
}

}  // namespace
}  // namespace nrt

using namespace nrt;

extern "C" nrt_status nrt_paths_export(const nrt_result* r, uint64_t* key_hi, uint64_t* key_lo,
                                       uint32_t* rep, double* power) {
  if (!r) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (power && !r->field_done) {
    ctx->last_error = "nrt_paths_export: the field is not computed (set materials)";
    return NRT_ERR_STATE;
  }
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (r->path_cap > 0) {
    export_paths_kernel<<<grid_of(r->path_cap, ctx->sm_count), 256, 0, ctx->stream>>>(
        (const PathRec*)r->paths, r->path_a, r->ctr + kCtrPaths, r->path_cap,
        r->n_pairs > 0 ? nullptr : r->ray_of_row, key_hi, key_lo, rep, power);
    count_launch();
  }
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  return NRT_OK;
}

extern "C" nrt_status nrt_shard_merge(nrt_ctx* ctx, int64_t n, const uint64_t* key_hi,
                                      const uint64_t* key_lo, const uint32_t* shard,
                                      const uint32_t* tried, const uint32_t* rep, int32_t rep_tries,
                                      const double* power, int32_t n_rx, uint8_t* win,
                                      double* power_out) {
  if (!ctx || n < 0 || n >= ((int64_t)1 << 32) - 1 || rep_tries < 0 || n_rx < 0 ||
      (n > 0 && (!key_hi || !key_lo || !shard || !rep || !win)) || (power_out && !power)) {
    if (ctx) ctx->last_error = "nrt_shard_merge: bad arguments";
    return NRT_ERR_ARG;
  }
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  if (power_out && n_rx > 0) NRT_CUDA_TRY(ctx, cudaMemsetAsync(power_out, 0, n_rx * sizeof(double), st));
  if (n == 0) return NRT_OK;
  const int sm = ctx->sm_count;
  NRT_CUDA_TRY(ctx, cudaMemsetAsync(win, 0, (size_t)n, st));
  uint32_t *perm = nullptr, *tperm = nullptr;
  uint64_t *k = nullptr, *tk = nullptr;
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&perm, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&tperm, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&k, n * 8, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&tk, n * 8, st));
  const unsigned g = grid_of(n, sm);
  iota_kernel<<<g, 256, 0, st>>>(perm, n);
  // least significant key first, each pass stable: shard, then lo, then hi
  gather64_kernel<uint32_t><<<g, 256, 0, st>>>(shard, perm, n, k);
  radix_sort_pairs(k, perm, tk, tperm, n, 32, st);
  gather64_kernel<uint64_t><<<g, 256, 0, st>>>(key_lo, perm, n, k);
  radix_sort_pairs(k, perm, tk, tperm, n, 64, st);
  gather64_kernel<uint64_t><<<g, 256, 0, st>>>(key_hi, perm, n, k);
  radix_sort_pairs(k, perm, tk, tperm, n, 64, st);
  merge_pick_kernel<<<g, 256, 0, st>>>(perm, n, key_hi, key_lo, tried, rep, rep_tries, power, n_rx,
                                       win, power_out);
  count_launch(5);
  cudaFreeAsync(perm, st);
  cudaFreeAsync(tperm, st);
  cudaFreeAsync(k, st);
  cudaFreeAsync(tk, st);
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  return NRT_OK;
}
