// Scene build (Sec. II-A): voxelise the augmented point cloud at resolution
// rho, group each voxel's points into a discretised point set (DPS) with an
// AABB inflated by the disc radius and a reception point at the mean
// position, and build a bounding-volume hierarchy over the DPS boxes.
//
// GB300 layout: points sorted along a Morton curve of their voxels (a stable
// LSD radix sort), disc records as two float4 streams (position + point id,
// normal + labels) so a DPS is one contiguous run read with 16-byte loads;
// the hierarchy is a binary radix tree over the DPS Morton codes (Karras
// 2012), each internal node holding both child boxes in 64 bytes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nrt_internal.h"

namespace nrt {
namespace {

__device__ __forceinline__ uint32_t f2sortable(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float sortable2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// min/max of positions (sortable encoding) + input validation flags
__global__ void bounds_kernel(const float* __restrict__ pos, const float* __restrict__ nrm,
                              int64_t n, uint32_t* __restrict__ mm, uint32_t* __restrict__ bad) {
  uint32_t lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, hi[3] = {0, 0, 0};
  uint32_t b = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float nn = 0.f;
    for (int k = 0; k < 3; ++k) {
      float p = pos[3 * i + k];
      if (!isfinite(p)) b |= 1u;
      uint32_t s = f2sortable(p);
      lo[k] = min(lo[k], s);
      hi[k] = max(hi[k], s);
      float q = nrm[3 * i + k];
      if (!isfinite(q)) b |= 2u;
      nn += q * q;
    }
    if (!(nn > 0.25f)) b |= 2u;  // zero or badly non-unit normal
  }
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], o));
      hi[k] = max(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], o));
    }
  }
  for (int o = 16; o > 0; o >>= 1) b |= __shfl_xor_sync(0xFFFFFFFFu, b, o);
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < 3; ++k) {
      atomicMin(&mm[k], lo[k]);
      atomicMax(&mm[3 + k], hi[k]);
    }
    if (b) atomicOr(bad, b);
  }
}

// Bounding box of every surface label's points (sortable encoding; labels
// are 16-bit): mm[6 * label + 0..2] min, [3..5] max.  Labels without points
// keep an empty box (min above max).
__global__ void label_bounds_kernel(const float* __restrict__ pos, const uint16_t* __restrict__ surf,
                                    int64_t n, uint32_t* __restrict__ mm) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t l = surf[i];
    for (int k = 0; k < 3; ++k) {
      const uint32_t u = f2sortable(pos[3 * i + k]);
      atomicMin(&mm[6 * l + k], u);
      atomicMax(&mm[6 * l + 3 + k], u);
    }
  }
}

// sortable bounds -> float4 (lo, hi) pairs grown by pad
__global__ void label_box_kernel(const uint32_t* __restrict__ mm, float pad, float4* __restrict__ box) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= 65536) return;
  const uint32_t* m = mm + 6 * l;
  if (m[0] > m[3]) {  // no points with this label: an empty box
    box[2 * l] = make_float4(1e30f, 1e30f, 1e30f, 0.f);
    box[2 * l + 1] = make_float4(-1e30f, -1e30f, -1e30f, 0.f);
    return;
  }
  box[2 * l] = make_float4(sortable2f(m[0]) - pad, sortable2f(m[1]) - pad, sortable2f(m[2]) - pad, 0.f);
  box[2 * l + 1] = make_float4(sortable2f(m[3]) + pad, sortable2f(m[4]) + pad, sortable2f(m[5]) + pad, 0.f);
}

__device__ __forceinline__ uint64_t spread3(uint64_t x) {
  x &= 0x1FFFFF;
  x = (x | x << 32) & 0x1F00000000FFFFull;
  x = (x | x << 16) & 0x1F0000FF0000FFull;
  x = (x | x << 8) & 0x100F00F00F00F00Full;
  x = (x | x << 4) & 0x10C30C30C30C30C3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

// voxel coordinates floor(fl32(fl32(p - bmin) / rho)) and their Morton code
__global__ void morton_kernel(const float* __restrict__ pos, int64_t n, float3 bmin, float rho,
                              uint64_t* __restrict__ key, uint32_t* __restrict__ idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v[3];
    const float b[3] = {bmin.x, bmin.y, bmin.z};
    for (int k = 0; k < 3; ++k) {
      float s = __fdiv_rn(__fsub_rn(pos[3 * i + k], b[k]), rho);
      v[k] = (uint64_t)(int64_t)floorf(s);
    }
    key[i] = spread3(v[0]) | (spread3(v[1]) << 1) | (spread3(v[2]) << 2);
    idx[i] = (uint32_t)i;
  }
}

__global__ void dps_flag_kernel(const uint64_t* __restrict__ key, int64_t n,
                                uint32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

__global__ void dps_begin_kernel(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ id,
                                 int64_t n, uint32_t* __restrict__ begin) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) begin[id[i]] = (uint32_t)i;
}

__global__ void disc_pack_kernel(const float* __restrict__ pos, const float* __restrict__ nrm,
                                 const uint16_t* __restrict__ surf, const uint8_t* __restrict__ mat,
                                 const uint32_t* __restrict__ order, int64_t n,
                                 float4* __restrict__ dp, float4* __restrict__ dn) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = order[i];
    dp[i] = make_float4(pos[3 * s], pos[3 * s + 1], pos[3 * s + 2], __int_as_float((int)s));
    const uint32_t lab = (uint32_t)surf[s] | ((uint32_t)mat[s] << 16);
    dn[i] = make_float4(nrm[3 * s], nrm[3 * s + 1], nrm[3 * s + 2], __uint_as_float(lab));
  }
}

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10C30C30C30C30C3ull;
  x = (x ^ (x >> 4)) & 0x100F00F00F00F00Full;
  x = (x ^ (x >> 8)) & 0x1F0000FF0000FFull;
  x = (x ^ (x >> 16)) & 0x1F00000000FFFFull;
  x = (x ^ (x >> 32)) & 0x1FFFFF;
  return (uint32_t)x;
}

// per DPS: range, voxel, Morton code, reception point, inflated AABB
__global__ void dps_reduce_kernel(const uint32_t* __restrict__ begin, int64_t n_dps, int64_t n,
                                  const float4* __restrict__ dp, const uint64_t* __restrict__ key,
                                  float pad, float3 bmin, float rho, uint2* __restrict__ range,
                                  int32_t* __restrict__ vox,
                                  uint64_t* __restrict__ dkey, float4* __restrict__ recv,
                                  float4* __restrict__ box, float4* __restrict__ center) {
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n_dps;
       d += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = begin[d];
    const uint32_t e = (d + 1 < n_dps) ? begin[d + 1] : (uint32_t)n;
    range[d] = make_uint2(b, e - b);
    const uint64_t k = key[b];
    dkey[d] = k;
    vox[3 * d] = (int32_t)compact3(k);
    vox[3 * d + 1] = (int32_t)compact3(k >> 1);
    vox[3 * d + 2] = (int32_t)compact3(k >> 2);
    float3 s = f3(0.f, 0.f, 0.f), lo = f3(1e30f, 1e30f, 1e30f), hi = f3(-1e30f, -1e30f, -1e30f);
    for (uint32_t i = b; i < e; ++i) {
      const float4 p = dp[i];
      s = s + xyz(p);
      lo = f3(fminf(lo.x, p.x), fminf(lo.y, p.y), fminf(lo.z, p.z));
      hi = f3(fmaxf(hi.x, p.x), fmaxf(hi.y, p.y), fmaxf(hi.z, p.z));
    }
    const float inv = 1.0f / (float)(e - b);
    recv[d] = make_float4(s.x * inv, s.y * inv, s.z * inv, 0.f);
    // local origin: the voxel's min corner, so that DPS lying on one
    // axis-aligned plane share the plane coordinate exactly
    center[d] = make_float4(__fadd_rn(bmin.x, __fmul_rn((float)vox[3 * d], rho)),
                            __fadd_rn(bmin.y, __fmul_rn((float)vox[3 * d + 1], rho)),
                            __fadd_rn(bmin.z, __fmul_rn((float)vox[3 * d + 2], rho)), 0.f);
    box[2 * d] = make_float4(lo.x - pad, lo.y - pad, lo.z - pad, 0.f);
    box[2 * d + 1] = make_float4(hi.x + pad, hi.y + pad, hi.z + pad, 0.f);
  }
}

// Disc positions relative to the min corner of their voxel: the difference
// of two nearby floats is exact, so a cast that forms (o - c) once per DPS
// makes the same rounding for every disc of the set, and that rounding
// cancels in the depth differences t_i - t_min of Eq. 4.
// id is the exclusive scan of the DPS-start flags, so point i belongs to DPS
// id[i] + flag[i] - 1.
__global__ void disc_localize_kernel(float4* __restrict__ dp, const uint32_t* __restrict__ id,
                                     const uint32_t* __restrict__ flag,
                                     const float4* __restrict__ center, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 c = center[id[i] + flag[i] - 1u];
    const float4 p = dp[i];
    dp[i] = make_float4(p.x - c.x, p.y - c.y, p.z - c.z, p.w);
  }
}

__device__ __forceinline__ int delta(const uint64_t* __restrict__ k, int64_t n, int64_t i,
                                     int64_t j) {
  if (j < 0 || j >= n) return -1;
  return __clzll(k[i] ^ k[j]);
}

// Binary radix tree over distinct sorted keys (Karras 2012): internal node i
// covers a key range; its split is the first position where the common
// prefix shortens.  Children >= 0 are internal nodes, < 0 leaves (~dps).
__global__ void karras_kernel(const uint64_t* __restrict__ k, int64_t n, int* __restrict__ child,
                              int* __restrict__ parent, int* __restrict__ leaf_parent) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n - 1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(k, n, i, i - d);
    int64_t lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
      if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(k, n, i, j);
    int64_t s = 0;
    int64_t t = l;
    do {
      t = (t + 1) >> 1;
      if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int64_t g = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    const int left = (lo == g) ? ~(int)g : (int)g;
    const int right = (hi == g + 1) ? ~(int)(g + 1) : (int)(g + 1);
    child[2 * i] = left;
    child[2 * i + 1] = right;
    if (left >= 0) parent[left] = (int)i; else leaf_parent[~left] = (int)i;
    if (right >= 0) parent[right] = (int)i; else leaf_parent[~right] = (int)i;
  }
}

// Bottom-up boxes: the second thread to reach a node merges its children.
__global__ void bvh_bounds_kernel(int64_t n_dps, const int* __restrict__ child,
                                  const int* __restrict__ parent, const int* __restrict__ leaf_parent,
                                  const float4* __restrict__ leaf_box, float4* node_box,
                                  unsigned int* visits, float4* __restrict__ nodes) {
  for (int64_t lf = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lf < n_dps;
       lf += (int64_t)gridDim.x * blockDim.x) {
    int node = leaf_parent[lf];
    for (int guard = 0; guard < 128 && node >= 0; ++guard) {
      __threadfence();
      if (atomicAdd(&visits[node], 1u) == 0u) break;
      __threadfence();
      float4 bx[4];
      for (int c = 0; c < 2; ++c) {
        const int ch = child[2 * node + c];
        if (ch < 0) {
          bx[2 * c] = leaf_box[2 * (int64_t)(~ch)];
          bx[2 * c + 1] = leaf_box[2 * (int64_t)(~ch) + 1];
        } else {
          bx[2 * c] = __ldcg(node_box + 2 * (int64_t)ch);
          bx[2 * c + 1] = __ldcg(node_box + 2 * (int64_t)ch + 1);
        }
      }
      const float4 L0 = bx[0], L1 = bx[1], R0 = bx[2], R1 = bx[3];
      nodes[4 * (int64_t)node + 0] = make_float4(L0.x, L0.y, L0.z, L1.x);
      nodes[4 * (int64_t)node + 1] = make_float4(L1.y, L1.z, R0.x, R0.y);
      nodes[4 * (int64_t)node + 2] = make_float4(R0.z, R1.x, R1.y, R1.z);
      nodes[4 * (int64_t)node + 3] =
          make_float4(__int_as_float(child[2 * node]), __int_as_float(child[2 * node + 1]), 0.f, 0.f);
      __stcg(node_box + 2 * (int64_t)node,
             make_float4(fminf(L0.x, R0.x), fminf(L0.y, R0.y), fminf(L0.z, R0.z), 0.f));
      __stcg(node_box + 2 * (int64_t)node + 1,
             make_float4(fmaxf(L1.x, R1.x), fmaxf(L1.y, R1.y), fmaxf(L1.z, R1.z), 0.f));
      __threadfence();
      node = node == 0 ? -1 : parent[node];
    }
  }
}

inline int grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 64);
}

}  // namespace

nrt_status build_scene(nrt_scene* s, const float* pos, const float* nrm, const uint16_t* surf,
                       const uint8_t* mat) {
  nrt_ctx* ctx = s->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t n = s->n;
  cudaEvent_t e0, e1;
  NRT_CUDA_TRY(ctx, cudaEventCreate(&e0));
  NRT_CUDA_TRY(ctx, cudaEventCreate(&e1));
  NRT_CUDA_TRY(ctx, cudaEventRecord(e0, st));

  uint32_t* mm = nullptr;  // 6 sortable bounds + 1 flag
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&mm, 8 * sizeof(uint32_t), st));
  const uint32_t init[8] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0, 0, 0, 0, 0};
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, st));
  bounds_kernel<<<grid_for(n), 256, 0, st>>>(pos, nrm, n, mm, mm + 6);
  uint32_t hm[8];
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(hm, mm, sizeof(hm), cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  cudaFreeAsync(mm, st);
  if (hm[6] & 1u) {
    ctx->last_error = "non-finite point position";
    return NRT_ERR_ARG;
  }
  if (hm[6] & 2u) {
    ctx->last_error = "zero or non-finite normal";
    return NRT_ERR_ARG;
  }
  auto dec = [](uint32_t u) {
    uint32_t b = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
    float f;
    memcpy(&f, &b, 4);
    return f;
  };
  float bmax[3];
  for (int k = 0; k < 3; ++k) {
    s->bmin[k] = dec(hm[k]);
    bmax[k] = dec(hm[3 + k]);
  }
  const float rho = s->params.rho;
  int bits = 1;
  for (int k = 0; k < 3; ++k) {
    const double span = ((double)bmax[k] - (double)s->bmin[k]) / rho + 2.0;
    while ((double)(1ull << bits) < span) ++bits;
  }
  if (bits > 21) {
    ctx->last_error = "scene spans more than 2^21 voxels along an axis";
    return NRT_ERR_ARG;
  }
  s->grid_bits = bits;

  uint64_t *key = nullptr, *tkey = nullptr;
  uint32_t *order = nullptr, *tord = nullptr, *flag = nullptr, *id = nullptr;
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&key, n * 8, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&tkey, n * 8, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&order, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&tord, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&flag, n * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&id, n * 4, st));
  morton_kernel<<<grid_for(n), 256, 0, st>>>(pos, n, make_float3(s->bmin[0], s->bmin[1], s->bmin[2]), rho, key, order);
  radix_sort_pairs(key, order, tkey, tord, n, 3 * bits, st);
  dps_flag_kernel<<<grid_for(n), 256, 0, st>>>(key, n, flag);
  scan_exclusive(flag, id, n, st);
  uint32_t last[2];
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(&last[0], id + n - 1, 4, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(&last[1], flag + n - 1, 4, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  const int64_t n_dps = (int64_t)last[0] + last[1];
  s->n_dps = n_dps;

  uint32_t* begin = nullptr;
  uint64_t* dkey = nullptr;
  float4* box = nullptr;
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&begin, n_dps * 4, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&dkey, n_dps * 8, st));
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&box, n_dps * 32, st));
  NRT_CUDA_TRY(ctx, cudaMalloc(&s->disc_p, n * sizeof(float4)));
  NRT_CUDA_TRY(ctx, cudaMalloc(&s->disc_n, n * sizeof(float4)));
  NRT_CUDA_TRY(ctx, cudaMalloc(&s->dps_range, n_dps * sizeof(uint2)));
  NRT_CUDA_TRY(ctx, cudaMalloc(&s->dps_vox, n_dps * 3 * sizeof(int32_t)));
  NRT_CUDA_TRY(ctx, cudaMalloc(&s->dps_recv, n_dps * sizeof(float4)));
  NRT_CUDA_TRY(ctx, cudaMalloc(&s->dps_center, n_dps * sizeof(float4)));
  dps_begin_kernel<<<grid_for(n), 256, 0, st>>>(flag, id, n, begin);
  disc_pack_kernel<<<grid_for(n), 256, 0, st>>>(pos, nrm, surf, mat, order, n, s->disc_p, s->disc_n);
  double ext = 0.0;
  for (int k = 0; k < 3; ++k) ext = std::max(ext, (double)bmax[k] - (double)s->bmin[k]);
  const float pad = s->params.r_p + (float)(1e-6 * ext) + 1e-6f;
  dps_reduce_kernel<<<grid_for(n_dps), 256, 0, st>>>(begin, n_dps, n, s->disc_p, key, pad,
                                                       make_float3(s->bmin[0], s->bmin[1], s->bmin[2]),
                                                       rho, s->dps_range, s->dps_vox, dkey, s->dps_recv,
                                                       box, s->dps_center);
  disc_localize_kernel<<<grid_for(n), 256, 0, st>>>(s->disc_p, id, flag, s->dps_center, n);
  // per surface label: the box of its discs (grown by the DPS boxes' pad and
  // 1e-4 m more, so that a ray-box test in float cannot drop a disc)
  {
    uint32_t* lmm = nullptr;
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&lmm, 65536 * 6 * sizeof(uint32_t), st));
    NRT_CUDA_TRY(ctx, cudaMemsetAsync(lmm, 0xFF, 65536 * 6 * sizeof(uint32_t), st));
    for (int k = 0; k < 3; ++k)  // max fields start at 0 (below every encoded value)
      NRT_CUDA_TRY(ctx, cudaMemset2DAsync(lmm + 3 + k, 6 * sizeof(uint32_t), 0, sizeof(uint32_t),
                                          65536, st));
    NRT_CUDA_TRY(ctx, cudaMalloc(&s->label_box, 65536 * 2 * sizeof(float4)));
    label_bounds_kernel<<<grid_for(n), 256, 0, st>>>(pos, surf, n, lmm);
    label_box_kernel<<<65536 / 256, 256, 0, st>>>(lmm, pad + 1e-4f, s->label_box);
    cudaFreeAsync(lmm, st);
  }
  // hierarchy
  const int64_t n_int = std::max<int64_t>(n_dps - 1, 1);
  NRT_CUDA_TRY(ctx, cudaMalloc(&s->nodes, n_int * 4 * sizeof(float4)));
  if (n_dps == 1) {
    s->root = ~0;
  } else {
    int *child = nullptr, *parent = nullptr, *leaf_parent = nullptr;
    float4* node_box = nullptr;
    unsigned int* visits = nullptr;
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&child, n_int * 2 * sizeof(int), st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&parent, n_int * sizeof(int), st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&leaf_parent, n_dps * sizeof(int), st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&node_box, n_int * 2 * sizeof(float4), st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&visits, n_int * sizeof(unsigned int), st));
    NRT_CUDA_TRY(ctx, cudaMemsetAsync(visits, 0, n_int * sizeof(unsigned int), st));
    NRT_CUDA_TRY(ctx, cudaMemsetAsync(parent, 0xFF, n_int * sizeof(int), st));
    karras_kernel<<<grid_for(n_dps), 256, 0, st>>>(dkey, n_dps, child, parent, leaf_parent);
    bvh_bounds_kernel<<<grid_for(n_dps), 256, 0, st>>>(n_dps, child, parent, leaf_parent, box,
                                                        node_box, visits, s->nodes);
    s->root = 0;
    cudaFreeAsync(child, st);
    cudaFreeAsync(parent, st);
    cudaFreeAsync(leaf_parent, st);
    cudaFreeAsync(node_box, st);
    cudaFreeAsync(visits, st);
    const nrt_status rc4 = collapse_bvh4(s, n_int, st);
    if (rc4 != NRT_OK) return rc4;
  }
  cudaFreeAsync(key, st);
  cudaFreeAsync(tkey, st);
  cudaFreeAsync(order, st);
  cudaFreeAsync(tord, st);
  cudaFreeAsync(flag, st);
  cudaFreeAsync(id, st);
  cudaFreeAsync(begin, st);
  cudaFreeAsync(dkey, st);
  cudaFreeAsync(box, st);
  NRT_CUDA_TRY(ctx, cudaEventRecord(e1, st));
  NRT_CUDA_TRY(ctx, cudaEventSynchronize(e1));
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  cudaEventElapsedTime(&s->build_ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return NRT_OK;
}

// 4-wide BVH collapsed (on the host) from the binary radix tree: a node takes
// its binary node's two children and opens the internal child with the
// largest box surface area until it holds four children or only leaves.
// Node layout, 8 float4: lo.x[4], lo.y[4], lo.z[4], hi.x[4], hi.y[4], hi.z[4],
// child[4] (>= 0 node, < 0 ~DPS, kEmptyChild unused), spare.  Replaces the
// binary nodes in s->nodes; the root is node 0.
nrt_status collapse_bvh4(nrt_scene* s, int64_t n_int, cudaStream_t st) {
  nrt_ctx* ctx = s->ctx;
  std::vector<float4> bin((size_t)n_int * 4);
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(bin.data(), s->nodes, bin.size() * sizeof(float4),
                                    cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  struct Child {
    int id;
    float lo[3], hi[3];
  };
  auto kids = [&](int node, Child* c) {
    const float4 a = bin[4 * node], b = bin[4 * node + 1], cc = bin[4 * node + 2], e = bin[4 * node + 3];
    int l, r;
    memcpy(&l, &e.x, 4);
    memcpy(&r, &e.y, 4);
    c[0] = Child{l, {a.x, a.y, a.z}, {a.w, b.x, b.y}};
    c[1] = Child{r, {b.z, b.w, cc.x}, {cc.y, cc.z, cc.w}};
  };
  auto area = [](const Child& c) {
    const float dx = c.hi[0] - c.lo[0], dy = c.hi[1] - c.lo[1], dz = c.hi[2] - c.lo[2];
    return dx * dy + dy * dz + dz * dx;
  };
  std::vector<float4> out;
  out.reserve((size_t)n_int * 4);
  std::vector<std::pair<int, int64_t>> queue;  // (binary node, BVH4 node)
  queue.push_back({0, 0});
  out.resize(8);
  for (size_t qi = 0; qi < queue.size(); ++qi) {
    const int bn = queue[qi].first;
    const int64_t slot = queue[qi].second;
    Child ch[4];
    int nc = 2;
    kids(bn, ch);
    while (nc < 4) {
      int best = -1;
      float ba = -1.0f;
      for (int i = 0; i < nc; ++i)
        if (ch[i].id >= 0 && area(ch[i]) > ba) {
          ba = area(ch[i]);
          best = i;
        }
      if (best < 0) break;
      Child two[2];
      kids(ch[best].id, two);
      ch[best] = two[0];
      ch[nc++] = two[1];
    }
    float lo[3][4], hi[3][4];
    int cid[4];
    for (int i = 0; i < 4; ++i) {
      if (i >= nc) {
        for (int k = 0; k < 3; ++k) lo[k][i] = hi[k][i] = 0.0f;
        cid[i] = kEmptyChild;
        continue;
      }
      for (int k = 0; k < 3; ++k) {
        lo[k][i] = ch[i].lo[k];
        hi[k][i] = ch[i].hi[k];
      }
      if (ch[i].id >= 0) {
        const int64_t ns = (int64_t)(out.size() / 8);
        out.resize(out.size() + 8);
        queue.push_back({ch[i].id, ns});
        cid[i] = (int)ns;
      } else {
        cid[i] = ch[i].id;
      }
    }
    float4* nd = out.data() + 8 * slot;
    for (int k = 0; k < 3; ++k) {
      nd[k] = make_float4(lo[k][0], lo[k][1], lo[k][2], lo[k][3]);
      nd[3 + k] = make_float4(hi[k][0], hi[k][1], hi[k][2], hi[k][3]);
    }
    float f[4];
    memcpy(f, cid, 16);
    nd[6] = make_float4(f[0], f[1], f[2], f[3]);
    nd[7] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float4* n4 = nullptr;
  NRT_CUDA_TRY(ctx, cudaMalloc(&n4, out.size() * sizeof(float4)));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(n4, out.data(), out.size() * sizeof(float4),
                                    cudaMemcpyHostToDevice, st));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  cudaFree(s->nodes);
  s->nodes = n4;
  s->n_nodes4 = (int64_t)(out.size() / 8);
  return NRT_OK;
}

SceneView scene_view(const nrt_scene* s) {
  SceneView v;
  v.disc_p = s->disc_p;
  v.disc_n = s->disc_n;
  v.dps_range = s->dps_range;
  v.dps_center = s->dps_center;
  v.label_box = s->label_box;
  v.recv = s->dps_recv;
  v.nodes = s->nodes;
  v.n_dps = (int)s->n_dps;
  v.root = s->root;
  v.rp2 = s->params.r_p * s->params.r_p;
  v.inv2rp2 = 1.0f / (2.0f * s->params.r_p * s->params.r_p);
  v.lambda_d = s->params.lambda_d;
  v.rho = s->params.rho;
  v.bmin = make_float3(s->bmin[0], s->bmin[1], s->bmin[2]);
  return v;
}

}  // namespace nrt
