// Device-side building blocks of the point-cloud radio ray tracer (sm_103a).
//
//  * the disc test and closest-hit query of Sec. II-C (Eq. 3, Eq. 4),
//  * software BVH traversal over DPS bounding boxes with a per-thread stack
//    in shared memory (GB300 has no RT cores),
//  * 128-bit path keys of Sec. II-B-4,
//  * complex arithmetic and the Fresnel coefficients used by the field.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nrt {

constexpr int kMaxDepth = 5;     // maximum interactions per path
// Traversal stack entries per thread: 27 x 8 B x 128 threads = 27 KB per
// block, 8 blocks (32 warps) per SM.  A deeper tree than the stack sets
// kErrStack and fails the call (the office scene's radix tree is 23 deep).
constexpr int kStackDepth = 27;
// unused child slot of a 4-wide BVH node (leaves are ~DPS >= -n_dps)
constexpr int kEmptyChild = (int)0x80000000;
constexpr float kC0 = 299792458.0f;
constexpr double kEps0 = 8.8541878128e-12;
constexpr uint32_t kNone = 0xFFFFFFFFu;

// device error bits (nrt_counters.error_flags)
enum : uint32_t {
  kErrStack = 1u << 0,       // traversal stack would overflow
  kErrHashFull = 1u << 1,    // hash probe limit reached
  kErrCandFull = 1u << 2,    // candidate buffer full
  kErrKeyFull = 1u << 3,     // more distinct keys than the key capacity
  kErrPathFull = 1u << 4,    // path buffer full
  kErrRecheck = 1u << 5,     // a representative refined twice came out differently
};

// ---------------------------------------------------------------- vector math
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float len3(float3 a) { return sqrtf(dot3(a, a)); }
__device__ __forceinline__ float3 unit3(float3 a) { return (1.0f / len3(a)) * a; }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  // Smith's algorithm keeps the quotient accurate when |b| components differ a lot.
  if (fabsf(b.x) >= fabsf(b.y)) {
    float r = b.y / b.x, den = b.x + b.y * r;
    return make_float2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  float r = b.x / b.y, den = b.x * r + b.y;
  return make_float2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
// principal square root (real part >= 0)
__device__ __forceinline__ float2 csqrt(float2 z) {
  float m = hypotf(z.x, z.y);
  if (m == 0.0f) return make_float2(0.0f, 0.0f);
  if (z.x >= 0.0f) {
    float t = sqrtf(0.5f * (m + z.x));
    return make_float2(t, z.y / (2.0f * t));
  }
  float t = sqrtf(0.5f * (m - z.x));
  return make_float2(fabsf(z.y) / (2.0f * t), copysignf(t, z.y));
}

// complex relative permittivity eta = eps_r - j sigma / (2 pi f eps0) (ITU-R P.2040)
__device__ __forceinline__ float2 permittivity(float eps_r, float sigma, float freq) {
  const float k = (float)(1.0 / (2.0 * 3.14159265358979323846 * kEps0));
  return make_float2(eps_r, -sigma * (k / freq));
}

// Fresnel reflection coefficient for incidence cosine c (pol 0 TE, 1 TM)
__device__ __forceinline__ float2 fresnel(float2 eta, float c, int pol) {
  float sin2 = 1.0f - c * c;
  float2 s = csqrt(make_float2(eta.x - sin2, eta.y));
  if (pol == 0) return cdiv(make_float2(c - s.x, -s.y), make_float2(c + s.x, s.y));
  float2 ec = cscale(c, eta);
  return cdiv(csub(ec, s), cadd(ec, s));
}

// d Gamma / d eta
__device__ __forceinline__ float2 dfresnel(float2 eta, float c, int pol) {
  float sin2 = 1.0f - c * c;
  float2 s = csqrt(make_float2(eta.x - sin2, eta.y));
  if (pol == 0) {
    float2 den = make_float2(c + s.x, s.y);
    return cdiv(make_float2(-c, 0.0f), cmul(s, cmul(den, den)));
  }
  float2 den = cadd(cscale(c, eta), s);
  float2 num = cscale(c, make_float2(eta.x - 2.0f * sin2, eta.y));
  return cdiv(num, cmul(s, cmul(den, den)));
}

// ---------------------------------------------------------------- scene view
// Discs are stored in DPS order (Morton order of the voxels); within a DPS in
// ascending point index.  disc_p.xyz is the position relative to the DPS's
// local origin dps_center, disc_p.w the original point index, disc_n.w the
// labels (surface | material << 16), both as raw bits.
struct SceneView {
  const float4* __restrict__ disc_p;
  const float4* __restrict__ disc_n;
  const uint2* __restrict__ dps_range;  // (first disc, count)
  const float4* __restrict__ dps_center;
  const float4* __restrict__ recv;      // reception point per DPS (DPS-directed launch)
  const float4* __restrict__ nodes;     // 4 float4 per internal node
  const float4* __restrict__ label_box; // [label][2]: box of each surface label's discs
  int n_dps;
  int root;        // >= 0 internal node, < 0 leaf ~dps
  float rp2;       // r_p^2
  float inv2rp2;   // 1 / (2 r_p^2)
  float lambda_d;
  float rho;
  float3 bmin;
};

struct Hit {
  float t;       // t of q_min (ray parameter of the closest disc hit)
  float tbar;    // Eq. 3 point q = o + tbar d (all q_i lie on the ray)
  float3 n;      // weighted normal facing the incoming ray
  int idx;       // point index of q_min (-1: miss)
  int dps;       // DPS of q_min
  uint32_t labels;
};

__device__ __forceinline__ int leaf_of(int c) { return ~c; }

// Whether the ray o + t d, t > tmin, can enter the box of surface label l
// (the same widened slab test as the traversal's): when it cannot, no disc
// with that label can be its closest hit.  *t_exit (optional) receives where
// the ray leaves the box, widened like the test: no disc of the label lies
// beyond it.
__device__ __forceinline__ bool ray_meets_label(const SceneView& S, float3 o, float3 d, float tmin,
                                                uint32_t l, float* t_exit = nullptr) {
  const float4 lo = __ldg(S.label_box + 2 * l), hi = __ldg(S.label_box + 2 * l + 1);
  const float3 inv = f3(1.0f / (fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x)),
                        1.0f / (fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y)),
                        1.0f / (fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z)));
  const float x0 = (lo.x - o.x) * inv.x, x1 = (hi.x - o.x) * inv.x;
  const float y0 = (lo.y - o.y) * inv.y, y1 = (hi.y - o.y) * inv.y;
  const float z0 = (lo.z - o.z) * inv.z, z1 = (hi.z - o.z) * inv.z;
  const float tin = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tmin));
  const float tout = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fmaxf(z0, z1));
  if (t_exit) *t_exit = tout * 1.000001f + 1e-6f;
  return tin <= tout * 1.000001f + 1e-6f;
}

// Closest disc hit along o + t d, t in (tmin, tmax), skipping DPS `skip`.
// any_hit: stop at the first disc hit found (shadow casts); a constant at
// most call sites, so the inlined copy drops the other case.
// weighted: also compute the Eq. 3 point and the weighted normal.
// stack / tstack point at this thread's column of a shared array laid out
// [depth][blockDim.x] (stride = blockDim.x) so that threads hit distinct banks.
// kSmem: how many entries that array holds; deeper entries, up to
// kStackDepth, go to a per-thread local array (a caller with register room
// for more blocks keeps fewer in shared memory; the default keeps all).
template <int kSmem = kStackDepth>
__device__ __forceinline__ Hit cast_ray(bool any_hit, const SceneView& S, float3 o, float3 d,
                                       int skip, float tmin, float tmax, bool weighted, int* stack,
                                       float* tstack, int stride, uint32_t* err) {
  constexpr bool kTwoLevel = kSmem < kStackDepth;
  Hit h;
  h.idx = -1;
  h.dps = -1;
  h.t = tmax;
  h.tbar = 0.0f;
  h.n = f3(0.f, 0.f, 0.f);
  h.labels = 0;
  int lstk[kTwoLevel ? kStackDepth - kSmem : 1];
  float ltstk[kTwoLevel ? kStackDepth - kSmem : 1];
  float best_t = tmax;
  int best_idx = -1;
  int best_leaf = -1;
  uint32_t best_lab = 0;
  const float3 inv = f3(1.0f / (fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x)),
                        1.0f / (fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y)),
                        1.0f / (fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z)));
  const float3 oi = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
  int node = S.root;
  int sp = 0;
  for (;;) {
    if (node >= 0) {
      // 4-wide node: slab tests of the four child boxes, then the nearest hit
      // child next and the others pushed farthest first
      const float4* nd = S.nodes + 8 * (size_t)node;
      const float4 lx = __ldg(nd + 0), ly = __ldg(nd + 1), lz = __ldg(nd + 2);
      const float4 hx = __ldg(nd + 3), hy = __ldg(nd + 4), hz = __ldg(nd + 5);
      const float4 cf = __ldg(nd + 6);
      const float blx[4] = {lx.x, lx.y, lx.z, lx.w}, bly[4] = {ly.x, ly.y, ly.z, ly.w};
      const float blz[4] = {lz.x, lz.y, lz.z, lz.w}, bhx[4] = {hx.x, hx.y, hx.z, hx.w};
      const float bhy[4] = {hy.x, hy.y, hy.z, hy.w}, bhz[4] = {hz.x, hz.y, hz.z, hz.w};
      const int cid[4] = {__float_as_int(cf.x), __float_as_int(cf.y), __float_as_int(cf.z),
                          __float_as_int(cf.w)};
      float te[4];
      int ce[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float x0 = fmaf(blx[c], inv.x, -oi.x), x1 = fmaf(bhx[c], inv.x, -oi.x);
        const float y0 = fmaf(bly[c], inv.y, -oi.y), y1 = fmaf(bhy[c], inv.y, -oi.y);
        const float z0 = fmaf(blz[c], inv.z, -oi.z), z1 = fmaf(bhz[c], inv.z, -oi.z);
        const float tin = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tmin));
        const float tout = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), best_t));
        // conservative comparison: widen by a relative 1e-6 so that float error
        // in the slab test never drops a box the ray grazes
        const bool hit = cid[c] != kEmptyChild && tin <= tout * 1.000001f + 1e-6f;
        te[c] = hit ? tin : __int_as_float(0x7f800000);
        ce[c] = hit ? cid[c] : kEmptyChild;
      }
      // sort the four (entry t, child) pairs by t: misses (+inf) go last
#define NRT_CSWAP(i, j)                                  \
  if (te[j] < te[i]) {                                   \
    const float tt = te[i];                              \
    te[i] = te[j];                                       \
    te[j] = tt;                                          \
    const int cc = ce[i];                                \
    ce[i] = ce[j];                                       \
    ce[j] = cc;                                          \
  }
      NRT_CSWAP(0, 1)
      NRT_CSWAP(2, 3)
      NRT_CSWAP(0, 2)
      NRT_CSWAP(1, 3)
      NRT_CSWAP(1, 2)
#undef NRT_CSWAP
      if (ce[0] != kEmptyChild) {
        bool over = false;
#pragma unroll
        for (int c = 3; c >= 1; --c) {
          if (ce[c] == kEmptyChild) continue;
          if (sp >= kStackDepth) {
            over = true;
            break;
          }
          if (!kTwoLevel || sp < kSmem) {
            stack[sp * stride] = ce[c];
            tstack[sp * stride] = te[c];
          } else {
            lstk[sp - kSmem] = ce[c];
            ltstk[sp - kSmem] = te[c];
          }
          ++sp;
        }
        if (over) {
          atomicOr(err, kErrStack);
          break;
        }
        node = ce[0];
        continue;
      }
    } else {
      const int dps = leaf_of(node);
      if (dps != skip) {
        const uint2 rg = __ldg(S.dps_range + dps);
        const float4 cc = __ldg(S.dps_center + dps);
        const float ox = o.x - cc.x, oy = o.y - cc.y, oz = o.z - cc.z;
        for (uint32_t i = rg.x; i < rg.x + rg.y; ++i) {
          const float4 P = __ldg(S.disc_p + i);
          const float wx = P.x - ox, wy = P.y - oy, wz = P.z - oz;
          // The plane point of a disc is at least as far from its centre as
          // the ray line is: skip discs whose centre is farther than r_p
          // from the line.  The perpendicular offset is formed by components
          // (relative error ~1e-4 at 20 m) and compared with a 1% margin, so
          // no disc the exact test below accepts is ever skipped.
          const float wd = wx * d.x + wy * d.y + wz * d.z;
          const float px = wx - wd * d.x, py = wy - wd * d.y, pz = wz - wd * d.z;
          if (px * px + py * py + pz * pz > S.rp2 * 1.01f) continue;
          const float4 N = __ldg(S.disc_n + i);
          const float num = wx * N.x + wy * N.y + wz * N.z;
          const float den = d.x * N.x + d.y * N.y + d.z * N.z;
          if (den == 0.0f) continue;
          const float t = __fdiv_rn(num, den);
          if (!(t > tmin) || t > best_t) continue;
          const float ex = t * d.x - wx, ey = t * d.y - wy, ez = t * d.z - wz;
          const float r2 = ex * ex + ey * ey + ez * ez;
          if (r2 > S.rp2) continue;
          const int idx = __float_as_int(P.w);
          if (t < best_t || idx < best_idx) {
            best_t = t;
            best_idx = idx;
            best_leaf = dps;
            best_lab = __float_as_uint(N.w);
          }
        }
        if (any_hit && best_idx >= 0) break;
      }
    }
    // pop, skipping subtrees that start beyond the current best hit
    bool found = false;
    while (sp > 0) {
      --sp;
      const bool in_smem = !kTwoLevel || sp < kSmem;
      if ((in_smem ? tstack[sp * stride] : ltstk[sp - kSmem]) <= best_t) {
        node = in_smem ? stack[sp * stride] : lstk[sp - kSmem];
        found = true;
        break;
      }
    }
    if (!found) break;
  }
  if (best_idx < 0) return h;
  h.t = best_t;
  h.idx = best_idx;
  h.dps = best_leaf;
  h.labels = best_lab;
  if (!weighted) return h;
  // Eq. 3 / Eq. 4 over the intersected discs of the DPS of q_min
  const uint2 rg = __ldg(S.dps_range + best_leaf);
  const float4 cc = __ldg(S.dps_center + best_leaf);
  const float ox = o.x - cc.x, oy = o.y - cc.y, oz = o.z - cc.z;
  float sw = 0.f, swt = 0.f;
  float3 sn = f3(0.f, 0.f, 0.f);
  for (uint32_t i = rg.x; i < rg.x + rg.y; ++i) {
    const float4 P = __ldg(S.disc_p + i);
    const float4 N = __ldg(S.disc_n + i);
    const float wx = P.x - ox, wy = P.y - oy, wz = P.z - oz;
    const float num = wx * N.x + wy * N.y + wz * N.z;
    const float den = d.x * N.x + d.y * N.y + d.z * N.z;
    if (den == 0.0f) continue;
    const float t = __fdiv_rn(num, den);
    if (!(t > tmin)) continue;
    const float ex = t * d.x - wx, ey = t * d.y - wy, ez = t * d.z - wz;
    const float r2 = ex * ex + ey * ey + ez * ez;
    if (r2 > S.rp2) continue;
    const float w = expf(-r2 * S.inv2rp2) * expf(-S.lambda_d * fabsf(t - best_t));
    sw += w;
    swt += w * t;
    sn = sn + w * xyz(N);
  }
  h.tbar = swt / sw;
  float3 n = unit3(sn);
  if (dot3(n, d) > 0.0f) n = -1.0f * n;
  h.n = n;
  return h;
}

// ---------------------------------------------------------------- launch
// Fibonacci sphere: z = 1 - (2i+1)/N, phi = 2 pi frac(i G / 2^64) with the
// 64-bit golden-angle constant G = round((2 - golden ratio) 2^64).  The
// fraction and the angle are evaluated once per ray in double precision and
// rounded to float, so the launch direction carries float rounding only.
__device__ __forceinline__ float3 fib_dir(uint32_t i, int64_t n) {
  const uint64_t G = 0x61C8864680B583EBull;
  const uint64_t u = (uint64_t)i * G;
  const double frac = (double)(u >> 11) * 1.1102230246251565e-16;  // 2^-53
  double s, c;
  sincospi(2.0 * frac, &s, &c);
  const double a = (2.0 * (double)i + 1.0) / (double)n;
  const double r = sqrt(fmax(a * (2.0 - a), 0.0));
  return f3((float)(r * c), (float)(r * s), (float)(1.0 - a));
}

// ---------------------------------------------------------------- keys
// hi = [rx:8 @56][diffuse:1 @55][k:3 @52][low 52]; see nrt.h.
__device__ __forceinline__ void make_key(int j, int diffuse, int k, const uint16_t* lab,
                                         const int* vox, uint64_t* hi, uint64_t* lo) {
  uint64_t h = ((uint64_t)(j & 0xFF) << 56) | ((uint64_t)(diffuse & 1) << 55) |
               ((uint64_t)(k & 7) << 52);
  uint64_t l = 0;
  const int nl = diffuse ? k - 1 : k;
  for (int m = 0; m < nl && m < 4; ++m) l |= (uint64_t)lab[m] << (16 * m);
  if (!diffuse && nl >= 5) h |= (uint64_t)lab[4];
  if (diffuse)
    h |= (uint64_t)(vox[0] & 0xFFFF) | ((uint64_t)(vox[1] & 0xFFFF) << 16) |
         ((uint64_t)(vox[2] & 0xFFFF) << 32);
  *hi = h;
  *lo = l;
}

// 64-bit hash of a key (the start of its probe sequence): the splitmix64
// finaliser applied to a combination of both words.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}
__device__ __forceinline__ uint64_t key_hash(uint64_t hi, uint64_t lo) {
  return mix64(hi ^ mix64(lo + 0x9E3779B97F4A7C15ull));
}

// voxel of a point, floor((q - bmin) / rho), as in the scene build
__device__ __forceinline__ void voxel_of(const SceneView& S, float3 q, int* v) {
  v[0] = (int)floorf(__fdiv_rn(__fsub_rn(q.x, S.bmin.x), S.rho));
  v[1] = (int)floorf(__fdiv_rn(__fsub_rn(q.y, S.bmin.y), S.rho));
  v[2] = (int)floorf(__fdiv_rn(__fsub_rn(q.z, S.bmin.z), S.rho));
}

// warp-aggregated atomic increment
__device__ __forceinline__ unsigned long long warp_inc(unsigned long long* ctr) {
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & ((1u << lane) - 1u));
}

}  // namespace nrt
