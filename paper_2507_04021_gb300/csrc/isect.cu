// Closest hits of arbitrary rays against the scene (nrt_cast), under the
// paper's disc model (Sec. II-C: ray/disc intersections, the Eq. 3 weighted
// point with the Eq. 4 weights) or under the SDF model of its prior work
// (Eq. 2), kept as an ablation of the intersection model.
//
// SDF model (a reading: the paper gives the Gaussian weight of Eq. 2 and says
// the prior work ray-marched a per-DPS signed distance function).  For DPS D,
// f_D(s) = sum_i w_i n_i.(s - p_i) / sum_i w_i, w_i = exp(-|p_i - s|^2 / (2 s^2))
// over D's points, defined where sum_i w_i >= e^-2.  Along the ray, D is
// marched over the ray's crossing of the bounding box of its points grown by
// 2 sigma: samples every sigma / 2 from the entry, the first pair with both
// samples defined and f > 0 >= f' (outside to inside) brackets the surface,
// 20 bisection steps refine it, the hit is the midpoint.  Each DPS is
// marched over its whole interval, so its root does not depend on the order
// in which DPS are visited.  The closest DPS hit wins (ties: smaller DPS);
// the normal is the normalised sum_i w_i n_i facing the ray, the labels
// those of D's point nearest to the hit.
#include <cmath>

#include "nrt_device.cuh"
#include "nrt_internal.h"

namespace nrt {
namespace {

constexpr int kCastThreads = 128;

struct CastOut {
  float* t;
  float* normal;
  int32_t* dps;
  uint32_t* labels;
};

__device__ __forceinline__ void store_miss(const CastOut& O, int64_t i) {
  if (O.t) O.t[i] = __int_as_float(0x7f800000);
  if (O.normal) O.normal[3 * i] = O.normal[3 * i + 1] = O.normal[3 * i + 2] = 0.0f;
  if (O.dps) O.dps[i] = -1;
  if (O.labels) O.labels[i] = 0;
}

__global__ void __launch_bounds__(kCastThreads)
    cast_disc_kernel(SceneView S, const float* __restrict__ o, const float* __restrict__ d, int64_t n,
                     float tmin, float tmax, CastOut O, uint32_t* err) {
  __shared__ int stk[kStackDepth * kCastThreads];
  __shared__ float tstk[kStackDepth * kCastThreads];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float3 oo = f3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
    const float3 dd = unit3(f3(d[3 * i], d[3 * i + 1], d[3 * i + 2]));
    const Hit h = cast_ray(false, S, oo, dd, -1, tmin, tmax, true, stk + threadIdx.x,
                                  tstk + threadIdx.x, kCastThreads, err);
    if (h.idx < 0) {
      store_miss(O, i);
      continue;
    }
    if (O.t) O.t[i] = h.tbar;
    if (O.normal) {
      O.normal[3 * i] = h.n.x;
      O.normal[3 * i + 1] = h.n.y;
      O.normal[3 * i + 2] = h.n.z;
    }
    if (O.dps) O.dps[i] = h.dps;
    if (O.labels) O.labels[i] = h.labels;
  }
}

// f and the weight sum of DPS [first, first + count) at x (relative to the
// DPS's local origin)
__device__ __forceinline__ void sdf_eval(const SceneView& S, uint2 rg, float3 x, float inv2s2,
                                         float* f, float* W) {
  float sw = 0.0f, sf = 0.0f;
  for (uint32_t i = rg.x; i < rg.x + rg.y; ++i) {
    const float4 P = __ldg(S.disc_p + i);
    const float4 N = __ldg(S.disc_n + i);
    const float vx = x.x - P.x, vy = x.y - P.y, vz = x.z - P.z;
    const float w = expf(-(vx * vx + vy * vy + vz * vz) * inv2s2);
    sw += w;
    sf += w * (N.x * vx + N.y * vy + N.z * vz);
  }
  *W = sw;
  *f = sw > 0.0f ? sf / sw : 0.0f;
}

// SDF root of DPS D on the ray within (t_lo, t_hi), or +inf.  The grid and
// the bracket are those of the DPS's whole interval; marching stops once a
// bracket starts beyond `stop` (the best hit so far), which cannot win.
__device__ float sdf_leaf(const SceneView& S, int D, float3 o, float3 d, float t_lo, float t_hi,
                          float stop, float sigma) {
  const uint2 rg = __ldg(S.dps_range + D);
  const float4 c = __ldg(S.dps_center + D);
  const float3 orl = f3(o.x - c.x, o.y - c.y, o.z - c.z);
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = rg.x; i < rg.x + rg.y; ++i) {
    const float4 P = __ldg(S.disc_p + i);
    lo[0] = fminf(lo[0], P.x), hi[0] = fmaxf(hi[0], P.x);
    lo[1] = fminf(lo[1], P.y), hi[1] = fmaxf(hi[1], P.y);
    lo[2] = fminf(lo[2], P.z), hi[2] = fmaxf(hi[2], P.z);
  }
  const float oc[3] = {orl.x, orl.y, orl.z}, dc[3] = {d.x, d.y, d.z};
  float t0 = t_lo, t1 = t_hi;
  for (int a = 0; a < 3; ++a) {
    const float l = lo[a] - 2.0f * sigma, u = hi[a] + 2.0f * sigma;
    if (dc[a] == 0.0f) {
      if (oc[a] < l || oc[a] > u) return INFINITY;
      continue;
    }
    float ta = (l - oc[a]) / dc[a], tb = (u - oc[a]) / dc[a];
    if (ta > tb) {
      const float tt = ta;
      ta = tb;
      tb = tt;
    }
    t0 = fmaxf(t0, ta);
    t1 = fminf(t1, tb);
  }
  if (!(t0 <= t1)) return INFINITY;
  const float h = 0.5f * sigma, inv2s2 = 1.0f / (2.0f * sigma * sigma);
  const float wmin = 0.1353352832366127f;  // e^-2
  float fa, Wa;
  sdf_eval(S, rg, orl + t0 * d, inv2s2, &fa, &Wa);
  const int n_steps = (int)floorf((t1 - t0) / h);
  for (int k = 0; k < n_steps; ++k) {
    const float ta = t0 + k * h, tb = t0 + (k + 1) * h;
    if (ta > stop) break;
    float fb, Wb;
    sdf_eval(S, rg, orl + tb * d, inv2s2, &fb, &Wb);
    if (Wa >= wmin && Wb >= wmin && fa > 0.0f && fb <= 0.0f) {
      float l = ta, u = tb;
      for (int it = 0; it < 20; ++it) {
        const float m = 0.5f * (l + u);
        float fm, Wm;
        sdf_eval(S, rg, orl + m * d, inv2s2, &fm, &Wm);
        if (fm > 0.0f) l = m;
        else u = m;
      }
      return 0.5f * (l + u);
    }
    fa = fb;
    Wa = Wb;
  }
  return INFINITY;
}

// Closest SDF hit over the DPS whose boxes the ray enters (4-wide BVH, nearest
// child first; leaf boxes are grown by pad when 2 sigma exceeds their r_p)
__global__ void __launch_bounds__(kCastThreads)
    cast_sdf_kernel(SceneView S, const float* __restrict__ o, const float* __restrict__ d, int64_t n,
                    float tmin, float tmax, float sigma, float pad, CastOut O, uint32_t* err) {
  __shared__ int stk_all[kStackDepth * kCastThreads];
  __shared__ float tstk_all[kStackDepth * kCastThreads];
  int* stack = stk_all + threadIdx.x;
  float* tstack = tstk_all + threadIdx.x;
  const int stride = kCastThreads;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float3 oo = f3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
    const float3 dd = unit3(f3(d[3 * i], d[3 * i + 1], d[3 * i + 2]));
    const float3 inv = f3(1.0f / (fabsf(dd.x) > 1e-20f ? dd.x : copysignf(1e-20f, dd.x)),
                          1.0f / (fabsf(dd.y) > 1e-20f ? dd.y : copysignf(1e-20f, dd.y)),
                          1.0f / (fabsf(dd.z) > 1e-20f ? dd.z : copysignf(1e-20f, dd.z)));
    float best_t = tmax;
    int best_D = -1;
    int node = S.root, sp = 0;
    bool overflow = false;
    for (;;) {
      if (node >= 0) {
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
        int nh = 0;
        for (int c = 0; c < 4; ++c) {
          if (cid[c] == kEmptyChild) continue;
          const float x0 = (blx[c] - pad - oo.x) * inv.x, x1 = (bhx[c] + pad - oo.x) * inv.x;
          const float y0 = (bly[c] - pad - oo.y) * inv.y, y1 = (bhy[c] + pad - oo.y) * inv.y;
          const float z0 = (blz[c] - pad - oo.z) * inv.z, z1 = (bhz[c] + pad - oo.z) * inv.z;
          const float tin = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), tmin));
          const float tout = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), best_t));
          if (tin <= tout * 1.000001f + 1e-6f) {
            // insertion by entry t (nearest first)
            int q = nh++;
            while (q > 0 && te[q - 1] > tin) {
              te[q] = te[q - 1];
              ce[q] = ce[q - 1];
              --q;
            }
            te[q] = tin;
            ce[q] = cid[c];
          }
        }
        if (nh > 0) {
          for (int c = nh - 1; c >= 1; --c) {
            if (sp >= kStackDepth) {
              overflow = true;
              break;
            }
            stack[sp * stride] = ce[c];
            tstack[sp * stride] = te[c];
            ++sp;
          }
          if (overflow) break;
          node = ce[0];
          continue;
        }
      } else {
        const int D = leaf_of(node);
        const float t = sdf_leaf(S, D, oo, dd, tmin, tmax, best_t, sigma);
        if (t < best_t || (t == best_t && best_D >= 0 && D < best_D)) {
          best_t = t;
          best_D = D;
        }
      }
      bool found = false;
      while (sp > 0) {
        --sp;
        if (tstack[sp * stride] <= best_t) {
          node = stack[sp * stride];
          found = true;
          break;
        }
      }
      if (!found) break;
    }
    if (overflow) atomicOr(err, kErrStack);
    if (best_D < 0) {
      store_miss(O, i);
      continue;
    }
    // weighted normal and the nearest point's labels at the hit
    const uint2 rg = __ldg(S.dps_range + best_D);
    const float4 c = __ldg(S.dps_center + best_D);
    const float3 q = f3(oo.x - c.x, oo.y - c.y, oo.z - c.z) + best_t * dd;
    const float inv2s2 = 1.0f / (2.0f * sigma * sigma);
    float3 sn = f3(0.f, 0.f, 0.f);
    float dmin = INFINITY;
    int imin = 0x7fffffff;
    uint32_t lab = 0;
    for (uint32_t k = rg.x; k < rg.x + rg.y; ++k) {
      const float4 P = __ldg(S.disc_p + k);
      const float4 N = __ldg(S.disc_n + k);
      const float vx = q.x - P.x, vy = q.y - P.y, vz = q.z - P.z;
      const float dd2 = vx * vx + vy * vy + vz * vz;
      sn = sn + expf(-dd2 * inv2s2) * xyz(N);
      const int idx = __float_as_int(P.w);
      if (dd2 < dmin || (dd2 == dmin && idx < imin)) {
        dmin = dd2;
        imin = idx;
        lab = __float_as_uint(N.w);
      }
    }
    float3 nn = unit3(sn);
    if (dot3(nn, dd) > 0.0f) nn = -1.0f * nn;
    if (O.t) O.t[i] = best_t;
    if (O.normal) {
      O.normal[3 * i] = nn.x;
      O.normal[3 * i + 1] = nn.y;
      O.normal[3 * i + 2] = nn.z;
    }
    if (O.dps) O.dps[i] = best_D;
    if (O.labels) O.labels[i] = lab;
  }
}

}  // namespace
}  // namespace nrt

using namespace nrt;

extern "C" nrt_status nrt_cast(nrt_scene* s, const float* o, const float* d, int64_t n,
                               const nrt_cast_params* p, float* t, float* normal, int32_t* dps,
                               uint32_t* labels) {
  if (!s || !p || n < 0 || (n > 0 && (!o || !d))) return NRT_ERR_ARG;
  nrt_ctx* ctx = s->ctx;
  if (n > ((int64_t)1 << 31)) {
    ctx->last_error = "at most 2^31 rays per call";
    return NRT_ERR_ARG;
  }
  if (p->model != NRT_ISECT_DISC && p->model != NRT_ISECT_SDF) {
    ctx->last_error = "unknown intersection model";
    return NRT_ERR_ARG;
  }
  if (p->model == NRT_ISECT_SDF && !(p->sigma > 0.0f && p->sigma < 1.0f)) {
    ctx->last_error = "SDF sigma must be in (0, 1) m";
    return NRT_ERR_ARG;
  }
  if (!(p->t_min >= 0.0f) || !(p->t_max > p->t_min)) {
    ctx->last_error = "need 0 <= t_min < t_max";
    return NRT_ERR_ARG;
  }
  if (n == 0) return NRT_OK;
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const SceneView S = scene_view(s);
  const CastOut O{t, normal, dps, labels};
  uint32_t* err = nullptr;
  NRT_CUDA_TRY(ctx, cudaMallocAsync(&err, 4, ctx->stream));
  NRT_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 4, ctx->stream));
  const int64_t blocks = std::min<int64_t>((n + kCastThreads - 1) / kCastThreads,
                                           (int64_t)ctx->sm_count * 16);
  if (p->model == NRT_ISECT_DISC) {
    cast_disc_kernel<<<(unsigned)blocks, kCastThreads, 0, ctx->stream>>>(S, o, d, n, p->t_min,
                                                                         p->t_max, O, err);
  } else {
    const float pad = fmaxf(0.0f, 2.0f * p->sigma - s->params.r_p) + 1e-6f;
    cast_sdf_kernel<<<(unsigned)blocks, kCastThreads, 0, ctx->stream>>>(S, o, d, n, p->t_min,
                                                                        p->t_max, p->sigma, pad, O,
                                                                        err);
  }
  count_launch();
  NRT_CUDA_TRY(ctx, cudaGetLastError());
  uint32_t herr = 0;
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, ctx->stream));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  cudaFreeAsync(err, ctx->stream);
  if (herr) {
    ctx->last_error = "traversal stack overflow";
    return NRT_ERR_OVERFLOW;
  }
  return NRT_OK;
}
