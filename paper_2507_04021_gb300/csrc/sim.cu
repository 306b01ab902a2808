// One simulation for one TX (Sec. II-B of the paper), as a sequence of
// kernels on the context stream:
//
//   vis_kernel       visibility from every RX to every DPS reception point
//   los_kernel       TX -> RX casts (LOS paths)
//   trace_kernel     Fibonacci launch; each ray reflected specularly at every
//                    hit (Eq. 3 point, weighted normal) up to the depth limit;
//                    per-bounce hit records
//   emit_kernel      path candidates (sphere or visibility capture) keyed by
//                    the 128-bit key of Sec. II-B-4 into an open-addressing
//                    hash table; min ray id per key
//   validate_*       per key, candidates in ray-id order until one validates:
//                    diffuse = shadow cast scatter point -> RX (Sec. II-B-1);
//                    specular = image-method minimiser of Eq. 1 on the
//                    interaction planes, then validation casts with t_a, t_d
//                    and up to kappa retries (Sec. II-B-2)
//   field_kernel     complex path coefficient and delay; per-RX power
//   adjoint_kernel   gradient of the received power w.r.t. per-label eps_r,
//                    sigma, S recomputed from the stored interaction sequences
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nrt_internal.h"

namespace nrt {
namespace {

constexpr int kTraceThreads = 128;
constexpr int kMaxProbe = 4096;

struct Table {
  unsigned long long* fp;  // 0 = empty
  uint64_t* hi;
  uint64_t* lo;
  uint32_t* minrow;
  uint32_t* kid;
  uint32_t* next;
  uint64_t mask;
};

struct KeyState {
  uint32_t* slot;    // [key] -> table slot
  uint32_t* cur;     // candidate row being validated
  uint32_t* tries;
  uint32_t* status;  // 0 pending, 1 valid, 2 invalid
};

struct Records {
  float4* q;  // q.xyz, segment length
  float4* n;  // normal.xyz (facing the incoming ray), cos_in
  float4* d;  // outgoing direction.xyz, dps (bits)
  int2* i;    // point index of q_min (-1: miss), labels (surf | mat << 16)
  int64_t n_rows;
  __device__ __forceinline__ int64_t at(int s, int64_t row) const {
    return (int64_t)s * n_rows + row;
  }
};

struct SimConst {
  float3 tx;
  int n_rx;
  int max_depth;
  int n_seg;
  int capture;
  int diffuse;
  int pol;
  int kappa;
  int rep_tries;
  float r_rx2;
  float t_min;
  float cos_ta;
  float t_d;
  float freq;
  float lambda;
  int64_t n_rays;
  int64_t vis_words;
};

__device__ __forceinline__ bool vis_bit(const uint32_t* vis, int64_t words, int j, int d) {
  return (__ldg(vis + (int64_t)j * words + (d >> 5)) >> (d & 31)) & 1u;
}

__device__ __forceinline__ void count_add(unsigned long long* c, unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(c, v);
}

#define NRT_STACK_DECL                                       \
  __shared__ int stk[kStackDepth * kTraceThreads];           \
  __shared__ float tstk[kStackDepth * kTraceThreads];        \
  int* my_stk = stk + threadIdx.x;                           \
  float* my_tstk = tstk + threadIdx.x;                       \
  uint32_t* err = (uint32_t*)(ctr + kCtrErr);

// ---------------------------------------------------------------- visibility
// One thread per (RX, DPS); a warp covers 32 consecutive DPS of one RX and
// writes one bit word.  Visible when nothing is hit before the reception
// point's voxel could begin, or the first hit lies in the DPS itself.
__global__ void __launch_bounds__(kTraceThreads)
    vis_kernel(SceneView S, SimConst C, const float4* __restrict__ rx,
               const float4* __restrict__ recv, uint32_t* __restrict__ vis,
               unsigned long long* ctr, float margin) {
  NRT_STACK_DECL
  const int64_t per_rx = C.vis_words * 32;
  const int64_t total = (int64_t)C.n_rx * per_rx;
  unsigned long long casts = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = base + threadIdx.x;
    bool bit = false;
    if (g < total) {
      const int j = (int)(g / per_rx);
      const int d = (int)(g - (int64_t)j * per_rx);
      if (d < S.n_dps) {
        const float3 o = xyz(__ldg(rx + j));
        const float3 v = xyz(__ldg(recv + d)) - o;
        const float s = len3(v);
        const float tmax = s - margin;
        if (tmax <= C.t_min) {
          bit = true;
        } else {
          const Hit h = cast_ray<false>(S, o, (1.0f / s) * v, -1, C.t_min, tmax, false, my_stk,
                                        my_tstk, kTraceThreads, err);
          ++casts;
          bit = h.idx < 0 || h.dps == d;
        }
      }
    }
    const unsigned word = __ballot_sync(0xFFFFFFFFu, bit);
    if ((threadIdx.x & 31) == 0 && g < total) vis[g >> 5] = word;
  }
  count_add(ctr + kCtrVisCasts, casts);
}

// ---------------------------------------------------------------- LOS
__global__ void __launch_bounds__(kTraceThreads)
    los_kernel(SceneView S, SimConst C, const float4* __restrict__ rx, PathRec* __restrict__ paths,
               unsigned long long* ctr, int64_t path_cap) {
  NRT_STACK_DECL
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C.n_rx) return;
  const float3 r = xyz(rx[j]);
  const float3 v = r - C.tx;
  const float s = len3(v);
  const Hit h = cast_ray<true>(S, C.tx, (1.0f / s) * v, -1, C.t_min, s, false, my_stk, my_tstk,
                               kTraceThreads, err);
  atomicAdd(ctr + kCtrLosCasts, 1ull);
  if (h.idx >= 0) return;
  const unsigned long long p = atomicAdd(ctr + kCtrPaths, 1ull);
  if ((int64_t)p >= path_cap) {
    atomicOr(err, kErrPathFull);
    return;
  }
  PathRec R;
  memset(&R, 0, sizeof(R));
  R.hi = (uint64_t)(j & 0xFF) << 56;
  R.lo = 0;
  R.rep = kNone;
  R.jtk = (uint32_t)j;
  R.length = s;
  R.geo = C.lambda / (4.0f * 3.14159265358979f * s);
  paths[p] = R;
}

// ---------------------------------------------------------------- trace
// One ray per thread; every interaction continues as a specular reflection
// (Sec. II-B: the ray count stays constant).  The next cast skips the DPS
// just hit.
__global__ void __launch_bounds__(kTraceThreads)
    trace_kernel(SceneView S, SimConst C, const uint32_t* __restrict__ ray_of_row,
                 const uint32_t* __restrict__ order, Records R, unsigned long long* ctr) {
  NRT_STACK_DECL
  unsigned long long segs = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < R.n_rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = order ? order[t] : t;
    const uint32_t ray = ray_of_row ? ray_of_row[row] : (uint32_t)row;
    float3 d = fib_dir(ray, C.n_rays);
    float3 o = C.tx;
    int skip = -1;
    for (int s = 0; s < C.n_seg; ++s) {
      const Hit h = cast_ray<false>(S, o, d, skip, C.t_min, __int_as_float(0x7f800000), true,
                                    my_stk, my_tstk, kTraceThreads, err);
      ++segs;
      const int64_t a = R.at(s, row);
      if (h.idx < 0) {
        R.i[a] = make_int2(-1, 0);
        break;
      }
      const float3 q = o + h.tbar * d;
      const float dn = dot3(d, h.n);
      float3 dout = d - (2.0f * dn) * h.n;
      dout = unit3(dout);
      R.q[a] = make_float4(q.x, q.y, q.z, h.tbar);
      R.n[a] = make_float4(h.n.x, h.n.y, h.n.z, fabsf(dn));
      R.d[a] = make_float4(dout.x, dout.y, dout.z, __int_as_float(h.dps));
      R.i[a] = make_int2(h.idx, (int)h.labels);
      o = q;
      d = dout;
      skip = h.dps;
    }
  }
  count_add(ctr + kCtrSegments, segs);
}

// ---------------------------------------------------------------- candidates
struct EmitArgs {
  Table T;
  uint2* cand;              // candidates (slot, row) at per-ray offsets
  const uint32_t* cand_off; // [launch index] first candidate of the ray
  uint32_t* cand_cnt;       // [launch index] candidates of the ray (count pass)
};

// Hash insert by one lane on behalf of the lanes holding the same key (same
// fingerprint); returns the slot.  No shared counters are touched: key ids
// are assigned afterwards from the table's occupancy.
__device__ __forceinline__ uint64_t insert_key(const EmitArgs& A, uint64_t hi, uint64_t lo,
                                               uint64_t f, unsigned long long* ctr) {
  uint64_t slot = f & A.T.mask;
  int probe = 0;
  for (; probe < kMaxProbe; ++probe) {
    const unsigned long long prev = atomicCAS(A.T.fp + slot, 0ull, (unsigned long long)f);
    if (prev == 0ull) {
      A.T.hi[slot] = hi;
      A.T.lo[slot] = lo;
      break;
    }
    if (prev == (unsigned long long)f) break;
    slot = (slot + 1) & A.T.mask;
  }
  if (probe == kMaxProbe) {
    atomicOr((uint32_t*)(ctr + kCtrErr), kErrHashFull);
    return ~0ull;
  }
  if (probe > 64) atomicMax(ctr + kCtrProbeMax, (unsigned long long)probe);
  return slot;
}

// One candidate per lane with pred set (all lanes of the warp call this
// together).  Lanes with equal keys are merged first: one lane inserts the
// key and records the group's lowest row; every lane still stores its own
// (slot, row) candidate, at its ray's next candidate position.  kCount only
// counts candidates per ray and per-warp distinct keys (an upper bound on
// the table's keys).
template <bool kCount>
__device__ __forceinline__ void warp_emit(const EmitArgs& A, bool pred, uint64_t hi, uint64_t lo,
                                          uint32_t row, unsigned long long* ctr, uint32_t& n_mine,
                                          unsigned long long& n_lead) {
  const unsigned act = __ballot_sync(0xFFFFFFFFu, pred);
  if (!act || !pred) return;
  const int lane = threadIdx.x & 31;
  const uint64_t f = key_fp(hi, lo);
  const unsigned peers = __match_any_sync(act, f);
  const int leader = __ffs(peers) - 1;
  if (kCount) {
    ++n_mine;
    if (lane == leader) ++n_lead;
    return;
  }
  const uint32_t minrow = __reduce_min_sync(peers, row);
  uint64_t slot = 0;
  if (lane == leader) {
    slot = insert_key(A, hi, lo, f, ctr);
    if (slot != ~0ull) atomicMin(A.T.minrow + slot, minrow);
  }
  slot = __shfl_sync(peers, slot, leader);
  if (slot == ~0ull) return;
  A.cand[n_mine++] = make_uint2((uint32_t)slot, row);
}

// Candidates of every ray (Sec. II-B): a warp walks 32 rays in launch order
// (neighbouring directions), bounce by bounce and RX by RX in lockstep, so
// that rays that found the same key merge before touching the hash table.
template <bool kCount>
__global__ void __launch_bounds__(256)
    emit_kernel(SceneView S, SimConst C, const float4* __restrict__ rx, Records R,
                const uint32_t* __restrict__ vis, const uint32_t* __restrict__ order, EmitArgs A,
                unsigned long long* ctr) {
  unsigned long long n_lead = 0, n_total = 0;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < R.n_rows; base += n_warps * 32) {
    const int64_t t = base + lane;
    const bool active = t < R.n_rows;
    const uint32_t row = active ? (order ? order[t] : (uint32_t)t) : 0u;
    uint32_t n_mine = (!kCount && active) ? A.cand_off[t] : 0u;
    uint16_t lab[kMaxDepth];
    bool alive = active;
    for (int s = 0; s < C.max_depth; ++s) {
      int2 ri = make_int2(-1, 0);
      float4 qq = make_float4(0.f, 0.f, 0.f, 0.f), dd = qq;
      if (alive) {
        const int64_t a = R.at(s, row);
        ri = R.i[a];
        if (ri.x >= 0) {
          qq = R.q[a];
          dd = R.d[a];
        }
      }
      alive = alive && ri.x >= 0;
      if (!__any_sync(0xFFFFFFFFu, alive)) break;
      const int k = s + 1;
      lab[s] = (uint16_t)(ri.y & 0xFFFF);
      if (C.capture == NRT_CAPTURE_VIS) {
        const int dps = __float_as_int(dd.w);
        int vox[3] = {0, 0, 0};
        if (alive) voxel_of(S, xyz(qq), vox);
        for (int j = 0; j < C.n_rx; ++j) {
          const bool v = alive && vis_bit(vis, C.vis_words, j, dps);
          uint64_t hi = 0, lo = 0;
          if (v) make_key(j, 0, k, lab, vox, &hi, &lo);
          warp_emit<kCount>(A, v, hi, lo, row, ctr, n_mine, n_lead);
          if (C.diffuse) {
            if (v) make_key(j, 1, k, lab, vox, &hi, &lo);
            warp_emit<kCount>(A, v, hi, lo, row, ctr, n_mine, n_lead);
          }
        }
      } else {
        // sphere capture on the segment leaving interaction k
        const float3 o = xyz(qq);
        const float3 dir = xyz(dd);
        float t_end = __int_as_float(0x7f800000);
        if (alive && s + 1 < C.n_seg) {
          const int64_t b = R.at(s + 1, row);
          if (R.i[b].x >= 0) t_end = R.q[b].w;
        }
        for (int j = 0; j < C.n_rx; ++j) {
          bool v = false;
          if (alive) {
            const float3 r = xyz(__ldg(rx + j));
            const float ts = fminf(fmaxf(dot3(r - o, dir), 0.0f), t_end);
            const float3 p = o + ts * dir - r;
            v = dot3(p, p) <= C.r_rx2;
          }
          uint64_t hi = 0, lo = 0;
          if (v) make_key(j, 0, k, lab, nullptr, &hi, &lo);
          warp_emit<kCount>(A, v, hi, lo, row, ctr, n_mine, n_lead);
        }
      }
    }
    if (kCount && active) {
      A.cand_cnt[t] = n_mine;
      n_total += n_mine;
    }
  }
  if (kCount) {
    count_add(ctr + kCtrCands, n_total);
    count_add(ctr + kCtrLeaders, n_lead);
  }
}

// Key ids from the table's occupancy: specular keys first, then diffuse.
__global__ void slot_flags_kernel(Table T, int64_t cap, uint32_t* __restrict__ fs,
                                  uint32_t* __restrict__ fd) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool used = T.fp[i] != 0ull;
    const bool diff = used && ((T.hi[i] >> 55) & 1ull);
    fs[i] = used && !diff;
    fd[i] = diff;
  }
}

__global__ void slot_assign_kernel(Table T, int64_t cap, const uint32_t* __restrict__ fs,
                                   const uint32_t* __restrict__ fd, const uint32_t* __restrict__ os,
                                   const uint32_t* __restrict__ od, uint32_t n_spec,
                                   uint32_t* __restrict__ key_slot, uint64_t* __restrict__ sort_key,
                                   uint32_t* __restrict__ sort_val,
                                   const uint32_t* __restrict__ launch_pos) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!fs[i] && !fd[i]) continue;
    const uint32_t kid = fs[i] ? os[i] : n_spec + od[i];
    T.kid[i] = kid;
    key_slot[kid] = (uint32_t)i;
    // validation order: launch position of the key's lowest row, so that a
    // warp validates keys found by neighbouring rays
    const uint32_t m = T.minrow[i];
    sort_key[kid] = launch_pos ? launch_pos[m] : m;
    sort_val[kid] = kid;
  }
}

__global__ void inverse_order_kernel(const uint32_t* __restrict__ order, int64_t n,
                                     uint32_t* __restrict__ pos) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    pos[order[t]] = (uint32_t)t;
}

// Every candidate re-derives its key from the hit records and compares it
// with the key stored in its slot: a 64-bit fingerprint collision between
// distinct keys is reported, never silently merged.
__global__ void verify_kernel(SceneView S, SimConst C, Records R, Table T, const uint2* __restrict__ cand,
                              int64_t n_cand, unsigned long long* ctr) {
  uint32_t* err = (uint32_t*)(ctr + kCtrErr);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cand;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint2 e = cand[c];
    const uint64_t hi = T.hi[e.x], lo = T.lo[e.x];
    const int j = (int)(hi >> 56);
    const int diffuse = (int)((hi >> 55) & 1);
    const int k = (int)((hi >> 52) & 7);
    uint16_t lab[kMaxDepth];
    for (int s = 0; s < k; ++s) lab[s] = (uint16_t)(R.i[R.at(s, e.y)].y & 0xFFFF);
    int vox[3] = {0, 0, 0};
    if (diffuse) voxel_of(S, xyz(R.q[R.at(k - 1, e.y)]), vox);
    uint64_t h2, l2;
    make_key(j, diffuse, k, lab, vox, &h2, &l2);
    if (h2 != hi || l2 != lo) atomicOr(err, kErrKeyMismatch);
  }
}

// ---------------------------------------------------------------- validation
struct ValArgs {
  Table T;
  KeyState K;
  Records R;
  const float4* rx;
  const uint32_t* ray_of_row;
  PathRec* paths;
  int64_t path_cap;
  uint32_t* next_list;  // keys still pending after this round
  int next_ctr;         // counter slot for next_list
};

__device__ __forceinline__ void finish_key(const ValArgs& A, uint32_t kid, bool valid,
                                           unsigned long long* ctr, const SimConst& C,
                                           const PathRec* rec) {
  uint32_t* err = (uint32_t*)(ctr + kCtrErr);
  if (valid) {
    A.K.status[kid] = 1;
    const unsigned long long p = warp_inc(ctr + kCtrPaths);
    if ((int64_t)p >= A.path_cap) {
      atomicOr(err, kErrPathFull);
      return;
    }
    A.paths[p] = *rec;
    return;
  }
  const uint32_t tr = A.K.tries[kid] + 1;
  A.K.tries[kid] = tr;
  if ((int)tr >= C.rep_tries) {
    A.K.status[kid] = 2;
  } else {
    A.K.status[kid] = 0;
    A.next_list[warp_inc(ctr + A.next_ctr)] = kid;
  }
}

// Diffuse: the candidate's own interaction points; the last one scatters
// toward the RX if the RX is in front of the surface and a cast from the
// scatter point (skipping its DPS) reaches the RX unobstructed (Sec. II-B-1).
__global__ void __launch_bounds__(kTraceThreads)
    validate_diffuse_kernel(SceneView S, SimConst C, ValArgs A, const uint32_t* __restrict__ list,
                            int64_t n_list, unsigned long long* ctr) {
  NRT_STACK_DECL
  unsigned long long casts = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_list;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t kid = list[i];
    const uint32_t slot = A.K.slot[kid];
    const uint32_t row = A.K.cur[kid];
    const uint64_t hi = A.T.hi[slot];
    const int j = (int)(hi >> 56);
    const int k = (int)((hi >> 52) & 7);
    const int64_t a = A.R.at(k - 1, row);
    const float4 qq = A.R.q[a], nn = A.R.n[a];
    const float3 q = xyz(qq), n = xyz(nn);
    const int dps = __float_as_int(A.R.d[a].w);
    const float3 u = xyz(A.rx[j]) - q;
    const float rs = len3(u);
    const float3 w = (1.0f / rs) * u;
    const float cs = dot3(n, w);
    bool valid = false;
    PathRec P;
    if (cs > 0.0f) {
      const Hit h = cast_ray<true>(S, q, w, dps, C.t_min, rs, false, my_stk, my_tstk,
                                   kTraceThreads, err);
      ++casts;
      valid = h.idx < 0;
    }
    if (valid) {
      memset(&P, 0, sizeof(P));
      P.hi = hi;
      P.lo = A.T.lo[slot];
      P.rep = row;
      P.jtk = (uint32_t)j | (1u << 8) | ((uint32_t)k << 9);
      float ri = 0.0f;
      uint64_t mats = 0;
      for (int m = 0; m < k; ++m) {
        const int64_t b = A.R.at(m, row);
        const float4 qm = A.R.q[b];
        P.pts[3 * m] = qm.x;
        P.pts[3 * m + 1] = qm.y;
        P.pts[3 * m + 2] = qm.z;
        ri += qm.w;
        P.cosv[m] = A.R.n[b].w;
        mats |= (uint64_t)((A.R.i[b].y >> 16) & 0xFF) << (8 * m);
      }
      P.mats_lo = (uint32_t)mats;
      P.mats_hi = (uint32_t)(mats >> 32);
      const float ci = nn.w;
      const float rho = S.rho;
      P.geo = C.lambda / (4.0f * 3.14159265358979f) *
              sqrtf(rho * rho * ci * cs / 3.14159265358979f) / (ri * rs);
      P.length = ri + rs;
    }
    finish_key(A, kid, valid, ctr, C, &P);
  }
  count_add(ctr + kCtrValCasts, casts);
}

// Specular: phase 1 solves Eq. 1 on the infinite planes (q_m, n_m) of the
// candidate's interactions; its minimiser with every reflection on the
// correct side of its plane is the image-method path (mirror the TX through
// the planes, back-trace from the RX).  Phase 2 casts I_{m-1} -> I_m and
// accepts the interaction when the hit is on the key's surface, its normal
// within t_a of the plane normal and the hit within t_d of the plane;
// otherwise that plane is replaced by the hit's and the solve retried (at
// most kappa times).  A hit on another surface, a miss or a failed side
// check ends the candidate.  Finally I_k -> RX must be clear.
// Coordinates are taken relative to the RX to keep float magnitudes small.
__global__ void __launch_bounds__(kTraceThreads)
    validate_specular_kernel(SceneView S, SimConst C, ValArgs A, const uint32_t* __restrict__ list,
                             int64_t n_list, unsigned long long* ctr) {
  NRT_STACK_DECL
  unsigned long long casts = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_list;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t kid = list[i];
    const uint32_t slot = A.K.slot[kid];
    const uint32_t row = A.K.cur[kid];
    const uint64_t hi = A.T.hi[slot], lo = A.T.lo[slot];
    const int j = (int)(hi >> 56);
    const int k = (int)((hi >> 52) & 7);
    uint32_t lab[kMaxDepth];
    for (int m = 0; m < 4; ++m) lab[m] = (uint32_t)((lo >> (16 * m)) & 0xFFFF);
    lab[4] = (uint32_t)(hi & 0xFFFF);
    const float3 rxp = xyz(A.rx[j]);
    float3 Pp[kMaxDepth], Pn[kMaxDepth];
    for (int m = 0; m < k; ++m) {
      const int64_t b = A.R.at(m, row);
      Pp[m] = xyz(A.R.q[b]) - rxp;
      Pn[m] = xyz(A.R.n[b]);
    }
    const float3 txl = C.tx - rxp;
    bool valid = false;
    float3 I[kMaxDepth + 2];
    uint32_t vmats[kMaxDepth];
    for (int attempt = 0; attempt <= C.kappa; ++attempt) {
      float3 img[kMaxDepth + 1];
      img[0] = txl;
      for (int m = 0; m < k; ++m)
        img[m + 1] = img[m] - (2.0f * dot3(img[m] - Pp[m], Pn[m])) * Pn[m];
      I[0] = txl;
      I[k + 1] = f3(0.f, 0.f, 0.f);
      float3 tgt = f3(0.f, 0.f, 0.f);
      bool ok = true;
      for (int m = k; m >= 1; --m) {
        const float3 dir = img[m] - tgt;
        const float den = dot3(dir, Pn[m - 1]);
        if (den == 0.0f) {
          ok = false;
          break;
        }
        const float u = dot3(Pp[m - 1] - tgt, Pn[m - 1]) / den;
        I[m] = tgt + u * dir;
        tgt = I[m];
      }
      if (!ok) break;
      for (int m = 1; m <= k && ok; ++m) {
        const float sa = dot3(I[m - 1] - I[m], Pn[m - 1]);
        const float sb = dot3(I[m + 1] - I[m], Pn[m - 1]);
        if (!(sa * sb > 0.0f)) ok = false;
      }
      if (!ok) break;
      int prev_dps = -1;
      int fail_m = -1;
      bool dead = false;
      float3 fq = f3(0.f, 0.f, 0.f), fn = f3(0.f, 0.f, 0.f);
      for (int m = 1; m <= k; ++m) {
        const float3 org = I[m - 1] + rxp;
        const float3 dir = unit3(I[m] - I[m - 1]);
        const Hit h = cast_ray<false>(S, org, dir, prev_dps, C.t_min, __int_as_float(0x7f800000),
                                      true, my_stk, my_tstk, kTraceThreads, err);
        ++casts;
        if (h.idx < 0 || (h.labels & 0xFFFFu) != lab[m - 1]) {
          dead = true;
          break;
        }
        const float3 qh = (org + h.tbar * dir) - rxp;
        const float c = fminf(1.0f, fabsf(dot3(Pn[m - 1], h.n)));
        const float dist = fabsf(dot3(qh - I[m], Pn[m - 1]));
        vmats[m - 1] = (h.labels >> 16) & 0xFFu;
        if (!(c >= C.cos_ta && dist <= C.t_d)) {
          fail_m = m;
          fq = qh;
          fn = h.n;
          break;
        }
        prev_dps = h.dps;
      }
      if (dead) break;
      if (fail_m > 0) {
        if (attempt == C.kappa) break;
        Pp[fail_m - 1] = fq;
        Pn[fail_m - 1] = fn;
        continue;
      }
      // last leg to the RX
      const float3 last = f3(0.f, 0.f, 0.f) - I[k];
      const float s = len3(last);
      const Hit hf = cast_ray<true>(S, I[k] + rxp, (1.0f / s) * last, prev_dps, C.t_min, s, false,
                                    my_stk, my_tstk, kTraceThreads, err);
      ++casts;
      valid = hf.idx < 0;
      break;
    }
    PathRec P;
    if (valid) {
      memset(&P, 0, sizeof(P));
      P.hi = hi;
      P.lo = lo;
      P.rep = row;
      P.jtk = (uint32_t)j | ((uint32_t)k << 9);
      float len = 0.0f;
      uint64_t mats = 0;
      for (int m = 0; m <= k; ++m) len += len3(I[m + 1] - I[m]);
      for (int m = 1; m <= k; ++m) {
        const float3 pw = I[m] + rxp;
        P.pts[3 * (m - 1)] = pw.x;
        P.pts[3 * (m - 1) + 1] = pw.y;
        P.pts[3 * (m - 1) + 2] = pw.z;
        P.cosv[m - 1] = fabsf(dot3(Pn[m - 1], unit3(I[m] - I[m - 1])));
        mats |= (uint64_t)vmats[m - 1] << (8 * (m - 1));
      }
      P.mats_lo = (uint32_t)mats;
      P.mats_hi = (uint32_t)(mats >> 32);
      P.length = len;
      P.geo = C.lambda / (4.0f * 3.14159265358979f * len);
    }
    finish_key(A, kid, valid, ctr, C, &P);
  }
  count_add(ctr + kCtrValCasts, casts);
}

// next candidate per pending key: the smallest row above the one just tried
__global__ void next_reset_kernel(const uint32_t* __restrict__ list, int64_t n, KeyState K, Table T) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    T.next[K.slot[list[i]]] = kNone;
}

// Next candidate per pending key: the smallest row above the one just tried.
// Candidates of keys that are settled, or not above their key's current row,
// are never needed again, so the survivors are compacted for the next round.
__global__ void next_scan_kernel(const uint2* __restrict__ cand, int64_t n_cand, KeyState K,
                                 Table T, uint2* __restrict__ out, unsigned long long* ctr) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cand;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint2 e = cand[c];
    const uint32_t kid = T.kid[e.x];
    if (K.status[kid] != 0 || e.y <= K.cur[kid]) continue;
    atomicMin(T.next + e.x, e.y);
    out[warp_inc(ctr + kCtrCompact)] = e;
  }
}

__global__ void next_apply_kernel(const uint32_t* __restrict__ list, int64_t n, KeyState K,
                                  Table T, uint32_t* __restrict__ out_list, unsigned long long* ctr,
                                  int out_ctr) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t kid = list[i];
    const uint32_t nx = T.next[K.slot[kid]];
    if (nx == kNone) {
      K.status[kid] = 2;
    } else {
      K.cur[kid] = nx;
      out_list[warp_inc(ctr + out_ctr)] = kid;
    }
  }
}

__global__ void key_init_kernel(int64_t n_keys, KeyState K, Table T) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_keys;
       i += (int64_t)gridDim.x * blockDim.x) {
    K.cur[i] = T.minrow[K.slot[i]];
    K.tries[i] = 0;
    K.status[i] = 0;
  }
}

// ---------------------------------------------------------------- ordering
// Paths ordered by (rx, type, k, representative row): deterministic output.
__global__ void path_sortkey_kernel(const PathRec* __restrict__ p, int64_t n,
                                    uint64_t* __restrict__ key, uint32_t* __restrict__ idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t jtk = p[i].jtk;
    const uint64_t j = jtk & 0xFF, ty = (jtk >> 8) & 1, k = (jtk >> 9) & 7;
    key[i] = (j << 36) | (ty << 35) | (k << 32) | (uint64_t)p[i].rep;
    idx[i] = (uint32_t)i;
  }
}

// per-RX range of the sorted paths: lower bounds of (j << 36) and ((j+1) << 36)
__global__ void rx_range_kernel(const uint64_t* __restrict__ key, int64_t n, int n_rx,
                                unsigned long long* __restrict__ cnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_rx) return;
  auto lower = [&](uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (key[mid] < v) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  cnt[j] = (unsigned long long)(lower((uint64_t)(j + 1) << 36) - lower((uint64_t)j << 36));
}

// Launch order: rows (rays in ascending id) sorted along a Morton curve of
// their Fibonacci-lattice cell (z band, azimuth), so that the 32 rays of a
// warp leave in neighbouring directions.
__device__ __forceinline__ uint32_t spread2(uint32_t x) {
  x &= 0xFFFF;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

__global__ void order_key_kernel(const uint32_t* __restrict__ ray_of_row, int64_t n, int64_t n_rays,
                                 uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = ray_of_row ? ray_of_row[c] : (uint64_t)c;
    const uint32_t zb = (uint32_t)min((2 * r + 1) * 32768ull / (uint64_t)n_rays, 65535ull);
    const uint32_t pb = (uint32_t)((r * 0x61C8864680B583EBull) >> 48);
    key[c] = (uint64_t)(spread2(zb) | (spread2(pb) << 1));
    val[c] = (uint32_t)c;
  }
}

__global__ void path_gather_kernel(const PathRec* __restrict__ src, const uint32_t* __restrict__ idx,
                                   int64_t n, PathRec* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

// ---------------------------------------------------------------- field
__device__ __forceinline__ int path_mat(const PathRec& P, int m) {
  const uint64_t mats = (uint64_t)P.mats_lo | ((uint64_t)P.mats_hi << 32);
  return (int)((mats >> (8 * m)) & 0xFF);
}

// a = geo * prod_m f_m Gamma_m(theta_m): f = sqrt(1 - S^2) for a specular
// reflection (effective roughness), f = S for the diffuse last interaction.
__global__ void field_kernel(const PathRec* __restrict__ P, int64_t n, const float* __restrict__ mat,
                             float freq, int pol, float2* __restrict__ a_out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const PathRec p = P[i];
    const int k = (p.jtk >> 9) & 7;
    const int diffuse = (p.jtk >> 8) & 1;
    float2 a = make_float2(p.geo, 0.0f);
    for (int m = 0; m < k; ++m) {
      const int l = path_mat(p, m);
      const float2 eta = permittivity(mat[l], mat[256 + l], freq);
      const float2 G = fresnel(eta, p.cosv[m], pol);
      const float Sl = mat[512 + l];
      const float f = (diffuse && m == k - 1) ? Sl : sqrtf(fmaxf(0.0f, 1.0f - Sl * Sl));
      a = cmul(a, cscale(f, G));
    }
    a_out[i] = a;
  }
}

// per-RX power: one block per RX over its contiguous range, fixed-order tree
__global__ void power_kernel(const float2* __restrict__ a, const int64_t* __restrict__ start,
                             const int64_t* __restrict__ count, double* __restrict__ power) {
  __shared__ double sh[256];
  const int j = blockIdx.x;
  const int64_t b = start[j], n = count[j];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 v = a[b + i];
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) power[j] = sh[0];
}

// ---------------------------------------------------------------- adjoint
// d|a|^2/dx = 2 Re(conj(a) da/dx); da/deta_l sums over the interactions with
// label l of (prod of the other factors) * f_m * dGamma/deta; deta/deps_r = 1,
// deta/dsigma = -j/(2 pi f eps0); dR/dS = -S/R, d(S Gamma)/dS = Gamma.
constexpr int kAdjThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kAdjThreads / 32; ++i) t += sh[i];
  return t;
}

__global__ void __launch_bounds__(kAdjThreads)
    adjoint_kernel(const PathRec* __restrict__ P, int64_t n, const float* __restrict__ mat,
                   float freq, int pol, const float* __restrict__ dLdP, int n_labels,
                   double* __restrict__ partial) {
  __shared__ double sh[kAdjThreads / 32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int k = 0, labs[kMaxDepth];
  float ge[kMaxDepth], gs[kMaxDepth], gc[kMaxDepth];
  if (i < n) {
    const PathRec p = P[i];
    k = (p.jtk >> 9) & 7;
    const int diffuse = (p.jtk >> 8) & 1;
    const int j = p.jtk & 0xFF;
    float2 fac[kMaxDepth], dfe[kMaxDepth], dfs[kMaxDepth];
    for (int m = 0; m < k; ++m) {
      const int l = path_mat(p, m);
      labs[m] = l;
      const float2 eta = permittivity(mat[l], mat[256 + l], freq);
      const float2 G = fresnel(eta, p.cosv[m], pol);
      const float2 dG = dfresnel(eta, p.cosv[m], pol);
      const float Sl = mat[512 + l];
      const bool last_d = diffuse && m == k - 1;
      const float R = sqrtf(fmaxf(0.0f, 1.0f - Sl * Sl));
      const float c = last_d ? Sl : R;
      fac[m] = cscale(c, G);
      dfe[m] = cscale(c, dG);
      dfs[m] = last_d ? G : cscale(R > 0.0f ? -Sl / R : 0.0f, G);
    }
    float2 a = make_float2(p.geo, 0.0f);
    for (int m = 0; m < k; ++m) a = cmul(a, fac[m]);
    const float w = 2.0f * dLdP[j];
    const float ks = (float)(1.0 / (2.0 * 3.14159265358979323846 * kEps0)) / freq;
    for (int m = 0; m < k; ++m) {
      float2 oth = make_float2(p.geo, 0.0f);
      for (int q = 0; q < k; ++q)
        if (q != m) oth = cmul(oth, fac[q]);
      const float2 ca = cconj(a);
      const float2 de = cmul(ca, cmul(oth, dfe[m]));
      const float2 ds = cmul(ca, cmul(oth, dfs[m]));
      ge[m] = w * de.x;
      gs[m] = w * (de.y * ks);  // Re(z * (-j ks)) = ks * Im(z)
      gc[m] = w * ds.x;
    }
  }
  for (int l = 0; l < n_labels; ++l) {
    double ve = 0.0, vs = 0.0, vc = 0.0;
    for (int m = 0; m < k; ++m)
      if (labs[m] == l) {
        ve += ge[m];
        vs += gs[m];
        vc += gc[m];
      }
    const double te = block_sum(ve, sh);
    const double ts = block_sum(vs, sh);
    const double tc = block_sum(vc, sh);
    if (threadIdx.x == 0) {
      partial[((int64_t)blockIdx.x * 3 + 0) * n_labels + l] = te;
      partial[((int64_t)blockIdx.x * 3 + 1) * n_labels + l] = ts;
      partial[((int64_t)blockIdx.x * 3 + 2) * n_labels + l] = tc;
    }
  }
}

__global__ void adjoint_reduce_kernel(const double* __restrict__ partial, int64_t n_blocks,
                                      int n_labels, float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n_labels) return;
  double s = 0.0;
  for (int64_t b = 0; b < n_blocks; ++b) s += partial[b * 3 * n_labels + t];
  out[t] = (float)s;
}

inline int blocks_for(int64_t n, int threads, int sm, int per_sm = 16) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm * per_sm));
}

SimConst make_const(const nrt_result* r) {
  SimConst C;
  C.tx = make_float3(r->tx[0], r->tx[1], r->tx[2]);
  C.n_rx = r->n_rx;
  C.max_depth = r->p.max_depth;
  C.n_seg = r->n_seg;
  C.capture = r->p.capture;
  C.diffuse = r->p.diffuse;
  C.pol = r->p.pol;
  C.kappa = r->p.kappa;
  C.rep_tries = r->p.rep_tries;
  C.r_rx2 = r->p.r_rx * r->p.r_rx;
  C.t_min = r->p.t_min;
  C.cos_ta = cosf(r->p.t_a_deg * 3.14159265358979f / 180.0f);
  C.t_d = r->p.t_d;
  C.freq = r->p.freq;
  C.lambda = (float)(299792458.0 / (double)r->p.freq);
  C.n_rays = r->p.n_rays;
  C.vis_words = r->vis_words;
  return C;
}

}  // namespace

#define TRY(expr) NRT_CUDA_TRY(ctx, expr)

// Allocate and run a full simulation into r (scene, params, rx, rows set).
nrt_status run_trace(nrt_result* r, const uint32_t* subset_d) {
  nrt_scene* sc = r->scene;
  nrt_ctx* ctx = sc->ctx;
  cudaStream_t st = ctx->stream;
  const int sm = ctx->sm_count;
  const SceneView S = scene_view(sc);
  const int64_t n = r->n_traced;
  r->n_seg = r->p.max_depth + (r->p.capture == NRT_CAPTURE_SPHERE ? 1 : 0);
  r->vis_words = (sc->n_dps + 31) / 32;
  SimConst C = make_const(r);
  launch_counter() = 0;
  for (int e = 0; e < 8; ++e) TRY(cudaEventCreate(&r->ev[e]));
  TRY(cudaEventRecord(r->ev[0], st));

  TRY(cudaMallocAsync(&r->ctr, kCtrCount * sizeof(unsigned long long), st));
  TRY(cudaMemsetAsync(r->ctr, 0, kCtrCount * sizeof(unsigned long long), st));
  unsigned long long* ctr = r->ctr;
  const float margin = 0.8660254037844386f * sc->params.rho + sc->params.r_p;

  // visibility matrix
  if (r->p.capture == NRT_CAPTURE_VIS) {
    TRY(cudaMallocAsync(&r->vis, (size_t)r->n_rx * r->vis_words * 4, st));
    const int64_t total = (int64_t)r->n_rx * r->vis_words * 32;
    vis_kernel<<<blocks_for(total, kTraceThreads, sm), kTraceThreads, 0, st>>>(
        S, C, r->rx, sc->dps_recv, r->vis, ctr, margin); count_launch();
  }
  TRY(cudaEventRecord(r->ev[1], st));

  // hit records (rows of never-reached bounces read as misses)
  const size_t nrec = (size_t)r->n_seg * n;
  TRY(cudaMallocAsync(&r->rec_q, nrec * sizeof(float4), st));
  TRY(cudaMallocAsync(&r->rec_n, nrec * sizeof(float4), st));
  TRY(cudaMallocAsync(&r->rec_d, nrec * sizeof(float4), st));
  TRY(cudaMallocAsync(&r->rec_i, nrec * sizeof(int2), st));
  TRY(cudaMemsetAsync(r->rec_i, 0xFF, nrec * sizeof(int2), st));
  Records R{r->rec_q, r->rec_n, r->rec_d, r->rec_i, n};

  // launch order (cached for the full launch)
  const uint32_t* order = nullptr;
  uint32_t* order_tmp = nullptr;
  if (subset_d || ctx->order_n != n) {
    uint64_t *ok, *tk;
    uint32_t *ov, *tv;
    TRY(cudaMallocAsync(&ok, n * 8, st));
    TRY(cudaMallocAsync(&tk, n * 8, st));
    TRY(cudaMallocAsync(&ov, n * 4, st));
    TRY(cudaMallocAsync(&tv, n * 4, st));
    order_key_kernel<<<blocks_for(n, 256, sm), 256, 0, st>>>(subset_d, n, r->p.n_rays, ok, ov); count_launch();
    radix_sort_pairs(ok, ov, tk, tv, n, 32, st);
    cudaFreeAsync(ok, st);
    cudaFreeAsync(tk, st);
    cudaFreeAsync(tv, st);
    if (subset_d) {
      order_tmp = ov;
    } else {
      if (ctx->order) cudaFreeAsync(ctx->order, st);
      ctx->order = ov;
      ctx->order_n = n;
    }
  }
  order = subset_d ? order_tmp : ctx->order;

  // LOS paths are written after the candidate count fixes the path buffer;
  // the cast itself is cheap and done then.
  TRY(cudaEventRecord(r->ev[2], st));
  trace_kernel<<<blocks_for(n, kTraceThreads, sm), kTraceThreads, 0, st>>>(S, C, subset_d, order, R, ctr); count_launch();
  TRY(cudaEventRecord(r->ev[3], st));

  // candidate count per ray -> candidate offsets and table size
  EmitArgs A{};
  uint32_t *cand_cnt, *cand_off;
  TRY(cudaMallocAsync(&cand_cnt, n * 4, st));
  TRY(cudaMallocAsync(&cand_off, n * 4, st));
  A.cand_cnt = cand_cnt;
  emit_kernel<true><<<blocks_for(n, 256, sm), 256, 0, st>>>(S, C, r->rx, R, r->vis, order, A, ctr); count_launch();
  scan_exclusive(cand_cnt, cand_off, n, st);
  unsigned long long cnt2[2] = {0, 0};
  TRY(cudaMemcpyAsync(&cnt2[0], ctr + kCtrCands, 8, cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&cnt2[1], ctr + kCtrLeaders, 8, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  const unsigned long long n_cand_h = cnt2[0], n_lead_h = cnt2[1];
  if (r->p.cand_capacity > 0 && (int64_t)n_cand_h > r->p.cand_capacity) {
    ctx->last_error = "more path candidates than cand_capacity";
    return NRT_ERR_OVERFLOW;
  }
  if (n_cand_h >= 0xFFFFFFFFull) {
    ctx->last_error = "more than 2^32 path candidates";
    return NRT_ERR_OVERFLOW;
  }
  const int64_t cand_cap = std::max<int64_t>((int64_t)n_cand_h, 1);
  // distinct keys <= per-warp distinct keys (n_lead) <= candidates
  const int64_t key_bound = std::max<int64_t>((int64_t)n_lead_h, 1);
  int64_t cap = r->p.key_capacity;
  if (cap <= 0) {
    cap = 1 << 12;
    while (cap < key_bound + key_bound / 2) cap <<= 1;
  }
  if (cap & (cap - 1)) {
    ctx->last_error = "key_capacity must be a power of two";
    return NRT_ERR_ARG;
  }
  const int64_t key_cap = std::min<int64_t>(cap, key_bound);
  Table T{};
  KeyState K{};
  uint32_t *spec_list, *diff_list, *list2_s, *list2_d;
  uint2 *cand, *cand2;
  TRY(cudaMallocAsync(&T.fp, cap * 8, st));
  TRY(cudaMallocAsync(&T.hi, cap * 8, st));
  TRY(cudaMallocAsync(&T.lo, cap * 8, st));
  TRY(cudaMallocAsync(&T.minrow, cap * 4, st));
  TRY(cudaMallocAsync(&T.kid, cap * 4, st));
  TRY(cudaMallocAsync(&T.next, cap * 4, st));
  TRY(cudaMemsetAsync(T.fp, 0, cap * 8, st));
  TRY(cudaMemsetAsync(T.minrow, 0xFF, cap * 4, st));
  T.mask = (uint64_t)cap - 1;
  TRY(cudaMallocAsync(&K.slot, key_cap * 4, st));
  TRY(cudaMallocAsync(&K.cur, key_cap * 4, st));
  TRY(cudaMallocAsync(&K.tries, key_cap * 4, st));
  TRY(cudaMallocAsync(&K.status, key_cap * 4, st));
  TRY(cudaMallocAsync(&spec_list, key_cap * 4, st));
  TRY(cudaMallocAsync(&diff_list, key_cap * 4, st));
  TRY(cudaMallocAsync(&list2_s, key_cap * 4, st));
  TRY(cudaMallocAsync(&list2_d, key_cap * 4, st));
  TRY(cudaMallocAsync(&cand, cand_cap * sizeof(uint2), st));
  TRY(cudaMallocAsync(&cand2, cand_cap * sizeof(uint2), st));
  A.T = T;
  A.cand = cand;
  A.cand_off = cand_off;
  emit_kernel<false><<<blocks_for(n, 256, sm), 256, 0, st>>>(S, C, r->rx, R, r->vis, order, A, ctr); count_launch();
  cudaFreeAsync(cand_cnt, st);
  cudaFreeAsync(cand_off, st);

  // key ids from the occupied slots (specular first), in launch order of
  // each key's lowest row within each type
  uint32_t *fs, *fd, *os, *od, *pos = nullptr, *tv;
  uint64_t *sk0, *tk0;
  uint32_t* sv0;
  TRY(cudaMallocAsync(&fs, cap * 4, st));
  TRY(cudaMallocAsync(&fd, cap * 4, st));
  TRY(cudaMallocAsync(&os, cap * 4, st));
  TRY(cudaMallocAsync(&od, cap * 4, st));
  slot_flags_kernel<<<blocks_for(cap, 256, sm), 256, 0, st>>>(T, cap, fs, fd); count_launch();
  scan_exclusive(fs, os, cap, st);
  scan_exclusive(fd, od, cap, st);
  uint32_t tail[4];
  TRY(cudaMemcpyAsync(&tail[0], os + cap - 1, 4, cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&tail[1], fs + cap - 1, 4, cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&tail[2], od + cap - 1, 4, cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&tail[3], fd + cap - 1, 4, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  int64_t n_spec = (int64_t)tail[0] + tail[1];
  int64_t n_diff = (int64_t)tail[2] + tail[3];
  const int64_t n_keys = n_spec + n_diff;
  if (n_keys > key_cap) {
    ctx->last_error = "hash table holds more keys than its bound";
    return NRT_ERR_OVERFLOW;
  }
  TRY(cudaMemsetAsync(ctr + kCtrKeys, 0, 8, st));
  const unsigned long long nk_h = (unsigned long long)n_keys;
  TRY(cudaMemcpyAsync(ctr + kCtrKeys, &nk_h, 8, cudaMemcpyHostToDevice, st));
  TRY(cudaMallocAsync(&sk0, std::max<int64_t>(n_keys, 1) * 8, st));
  TRY(cudaMallocAsync(&tk0, std::max<int64_t>(n_keys, 1) * 8, st));
  TRY(cudaMallocAsync(&sv0, std::max<int64_t>(n_keys, 1) * 4, st));
  TRY(cudaMallocAsync(&tv, std::max<int64_t>(n_keys, 1) * 4, st));
  if (order) {
    TRY(cudaMallocAsync(&pos, n * 4, st));
    inverse_order_kernel<<<blocks_for(n, 256, sm), 256, 0, st>>>(order, n, pos); count_launch();
  }
  slot_assign_kernel<<<blocks_for(cap, 256, sm), 256, 0, st>>>(T, cap, fs, fd, os, od, (uint32_t)n_spec,
                                                               K.slot, sk0, sv0, pos); count_launch();
  if (n_spec > 1) radix_sort_pairs(sk0, sv0, tk0, tv, n_spec, 32, st);
  if (n_diff > 1) radix_sort_pairs(sk0 + n_spec, sv0 + n_spec, tk0, tv, n_diff, 32, st);
  if (n_spec) TRY(cudaMemcpyAsync(spec_list, sv0, n_spec * 4, cudaMemcpyDeviceToDevice, st));
  if (n_diff) TRY(cudaMemcpyAsync(diff_list, sv0 + n_spec, n_diff * 4, cudaMemcpyDeviceToDevice, st));
  cudaFreeAsync(fs, st);
  cudaFreeAsync(fd, st);
  cudaFreeAsync(os, st);
  cudaFreeAsync(od, st);
  cudaFreeAsync(sk0, st);
  cudaFreeAsync(tk0, st);
  cudaFreeAsync(sv0, st);
  cudaFreeAsync(tv, st);
  if (pos) cudaFreeAsync(pos, st);
  int64_t n_cand = (int64_t)n_cand_h;
  verify_kernel<<<blocks_for(n_cand, 256, sm), 256, 0, st>>>(S, C, R, T, cand, n_cand, ctr); count_launch();
  key_init_kernel<<<blocks_for(n_keys, 256, sm), 256, 0, st>>>(n_keys, K, T); count_launch();

  // path buffer: at most one path per key, plus LOS
  r->path_cap = n_keys + r->n_rx;
  PathRec* raw = nullptr;
  TRY(cudaMallocAsync(&raw, r->path_cap * sizeof(PathRec), st));
  los_kernel<<<(r->n_rx + kTraceThreads - 1) / kTraceThreads, kTraceThreads, 0, st>>>(
      S, C, r->rx, raw, ctr, r->path_cap); count_launch();
  TRY(cudaEventRecord(r->ev[4], st));

  // validation rounds: candidates in row (= ray id) order until one validates
  ValArgs V{};
  V.T = T;
  V.K = K;
  V.R = R;
  V.rx = r->rx;
  V.ray_of_row = subset_d;
  V.paths = raw;
  V.path_cap = r->path_cap;
  uint32_t *cur_s = spec_list, *cur_d = diff_list, *nxt_s = list2_s, *nxt_d = list2_d;
  uint2 *cand_cur = cand, *cand_nxt = cand2;
  for (int round = 0; round < r->p.rep_tries && (n_spec > 0 || n_diff > 0); ++round) {
    TRY(cudaMemsetAsync(ctr + kCtrKeysSpec, 0, 16, st));  // spec + diff next counters
    if (n_spec > 0) {
      V.next_list = nxt_s;
      V.next_ctr = kCtrKeysSpec;
      validate_specular_kernel<<<blocks_for(n_spec, kTraceThreads, sm), kTraceThreads, 0, st>>>(
          S, C, V, cur_s, n_spec, ctr); count_launch();
    }
    if (n_diff > 0) {
      V.next_list = nxt_d;
      V.next_ctr = kCtrKeysDiff;
      validate_diffuse_kernel<<<blocks_for(n_diff, kTraceThreads, sm), kTraceThreads, 0, st>>>(
          S, C, V, cur_d, n_diff, ctr); count_launch();
    }
    unsigned long long nn[2];
    TRY(cudaMemcpyAsync(nn, ctr + kCtrKeysSpec, 16, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    n_spec = (int64_t)nn[0];
    n_diff = (int64_t)nn[1];
    if (n_spec + n_diff == 0 || round + 1 >= r->p.rep_tries) break;
    // next candidate rows for the keys still pending
    if (n_spec) next_reset_kernel<<<blocks_for(n_spec, 256, sm), 256, 0, st>>>(nxt_s, n_spec, K, T); count_launch();
    if (n_diff) next_reset_kernel<<<blocks_for(n_diff, 256, sm), 256, 0, st>>>(nxt_d, n_diff, K, T); count_launch();
    TRY(cudaMemsetAsync(ctr + kCtrCompact, 0, 8, st));
    next_scan_kernel<<<blocks_for(n_cand, 256, sm), 256, 0, st>>>(cand_cur, n_cand, K, T, cand_nxt, ctr); count_launch();
    std::swap(cand_cur, cand_nxt);
    TRY(cudaMemsetAsync(ctr + kCtrKeysSpec, 0, 16, st));
    if (n_spec)
      next_apply_kernel<<<blocks_for(n_spec, 256, sm), 256, 0, st>>>(nxt_s, n_spec, K, T, cur_s, ctr,
                                                                    kCtrKeysSpec); count_launch();
    if (n_diff)
      next_apply_kernel<<<blocks_for(n_diff, 256, sm), 256, 0, st>>>(nxt_d, n_diff, K, T, cur_d, ctr,
                                                                    kCtrKeysDiff); count_launch();
    unsigned long long ncmp = 0;
    TRY(cudaMemcpyAsync(nn, ctr + kCtrKeysSpec, 16, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(&ncmp, ctr + kCtrCompact, 8, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    n_spec = (int64_t)nn[0];
    n_diff = (int64_t)nn[1];
    n_cand = (int64_t)ncmp;
  }
  TRY(cudaEventRecord(r->ev[5], st));

  // deterministic order of the paths, then the field
  unsigned long long hc[kCtrCount];
  TRY(cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  r->n_paths = std::min<int64_t>((int64_t)hc[kCtrPaths], r->path_cap);
  const int64_t np = r->n_paths;
  uint64_t *sk, *tk;
  uint32_t *si, *ti;
  TRY(cudaMallocAsync(&sk, std::max<int64_t>(np, 1) * 8, st));
  TRY(cudaMallocAsync(&tk, std::max<int64_t>(np, 1) * 8, st));
  TRY(cudaMallocAsync(&si, std::max<int64_t>(np, 1) * 4, st));
  TRY(cudaMallocAsync(&ti, std::max<int64_t>(np, 1) * 4, st));
  TRY(cudaMallocAsync(&r->paths, std::max<int64_t>(np, 1) * sizeof(PathRec), st));
  if (np > 0) {
    path_sortkey_kernel<<<blocks_for(np, 256, sm), 256, 0, st>>>(raw, np, sk, si); count_launch();
    radix_sort_pairs(sk, si, tk, ti, np, 44, st);
    path_gather_kernel<<<blocks_for(np, 256, sm), 256, 0, st>>>(raw, si, np, (PathRec*)r->paths); count_launch();
  }
  // per-RX ranges (paths are sorted by RX first)
  unsigned long long* rxc = nullptr;
  TRY(cudaMallocAsync(&rxc, r->n_rx * 8, st));
  TRY(cudaMemsetAsync(rxc, 0, r->n_rx * 8, st));
  if (np > 0) {
    rx_range_kernel<<<(r->n_rx + 63) / 64, 64, 0, st>>>(sk, np, r->n_rx, rxc); count_launch();
  }
  std::vector<unsigned long long> rxh(r->n_rx);
  TRY(cudaMemcpyAsync(rxh.data(), rxc, r->n_rx * 8, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  cudaFreeAsync(rxc, st);
  r->rx_count = new int64_t[r->n_rx]();
  r->rx_start = new int64_t[r->n_rx]();
  for (int j = 0; j < r->n_rx; ++j) r->rx_count[j] = (int64_t)rxh[j];
  for (int j = 1; j < r->n_rx; ++j) r->rx_start[j] = r->rx_start[j - 1] + r->rx_count[j - 1];
  cudaFreeAsync(sk, st);
  cudaFreeAsync(tk, st);
  cudaFreeAsync(si, st);
  cudaFreeAsync(ti, st);
  cudaFreeAsync(raw, st);
  cudaFreeAsync(T.fp, st);
  cudaFreeAsync(T.hi, st);
  cudaFreeAsync(T.lo, st);
  cudaFreeAsync(T.minrow, st);
  cudaFreeAsync(T.kid, st);
  cudaFreeAsync(T.next, st);
  cudaFreeAsync(K.slot, st);
  cudaFreeAsync(K.cur, st);
  cudaFreeAsync(K.tries, st);
  cudaFreeAsync(K.status, st);
  cudaFreeAsync(spec_list, st);
  cudaFreeAsync(diff_list, st);
  cudaFreeAsync(list2_s, st);
  cudaFreeAsync(list2_d, st);
  cudaFreeAsync(cand, st);
  cudaFreeAsync(cand2, st);
  if (order_tmp) cudaFreeAsync(order_tmp, st);
  TRY(cudaMallocAsync(&r->path_a, std::max<int64_t>(np, 1) * sizeof(float2), st));
  TRY(cudaMallocAsync(&r->power, r->n_rx * sizeof(double), st));
  nrt_status fst = run_field(r);
  if (fst != NRT_OK) return fst;
  TRY(cudaEventRecord(r->ev[6], st));
  TRY(cudaEventRecord(r->ev[7], st));
  TRY(cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  TRY(cudaGetLastError());
  nrt_counters& c = r->counters;
  c.rays = n;
  c.segments = (int64_t)hc[kCtrSegments];
  c.vis_casts = (int64_t)hc[kCtrVisCasts];
  c.los_casts = (int64_t)hc[kCtrLosCasts];
  c.validation_casts = (int64_t)hc[kCtrValCasts];
  c.candidates = (int64_t)hc[kCtrCands];
  c.keys = (int64_t)hc[kCtrKeys];
  c.paths = r->n_paths;
  c.n_dps = sc->n_dps;
  c.hash_probes_max = (int64_t)hc[kCtrProbeMax];
  c.error_flags = (int64_t)(hc[kCtrErr] & 0xFFFFFFFFull);
  c.kernel_launches = launch_counter();
  if (c.error_flags & (kErrHashFull | kErrCandFull | kErrPathFull | kErrKeyMismatch)) {
    ctx->last_error = "device buffer overflow or key fingerprint collision (flags " +
                      std::to_string(c.error_flags) + ")";
    return NRT_ERR_OVERFLOW;
  }
  if (c.error_flags & kErrStack) {
    ctx->last_error = "traversal stack overflow";
    return NRT_ERR_OVERFLOW;
  }
  return NRT_OK;
}

nrt_status run_field(nrt_result* r) {
  nrt_scene* sc = r->scene;
  nrt_ctx* ctx = sc->ctx;
  cudaStream_t st = ctx->stream;
  if (!sc->have_materials) {
    r->field_done = false;
    return NRT_OK;  // field computed once materials are set
  }
  const int64_t np = r->n_paths;
  if (np > 0)
    field_kernel<<<blocks_for(np, 256, ctx->sm_count), 256, 0, st>>>(
        (const PathRec*)r->paths, np, sc->mat, r->p.freq, r->p.pol, r->path_a); count_launch();
  int64_t *start_d, *count_d;
  TRY(cudaMallocAsync(&start_d, r->n_rx * 8, st));
  TRY(cudaMallocAsync(&count_d, r->n_rx * 8, st));
  TRY(cudaMemcpyAsync(start_d, r->rx_start, r->n_rx * 8, cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(count_d, r->rx_count, r->n_rx * 8, cudaMemcpyHostToDevice, st));
  power_kernel<<<r->n_rx, 256, 0, st>>>(r->path_a, start_d, count_d, r->power); count_launch();
  cudaFreeAsync(start_d, st);
  cudaFreeAsync(count_d, st);
  TRY(cudaGetLastError());
  r->field_done = true;
  return NRT_OK;
}

nrt_status run_backward(nrt_result* r, const float* dL_dP_h, float* g_eps, float* g_sig,
                        float* g_sca) {
  nrt_scene* sc = r->scene;
  nrt_ctx* ctx = sc->ctx;
  cudaStream_t st = ctx->stream;
  const int L = sc->n_labels;
  const int64_t np = r->n_paths;
  const int64_t nb = std::max<int64_t>(1, (np + kAdjThreads - 1) / kAdjThreads);
  float *dldp, *out;
  double* partial;
  TRY(cudaMallocAsync(&dldp, r->n_rx * 4, st));
  TRY(cudaMallocAsync(&out, 3 * L * 4, st));
  TRY(cudaMallocAsync(&partial, nb * 3 * L * 8, st));
  TRY(cudaMemcpyAsync(dldp, dL_dP_h, r->n_rx * 4, cudaMemcpyHostToDevice, st));
  TRY(cudaMemsetAsync(partial, 0, nb * 3 * L * 8, st));
  if (np > 0)
    adjoint_kernel<<<(unsigned)nb, kAdjThreads, 0, st>>>((const PathRec*)r->paths, np, sc->mat,
                                                         r->p.freq, r->p.pol, dldp, L, partial); count_launch();
  adjoint_reduce_kernel<<<(3 * L + 127) / 128, 128, 0, st>>>(partial, nb, L, out); count_launch();
  std::vector<float> h(3 * L);
  TRY(cudaMemcpyAsync(h.data(), out, 3 * L * 4, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  cudaFreeAsync(dldp, st);
  cudaFreeAsync(out, st);
  cudaFreeAsync(partial, st);
  for (int l = 0; l < L; ++l) {
    if (g_eps) g_eps[l] = h[l];
    if (g_sig) g_sig[l] = h[L + l];
    if (g_sca) g_sca[l] = h[2 * L + l];
  }
  TRY(cudaGetLastError());
  return NRT_OK;
}

}  // namespace nrt
