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

}  // namespace

// Debug builds (-DNRT_CHECK_BOUNDS): computed indices are range-checked; the
// first violation is recorded (kernel code << 48 | index) and the access
// skipped, so that an indexing fault shows up as a report, not a GPU fault.
struct DbgCaps {
  int64_t table, keys, cand, paths, rows, nrx;
};
#ifdef NRT_CHECK_BOUNDS
__device__ DbgCaps g_dbg_caps;
__device__ unsigned long long g_dbg_word;
#define NRT_GUARD(cond, code, val)                                                           \
  if (!(cond)) {                                                                             \
    atomicCAS(&g_dbg_word, 0ull,                                                             \
              ((unsigned long long)(code) << 48) | ((unsigned long long)(val)&0xFFFFFFFFFFFFull)); \
    continue;                                                                                \
  }
// record-only variant for warp-synchronous code: evaluates to cond
#define NRT_OK_IDX(cond, code, val)                                                            \
  ((cond) ? true                                                                             \
          : (atomicCAS(&g_dbg_word, 0ull,                                                    \
                       ((unsigned long long)(code) << 48) |                                  \
                           ((unsigned long long)(val)&0xFFFFFFFFFFFFull)),                   \
             false))
#else
#define NRT_GUARD(cond, code, val)
#define NRT_OK_IDX(cond, code, val) true
#endif

// Debug builds only: the capacities the guards compare against.
inline cudaError_t dbg_set_caps(int64_t table, int64_t keys, int64_t cand, int64_t paths,
                                int64_t rows, int64_t nrx, cudaStream_t st) {
#ifdef NRT_CHECK_BOUNDS
  DbgCaps dc{table, keys, cand, paths, rows, nrx};
  const unsigned long long zero = 0;
  cudaError_t e = cudaMemcpyToSymbolAsync(g_dbg_caps, &dc, sizeof(dc), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && table < 0)
    e = cudaMemcpyToSymbolAsync(g_dbg_word, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
  return e;
#else
  (void)table, (void)keys, (void)cand, (void)paths, (void)rows, (void)nrx, (void)st;
  return cudaSuccess;
#endif
}

namespace {

// One hash slot is the whole 128-bit key (16 bytes, two slots per 32-byte
// sector), claimed by one 128-bit compare-and-swap, so two distinct keys
// never share a slot.  All-ones is the empty key (no key has all three bits
// of its k field set), so one 0xFF fill initialises the table.  Key ids live
// in a separate array, kid[slot], written once the table is complete: the
// candidate pass reads 4 bytes per candidate from it instead of a bucket.
struct alignas(16) Key128 {
  unsigned long long hi, lo;
};
static_assert(sizeof(Key128) == 16, "Key128 layout");
__device__ __forceinline__ bool key_empty(uint64_t hi, uint64_t lo) {
  return hi == ~0ull && lo == ~0ull;
}

struct Table {
  Key128* b;      // [slot] key; all-ones = empty
  uint32_t* kid;  // [slot] key id of an occupied slot
  uint64_t mask;
};
// candidate slot of a key the full table could not take (tables hold at most
// 2^31 slots, so no slot index reaches it)
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;
constexpr int64_t kMaxTable = 1ll << 31;

struct KeyState {
  uint32_t* slot;    // [key] -> table slot
  uint32_t* cur;     // candidate row being validated
  uint32_t* pos;     // its position in the sorted candidate array
  uint32_t* end;     // end of the key's run in the sorted candidate array
  uint32_t* tries;   // candidates that failed (before the valid one)
  uint32_t* status;  // 0 pending, 1 valid, 2 invalid
};

// Candidates sorted once by (key id, row): a key's candidates form one run in
// ray order, so its next candidate is the next element of the run.
struct SortedCand {
  const uint64_t* key;  // (key id << row_bits) | row
  const unsigned long long* n_p;
  int64_t cap;
  int row_bits;
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
  int launch;  // NRT_LAUNCH_FIB or NRT_LAUNCH_DPS
  // batch mode: rows are grouped by pair (pair j owns rows pair_start[j] ..
  // pair_start[j+1]-1, a Fibonacci launch of pair_rays[j] rays from
  // tx_pair[j]); one shared physical RX; the RX field of a key holds j.
  int batch;
  int n_pairs;
  const float4* tx_pair;
  const uint32_t* pair_start;
  const int64_t* pair_rays;
};

__device__ __forceinline__ int pair_of_row(const SimConst& C, uint32_t row) {
  int lo = 0, hi = C.n_pairs;  // largest j with pair_start[j] <= row
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(C.pair_start + mid) <= row) lo = mid;
    else hi = mid;
  }
  return lo;
}

// TX of key/pair j (batch) or the simulation's TX
__device__ __forceinline__ float3 tx_of(const SimConst& C, int j) {
  return C.batch ? xyz(__ldg(C.tx_pair + j)) : C.tx;
}

__device__ __forceinline__ bool vis_bit(const uint32_t* vis, int64_t words, int j, int d) {
  return (__ldg(vis + (int64_t)j * words + (d >> 5)) >> (d & 31)) & 1u;
}

__device__ __forceinline__ void count_add(unsigned long long* c, unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(c, v);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Batch latency bookkeeping: lanes whose unit of work for pair `pj` ended
// (a traced ray, a validated key) subtract it from the pair's count, one
// atomic per pair and warp step; the lane that takes the count to zero
// stamps the pair's completion time.  All active lanes call it together.
__device__ __forceinline__ void pair_units_done(bool ended, int pj, unsigned long long* left,
                                                unsigned long long* stamp) {
  const unsigned act = __activemask();
  const unsigned em = __ballot_sync(act, ended);
  if (!ended) return;
  const unsigned peers = __match_any_sync(em, pj);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) {
    const unsigned long long n = (unsigned long long)__popc(peers);
    if (atomicAdd(left + pj, 0ull - n) == n) stamp[pj] = global_ns();
  }
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
__global__ void __launch_bounds__(kTraceThreads, 8)
    vis_kernel(SceneView S, SimConst C, const float4* __restrict__ rx,
               const float4* __restrict__ recv, uint32_t* __restrict__ vis,
               unsigned long long* ctr, float margin) {
  // 12 stack entries in shared memory (the rest in local memory): the
  // kernel's registers allow more blocks per SM than 27 entries would
  constexpr int kVisSmem = 12;
  __shared__ int stk[kVisSmem * kTraceThreads];
  __shared__ float tstk[kVisSmem * kTraceThreads];
  int* my_stk = stk + threadIdx.x;
  float* my_tstk = tstk + threadIdx.x;
  uint32_t* err = (uint32_t*)(ctr + kCtrErr);
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
          const Hit h = cast_ray<kVisSmem>(false, S, o, (1.0f / s) * v, -1, C.t_min, tmax, false,
                                           my_stk, my_tstk, kTraceThreads, err);
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
__global__ void __launch_bounds__(kTraceThreads, 8)
    los_kernel(SceneView S, SimConst C, const float4* __restrict__ rx, PathRec* __restrict__ paths,
               unsigned long long* ctr, int64_t path_cap) {
  NRT_STACK_DECL
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (C.batch ? C.n_pairs : C.n_rx)) return;
  const float3 r = xyz(rx[C.batch ? 0 : j]);
  const float3 txp = tx_of(C, j);
  const float3 v = r - txp;
  const float s = len3(v);
  const Hit h = cast_ray(true, S, txp, (1.0f / s) * v, -1, C.t_min, s, false, my_stk, my_tstk,
                               kTraceThreads, err);
  atomicAdd(ctr + kCtrLosCasts, 1ull);
  if (h.idx >= 0) return;
  const unsigned long long p = warp_inc(ctr + kCtrPaths);
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

// ---------------------------------------------------------------- diffraction
// Single-bounce edge diffraction (Sec. II-B-3): one thread per (edge, RX)
// (batch: per (edge, pair)).  The diffraction point is the exact minimiser
// of |TX - D| + |D - RX| on the edge line (unfold the half-planes through the
// edge into one plane; the straight line crosses the edge at
// t = (a_t b_r + a_r b_t) / (b_t + b_r), a the position along the edge, b the
// distance from it), kept strictly inside the segment with TX and RX
// outside the wedge; each end then casts toward D and must not hit anything
// closer than rho before it.  The geometry and the UTD wedge terms
// (Kouyoumjian-Pathak, Luebbers' weighting of the reflection-boundary terms)
// are evaluated in FP64: they are material independent, so they are stored
// once per path and the field kernel only applies the face reflection
// coefficients.  Record layout of a diffracted path: pts[0..2] = D,
// pts[3..8] = K (T1 + T2), K T3, K T4 (complex), pts[9..10] = the vector-model
// projections (v_s, v_h), cosv[0..1] = the face incidence cosines,
// mats = face 0 | face n << 8, rep = the edge index.
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zsc(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zexpj(double t) {
  double sn, cs;
  sincos(t, &sn, &cs);
  return make_double2(cs, sn);
}

// F(x) = j sqrt(pi x) e^{j(x - pi/4)} erfc(e^{j pi/4} sqrt x) (the UTD transition
// function): the power series of erf for x <= 20, the asymptotic series
// sum_n t_n, t_n = t_{n-1} j (2n - 1) / (2x), beyond (both ~1e-8 relative at
// the switch)
__device__ double2 utd_transition(double x) {
  if (!(x > 0.0)) return make_double2(0.0, 0.0);
  if (x > 20.0) {
    double2 sum = make_double2(1.0, 0.0), t = sum;
    for (int n = 1; n < 64; ++n) {
      const double2 nt = zmul(t, make_double2(0.0, (2.0 * n - 1.0) / (2.0 * x)));
      if (hypot(nt.x, nt.y) > hypot(t.x, t.y)) break;
      t = nt;
      sum = zadd(sum, t);
      if (hypot(t.x, t.y) < 1e-17) break;
    }
    return sum;
  }
  // erf(z) = 2/sqrt(pi) z sum_n (-z^2)^n / (n! (2n + 1)), z^2 = j x
  double2 c = make_double2(1.0, 0.0), acc = c;
  for (int n = 1; n < 200; ++n) {
    c = zsc(1.0 / n, zmul(c, make_double2(0.0, -x)));
    const double2 term = zsc(1.0 / (2.0 * n + 1.0), c);
    acc = zadd(acc, term);
    if (n > x && hypot(term.x, term.y) < 1e-17 * hypot(acc.x, acc.y)) break;
  }
  const double u = sqrt(x);
  const double2 z = zsc(u, make_double2(0.70710678118654752440, 0.70710678118654752440));
  const double2 erf_z = zsc(1.12837916709551257390, zmul(z, acc));  // 2 / sqrt(pi)
  const double2 erfc_z = make_double2(1.0 - erf_z.x, -erf_z.y);
  const double2 pre = zmul(make_double2(0.0, sqrt(3.14159265358979323846 * x)),
                           zexpj(x - 0.25 * 3.14159265358979323846));
  return zmul(pre, erfc_z);
}

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 d3(float3 v) { return {v.x, v.y, v.z}; }
__device__ __forceinline__ D3 d3(float4 v) { return {v.x, v.y, v.z}; }
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 dadd(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 dmul(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double ddot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double dlen(D3 a) { return sqrt(ddot(a, a)); }
__device__ __forceinline__ D3 dunit(D3 a) { return dmul(1.0 / dlen(a), a); }
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ D3 dtheta(D3 d) {  // theta^ about +z (x^ on the axis)
  const double h = sqrt(d.x * d.x + d.y * d.y);
  if (h < 1e-12) return {1.0, 0.0, 0.0};
  return {d.z * d.x / h, d.z * d.y / h, -h};
}

__global__ void __launch_bounds__(kTraceThreads)
    diffraction_kernel(SceneView S, SimConst C, const float4* __restrict__ rx,
                       const float4* __restrict__ edges, int64_t n_edges, PathRec* __restrict__ paths,
                       unsigned long long* ctr, int64_t path_cap) {
  NRT_STACK_DECL
  const double kPiD = 3.14159265358979323846;
  const int nj = C.batch ? C.n_pairs : C.n_rx;
  unsigned long long casts = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_edges * nj;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / nj;
    const int j = (int)(q - e * nj);
    const float4 ea = __ldg(edges + 4 * e), eb = __ldg(edges + 4 * e + 1);
    const D3 A = d3(ea), n0 = d3(__ldg(edges + 4 * e + 2)), n1 = d3(__ldg(edges + 4 * e + 3));
    const float3 txf = tx_of(C, j), rxf = xyz(__ldg(rx + (C.batch ? 0 : j)));
    const D3 T = d3(txf), R = d3(rxf);
    const D3 ev = dsub(d3(eb), A);
    const double len = dlen(ev);
    const D3 eu = dmul(1.0 / len, ev);
    const double at = ddot(dsub(T, A), eu), ar = ddot(dsub(R, A), eu);
    const double bt = dlen(dsub(dsub(T, A), dmul(at, eu))), br = dlen(dsub(dsub(R, A), dmul(ar, eu)));
    if (!(bt + br > 0.0)) continue;
    const double tp = (at * br + ar * bt) / (bt + br);
    if (!(tp > 0.0 && tp < len)) continue;
    const D3 D = dadd(A, dmul(tp, eu));
    if (!(fmax(ddot(dsub(T, D), n0), ddot(dsub(T, D), n1)) > 0.0)) continue;
    if (!(fmax(ddot(dsub(R, D), n0), ddot(dsub(R, D), n1)) > 0.0)) continue;
    const double s_in = dlen(dsub(D, T)), s_out = dlen(dsub(R, D));
    const D3 si = dmul(1.0 / s_in, dsub(D, T)), so = dmul(1.0 / s_out, dsub(R, D));
    const double cb = ddot(si, eu);
    const double sinb = sqrt(fmax(0.0, 1.0 - cb * cb));
    if (!(sinb > 0.0)) continue;
    // visibility of the edge point from the TX, then from the RX
    bool vis = true;
    const float3 Df = make_float3((float)D.x, (float)D.y, (float)D.z);
    const float3 ends[2] = {txf, rxf};
    const double dist[2] = {s_in, s_out};
    for (int t = 0; t < 2 && vis; ++t) {
      const float tmax = (float)(dist[t] - (double)S.rho);
      if (!(tmax > C.t_min)) continue;
      const Hit h = cast_ray(true, S, ends[t], unit3(Df - ends[t]), -1, C.t_min, tmax, false, my_stk,
                                   my_tstk, kTraceThreads, err);
      ++casts;
      vis = h.idx < 0;
    }
    if (!vis) continue;
    // wedge frame: t0 in face 0 pointing away from the edge; exterior angle n pi
    D3 t0 = dunit(dcross(n0, eu));
    if (ddot(t0, n1) > 0.0) t0 = dmul(-1.0, t0);
    D3 t1 = dunit(dcross(n1, eu));
    if (ddot(t1, n0) > 0.0) t1 = dmul(-1.0, t1);
    const double nw = 2.0 - acos(fmin(1.0, fmax(-1.0, ddot(t0, t1)))) / kPiD;
    auto angle = [&](D3 x) {
      const D3 v = dsub(x, D);
      const D3 vp = dsub(v, dmul(ddot(v, eu), eu));
      double ph = atan2(ddot(vp, n0), ddot(vp, t0));
      return ph < 0.0 ? ph + 2.0 * kPiD : ph;
    };
    const double phi_in = angle(T), phi_out = angle(R);
    const double k = 2.0 * kPiD * (double)C.freq / 299792458.0;
    const double L = s_in * s_out * sinb * sinb / (s_in + s_out);
    auto term = [&](double beta, int sgn) {  // cot((pi + sgn beta) / 2n) F(kL a^{sgn}(beta))
      const double N = rint((beta + sgn * kPiD) / (2.0 * kPiD * nw));
      const double c = cos((2.0 * kPiD * nw * N - beta) / 2.0);
      const double v = (kPiD + sgn * beta) / (2.0 * nw);
      return zsc(cos(v) / sin(v), utd_transition(k * L * 2.0 * c * c));
    };
    const double bm = phi_out - phi_in, bp = phi_out + phi_in;
    const double2 Kc = zsc(-1.0 / (2.0 * nw * sqrt(2.0 * kPiD * k) * sinb),
                           zexpj(-0.25 * kPiD));
    const double2 t12 = zmul(Kc, zadd(term(bm, +1), term(bm, -1)));
    const double2 t3 = zmul(Kc, term(bp, -1));
    const double2 t4 = zmul(Kc, term(bp, +1));
    // vector model: edge-fixed bases of the incident and diffracted rays
    const D3 fi = dmul(-1.0, dunit(dcross(eu, si))), bi = dcross(fi, si);
    const D3 fo = dunit(dcross(eu, so)), bo = dcross(fo, so);
    const D3 tht = dtheta(si), thr = dtheta(dmul(-1.0, so));
    const unsigned long long p = warp_inc(ctr + kCtrPaths);
    if ((int64_t)p >= path_cap) {
      atomicOr(err, kErrPathFull);
      continue;
    }
    PathRec P;
    memset(&P, 0, sizeof(P));
    P.hi = ((uint64_t)(j & 0xFF) << 56) | (1ull << 52) | (1ull << 51);
    P.lo = (uint64_t)e;
    P.rep = (uint32_t)e;
    P.jtk = (uint32_t)j | (1u << 9) | (1u << 12);
    P.length = (float)(s_in + s_out);
    P.geo = (float)(((double)C.lambda) / (4.0 * kPiD * sqrt(s_in * s_out * (s_in + s_out))));
    P.cosv[0] = (float)(sinb * sin(phi_in));
    P.cosv[1] = (float)(sinb * sin(nw * kPiD - phi_out));
    P.mats_lo = (uint32_t)(__float_as_int(ea.w) & 0xFF) | ((uint32_t)(__float_as_int(eb.w) & 0xFF) << 8);
    P.pts[0] = Df.x;
    P.pts[1] = Df.y;
    P.pts[2] = Df.z;
    P.pts[3] = (float)t12.x;
    P.pts[4] = (float)t12.y;
    P.pts[5] = (float)t3.x;
    P.pts[6] = (float)t3.y;
    P.pts[7] = (float)t4.x;
    P.pts[8] = (float)t4.y;
    P.pts[9] = (float)(-ddot(thr, bo) * ddot(tht, bi));
    P.pts[10] = (float)(-ddot(thr, fo) * ddot(tht, fi));
    paths[p] = P;
  }
  count_add(ctr + kCtrDfrCasts, casts);
}

// ---------------------------------------------------------------- trace
// One ray per thread; every interaction continues as a specular reflection
// (Sec. II-B: the ray count stays constant).  The next cast skips the DPS
// just hit.
__device__ __forceinline__ unsigned trace_row(const SceneView& S, const SimConst& C,
                                              const uint32_t* __restrict__ ray_of_row,
                                              const Records& R, int64_t row, int* stk, float* tstk,
                                              uint32_t* err);

__device__ __forceinline__ void ray_start(const SceneView& S, const SimConst& C,
                                          const uint32_t* __restrict__ ray_of_row, int64_t row,
                                          float3* o, float3* d);

// Every interaction continues as a specular reflection (Sec. II-B: the ray
// count stays constant); the next cast skips the DPS just hit.  Scheduling:
// one loop step is one bounce of the lane's current ray; a lane whose ray
// has ended (a miss or the last segment) takes the next ray of the launch
// order from a counter (one warp-aggregated atomic per fetch), so rays that
// escape early do not leave their lanes idle while the warp's longest ray
// finishes.  Each ray's casts are those of a ray-at-a-time loop.
// Batches: pair_left[j] counts pair j's rays still in flight (set before the
// launch); the lane that ends its last ray stamps pair_done[j].
__global__ void __launch_bounds__(kTraceThreads, 8)
    trace_kernel(SceneView S, SimConst C, const uint32_t* __restrict__ ray_of_row,
                 const uint32_t* __restrict__ order, Records R, unsigned long long* __restrict__ fetch,
                 unsigned long long* ctr, unsigned long long* pair_left,
                 unsigned long long* pair_done) {
  NRT_STACK_DECL
  unsigned long long segs = 0;
  const int lane = threadIdx.x & 31;
  bool have = false;
  int64_t row = 0;
  float3 o = C.tx, d = C.tx;
  int skip = -1, seg = 0;
  for (;;) {
    if (!have) {
      const unsigned mask = __activemask();
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(fetch, (unsigned long long)__popc(mask));
      base = __shfl_sync(mask, base, leader);
      const int64_t t = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
      if (t >= R.n_rows) break;
      row = order ? order[t] : t;
      NRT_GUARD(row >= 0 && row < g_dbg_caps.rows, 25, row)
      ray_start(S, C, ray_of_row, row, &o, &d);
      skip = -1;
      seg = 0;
      have = true;
    }
    const Hit h = cast_ray(false, S, o, d, skip, C.t_min, __int_as_float(0x7f800000), true, my_stk,
                                  my_tstk, kTraceThreads, err);
    ++segs;
    const int64_t a = R.at(seg, row);
    bool ended = true;
    if (h.idx < 0) {
      R.i[a] = make_int2(-1, 0);
    } else {
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
      ended = ++seg >= C.n_seg;
    }
    if (pair_left) pair_units_done(ended, pair_of_row(C, (uint32_t)row), pair_left, pair_done);
    have = !ended;
  }
  count_add(ctr + kCtrSegments, segs);
}

// ---------------------------------------------------------------- candidates
struct EmitArgs {
  Table T;
  uint64_t cand_cap;
  uint2* cand;              // candidates (slot, row) at per-ray offsets, rows ascending
  const uint32_t* cand_off; // [row] first candidate of the ray
  uint32_t* cand_cnt;       // [row] candidates of the ray (count pass)
  const uint32_t* key_status;  // label pass: validation status per key id
  uint8_t* labels;             // label pass: [row] member of a valid specular key
};

enum { kModeEmit = 0, kModeCount = 1, kModeLabel = 2 };

// Slot of an existing key, or ~0 (label pass; the table is complete).
__device__ __forceinline__ uint64_t find_key(const EmitArgs& A, uint64_t hi, uint64_t lo,
                                             uint64_t f) {
  uint64_t slot = f & A.T.mask;
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    const Key128 g = A.T.b[slot];
    if (key_empty(g.hi, g.lo)) return ~0ull;
    if (g.hi == hi && g.lo == lo) return slot;
    slot = (slot + 1) & A.T.mask;
  }
  return ~0ull;
}

// Hash insert by one lane on behalf of the lanes holding the same key;
// returns the slot.  The probe sequence starts at the key's hash f; a slot
// is claimed, or found to hold the key already, by one 128-bit
// compare-and-swap.  No shared counters are touched: key ids are assigned
// afterwards from the table's occupancy.
__device__ __forceinline__ uint64_t insert_key(const EmitArgs& A, uint64_t hi, uint64_t lo,
                                               uint64_t f, unsigned long long* ctr) {
  uint64_t slot = f & A.T.mask;
  const Key128 empty{~0ull, ~0ull}, mine{hi, lo};
  int probe = 0;
  for (; probe < kMaxProbe; ++probe) {
    const Key128 prev = atomicCAS(&A.T.b[slot], empty, mine);
    if (key_empty(prev.hi, prev.lo) || (prev.hi == hi && prev.lo == lo)) break;
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
// key; every lane still stores its own (slot, row) candidate, at its ray's
// next candidate position.  The count
// mode only counts candidates per ray and per-warp distinct keys (an upper
// bound on the table's keys); the label mode sets n_mine to 1 when the key
// is a validated specular key.
template <int kMode>
__device__ __forceinline__ void warp_emit(const EmitArgs& A, bool pred, uint64_t hi, uint64_t lo,
                                          uint32_t row, unsigned long long* ctr, uint32_t& n_mine,
                                          unsigned long long& n_lead) {
  const unsigned act = __ballot_sync(0xFFFFFFFFu, pred);
  if (!act || !pred) return;
  const int lane = threadIdx.x & 31;
  const uint64_t f = key_hash(hi, lo);
  if (kMode == kModeLabel) {
    if ((hi >> 55) & 1ull) return;  // specular keys only
    const uint64_t slot = find_key(A, hi, lo, f);
    if (slot != ~0ull && A.key_status[A.T.kid[slot]] == 1u) n_mine = 1u;
    return;
  }
  const unsigned peers = __match_any_sync(act, hi) & __match_any_sync(act, lo);  // equal keys
  const int leader = __ffs(peers) - 1;
  if (kMode == kModeCount) {
    ++n_mine;
    if (lane == leader) ++n_lead;
    return;
  }
  uint64_t slot = 0;
  if (lane == leader) slot = insert_key(A, hi, lo, f, ctr);
  slot = __shfl_sync(peers, slot, leader);
  // a full table (flagged by insert_key) still fills the position the count
  // pass reserved, with slot kNoSlot, so that no candidate entry below the
  // count is left unwritten; cand_key_kernel gives it no key
  const uint32_t s32 = slot == ~0ull ? kNoSlot : (uint32_t)slot;
  if (n_mine < A.cand_cap) A.cand[n_mine] = make_uint2(s32, row);
  else atomicOr((uint32_t*)(ctr + kCtrErr), kErrCandFull);
  ++n_mine;
}

// Candidates of every ray (Sec. II-B): a warp walks 32 rays in launch order
// (neighbouring directions), bounce by bounce and RX by RX in lockstep, so
// that rays that found the same key merge before touching the hash table.
template <int kMode>
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
    bool active = t < R.n_rows;
    uint32_t row = active ? (order ? order[t] : (uint32_t)t) : 0u;
    if (active && !NRT_OK_IDX(row < g_dbg_caps.rows, 26, row)) {
      active = false;
      row = 0u;
    }
    uint32_t n_mine = (kMode == kModeEmit && active) ? A.cand_off[row] : 0u;
    const int pair_j = (C.batch && active) ? pair_of_row(C, row) : 0;
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
        const int n_j = C.batch ? 1 : C.n_rx;
        for (int jv = 0; jv < n_j; ++jv) {
          const bool v = alive && vis_bit(vis, C.vis_words, jv, dps);
          const int j = C.batch ? pair_j : jv;
          uint64_t hi = 0, lo = 0;
          if (v) make_key(j, 0, k, lab, vox, &hi, &lo);
          warp_emit<kMode>(A, v, hi, lo, row, ctr, n_mine, n_lead);
          if (C.diffuse) {
            if (v) make_key(j, 1, k, lab, vox, &hi, &lo);
            warp_emit<kMode>(A, v, hi, lo, row, ctr, n_mine, n_lead);
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
          warp_emit<kMode>(A, v, hi, lo, row, ctr, n_mine, n_lead);
        }
      }
    }
    if (kMode == kModeLabel && active) A.labels[row] = (uint8_t)n_mine;
    if (kMode == kModeCount && active) {
      A.cand_cnt[row] = n_mine;
      n_total += n_mine;
    }
  }
  if (kMode == kModeCount) {
    count_add(ctr + kCtrCands, n_total);
    count_add(ctr + kCtrLeaders, n_lead);
  }
}

// Key ids from the table's occupancy: specular keys first, then diffuse,
// each in slot order.  The table is cut into tiles of kSlotTile slots, one
// block each; thread t of a block owns the kSlotPer consecutive slots from
// t * kSlotPer.  A first pass counts each tile's keys of both types, the
// tile counts are scanned, and the assigning pass ranks the slots inside
// its tile with a block-wide scan -- no per-slot flag or offset arrays.
constexpr int kSlotThreads = 256;
constexpr int kSlotPer = 16;
constexpr int kSlotTile = kSlotThreads * kSlotPer;

// occupancy masks of the calling thread's slots (bit r: slot first + r)
__device__ __forceinline__ void slot_masks(const Table& T, int64_t cap, int64_t first,
                                           uint32_t* ms, uint32_t* md) {
  uint32_t s = 0, d = 0;
  for (int r = 0; r < kSlotPer; ++r) {
    const int64_t i = first + r;
    if (i >= cap) break;
    const Key128 g = T.b[i];
    if (key_empty(g.hi, g.lo)) continue;
    if ((g.hi >> 55) & 1ull) d |= 1u << r;
    else s |= 1u << r;
  }
  *ms = s;
  *md = d;
}

// Exclusive block-wide prefix of v (two 16-bit counts packed in one word:
// a tile holds at most kSlotTile = 4096 keys of each type) and the block
// total.  All kSlotThreads threads call it.
__device__ __forceinline__ uint32_t block_prefix(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sum[kSlotThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
  uint32_t before = 0, all = 0;
  for (int k = 0; k < kSlotThreads / 32; ++k) {
    if (k < w) before += warp_sum[k];
    all += warp_sum[k];
  }
  __syncthreads();  // warp_sum may be reused by a later call
  *total = all;
  return before + x - v;
}

__global__ void __launch_bounds__(kSlotThreads)
    slot_count_kernel(Table T, int64_t cap, uint32_t* __restrict__ tile_s,
                      uint32_t* __restrict__ tile_d) {
  const int64_t first = (int64_t)blockIdx.x * kSlotTile + (int64_t)threadIdx.x * kSlotPer;
  uint32_t ms, md, total;
  slot_masks(T, cap, first, &ms, &md);
  block_prefix((uint32_t)__popc(ms) | ((uint32_t)__popc(md) << 16), &total);
  if (threadIdx.x == 0) {
    tile_s[blockIdx.x] = total & 0xFFFFu;
    tile_d[blockIdx.x] = total >> 16;
  }
}

// 10 bits per axis interleaved (x lowest)
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
  x &= 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__global__ void __launch_bounds__(kSlotThreads)
    slot_assign_kernel(Table T, int64_t cap, const uint32_t* __restrict__ tile_os,
                       const uint32_t* __restrict__ tile_od,
                       const unsigned long long* __restrict__ counts,
                       uint32_t* __restrict__ key_slot, int64_t key_cap) {
  const uint32_t n_spec = (uint32_t)counts[0];  // diffuse ids follow the specular ones
  const int64_t first = (int64_t)blockIdx.x * kSlotTile + (int64_t)threadIdx.x * kSlotPer;
  uint32_t ms, md, total;
  slot_masks(T, cap, first, &ms, &md);
  const uint32_t pre =
      block_prefix((uint32_t)__popc(ms) | ((uint32_t)__popc(md) << 16), &total);
  uint32_t next_s = tile_os[blockIdx.x] + (pre & 0xFFFFu);
  uint32_t next_d = n_spec + tile_od[blockIdx.x] + (pre >> 16);
  for (int r = 0; r < kSlotPer; ++r) {
    const bool spec = (ms >> r) & 1u, diff = (md >> r) & 1u;
    if (!spec && !diff) continue;
    const int64_t i = first + r;
    const uint32_t kid = spec ? next_s++ : next_d++;
    T.kid[i] = kid;  // ids at or past key_cap: keys over capacity, reported by key_count
    if ((int64_t)kid < key_cap) key_slot[kid] = (uint32_t)i;
  }
}

// Validation order of a key: type, the coarse Morton code of the voxel of its
// lowest row's last interaction point (the lowest row is the first
// candidate of the key's run), the RX (pair), then the fine Morton code (the
// low fb bits).  Diffuse keys take fb = 0 (voxel, then RX): a
// warp's shadow casts leave one voxel toward the receivers, so the region's
// BVH nodes and discs are read once for all receivers.  Specular keys take
// cells of 16 voxels per axis (fb = 12), then the RX: a warp's image-method
// legs run from one region toward one receiver and share the nodes along the
// way.  Measured on the office simulation, validation time: 15.1 ms with
// fb = 0 for both, 14.3 ms with 12 for both, 14.0 ms with 12 / 0 (specular
// flat from 9 to 15; RX-first order, fb = mb, 15.4 ms).  The fields are
// packed tight (jb bits of RX, mb = 3 x grid bits of Morton code, one type
// bit) so that the sort takes as few 8-bit passes as the scene needs.
// Batches also count each pair's keys into pair_keys (NULL otherwise).
__global__ void val_order_kernel(SceneView S, Records R, Table T, KeyState K,
                                 const unsigned long long* __restrict__ counts,
                                 uint64_t* __restrict__ sort_key, uint32_t* __restrict__ sort_val,
                                 int jb, int mb, int fb_spec, unsigned long long* pair_keys) {
  const int64_t n_keys = (int64_t)counts[2];
  for (int64_t kid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; kid < n_keys;
       kid += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t slot = K.slot[kid];
    NRT_GUARD(slot < g_dbg_caps.table, 2, slot)
    const uint32_t m = K.cur[kid];  // lowest row: the first candidate of the key's run
    NRT_GUARD(m < g_dbg_caps.rows, 27, m)
    const uint64_t hi = T.b[slot].hi;
    const bool spec = !((hi >> 55) & 1ull);
    const int k = (int)((hi >> 52) & 7);
    int vox[3] = {0, 0, 0};
    if (k >= 1) voxel_of(S, xyz(R.q[R.at(k - 1, m)]), vox);
    const int vmax = (1 << (mb / 3)) - 1;  // Morton fields stay inside their mb bits
    const uint32_t mort = spread3((uint32_t)min(max(vox[0], 0), vmax)) |
                          (spread3((uint32_t)min(max(vox[1], 0), vmax)) << 1) |
                          (spread3((uint32_t)min(max(vox[2], 0), vmax)) << 2);
    const int fb = spec ? fb_spec : 0;
    const uint64_t fine = (uint64_t)mort & ((1ull << fb) - 1ull);
    sort_key[kid] = ((uint64_t)(spec ? 0u : 1u) << (jb + mb)) | ((uint64_t)(mort >> fb) << (jb + fb)) |
                    ((hi >> 56) << fb) | fine;
    sort_val[kid] = (uint32_t)kid;
    if (pair_keys) atomicAdd(pair_keys + (hi >> 56), 1ull);
  }
}

// key counts from the tile-count scan tails: [0] specular, [1] diffuse, [2]
// all, clamped to the key capacity.  More keys than that (possible only
// when the capacity was fixed ahead of the trace, as for a recorded graph)
// raise kErrKeyFull; keys with ids at or past the capacity are left out.
__global__ void key_count_kernel(const uint32_t* __restrict__ fs, const uint32_t* __restrict__ fd,
                                 const uint32_t* __restrict__ os, const uint32_t* __restrict__ od,
                                 int64_t n, int64_t key_cap, unsigned long long* __restrict__ out,
                                 unsigned long long* __restrict__ ctr) {
  const unsigned long long ns = (unsigned long long)os[n - 1] + fs[n - 1];
  const unsigned long long nd = (unsigned long long)od[n - 1] + fd[n - 1];
  const unsigned long long cap = (unsigned long long)key_cap;
  if (ns + nd > cap) atomicOr((uint32_t*)(ctr + kCtrErr), kErrKeyFull);
  const unsigned long long ns_c = ns < cap ? ns : cap;
  const unsigned long long all = ns + nd < cap ? ns + nd : cap;
  out[0] = ns_c;
  out[1] = all - ns_c;
  out[2] = all;
}

// keys sorted by (type, launch position): specular ids first, then diffuse
__global__ void split_lists_kernel(const uint32_t* __restrict__ sorted, int64_t cap,
                                   const unsigned long long* __restrict__ counts,
                                   uint32_t* __restrict__ spec, uint32_t* __restrict__ diff) {
  const int64_t ns = (int64_t)counts[0], nk = (int64_t)counts[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < min(nk, cap);
       i += (int64_t)gridDim.x * blockDim.x) {
    NRT_GUARD(sorted[i] < g_dbg_caps.keys, 3, sorted[i])
    if (i < ns) spec[i] = sorted[i];
    else diff[i - ns] = sorted[i];
  }
}

// Candidates (slot, row) -> sort keys (key id << row_bits) | row, in place:
// sorting on the key id takes ceil(log2(keys)) bits instead of the table's.
__global__ void cand_key_kernel(Table T, uint2* cand, const unsigned long long* __restrict__ n_cand_p,
                                int64_t cap, int row_bits, int64_t key_cap) {
  const int64_t n_cand = min((int64_t)*n_cand_p, cap);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cand;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint2 e = cand[c];
    NRT_GUARD(e.x == kNoSlot || e.x < g_dbg_caps.table, 21, e.x)
    NRT_GUARD(e.y < g_dbg_caps.rows, 22, e.y)
    // a key over capacity (or a candidate the full table could not take)
    // gets all ones: its id field sorts after every id below key_cap
    // (2^kid_bits > key_cap) and matches none of them
    const uint32_t kid = (uint64_t)e.x <= T.mask ? T.kid[e.x] : 0xFFFFFFFFu;
    reinterpret_cast<uint64_t*>(cand)[c] =
        (int64_t)kid < key_cap ? ((uint64_t)kid << row_bits) | (uint64_t)e.y : ~0ull;
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
  SortedCand SC;  // each key's candidates, one run per slot in ray order
  unsigned long long* pair_keys;   // batches: keys of pair j still being validated
  unsigned long long* pair_ready;  // batches: pair j's last key finished (stamp)
};

// Outcome of one try of key kid (candidate row *row at position *pos of the
// sorted candidates): a valid path is recorded; otherwise the key moves to
// its next candidate -- the next element of its run, i.e. the next larger
// ray id -- unless it has no candidate left or used rep_tries (> 0) tries.
// Returns true when the key is finished.
__device__ __forceinline__ bool key_try(const ValArgs& A, uint32_t kid, bool valid,
                                        const PathRec* rec, uint32_t* row, uint32_t* pos,
                                        unsigned long long* ctr, const SimConst& C) {
  uint32_t* err = (uint32_t*)(ctr + kCtrErr);
  if (valid) {
    A.K.status[kid] = 1;
    const unsigned long long p = warp_inc(ctr + kCtrPaths);
    if ((int64_t)p >= A.path_cap) {
      atomicOr(err, kErrPathFull);
      return true;
    }
    A.paths[p] = *rec;
    return true;
  }
  const uint32_t tr = A.K.tries[kid] + 1;
  A.K.tries[kid] = tr;
  if (C.rep_tries > 0 && (int)tr >= C.rep_tries) {
    A.K.status[kid] = 2;
    return true;
  }
  const int64_t n_cand = min((int64_t)*A.SC.n_p, A.SC.cap);
  const int64_t q = (int64_t)*pos + 1;
  const uint64_t e = q < n_cand ? A.SC.key[q] : ~0ull;
  if (q >= n_cand || (e >> A.SC.row_bits) != (uint64_t)kid) {
    A.K.status[kid] = 2;
    return true;
  }
  *row = (uint32_t)(e & ((1ull << A.SC.row_bits) - 1ull));
  *pos = (uint32_t)q;
  A.K.cur[kid] = *row;
  A.K.pos[kid] = *pos;
  return false;
}

// next key of a list for the calling lane (one warp-aggregated atomic per
// fetch); returns its position or -1 when the list is exhausted
__device__ __forceinline__ int64_t fetch_next(unsigned long long* fetch, int64_t n) {
  const int lane = threadIdx.x & 31;
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(fetch, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  const int64_t i = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
  return i < n ? i : -1;
}

// Diffuse: the candidate's own interaction points; the last one scatters
// toward the RX if the RX is in front of the surface and a cast from the
// scatter point (skipping its DPS) reaches the RX unobstructed (Sec. II-B-1).
// One loop step is one try (one shadow cast); a lane walks its key's
// candidates in ray order and takes the next key of the list when the key is
// finished.
__global__ void __launch_bounds__(kTraceThreads, 6)
    validate_diffuse_kernel(SceneView S, SimConst C, ValArgs A, const uint32_t* __restrict__ list,
                            const unsigned long long* __restrict__ n_list_p,
                            unsigned long long* __restrict__ fetch, unsigned long long* ctr) {
  NRT_STACK_DECL
  unsigned long long casts = 0;
  const int64_t n_list = (int64_t)*n_list_p;
  bool have = false;
  uint32_t kid = 0, slot = 0, row = 0, pos = 0;
  for (;;) {
    if (!have) {
      const int64_t i = fetch_next(fetch, n_list);
      if (i < 0) break;
      kid = list[i];
      NRT_GUARD(kid < g_dbg_caps.keys, 5, kid)
      slot = A.K.slot[kid];
      NRT_GUARD(slot < g_dbg_caps.table, 6, slot)
      row = A.K.cur[kid];
      pos = A.K.pos[kid];
      have = true;
    }
    NRT_GUARD(row < g_dbg_caps.rows, 7, row)
    const uint64_t hi = A.T.b[slot].hi;
    const int j = (int)(hi >> 56);
    const int k = (int)((hi >> 52) & 7);
    NRT_GUARD(k >= 1 && k <= C.max_depth, 8, k)
    const int64_t a = A.R.at(k - 1, row);
    const float4 qq = A.R.q[a], nn = A.R.n[a];
    const float3 q = xyz(qq), n = xyz(nn);
    const int dps = __float_as_int(A.R.d[a].w);
    const float3 u = xyz(A.rx[C.batch ? 0 : j]) - q;
    const float rs = len3(u);
    const float3 w = (1.0f / rs) * u;
    const float cs = dot3(n, w);
    bool valid = false;
    PathRec P;
    if (cs > 0.0f) {
      const Hit h = cast_ray(true, S, q, w, dps, C.t_min, rs, false, my_stk, my_tstk,
                                   kTraceThreads, err);
      ++casts;
      valid = h.idx < 0;
    }
    if (valid) {
      memset(&P, 0, sizeof(P));
      P.hi = hi;
      P.lo = A.T.b[slot].lo;
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
      P.nd[0] = n.x;
      P.nd[1] = n.y;
      P.nd[2] = n.z;
      const float ci = nn.w;
      const float rho = S.rho;
      P.geo = C.lambda / (4.0f * 3.14159265358979f) *
              sqrtf(rho * rho * ci * cs / 3.14159265358979f) / (ri * rs);
      P.length = ri + rs;
    }
    const bool fin = key_try(A, kid, valid, &P, &row, &pos, ctr, C);
    if (A.pair_keys) pair_units_done(fin, j, A.pair_keys, A.pair_ready);
    if (fin) have = false;
  }
  count_add(ctr + kCtrValCasts, casts);
  count_add(ctr + kCtrDiffCasts, casts);
}

// Specular (Sec. II-B-2), one candidate: phase 1 solves Eq. 1 on the
// infinite planes (q_m, n_m) of the candidate's interactions; its minimiser
// with every reflection on the correct side of its plane is the image-method
// path (mirror the TX through the planes, back-trace from the RX).  Phase 2
// casts I_{m-1} -> I_m and accepts the interaction when the hit is on the
// key's surface, its normal within t_a of the plane normal and the hit within
// t_d of the plane; otherwise that plane is replaced by the hit's and the
// solve retried (at most kappa times).  A hit on another surface, a miss or
// a failed side check ends the candidate.  Finally I_k -> RX must be clear.
// Coordinates are taken relative to the RX to keep float magnitudes small.
// Returns whether the candidate validates; with P, its path record.  Used by
// the item pass and by the per-key finish, so both take the same decisions.
// best (the item pass): the key's lowest valid rank so far; once it drops
// below this candidate's rank the candidate cannot be the key's path, so it
// stops before its next cast (exact: only the lowest valid rank is kept).
// stage at which a candidate ended (counters): before any cast, at its
// first leg's cast, later (or valid)
enum : int { kSpecNoCast = 0, kSpecLeg1 = 1, kSpecLater = 2 };

// Image-method points of one attempt (Eq. 1), relative to the RX: I[0] the
// TX (txl), I[k + 1] the RX (the origin), I[1..k] on the planes (Pp, Pn)
// found backwards from the RX through the mirrored TX images; false when a
// leg is parallel to its plane or a point's neighbours lie on opposite
// sides of its plane (no specular reflection there).  Shared by every
// refinement path so that all take the same decisions.
__device__ __forceinline__ bool spec_points(float3 txl, const float3* Pp, const float3* Pn, int k,
                                            float3* I) {
  float3 img[kMaxDepth + 1];
  img[0] = txl;
  for (int m = 0; m < k; ++m)
    img[m + 1] = img[m] - (2.0f * dot3(img[m] - Pp[m], Pn[m])) * Pn[m];
  I[0] = txl;
  I[k + 1] = f3(0.f, 0.f, 0.f);
  float3 tgt = f3(0.f, 0.f, 0.f);
  for (int m = k; m >= 1; --m) {
    const float3 dir = img[m] - tgt;
    const float den = dot3(dir, Pn[m - 1]);
    if (den == 0.0f) return false;
    const float u = dot3(Pp[m - 1] - tgt, Pn[m - 1]) / den;
    I[m] = tgt + u * dir;
    tgt = I[m];
  }
  for (int m = 1; m <= k; ++m) {
    const float sa = dot3(I[m - 1] - I[m], Pn[m - 1]);
    const float sb = dot3(I[m + 1] - I[m], Pn[m - 1]);
    if (!(sa * sb > 0.0f)) return false;
  }
  return true;
}

// Leg m of an attempt: from I[m - 1] towards I[m], in scene coordinates.
__device__ __forceinline__ void spec_leg_ray(const float3* I, int m, float3 rxp, float3* org,
                                             float3* dir) {
  *org = I[m - 1] + rxp;
  *dir = unit3(I[m] - I[m - 1]);
}

// Whether a leg's closest hit (on the key's surface) is the interaction the
// plane predicts: its weighted normal within t_a of the plane's and its
// Eq. 3 point within t_d of the plane (Table I thresholds).  *qh receives the
// hit point relative to the RX, the plane point of a retry.
__device__ __forceinline__ bool spec_hit_fits(const SimConst& C, float3 org, float3 dir, float3 rxp,
                                              float tbar, float3 hn, float3 Im, float3 Pnm,
                                              float3* qh) {
  *qh = (org + tbar * dir) - rxp;
  const float c = fminf(1.0f, fabsf(dot3(Pnm, hn)));
  const float dist = fabsf(dot3(*qh - Im, Pnm));
  return c >= C.cos_ta && dist <= C.t_d;
}

// The final leg: from I[k] to the RX (an any-hit cast over its length).
__device__ __forceinline__ void spec_final_ray(const float3* I, int k, float3 rxp, float3* org,
                                               float3* dir, float* len) {
  const float3 last = f3(0.f, 0.f, 0.f) - I[k];
  *len = len3(last);
  *org = I[k] + rxp;
  *dir = (1.0f / *len) * last;
}

// A candidate's starting planes (its own interaction points and weighted
// normals, relative to the RX) and the key's surface label per interaction.
__device__ __forceinline__ void spec_load(const ValArgs& A, uint64_t hi, uint64_t lo, uint32_t row,
                                          int k, float3 rxp, float3* Pp, float3* Pn, uint32_t* lab) {
  for (int m = 0; m < k; ++m) {
    const int64_t b = A.R.at(m, row);
    Pp[m] = xyz(A.R.q[b]) - rxp;
    Pn[m] = xyz(A.R.n[b]);
  }
  for (int m = 0; m < 4; ++m) lab[m] = (uint32_t)((lo >> (16 * m)) & 0xFFFF);
  lab[4] = (uint32_t)(hi & 0xFFFF);
}

__device__ __forceinline__ bool spec_candidate(const SceneView& S, const SimConst& C,
                                               const ValArgs& A, uint64_t hi, uint64_t lo,
                                               uint32_t row, int* my_stk, float* my_tstk,
                                               uint32_t* err, unsigned long long& casts,
                                               unsigned long long& pruned, PathRec* P,
                                               int* stage = nullptr, const uint32_t* best = nullptr,
                                               uint32_t kid = 0, uint32_t rank = 0) {
  const int j = (int)(hi >> 56);
  const int k = (int)((hi >> 52) & 7);
  const float3 rxp = xyz(A.rx[C.batch ? 0 : j]);
  const float3 txl = tx_of(C, j) - rxp;
  float3 Pp[kMaxDepth], Pn[kMaxDepth];
  uint32_t lab[kMaxDepth];
  spec_load(A, hi, lo, row, k, rxp, Pp, Pn, lab);
  float3 I[kMaxDepth + 2];
  uint32_t vmats[kMaxDepth];
  int prev_dps = -1;
  const unsigned long long casts0 = casts;
  if (stage) *stage = kSpecNoCast;
  for (int attempt = 0;; ++attempt) {
    if (best && attempt > 0 && *(volatile const uint32_t*)(best + kid) < rank) return false;
    if (!spec_points(txl, Pp, Pn, k, I)) return false;
    prev_dps = -1;
    int fail_m = -1;
    float3 fq = f3(0.f, 0.f, 0.f), fn = f3(0.f, 0.f, 0.f);
    for (int m = 1; m <= k; ++m) {
      float3 org, dir;
      spec_leg_ray(I, m, rxp, &org, &dir);
      // a leg whose ray cannot reach the key's surface at this interaction
      // ends the candidate without a cast (its closest hit would be another
      // surface or nothing)
      // and a leg's search ends where its ray leaves that box: a hit beyond
      // is on another surface, which ends the candidate as nothing found does
      if (best && m > 1 && *(volatile const uint32_t*)(best + kid) < rank) return false;
      float t_exit;
      if (!ray_meets_label(S, org, dir, C.t_min, lab[m - 1], &t_exit)) {
        ++pruned;
        return false;
      }
      const Hit h = cast_ray(false, S, org, dir, prev_dps, C.t_min, t_exit, true, my_stk, my_tstk,
                             kTraceThreads, err);
      ++casts;
      if (stage) *stage = casts - casts0 == 1 ? kSpecLeg1 : kSpecLater;
      if (h.idx < 0 || (h.labels & 0xFFFFu) != lab[m - 1]) return false;
      if (stage) *stage = kSpecLater;
      float3 qh;
      const bool fits = spec_hit_fits(C, org, dir, rxp, h.tbar, h.n, I[m], Pn[m - 1], &qh);
      vmats[m - 1] = (h.labels >> 16) & 0xFFu;
      if (!fits) {
        fail_m = m;
        fq = qh;
        fn = h.n;
        break;
      }
      prev_dps = h.dps;
    }
    if (fail_m > 0) {
      if (attempt == C.kappa) return false;
      Pp[fail_m - 1] = fq;  // retry with the hit's plane
      Pn[fail_m - 1] = fn;
      continue;
    }
    break;
  }
  if (best && *(volatile const uint32_t*)(best + kid) < rank) return false;
  // last leg to the RX
  float3 forg, fdir;
  float sl;
  spec_final_ray(I, k, rxp, &forg, &fdir, &sl);
  const Hit hf = cast_ray(true, S, forg, fdir, prev_dps, C.t_min, sl, false, my_stk, my_tstk,
                          kTraceThreads, err);
  ++casts;
  if (stage) *stage = kSpecLater;
  if (hf.idx >= 0) return false;
  if (P) {
    memset(P, 0, sizeof(*P));
    P->hi = hi;
    P->lo = lo;
    P->rep = row;
    P->jtk = (uint32_t)j | ((uint32_t)k << 9);
    float len = 0.0f;
    uint64_t mats = 0;
    for (int m = 0; m <= k; ++m) len += len3(I[m + 1] - I[m]);
    for (int m = 1; m <= k; ++m) {
      const float3 pw = I[m] + rxp;
      P->pts[3 * (m - 1)] = pw.x;
      P->pts[3 * (m - 1) + 1] = pw.y;
      P->pts[3 * (m - 1) + 2] = pw.z;
      P->cosv[m - 1] = fabsf(dot3(Pn[m - 1], unit3(I[m] - I[m - 1])));
      mats |= (uint64_t)vmats[m - 1] << (8 * (m - 1));
    }
    P->mats_lo = (uint32_t)mats;
    P->mats_hi = (uint32_t)(mats >> 32);
    P->length = len;
    P->geo = C.lambda / (4.0f * 3.14159265358979f * len);
  }
  return true;
}

// Specular keys are validated over all their candidates at once (the
// paper refines every candidate, Sec. II-B-2, and keeps one path per key,
// Sec. II-B-4): items = (key, candidate) pairs, the candidates of each key
// in ray order, keys in validation order.  spec_count / scan / spec_expand
// lay the items out; the item pass refines each and keeps, per key, the
// lowest rank (position in the key's run) that validates; spec_finish
// writes the representative's path.  With rep_tries > 0 only the first
// rep_tries candidates of a key are items.
__device__ __forceinline__ uint32_t key_items(const KeyState& K, uint32_t kid, int rep_tries) {
  const uint32_t len = K.end[kid] - K.pos[kid];
  return rep_tries > 0 ? min(len, (uint32_t)rep_tries) : len;
}

// A key's first kHeadItems candidates are its head items, the rest its tail
// items; the item array holds every key's head, then every key's tail, so
// that a key with a valid candidate among its first ones usually knows it
// before its tail starts (and skips it).  The office's valid specular keys
// win at ranks up to tens of thousands; 2048 measured best (8 to 16384).
constexpr uint32_t kHeadItems = 2048;

__global__ void spec_count_kernel(KeyState K, const uint32_t* __restrict__ list,
                                  const unsigned long long* __restrict__ n_list_p, int rep_tries,
                                  uint32_t* __restrict__ cnt_h, uint32_t* __restrict__ cnt_t,
                                  uint32_t* __restrict__ best, uint32_t* __restrict__ hleft) {
  const int64_t n = (int64_t)*n_list_p;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t kid = list[q];
    NRT_GUARD(kid < g_dbg_caps.keys, 9, kid)
    const uint32_t m = key_items(K, kid, rep_tries);
    cnt_h[q] = min(m, kHeadItems);
    cnt_t[q] = m - min(m, kHeadItems);
    best[kid] = kNone;
    hleft[kid] = min(m, kHeadItems);
  }
}

// one warp per key: the key's items are candidate positions pos .. pos + m
// - 1, the head ones at off_h[q] and the tail ones after every key's head
__global__ void spec_expand_kernel(KeyState K, const uint32_t* __restrict__ list,
                                   const unsigned long long* __restrict__ n_list_p,
                                   const uint32_t* __restrict__ cnt_h, const uint32_t* __restrict__ off_h,
                                   const uint32_t* __restrict__ cnt_t, const uint32_t* __restrict__ off_t,
                                   uint32_t* __restrict__ items, int64_t item_cap,
                                   unsigned long long* __restrict__ n_items) {
  const int64_t n = (int64_t)*n_list_p;
  if (n <= 0) return;
  const int64_t heads = (int64_t)off_h[n - 1] + cnt_h[n - 1];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < n; q += n_warps) {
    const uint32_t kid = list[q];
    const uint32_t c0 = K.pos[kid], mh = cnt_h[q], mt = cnt_t[q];
    const int64_t oh = off_h[q], ot = heads + off_t[q];
    for (uint32_t t = lane; t < mh; t += 32)
      if (oh + t < item_cap) items[oh + t] = c0 + t;
    for (uint32_t t = lane; t < mt; t += 32)
      if (ot + t < item_cap) items[ot + t] = c0 + kHeadItems + t;
    if (q == n - 1 && lane == 0) *n_items = min(ot + mt, item_cap);
  }
}

// Item pass: lanes take items in order (one warp-aggregated atomic per
// fetch); an item ranked after a key's already-found valid candidate is
// skipped (it cannot be the lowest).
__global__ void __launch_bounds__(kTraceThreads, 5)
    validate_specular_items_kernel(SceneView S, SimConst C, ValArgs A,
                                   const uint32_t* __restrict__ items,
                                   const unsigned long long* __restrict__ n_items_p,
                                   uint32_t* __restrict__ best, unsigned long long* __restrict__ fetch,
                                   unsigned long long* ctr) {
  NRT_STACK_DECL
  unsigned long long casts = 0, pruned = 0, evaluated = 0, no_cast = 0, at_leg1 = 0;
  const int64_t n_items = (int64_t)*n_items_p;
  const uint64_t row_mask = (1ull << A.SC.row_bits) - 1ull;
  for (;;) {
    const int64_t i = fetch_next(fetch, n_items);
    if (i < 0) break;
    const uint32_t c = items[i];
    NRT_GUARD(c < g_dbg_caps.cand, 23, c)
    const uint64_t e = A.SC.key[c];
    const uint32_t kid = (uint32_t)(e >> A.SC.row_bits);
    NRT_GUARD(kid < g_dbg_caps.keys, 9, kid)
    const uint32_t row = (uint32_t)(e & row_mask);
    NRT_GUARD(row < g_dbg_caps.rows, 11, row)
    const uint32_t rank = c - A.K.pos[kid];
    if (*(volatile uint32_t*)(best + kid) < rank) continue;
    const uint32_t slot = A.K.slot[kid];
    NRT_GUARD(slot < g_dbg_caps.table, 10, slot)
    const uint64_t hi = A.T.b[slot].hi, lo = A.T.b[slot].lo;
    NRT_GUARD(((hi >> 52) & 7) >= 1 && ((hi >> 52) & 7) <= (uint64_t)C.max_depth, 12, hi >> 52)
    int stage = kSpecLater;
    ++evaluated;
    if (spec_candidate(S, C, A, hi, lo, row, my_stk, my_tstk, err, casts, pruned, nullptr, &stage,
                       best, kid, rank))
      atomicMin(best + kid, rank);
    no_cast += stage == kSpecNoCast;
    at_leg1 += stage == kSpecLeg1;
  }
  count_add(ctr + kCtrValCasts, casts);
  count_add(ctr + kCtrPrunedLegs, pruned);
  count_add(ctr + kCtrSpecItems, evaluated);
  count_add(ctr + kCtrSpecNoCast, no_cast);
  count_add(ctr + kCtrSpecLeg1, at_leg1);
}

// Specular refinement as waves.  The item pass above runs each candidate's
// whole retry chain in one lane: its refinement state (planes, image-method
// points) stays in registers across every cast, so the pass runs at 96
// registers and 5 blocks per SM, and lanes set up new items while their
// neighbours traverse.  Here a candidate's state lives in one of up to
// kSpecSlots slots in device memory, and each wave is three launches:
//   spec_wave_advance_kernel: consumes the last wave's hit of every live slot
//     and moves its candidate on -- to its next leg, a retry with the hit's
//     plane, its final leg, or its end -- with the helpers spec_candidate
//     uses and the same early stops (a candidate stops before its next cast
//     once its key's lowest valid rank is below its own); a slot whose
//     candidate ended takes the next items in item order until one needs a
//     cast; the next leg of every live slot is queued;
//   spec_wave_cast_kernel: the queued final legs (any hit; first, so that
//     the long ones overlap the rest) and legs (closest hit, weighted), in a
//     kernel that holds no refinement state (64 registers, 8 blocks per SM).
// The decisions per candidate are those of spec_candidate, so the lowest
// valid rank of every key -- the only thing kept -- is the same.
// With millions of slots every head item is taken within the first waves,
// before most keys have found their lowest valid rank; a tail item whose
// key still has head candidates in slots is therefore deferred to a second
// list, which opens once the first is exhausted and fewer than one slot in
// 16 holds a head candidate.  Once every item is taken and a wave queues
// fewer than kHandoffLegs casts, the waves stop (the later launches return
// at once) and spec_resume_kernel runs the candidates still in slots to
// their end, one lane each, without a kernel boundary per leg; the item
// pass then takes whatever items the kSpecWaves waves left (none, unless
// the work outgrew them).
constexpr int64_t kSpecSlots = 1 << 22;
constexpr int kSpecWaves = 32;
constexpr unsigned long long kHandoffLegs = 1ull << 18;

enum : int { kSlotEmpty = 0, kSlotLeg = 1, kSlotFinal = 2 };

// wave counters (index + wave % 3): legs queued, final legs queued, their
// fetch counters; the deferred list's count, fetch counter and open flag;
// the stop flag; the resume pass's fetch counter; head candidates placed in
// slots and ended there
enum : int { kWcLegs = 0, kWcFinal = 3, kWcLegFetch = 6, kWcFinalFetch = 9, kWcDefer = 12,
             kWcDeferFetch = 13, kWcDeferOpen = 14, kWcStop = 15, kWcResume = 16,
             kWcHeadsIn = 17, kWcHeadsOut = 18, kWcN = 19 };

struct SpecSlots {
  uint32_t* kid;
  uint32_t* rank;
  ulonglong2* key;  // key words (hi, lo)
  int4* ctl;        // attempt, leg m, DPS of the last hit (-1), phase
  float* pl;        // [6 kMaxDepth][n]: plane t's point (3 floats), normal (3)
  float* im;        // [3 kMaxDepth][n]: image-method points I[1..k]
  float4* hq;       // last hit: tbar, weighted normal
  int2* hd;         // last hit: DPS (-1: nothing hit), labels
  float4* q;        // queued legs [2][n]: (origin, t_max), (direction, DPS skipped)
  uint32_t* qs;     // their slots
  float4* qa;       // queued final legs, same layout
  uint32_t* qas;
  uint32_t* defer;  // deferred tail items [cand]
  uint32_t* hleft;  // per key: head candidates not yet finished
  unsigned long long* wc;  // kWcN counters
  int64_t n;
};

// component block b (3 floats) of slot s in a [3 b + c][n] array
__device__ __forceinline__ float3 slot_f3(const float* a, int64_t n, int64_t s, int b) {
  const float* p = a + (int64_t)(3 * b) * n + s;
  return f3(p[0], p[n], p[2 * n]);
}

__device__ __forceinline__ void slot_put3(float* a, int64_t n, int64_t s, int b, float3 v) {
  float* p = a + (int64_t)(3 * b) * n + s;
  p[0] = v.x;
  p[n] = v.y;
  p[2 * n] = v.z;
}

// surface label of interaction t (0-based) of a specular key
__device__ __forceinline__ uint32_t key_label(uint64_t hi, uint64_t lo, int t) {
  return t < 4 ? (uint32_t)((lo >> (16 * t)) & 0xFFFF) : (uint32_t)(hi & 0xFFFF);
}

// one queue entry per live slot: warp-aggregated position in this wave's queue
__device__ __forceinline__ void slot_queue(float4* q, uint32_t* qs, unsigned long long* count,
                                           int64_t s, float3 org, float t_max, float3 dir,
                                           int skip) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  const int64_t i = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
  q[2 * i] = make_float4(org.x, org.y, org.z, t_max);
  q[2 * i + 1] = make_float4(dir.x, dir.y, dir.z, __int_as_float(skip));
  qs[i] = (uint32_t)s;
}

// a leg or final leg to cast next
struct SlotRay {
  float3 org, dir;
  float t_max;
  int skip;
};

struct SpecCounts {
  unsigned long long pruned = 0, evaluated = 0, no_cast = 0, at_leg1 = 0;
  unsigned long long heads_in = 0, heads_out = 0;
};

// appends c to the deferred list (warp-aggregated)
__device__ __forceinline__ void defer_push(const SpecSlots& Q, uint32_t c) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(Q.wc + kWcDefer, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  Q.defer[base + __popc(mask & ((1u << lane) - 1u))] = c;
}

// Consumes the hit of slot s's last cast and moves its candidate on, as
// spec_candidate does after that cast; returns the phase of its next cast
// (its ray in *ray), or kSlotEmpty when the candidate ended.  The slot's
// phase is written either way; a head candidate that ended is counted off
// its key's hleft.
__device__ __forceinline__ int slot_advance(const SceneView& S, const SimConst& C,
                                            const ValArgs& A, const SpecSlots& Q, int64_t s,
                                            uint32_t* best, SlotRay* ray, SpecCounts& cnt) {
  const int4 ctl = Q.ctl[s];
  int attempt = ctl.x, m = ctl.y, prev = ctl.z;
  const uint32_t kid = Q.kid[s], rank = Q.rank[s];
  int next = kSlotEmpty;
  if (ctl.w == kSlotFinal) {
    if (Q.hd[s].x < 0) atomicMin(best + kid, rank);  // nothing in the way: valid
  } else {
    const ulonglong2 kw = Q.key[s];
    const int j = (int)(kw.x >> 56);
    const int k = (int)((kw.x >> 52) & 7);
    const float3 rxp = xyz(A.rx[C.batch ? 0 : j]);
    const float3 txl = tx_of(C, j) - rxp;
    const int2 hd = Q.hd[s];
    if (hd.x < 0 || ((uint32_t)hd.y & 0xFFFFu) != key_label(kw.x, kw.y, m - 1)) {
      cnt.at_leg1 += attempt == 0 && m == 1;  // ended at its first cast
    } else {
      float3 J[2];  // I[m - 1], I[m]
      J[0] = m == 1 ? txl : slot_f3(Q.im, Q.n, s, m - 2);
      J[1] = slot_f3(Q.im, Q.n, s, m - 1);
      const float4 hq = Q.hq[s];
      const float3 hn = f3(hq.y, hq.z, hq.w);
      float3 org, dir, qh;
      spec_leg_ray(J, 1, rxp, &org, &dir);
      if (!spec_hit_fits(C, org, dir, rxp, hq.x, hn, J[1], slot_f3(Q.pl, Q.n, s, 2 * m - 1), &qh)) {
        if (attempt < C.kappa) {
          ++attempt;  // retry with the hit's plane
          if (!(*(volatile const uint32_t*)(best + kid) < rank)) {
            float3 Pp[kMaxDepth], Pn[kMaxDepth], I[kMaxDepth + 2];
            for (int t = 0; t < k; ++t) {
              Pp[t] = slot_f3(Q.pl, Q.n, s, 2 * t);
              Pn[t] = slot_f3(Q.pl, Q.n, s, 2 * t + 1);
            }
            Pp[m - 1] = qh;
            Pn[m - 1] = hn;
            if (spec_points(txl, Pp, Pn, k, I)) {
              slot_put3(Q.pl, Q.n, s, 2 * m - 2, qh);
              slot_put3(Q.pl, Q.n, s, 2 * m - 1, hn);
              for (int t = 1; t <= k; ++t) slot_put3(Q.im, Q.n, s, t - 1, I[t]);
              m = 1;
              prev = -1;
              spec_leg_ray(I, 1, rxp, &ray->org, &ray->dir);
              next = kSlotLeg;
            }
          }
        }
      } else {
        prev = hd.x;
        ++m;
        if (!(*(volatile const uint32_t*)(best + kid) < rank)) {
          if (m <= k) {
            J[0] = J[1];
            J[1] = slot_f3(Q.im, Q.n, s, m - 1);
            spec_leg_ray(J, 1, rxp, &ray->org, &ray->dir);
            next = kSlotLeg;
          } else {
            spec_final_ray(J + 1, 0, rxp, &ray->org, &ray->dir, &ray->t_max);
            next = kSlotFinal;
          }
        }
      }
      if (next == kSlotLeg && !ray_meets_label(S, ray->org, ray->dir, C.t_min,
                                               key_label(kw.x, kw.y, m - 1), &ray->t_max)) {
        ++cnt.pruned;
        next = kSlotEmpty;
      }
    }
  }
  ray->skip = prev;
  if (next == kSlotEmpty && rank < kHeadItems) {
    atomicSub(Q.hleft + kid, 1u);
    ++cnt.heads_out;
  }
  Q.ctl[s] = make_int4(attempt, m, prev, next);
  return next;
}

// One item for the empty slot s, in item order: the next of the first list,
// or, once that is exhausted and the deferred list is open (no deferral
// can follow), of the deferred list.  Returns kTakePlaced (the item is in
// the slot, its first leg in *ray), kTakeAgain (the item needed no cast,
// was skipped or deferred) or kTakeNone (no item for now).  A tail item
// whose key still has head candidates in slots is deferred.
enum : int { kTakeNone = 0, kTakePlaced = 1, kTakeAgain = 2 };

__device__ __forceinline__ int slot_take(const SceneView& S, const SimConst& C, const ValArgs& A,
                                         const SpecSlots& Q, int64_t s,
                                         const uint32_t* __restrict__ items, int64_t n_items,
                                         unsigned long long* fetch, bool defer_open,
                                         uint32_t* best, SlotRay* ray, SpecCounts& cnt) {
  uint32_t c;
  bool deferred = false;
  if (*(volatile unsigned long long*)fetch < (unsigned long long)n_items) {
    const int64_t i = fetch_next(fetch, n_items);
    if (i < 0) return kTakeAgain;  // the last ones went to other lanes
    c = items[i];
  } else {
    if (!defer_open) return kTakeNone;
    const int64_t nd = (int64_t)*(volatile unsigned long long*)(Q.wc + kWcDefer);
    if ((int64_t)*(volatile unsigned long long*)(Q.wc + kWcDeferFetch) >= nd) return kTakeNone;
    const int64_t i = fetch_next(Q.wc + kWcDeferFetch, nd);
    if (i < 0) return kTakeNone;
    c = Q.defer[i];
    deferred = true;
  }
  if (!NRT_OK_IDX(c < g_dbg_caps.cand, 31, c)) return kTakeAgain;
  const uint64_t row_mask = (1ull << A.SC.row_bits) - 1ull;
  const uint64_t e = A.SC.key[c];
  const uint32_t kid = (uint32_t)(e >> A.SC.row_bits);
  if (!NRT_OK_IDX(kid < g_dbg_caps.keys, 32, kid)) return kTakeAgain;
  const uint32_t row = (uint32_t)(e & row_mask);
  if (!NRT_OK_IDX(row < g_dbg_caps.rows, 33, row)) return kTakeAgain;
  const uint32_t rank = c - A.K.pos[kid];
  const bool head = rank < kHeadItems;
  if (*(volatile const uint32_t*)(best + kid) < rank) {
    if (head) atomicSub(Q.hleft + kid, 1u);
    return kTakeAgain;
  }
  if (!head && !deferred && *(volatile const uint32_t*)(Q.hleft + kid) > 0) {
    defer_push(Q, c);
    return kTakeAgain;
  }
  const uint32_t slot = A.K.slot[kid];
  if (!NRT_OK_IDX(slot < g_dbg_caps.table, 34, slot)) return kTakeAgain;
  const uint64_t hi = A.T.b[slot].hi, lo = A.T.b[slot].lo;
  const int k = (int)((hi >> 52) & 7);
  if (!NRT_OK_IDX(k >= 1 && k <= C.max_depth, 35, k)) return kTakeAgain;
  const int j = (int)(hi >> 56);
  ++cnt.evaluated;
  const float3 rxp = xyz(A.rx[C.batch ? 0 : j]);
  const float3 txl = tx_of(C, j) - rxp;
  float3 Pp[kMaxDepth], Pn[kMaxDepth], I[kMaxDepth + 2];
  uint32_t lab[kMaxDepth];
  spec_load(A, hi, lo, row, k, rxp, Pp, Pn, lab);
  bool cast = spec_points(txl, Pp, Pn, k, I);
  if (cast) {
    spec_leg_ray(I, 1, rxp, &ray->org, &ray->dir);
    cast = ray_meets_label(S, ray->org, ray->dir, C.t_min, lab[0], &ray->t_max);
    cnt.pruned += !cast;
  }
  if (!cast) {
    ++cnt.no_cast;
    if (head) atomicSub(Q.hleft + kid, 1u);
    return kTakeAgain;
  }
  Q.kid[s] = kid;
  Q.rank[s] = rank;
  Q.key[s] = make_ulonglong2(hi, lo);
  for (int t = 0; t < k; ++t) {
    slot_put3(Q.pl, Q.n, s, 2 * t, Pp[t]);
    slot_put3(Q.pl, Q.n, s, 2 * t + 1, Pn[t]);
    slot_put3(Q.im, Q.n, s, t, I[t + 1]);
  }
  ray->skip = -1;
  Q.ctl[s] = make_int4(0, 1, -1, kSlotLeg);
  cnt.heads_in += head;
  return kTakePlaced;
}

__global__ void __launch_bounds__(kTraceThreads, 4)
    spec_wave_advance_kernel(SceneView S, SimConst C, ValArgs A, SpecSlots Q,
                             const uint32_t* __restrict__ items,
                             const unsigned long long* __restrict__ n_items_p,
                             uint32_t* __restrict__ best, unsigned long long* __restrict__ fetch,
                             unsigned long long* ctr, int w) {
  const int cur = w % 3, nxt = (w + 1) % 3;
  // the next wave's counters (their last user was wave w - 2)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Q.wc[kWcLegs + nxt] = 0;
    Q.wc[kWcFinal + nxt] = 0;
    Q.wc[kWcLegFetch + nxt] = 0;
    Q.wc[kWcFinalFetch + nxt] = 0;
  }
  if (Q.wc[kWcStop]) return;  // set by the last wave's cast kernel
  const bool defer_open = Q.wc[kWcDeferOpen] != 0;
  const int64_t n_items = (int64_t)*n_items_p;
  SpecCounts cnt;
  // whole warps step through the slots together, so that the refill below
  // takes items with one fetch per warp and refill step
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < Q.n;
       base += stride) {
    const int64_t s = base + (threadIdx.x & 31);
    const bool valid = s < Q.n;
    SlotRay ray;
    int next = kSlotEmpty;
    if (valid && Q.ctl[s].w != kSlotEmpty) next = slot_advance(S, C, A, Q, s, best, &ray, cnt);
    bool need = valid && next == kSlotEmpty;
    __syncwarp();
    while (__any_sync(0xFFFFFFFFu, need)) {
      if (need) {
        const int r = slot_take(S, C, A, Q, s, items, n_items, fetch, defer_open, best, &ray, cnt);
        if (r == kTakePlaced) next = kSlotLeg;
        need = r == kTakeAgain;
      }
    }
    if (next == kSlotLeg)
      slot_queue(Q.q, Q.qs, Q.wc + kWcLegs + cur, s, ray.org, ray.t_max, ray.dir, ray.skip);
    else if (next == kSlotFinal)
      slot_queue(Q.qa, Q.qas, Q.wc + kWcFinal + cur, s, ray.org, ray.t_max, ray.dir, ray.skip);
  }
  count_add(ctr + kCtrPrunedLegs, cnt.pruned);
  count_add(ctr + kCtrSpecItems, cnt.evaluated);
  count_add(ctr + kCtrSpecNoCast, cnt.no_cast);
  count_add(ctr + kCtrSpecLeg1, cnt.at_leg1);
  count_add(Q.wc + kWcHeadsIn, cnt.heads_in);
  count_add(Q.wc + kWcHeadsOut, cnt.heads_out);
}

// The wave's queued casts: the final legs first (any hit between I[k] and
// the RX; some graze a surface for metres, and started first they overlap
// the rest), then the legs (closest hit up to the exit of the key's surface
// box, weighted: Eq. 3/4), as spec_candidate casts them.  Its first thread
// also decides for the next wave: the deferred list opens once the first
// list is exhausted and fewer than one slot in 16 holds a head candidate;
// the waves stop once both lists are taken and this wave queued fewer than
// kHandoffLegs casts.
__global__ void __launch_bounds__(kTraceThreads, 8)
    spec_wave_cast_kernel(SceneView S, SimConst C, SpecSlots Q,
                          const unsigned long long* __restrict__ fetch,
                          const unsigned long long* __restrict__ n_items_p, unsigned long long* ctr,
                          int w) {
  NRT_STACK_DECL
  const int cur = w % 3;
  const unsigned long long nl = Q.wc[kWcLegs + cur], nf = Q.wc[kWcFinal + cur];
  if (blockIdx.x == 0 && threadIdx.x == 0 && !Q.wc[kWcStop] && *fetch >= *n_items_p) {
    if (Q.wc[kWcDeferOpen] == 0) {
      if (Q.wc[kWcHeadsIn] - Q.wc[kWcHeadsOut] <= (unsigned long long)(Q.n / 16))
        Q.wc[kWcDeferOpen] = 1;
    } else if (Q.wc[kWcDeferFetch] >= Q.wc[kWcDefer] && nl + nf < kHandoffLegs) {
      Q.wc[kWcStop] = 1;
    }
  }
  if (nl + nf == 0) return;
  unsigned long long casts = 0;
  bool finals = nf > 0;
  for (;;) {
    if (finals) {
      const int64_t i = fetch_next(Q.wc + kWcFinalFetch + cur, (int64_t)nf);
      if (i >= 0) {
        const uint32_t s = Q.qas[i];
        NRT_GUARD(s < Q.n, 37, s)
        const float4 a = Q.qa[2 * i], b = Q.qa[2 * i + 1];
        const Hit h = cast_ray(true, S, xyz(a), xyz(b), __float_as_int(b.w), C.t_min, a.w, false,
                               my_stk, my_tstk, kTraceThreads, err);
        ++casts;
        Q.hd[s] = make_int2(h.dps, (int)h.labels);
        continue;
      }
      finals = false;
    }
    const int64_t i = fetch_next(Q.wc + kWcLegFetch + cur, (int64_t)nl);
    if (i < 0) break;
    const uint32_t s = Q.qs[i];
    NRT_GUARD(s < Q.n, 36, s)
    const float4 a = Q.q[2 * i], b = Q.q[2 * i + 1];
    const Hit h = cast_ray(false, S, xyz(a), xyz(b), __float_as_int(b.w), C.t_min, a.w, true, my_stk,
                           my_tstk, kTraceThreads, err);
    ++casts;
    Q.hq[s] = make_float4(h.tbar, h.n.x, h.n.y, h.n.z);
    Q.hd[s] = make_int2(h.dps, (int)h.labels);
  }
  count_add(ctr + kCtrValCasts, casts);
}

// After the waves: each candidate still in a slot runs to its end in one
// lane (its pending hit first, then cast by cast).
__global__ void __launch_bounds__(kTraceThreads, 5)
    spec_resume_kernel(SceneView S, SimConst C, ValArgs A, SpecSlots Q, uint32_t* __restrict__ best,
                       unsigned long long* ctr) {
  NRT_STACK_DECL
  SpecCounts cnt;
  unsigned long long casts = 0;
  for (;;) {
    const int64_t s = fetch_next(Q.wc + kWcResume, Q.n);
    if (s < 0) break;
    if (Q.ctl[s].w == kSlotEmpty) continue;
    for (;;) {
      SlotRay ray;
      const int next = slot_advance(S, C, A, Q, s, best, &ray, cnt);
      if (next == kSlotEmpty) break;
      Hit h;
      if (next == kSlotLeg)
        h = cast_ray(false, S, ray.org, ray.dir, ray.skip, C.t_min, ray.t_max, true, my_stk, my_tstk,
                     kTraceThreads, err);
      else
        h = cast_ray(true, S, ray.org, ray.dir, ray.skip, C.t_min, ray.t_max, false, my_stk, my_tstk,
                     kTraceThreads, err);
      ++casts;
      Q.hq[s] = make_float4(h.tbar, h.n.x, h.n.y, h.n.z);
      Q.hd[s] = make_int2(h.dps, (int)h.labels);
    }
  }
  count_add(ctr + kCtrValCasts, casts);
  count_add(ctr + kCtrPrunedLegs, cnt.pruned);
  count_add(ctr + kCtrSpecLeg1, cnt.at_leg1);
}

// Per specular key: the lowest valid rank is the representative (its path
// recorded by refining it once more, with the same function); the key's
// status, tries and representative row follow the ray-order rule.
__global__ void __launch_bounds__(kTraceThreads)
    spec_finish_kernel(SceneView S, SimConst C, ValArgs A, const uint32_t* __restrict__ list,
                       const unsigned long long* __restrict__ n_list_p,
                       const uint32_t* __restrict__ best, unsigned long long* ctr) {
  NRT_STACK_DECL
  unsigned long long casts = 0;
  const int64_t n = (int64_t)*n_list_p;
  const uint64_t row_mask = (1ull << A.SC.row_bits) - 1ull;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = base + threadIdx.x;
    bool fin = false;
    int j = 0;
    if (q < n) {
      const uint32_t kid = list[q];
      const uint32_t b = best[kid];
      const uint32_t slot = A.K.slot[kid];
      const uint64_t hi = A.T.b[slot].hi, lo = A.T.b[slot].lo;
      j = (int)(hi >> 56);
      fin = true;
      if (b != kNone) {
        const uint32_t c = A.K.pos[kid] + b;
        const uint32_t row = (uint32_t)(A.SC.key[c] & row_mask);
        PathRec P;
        unsigned long long pruned = 0;
        if (spec_candidate(S, C, A, hi, lo, row, my_stk, my_tstk, err, casts, pruned, &P)) {
          A.K.status[kid] = 1;
          A.K.tries[kid] = b;
          A.K.cur[kid] = row;
          A.K.pos[kid] = c;
          const unsigned long long p = atomicAdd(ctr + kCtrPaths, 1ull);
          if ((int64_t)p < A.path_cap) A.paths[p] = P;
          else atomicOr(err, kErrPathFull);
        } else {
          atomicOr(err, kErrRecheck);  // the same refinement decided otherwise
          A.K.status[kid] = 2;
        }
      } else {
        A.K.status[kid] = 2;
        A.K.tries[kid] = key_items(A.K, kid, C.rep_tries);
      }
    }
    if (A.pair_keys) pair_units_done(fin, j, A.pair_keys, A.pair_ready);
  }
  count_add(ctr + kCtrValCasts, casts);
}

// Every key starts at the first (lowest-row) candidate of its run.  cur, pos,
// tries and status are zeroed beforehand, so a key left without a run (a
// result that overflowed its candidate capacity reports an error) still
// points at a candidate inside the arrays.
__global__ void run_start_kernel(SortedCand SC, KeyState K, int64_t key_cap) {
  const int64_t n = min((int64_t)*SC.n_p, SC.cap);
  const uint64_t row_mask = (1ull << SC.row_bits) - 1ull;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t e = SC.key[c];
    const uint64_t kid = e >> SC.row_bits;
    if (kid >= (uint64_t)key_cap) continue;  // candidates of keys over capacity
    if (c == 0 || (SC.key[c - 1] >> SC.row_bits) != kid) {
      K.pos[kid] = (uint32_t)c;
      K.cur[kid] = (uint32_t)(e & row_mask);
    }
    if (c == n - 1 || (SC.key[c + 1] >> SC.row_bits) != kid) K.end[kid] = (uint32_t)(c + 1);
  }
}


// Per-key summaries for merging ray-range shards: candidates tried (the
// valid one included) and the ray id of the validated candidate.
__global__ void key_summary_kernel(const unsigned long long* __restrict__ n_keys_p, KeyState K,
                                   Table T, const uint32_t* __restrict__ ray_of_row,
                                   uint64_t* __restrict__ hi, uint64_t* __restrict__ lo,
                                   uint32_t* __restrict__ tried, uint32_t* __restrict__ rep) {
  const int64_t n_keys = (int64_t)*n_keys_p;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_keys;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t slot = K.slot[i];
    hi[i] = T.b[slot].hi;
    lo[i] = T.b[slot].lo;
    const bool valid = K.status[i] == 1u;
    tried[i] = K.tries[i] + (valid ? 1u : 0u);
    const uint32_t row = K.cur[i];
    rep[i] = valid ? (ray_of_row ? ray_of_row[row] : row) : 0xFFFFFFFFu;
  }
}


// ---------------------------------------------------------------- ordering
// Paths ordered by (rx, type, k, representative row): deterministic output.
// key = [rx][type][k][representative row in row_bits bits] (LOS, the only
// k = 0 path of an RX, keeps its masked kNone); bits row_bits + 12
__global__ void path_sortkey_kernel(const PathRec* __restrict__ p,
                                    const unsigned long long* __restrict__ n_p, int64_t cap,
                                    int row_bits, uint64_t* __restrict__ key,
                                    uint32_t* __restrict__ idx) {
  const int64_t n = min((int64_t)*n_p, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    idx[i] = (uint32_t)i;
    const uint32_t jtk = p[i].jtk;
    const bool dfr = (jtk >> 12) & 1;  // diffracted paths last: class (1, 6)
    const uint64_t j = jtk & 0xFF, ty = dfr ? 1 : (jtk >> 8) & 1, k = dfr ? 6 : (jtk >> 9) & 7;
    key[i] = (j << (row_bits + 4)) | (ty << (row_bits + 3)) | (k << row_bits) |
             ((uint64_t)p[i].rep & ((1ull << row_bits) - 1ull));
  }
}

// per-RX range of the sorted paths: lower bounds of (j << 36) and ((j+1) << 36)
__global__ void rx_range_kernel(const uint64_t* __restrict__ key,
                                const unsigned long long* __restrict__ n_p, int64_t cap, int n_rx,
                                int rx_shift, int64_t* __restrict__ start, int64_t* __restrict__ cnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_rx) return;
  const int64_t n = min((int64_t)*n_p, cap);
  auto lower = [&](uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (key[mid] < v) lo = mid + 1;
      else hi = mid;
    }
    return lo;
  };
  const int64_t a = lower((uint64_t)j << rx_shift);
  start[j] = a;
  cnt[j] = lower((uint64_t)(j + 1) << rx_shift) - a;
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

__global__ void order_key_kernel(SimConst C, const uint32_t* __restrict__ ray_of_row, int64_t n,
                                 int64_t n_rays, uint64_t* __restrict__ key,
                                 uint32_t* __restrict__ val) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = ray_of_row ? ray_of_row[c] : (uint64_t)c;
    uint64_t nr = (uint64_t)n_rays, hi = 0;
    if (C.batch) {
      const int pj = pair_of_row(C, (uint32_t)c);
      r = (uint64_t)c - C.pair_start[pj];
      nr = (uint64_t)C.pair_rays[pj];
      hi = (uint64_t)pj << 32;
    }
    const uint32_t zb = (uint32_t)min((2 * r + 1) * 32768ull / nr, 65535ull);
    const uint32_t pb = (uint32_t)((r * 0x61C8864680B583EBull) >> 48);
    key[c] = hi | (uint64_t)(spread2(zb) | (spread2(pb) << 1));
    val[c] = (uint32_t)c;
  }
}

// sorted paths: only the first n entries hold paths (padding sorts last)
__global__ void path_gather_kernel(const PathRec* __restrict__ src, const uint32_t* __restrict__ idx,
                                   const unsigned long long* __restrict__ n_p, int64_t cap,
                                   PathRec* __restrict__ dst) {
  const int64_t n = min((int64_t)*n_p, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    NRT_GUARD(idx[i] < g_dbg_caps.paths, 20, idx[i])
    dst[i] = src[idx[i]];
  }
}

// ---------------------------------------------------------------- field

// ---------------------------------------------------------------- vector polarisation
// pol = NRT_POL_VECTOR.  TX and RX radiate / receive along theta^ (spherical
// basis about +z).  Each interaction m has an incoming direction d_m, an
// outgoing d_{m+1} and a normal n_m (specular: along d_{m+1} - d_m; diffuse
// last interaction: the scatter point's surface normal).  Its field basis is
// s = unit(d_m x n_m) across the plane of incidence and p = s x d (in: d_m,
// out: d_{m+1}); the s component is scaled by c Gamma_TE, the p component by
// c Gamma_TM (c = R, or S at a diffuse last interaction).  Between two
// interactions the outgoing basis of m is re-expressed in the incoming basis
// of m+1 by a real 2x2 matrix, both bases spanning the plane normal to
// d_{m+1}.  a = geo r^T D_k B_{k-1} ... B_1 D_1 e0 (e0, r: the TX and RX
// polarisation in the first and last basis).  LOS: theta^(u) . theta^(-u) = 1.
struct PathFrame {
  float3 tx;              // the simulation's TX
  const float4* tx_pair;  // batch: TX of pair j
  const float4* rx;       // physical receivers (batch: one)
  int batch;
};

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// theta^ along the unit direction d; x^ on the z axis
__device__ __forceinline__ float3 theta_unit(float3 d) {
  const float h = sqrtf(d.x * d.x + d.y * d.y);
  if (h < 1e-12f) return f3(1.0f, 0.0f, 0.0f);
  const float c = d.z / h;
  return f3(c * d.x, c * d.y, -h);
}

// s^ across the plane of incidence; at (near) normal incidence, where the
// plane is undefined and Gamma_TM = -Gamma_TE, any unit vector across d_in
__device__ __forceinline__ float3 across_unit(float3 din, float3 n) {
  const float3 s = cross3(din, n);
  const float l = len3(s);
  if (l < 1e-4f)
    return unit3(cross3(din, fabsf(din.z) < 0.9f ? f3(0.0f, 0.0f, 1.0f) : f3(1.0f, 0.0f, 0.0f)));
  return (1.0f / l) * s;
}

struct JonesGeom {
  float e0[2];                 // TX polarisation in the first incoming basis
  float B[kMaxDepth - 1][4];   // outgoing basis of m -> incoming basis of m+1 (row-major)
  float r[2];                  // RX polarisation in the last outgoing basis
};

__device__ __forceinline__ void jones_geom(const PathRec& p, int k, int diffuse, float3 tx,
                                           float3 rx, JonesGeom& J) {
  float3 q = f3(p.pts[0], p.pts[1], p.pts[2]);
  float3 din = unit3(q - tx);
  float3 s_prev = f3(0.f, 0.f, 0.f), po_prev = s_prev;
#pragma unroll
  for (int m = 0; m < kMaxDepth; ++m) {
    if (m < k) {
      const float3 nxt = m + 1 < k ? f3(p.pts[3 * m + 3], p.pts[3 * m + 4], p.pts[3 * m + 5]) : rx;
      const float3 dout = unit3(nxt - q);
      const float3 n = (diffuse && m == k - 1) ? f3(p.nd[0], p.nd[1], p.nd[2]) : unit3(dout - din);
      const float3 s = across_unit(din, n);
      const float3 pin = cross3(s, din);
      if (m == 0) {
        const float3 t = theta_unit(din);
        J.e0[0] = dot3(t, s);
        J.e0[1] = dot3(t, pin);
      } else {
        J.B[m - 1][0] = dot3(s, s_prev);
        J.B[m - 1][1] = dot3(s, po_prev);
        J.B[m - 1][2] = dot3(pin, s_prev);
        J.B[m - 1][3] = dot3(pin, po_prev);
      }
      s_prev = s;
      po_prev = cross3(s, dout);
      din = dout;
      q = nxt;
    }
  }
  const float3 t = theta_unit(-1.0f * din);
  J.r[0] = dot3(t, s_prev);
  J.r[1] = dot3(t, po_prev);
}

__device__ __forceinline__ float3 frame_tx(const PathFrame& F, int j) {
  return F.batch ? xyz(__ldg(F.tx_pair + j)) : F.tx;
}
__device__ __forceinline__ float3 frame_rx(const PathFrame& F, int j) {
  return xyz(__ldg(F.rx + (F.batch ? 0 : j)));
}

// Diffracted path: D = K(T1 + T2) + R0 K T3 + Rn K T4 with the stored
// material-independent terms (soft / TE coefficients for pol 0, hard / TM
// for pol 1, v_s D_s + v_h D_h for the vector model); a = geo D.  dD
// (optional): dD/deta of face 0 and face n.
__device__ __forceinline__ float2 diffraction_factor(const PathRec& p, const float* __restrict__ mat,
                                                     float freq, int pol, float2* dD) {
  const float2 t12 = make_float2(p.pts[3], p.pts[4]), t3 = make_float2(p.pts[5], p.pts[6]);
  const float2 t4 = make_float2(p.pts[7], p.pts[8]);
  const int l0 = path_mat(p, 0), l1 = path_mat(p, 1);
  const float2 eta0 = permittivity(mat[l0], mat[256 + l0], freq);
  const float2 eta1 = permittivity(mat[l1], mat[256 + l1], freq);
  float2 Dsum = make_float2(0.f, 0.f), g0 = Dsum, g1 = Dsum;
  for (int t = 0; t < 2; ++t) {
    const float v = pol == 2 ? p.pts[9 + t] : (t == pol ? 1.0f : 0.0f);
    if (v == 0.0f) continue;
    const float2 Dt = cadd(t12, cadd(cmul(fresnel(eta0, p.cosv[0], t), t3),
                                     cmul(fresnel(eta1, p.cosv[1], t), t4)));
    Dsum = cadd(Dsum, cscale(v, Dt));
    if (dD) {
      g0 = cadd(g0, cscale(v, cmul(dfresnel(eta0, p.cosv[0], t), t3)));
      g1 = cadd(g1, cscale(v, cmul(dfresnel(eta1, p.cosv[1], t), t4)));
    }
  }
  if (dD) {
    dD[0] = g0;
    dD[1] = g1;
  }
  return Dsum;
}

// a = geo * prod_m f_m Gamma_m(theta_m): f = sqrt(1 - S^2) for a specular
// reflection (effective roughness), f = S for the diffuse last interaction;
// the vector model replaces the product by the 2x2 chain above.
__global__ void field_kernel(const PathRec* __restrict__ P, const unsigned long long* __restrict__ n_p,
                             int64_t cap, const float* __restrict__ mat, float freq, int pol,
                             PathFrame F, float2* __restrict__ a_out) {
  const int64_t n = min((int64_t)*n_p, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const PathRec p = P[i];
    const int k = (p.jtk >> 9) & 7;
    const int diffuse = (p.jtk >> 8) & 1;
    float2 a = make_float2(p.geo, 0.0f);
    if ((p.jtk >> 12) & 1) {
      a = cscale(p.geo, diffraction_factor(p, mat, freq, pol, nullptr));
    } else if (pol == 2) {
      if (k > 0) {
        const int j = p.jtk & 0xFF;
        JonesGeom J;
        jones_geom(p, k, diffuse, frame_tx(F, j), frame_rx(F, j), J);
        float2 v0 = make_float2(J.e0[0], 0.0f), v1 = make_float2(J.e0[1], 0.0f);
#pragma unroll
        for (int m = 0; m < kMaxDepth; ++m) {
          if (m < k) {
            float2 D[2];
            interaction_factors(p, m, k, diffuse, mat, freq, pol, D, nullptr, nullptr);
            v0 = cmul(v0, D[0]);
            v1 = cmul(v1, D[1]);
            if (m + 1 < k) {
              const float2 u0 = cadd(cscale(J.B[m][0], v0), cscale(J.B[m][1], v1));
              const float2 u1 = cadd(cscale(J.B[m][2], v0), cscale(J.B[m][3], v1));
              v0 = u0;
              v1 = u1;
            }
          }
        }
        a = cscale(p.geo, cadd(cscale(J.r[0], v0), cscale(J.r[1], v1)));
      }
    } else {
      for (int m = 0; m < k; ++m) {
        float2 D[1];
        interaction_factors(p, m, k, diffuse, mat, freq, pol, D, nullptr, nullptr);
        a = cmul(a, D[0]);
      }
    }
    a_out[i] = a;
  }
}

// P_j = sum |a|^2 over RX j's paths in two fixed-order levels (the same
// result on every run): kPowerChunks blocks per RX write partial sums, then
// one pass adds each RX's partials in order.
constexpr int kPowerChunks = 64;
__global__ void power_partial_kernel(const float2* __restrict__ a, const int64_t* __restrict__ start,
                                     const int64_t* __restrict__ count, double* __restrict__ partial) {
  __shared__ double sh[256];
  const int j = blockIdx.y;
  const int64_t b = start[j], n = count[j];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    NRT_GUARD(b + i < g_dbg_caps.paths, 24, b + i)
    const float2 v = a[b + i];
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)j * kPowerChunks + blockIdx.x] = sh[0];
}

__global__ void power_sum_kernel(const double* __restrict__ partial, int n_rx,
                                 double* __restrict__ power) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_rx) return;
  double s = 0.0;
  for (int c = 0; c < kPowerChunks; ++c) s += partial[(int64_t)j * kPowerChunks + c];
  power[j] = s;
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

// wpath (optional): per-path complex weights W_p of a loss whose gradient is
// sum_p Re(W_p da_p/dtheta); without it W_p = 2 dL/dP_j conj(a_p) (power loss).
//
// Vector model: a / geo is linear in each interaction's (D_TE, D_TM); its
// partials are (row vector after m) x (field entering m), component-wise,
// from one forward and one backward sweep over the 2x2 chain.
__global__ void __launch_bounds__(kAdjThreads)
    adjoint_kernel(const PathRec* __restrict__ P, int64_t n, const float* __restrict__ mat,
                   float freq, int pol, PathFrame F, const float* __restrict__ dLdP,
                   const double2* __restrict__ wpath, int n_labels, double* __restrict__ partial) {
  __shared__ double sh[kAdjThreads / 32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int k = 0, labs[kMaxDepth];
  float ge[kMaxDepth], gs[kMaxDepth], gc[kMaxDepth];
  if (i < n) {
    const PathRec p = P[i];
    k = (p.jtk >> 9) & 7;
    const int diffuse = (p.jtk >> 8) & 1;
    const int j = p.jtk & 0xFF;
    // da/deta_m and da/dS_m (before the loss weight)
    float2 dae[kMaxDepth], das[kMaxDepth];
    float2 a = make_float2(p.geo, 0.0f);
    if ((p.jtk >> 12) & 1) {  // diffracted: the two faces' coefficients, no S
      float2 dD[2];
      a = cscale(p.geo, diffraction_factor(p, mat, freq, pol, dD));
      k = 2;
      labs[0] = path_mat(p, 0);
      labs[1] = path_mat(p, 1);
      dae[0] = cscale(p.geo, dD[0]);
      dae[1] = cscale(p.geo, dD[1]);
      das[0] = das[1] = make_float2(0.f, 0.f);
    } else if (pol == 2) {
      if (k > 0) {
        JonesGeom J;
        jones_geom(p, k, diffuse, frame_tx(F, j), frame_rx(F, j), J);
        float2 D[kMaxDepth][2], De[kMaxDepth][2], Ds[kMaxDepth][2], fw[kMaxDepth][2];
        float2 v0 = make_float2(J.e0[0], 0.0f), v1 = make_float2(J.e0[1], 0.0f);
#pragma unroll
        for (int m = 0; m < kMaxDepth; ++m) {
          if (m < k) {
            labs[m] = path_mat(p, m);
            interaction_factors(p, m, k, diffuse, mat, freq, pol, D[m], De[m], Ds[m]);
            fw[m][0] = v0;
            fw[m][1] = v1;
            v0 = cmul(v0, D[m][0]);
            v1 = cmul(v1, D[m][1]);
            if (m + 1 < k) {
              const float2 u0 = cadd(cscale(J.B[m][0], v0), cscale(J.B[m][1], v1));
              const float2 u1 = cadd(cscale(J.B[m][2], v0), cscale(J.B[m][3], v1));
              v0 = u0;
              v1 = u1;
            }
          }
        }
        a = cscale(p.geo, cadd(cscale(J.r[0], v0), cscale(J.r[1], v1)));
        float2 w0 = make_float2(p.geo * J.r[0], 0.0f), w1 = make_float2(p.geo * J.r[1], 0.0f);
#pragma unroll
        for (int m = kMaxDepth - 1; m >= 0; --m) {
          if (m < k) {
            const float2 x0 = cmul(w0, fw[m][0]), x1 = cmul(w1, fw[m][1]);
            dae[m] = cadd(cmul(x0, De[m][0]), cmul(x1, De[m][1]));
            das[m] = cadd(cmul(x0, Ds[m][0]), cmul(x1, Ds[m][1]));
            if (m > 0) {  // w <- w D_m B_{m-1}
              const float2 y0 = cmul(w0, D[m][0]), y1 = cmul(w1, D[m][1]);
              w0 = cadd(cscale(J.B[m - 1][0], y0), cscale(J.B[m - 1][2], y1));
              w1 = cadd(cscale(J.B[m - 1][1], y0), cscale(J.B[m - 1][3], y1));
            }
          }
        }
      }
    } else {
      float2 fac[kMaxDepth], dfe[kMaxDepth], dfs[kMaxDepth];
      for (int m = 0; m < k; ++m) {
        labs[m] = path_mat(p, m);
        interaction_factors(p, m, k, diffuse, mat, freq, pol, &fac[m], &dfe[m], &dfs[m]);
      }
      for (int m = 0; m < k; ++m) a = cmul(a, fac[m]);
      for (int m = 0; m < k; ++m) {
        float2 oth = make_float2(p.geo, 0.0f);
        for (int q = 0; q < k; ++q)
          if (q != m) oth = cmul(oth, fac[q]);
        dae[m] = cmul(oth, dfe[m]);
        das[m] = cmul(oth, dfs[m]);
      }
    }
    float2 W;
    if (wpath) {
      const double2 wd = wpath[i];
      W = make_float2((float)wd.x, (float)wd.y);
    } else {
      W = cscale(2.0f * dLdP[j], cconj(a));
    }
    const float ks = (float)(1.0 / (2.0 * 3.14159265358979323846 * kEps0)) / freq;
    for (int m = 0; m < k; ++m) {
      const float2 de = cmul(W, dae[m]);
      const float2 ds = cmul(W, das[m]);
      ge[m] = de.x;
      gs[m] = de.y * ks;  // Re(z * (-j ks)) = ks * Im(z)
      gc[m] = ds.x;
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

// path records reserved for diffracted paths: one per (edge, RX or pair)
int64_t diffraction_slots(const nrt_result* r) {
  if (!r->p.diffraction) return 0;
  return r->scene->n_edges * (r->n_pairs > 0 ? r->n_pairs : r->n_rx_phys);
}

PathFrame path_frame(const nrt_result* r) {
  PathFrame F;
  F.tx = make_float3(r->tx[0], r->tx[1], r->tx[2]);
  F.tx_pair = r->tx_pair;
  F.rx = r->rx;
  F.batch = r->n_pairs > 0 ? 1 : 0;
  return F;
}

inline int blocks_for(int64_t n, int threads, int sm, int per_sm = 16) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm * per_sm));
}

SimConst make_const(const nrt_result* r) {
  SimConst C;
  C.tx = make_float3(r->tx[0], r->tx[1], r->tx[2]);
  C.n_rx = r->n_rx_phys;
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
  C.launch = r->p.launch;
  C.vis_words = r->vis_words;
  C.batch = r->n_pairs > 0 ? 1 : 0;
  C.n_pairs = r->n_pairs;
  C.tx_pair = r->tx_pair;
  C.pair_start = r->pair_start;
  C.pair_rays = r->pair_rays;
  return C;
}

// Origin and direction of the ray of `row`: the Fibonacci sphere, or
// (Sec. II-B) toward the reception point of DPS `ray` (the DPS are stored in
// voxel Morton order); batch rows take their pair's TX and launch size.
__device__ __forceinline__ void ray_start(const SceneView& S, const SimConst& C,
                                          const uint32_t* __restrict__ ray_of_row, int64_t row,
                                          float3* o_out, float3* d_out) {
  uint32_t ray = ray_of_row ? ray_of_row[row] : (uint32_t)row;
  int64_t n_launch = C.n_rays;
  float3 o = C.tx;
  if (C.batch) {
    const int pj = pair_of_row(C, (uint32_t)row);
    ray = (uint32_t)row - __ldg(C.pair_start + pj);
    n_launch = __ldg(C.pair_rays + pj);
    o = xyz(__ldg(C.tx_pair + pj));
  }
  *o_out = o;
  *d_out = C.launch == NRT_LAUNCH_DPS ? unit3(xyz(__ldg(S.recv + ray)) - o) : fib_dir(ray, n_launch);
}

// One ray: launch, closest hit per bounce, specular continuation; the hit
// records go to the ray's row.  Returns the segments cast.
__device__ __forceinline__ unsigned trace_row(const SceneView& S, const SimConst& C,
                                              const uint32_t* __restrict__ ray_of_row,
                                              const Records& R, int64_t row, int* stk, float* tstk,
                                              uint32_t* err) {
  float3 o, d;
  ray_start(S, C, ray_of_row, row, &o, &d);
  int skip = -1;
  unsigned segs = 0;
  for (int s = 0; s < C.n_seg; ++s) {
    const Hit h = cast_ray(false, S, o, d, skip, C.t_min, __int_as_float(0x7f800000), true, stk,
                                  tstk, kTraceThreads, err);
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
  return segs;
}

// Batch trace as one persistent launch: warps pull work items of `packet`
// rays of one pair from a queue (uneven budgets balance themselves); the warp
// that finishes a pair's last item stamps the pair's completion time.
__global__ void __launch_bounds__(kTraceThreads, 8)
    trace_persistent_kernel(SceneView S, SimConst C, const uint32_t* __restrict__ order, Records R,
                            const uint32_t* __restrict__ chunk_start, int packet,
                            unsigned long long* queue, unsigned long long* stamps,
                            unsigned long long* ctr) {
  NRT_STACK_DECL
  const int lane = threadIdx.x & 31;
  const uint32_t n_chunks = __ldg(chunk_start + C.n_pairs);
  unsigned long long segs = 0;
  for (int guard = 0; guard < (1 << 30); ++guard) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(queue, 1ull);
    c = __shfl_sync(0xFFFFFFFFu, c, 0);
    if (c >= n_chunks) break;
    int lo = 0, hi = C.n_pairs;  // pair of chunk c
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(chunk_start + mid) <= c) lo = mid;
      else hi = mid;
    }
    const int pj = lo;
    const int64_t t0 = (int64_t)__ldg(C.pair_start + pj) + (int64_t)(c - __ldg(chunk_start + pj)) * packet;
    const int64_t t1 = min(t0 + packet, (int64_t)__ldg(C.pair_start + pj + 1));
    for (int64_t t = t0 + lane; t < t1; t += 32) {
      const int64_t row = order ? order[t] : t;
      segs += trace_row(S, C, nullptr, R, row, my_stk, my_tstk, err);
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      if (atomicAdd(queue + 1 + pj, ~0ull) == 1ull) stamps[1 + pj] = global_ns();  // -1
    }
  }
  count_add(ctr + kCtrSegments, segs);
}

__global__ void queue_init_kernel(const uint32_t* __restrict__ chunk_start, int n_pairs,
                                  unsigned long long* __restrict__ queue) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) queue[0] = 0ull;
  if (j < n_pairs) queue[1 + j] = chunk_start[j + 1] - chunk_start[j];
}

// Batch latency state before the trace: stamps[0] = start, the per-pair
// stamps cleared, rays in flight per pair = its budget, keys per pair = 0
// (counted once key ids exist).  queue layout: [0] work head, [1 + j] chunks
// left, [1 + P + j] rays left, [1 + 2P + j] keys left; stamps: [0] start,
// [1 + j] pair j traced, [1 + P + j] pair j's keys validated.
__global__ void batch_stamp_init_kernel(SimConst C, unsigned long long* __restrict__ queue,
                                        unsigned long long* __restrict__ stamps) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int P = C.n_pairs;
  if (j == 0) stamps[0] = global_ns();
  if (j < P) {
    queue[1 + P + j] = (unsigned long long)(__ldg(C.pair_start + j + 1) - __ldg(C.pair_start + j));
    queue[1 + 2 * P + j] = 0ull;
    stamps[1 + j] = 0ull;
    stamps[1 + P + j] = 0ull;
  }
}

// pairs without keys have their paths validated as soon as validation starts
__global__ void pair_nokey_stamp_kernel(int n_pairs, const unsigned long long* __restrict__ keys_left,
                                        unsigned long long* __restrict__ stamps) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n_pairs && keys_left[j] == 0ull) stamps[1 + n_pairs + j] = global_ns();
}

}  // namespace

#define TRY(expr) NRT_CUDA_TRY(ctx, expr)

namespace {

struct Caps {
  int64_t cand = 1, keys = 1, table = 4096, paths = 1;
};

// Pipeline buffers.  Normal simulations allocate them for one call; a batch
// graph keeps them for every replay.
struct Work {
  Caps caps;
  Table T{};
  KeyState K{};
  uint32_t *spec_list = nullptr, *diff_list = nullptr;
  uint32_t *spec_cnt = nullptr, *spec_off = nullptr, *spec_best = nullptr;  // [keys]
  uint32_t *spec_cnt_t = nullptr, *spec_off_t = nullptr;  // tail item counts, offsets [keys]
  uint32_t* items = nullptr;  // specular (key, candidate) items [cand]
  SpecSlots sw{};             // refinement state of the specular waves
  uint2 *cand = nullptr, *cand2 = nullptr;
  uint32_t *cand_cnt = nullptr, *cand_off = nullptr;
  uint32_t *fs = nullptr, *fd = nullptr, *os = nullptr, *od = nullptr;  // per-tile key counts, scans
  uint64_t *sk0 = nullptr, *tk0 = nullptr;
  uint32_t *sv0 = nullptr, *tv = nullptr;
  PathRec* raw = nullptr;
  uint64_t *psk = nullptr, *ptk = nullptr;
  uint32_t *psi = nullptr, *pti = nullptr;
  unsigned long long* cnt = nullptr;  // key counts and work counters
  uint32_t* order = nullptr;          // launch order owned by this call (subset / batch)
};

// key counts and work-fetch counters in Work::cnt
enum { kCntSpec = 0, kCntDiff, kCntKeys, kCntFetchS, kCntFetchD, kCntItems, kCntN };

template <class T>
cudaError_t dalloc(T** p, int64_t n, cudaStream_t st) {
  return cudaMallocAsync((void**)p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), st);
}

nrt_status alloc_work(nrt_ctx* ctx, Work& W, const Caps& c, int64_t n_rows, cudaStream_t st) {
  W.caps = c;
  TRY(dalloc(&W.T.b, c.table, st));
  TRY(dalloc(&W.T.kid, c.table, st));
  W.T.mask = (uint64_t)c.table - 1;
  TRY(dalloc(&W.K.slot, c.keys, st));
  TRY(dalloc(&W.K.cur, c.keys, st));
  TRY(dalloc(&W.K.pos, c.keys, st));
  TRY(dalloc(&W.K.end, c.keys, st));
  TRY(dalloc(&W.spec_cnt, c.keys, st));
  TRY(dalloc(&W.spec_off, c.keys, st));
  TRY(dalloc(&W.spec_cnt_t, c.keys, st));
  TRY(dalloc(&W.spec_off_t, c.keys, st));
  TRY(dalloc(&W.spec_best, c.keys, st));
  TRY(dalloc(&W.items, c.cand, st));
  TRY(dalloc(&W.K.tries, c.keys, st));
  TRY(dalloc(&W.K.status, c.keys, st));
  TRY(dalloc(&W.spec_list, c.keys, st));
  TRY(dalloc(&W.diff_list, c.keys, st));
  TRY(dalloc(&W.cand, c.cand, st));
  TRY(dalloc(&W.cand2, c.cand, st));
  if (!W.cand_cnt) TRY(dalloc(&W.cand_cnt, n_rows, st));
  if (!W.cand_off) TRY(dalloc(&W.cand_off, n_rows, st));
  const int64_t n_tiles = (c.table + kSlotTile - 1) / kSlotTile;  // per-tile key counts
  TRY(dalloc(&W.fs, n_tiles, st));
  TRY(dalloc(&W.fd, n_tiles, st));
  TRY(dalloc(&W.os, n_tiles, st));
  TRY(dalloc(&W.od, n_tiles, st));
  TRY(dalloc(&W.sk0, c.keys, st));
  TRY(dalloc(&W.tk0, c.keys, st));
  TRY(dalloc(&W.sv0, c.keys, st));
  TRY(dalloc(&W.tv, c.keys, st));
  TRY(dalloc(&W.raw, c.paths, st));
  TRY(dalloc(&W.psk, c.paths, st));
  TRY(dalloc(&W.ptk, c.paths, st));
  TRY(dalloc(&W.psi, c.paths, st));
  TRY(dalloc(&W.pti, c.paths, st));
  TRY(dalloc(&W.cnt, kCntN, st));
  SpecSlots& Q = W.sw;
  Q.n = std::min<int64_t>(c.cand, kSpecSlots);
  TRY(dalloc(&Q.kid, Q.n, st));
  TRY(dalloc(&Q.rank, Q.n, st));
  TRY(dalloc(&Q.key, Q.n, st));
  TRY(dalloc(&Q.ctl, Q.n, st));
  TRY(dalloc(&Q.pl, 6 * kMaxDepth * Q.n, st));
  TRY(dalloc(&Q.im, 3 * kMaxDepth * Q.n, st));
  TRY(dalloc(&Q.hq, Q.n, st));
  TRY(dalloc(&Q.hd, Q.n, st));
  TRY(dalloc(&Q.q, 2 * Q.n, st));
  TRY(dalloc(&Q.qs, Q.n, st));
  TRY(dalloc(&Q.qa, 2 * Q.n, st));
  TRY(dalloc(&Q.qas, Q.n, st));
  TRY(dalloc(&Q.defer, c.cand, st));
  TRY(dalloc(&Q.hleft, c.keys, st));
  TRY(dalloc(&Q.wc, kWcN, st));
  return NRT_OK;
}

void release_work(Work& W, cudaStream_t st) {
  void* ptrs[] = {W.T.b, W.T.kid, W.K.slot, W.K.cur, W.K.pos, W.K.end, W.spec_cnt, W.spec_off,
                  W.spec_cnt_t, W.spec_off_t,
                  W.spec_best, W.items,
                  W.K.tries, W.K.status, W.spec_list, W.diff_list, W.cand,
                  W.cand2, W.cand_cnt, W.cand_off, W.fs, W.fd, W.os, W.od, W.sk0, W.tk0,
                  W.sv0, W.tv, W.raw, W.psk, W.ptk, W.psi, W.pti, W.cnt, W.order,
                  W.sw.kid, W.sw.rank, W.sw.key, W.sw.ctl, W.sw.pl, W.sw.im, W.sw.hq, W.sw.hd,
                  W.sw.q, W.sw.qs, W.sw.qa, W.sw.qas, W.sw.defer, W.sw.hleft, W.sw.wc};
  for (void* q : ptrs)
    if (q) cudaFreeAsync(q, st);
  W = Work();
}

// Result-owned buffers: records, counters, visibility and per-RX arrays once;
// the path buffers (re)sized to the caps when with_paths is set.
nrt_status alloc_result(nrt_result* r, const Caps& c, bool with_paths) {
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  const size_t nrec = (size_t)r->n_seg * r->n_traced;
  if (!r->ctr) TRY(dalloc(&r->ctr, kCtrCount, st));
  if (!r->rec_q) {
    TRY(dalloc(&r->rec_q, nrec, st));
    TRY(dalloc(&r->rec_n, nrec, st));
    TRY(dalloc(&r->rec_d, nrec, st));
    TRY(dalloc(&r->rec_i, nrec, st));
  }
  if (!r->vis && r->p.capture == NRT_CAPTURE_VIS)
    TRY(dalloc(&r->vis, (int64_t)r->n_rx_phys * r->vis_words, st));
  if (!r->power) TRY(dalloc(&r->power, r->n_rx, st));
  if (!r->power_part) TRY(dalloc(&r->power_part, (int64_t)r->n_rx * kPowerChunks, st));
  if (!r->rx_start_d) TRY(dalloc(&r->rx_start_d, r->n_rx, st));
  if (!r->rx_count_d) TRY(dalloc(&r->rx_count_d, r->n_rx, st));
  if (r->p.ray_labels && !r->labels) TRY(dalloc(&r->labels, r->n_traced, st));
  if (with_paths && r->p.keep_keys) {
    void* old[] = {r->key_hi, r->key_lo, r->key_tried, r->key_rep};
    for (void* q : old)
      if (q) cudaFreeAsync(q, st);
    r->key_cap = c.keys;
    TRY(dalloc(&r->key_hi, c.keys, st));
    TRY(dalloc(&r->key_lo, c.keys, st));
    TRY(dalloc(&r->key_tried, c.keys, st));
    TRY(dalloc(&r->key_rep, c.keys, st));
  }
  if (with_paths) {
    if (r->paths) cudaFreeAsync(r->paths, st);
    if (r->path_a) cudaFreeAsync(r->path_a, st);
    r->path_cap = c.paths;
    TRY(dalloc((PathRec**)&r->paths, c.paths, st));
    TRY(dalloc(&r->path_a, c.paths, st));
  }
  return NRT_OK;
}

// Launch order: rows sorted by the Morton code of their Fibonacci cell (batch:
// within each pair).  The full single-TX launch is cached in the context.
nrt_status make_order(nrt_result* r, const SimConst& C, const uint32_t* subset_d, Work& W,
                      const uint32_t** order) {
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t n = r->n_traced;
  const int sm = ctx->sm_count;
  if (C.launch == NRT_LAUNCH_DPS) {  // DPS order is already Morton order
    *order = nullptr;
    return NRT_OK;
  }
  const bool cacheable = !subset_d && !C.batch;
  if (cacheable && ctx->order_n == n && ctx->order) {
    *order = ctx->order;
    return NRT_OK;
  }
  uint64_t *ok, *tk;
  uint32_t *ov, *tv;
  TRY(dalloc(&ok, n, st));
  TRY(dalloc(&tk, n, st));
  TRY(dalloc(&ov, n, st));
  TRY(dalloc(&tv, n, st));
  order_key_kernel<<<blocks_for(n, 256, sm), 256, 0, st>>>(C, subset_d, n, r->p.n_rays, ok, ov); count_launch();
  radix_sort_pairs(ok, ov, tk, tv, n, C.batch ? 40 : 32, st);
  cudaFreeAsync(ok, st);
  cudaFreeAsync(tk, st);
  cudaFreeAsync(tv, st);
  if (cacheable) {
    if (ctx->order) cudaFreeAsync(ctx->order, st);
    ctx->order = ov;
    ctx->order_n = n;
  } else {
    W.order = ov;
  }
  *order = ov;
  return NRT_OK;
}

// Everything after the candidate count, with counts kept on the device so
// that the sequence can also be recorded into a CUDA graph.
nrt_status enqueue_rest(nrt_result* r, Work& W, const SceneView& S, const SimConst& C,
                        const uint32_t* order) {
  nrt_scene* sc = r->scene;
  nrt_ctx* ctx = sc->ctx;
  cudaStream_t st = ctx->stream;
  const int sm = ctx->sm_count;
  const int64_t n = r->n_traced;
  const Caps& c = W.caps;
  unsigned long long* ctr = r->ctr;
  Records R{r->rec_q, r->rec_n, r->rec_d, r->rec_i, n};

  TRY(cudaMemsetAsync(W.T.b, 0xFF, c.table * sizeof(Key128), st));
  TRY(cudaMemsetAsync(W.cnt, 0, kCntN * 8, st));
  EmitArgs A{};
  A.T = W.T;
  A.cand_cap = (uint64_t)c.cand;
  A.cand = W.cand;
  A.cand_off = W.cand_off;
  emit_kernel<kModeEmit><<<blocks_for(n, 256, sm), 256, 0, st>>>(S, C, r->rx, R, r->vis, order, A, ctr); count_launch();

  // key ids from the occupied slots, specular first, each type in launch
  // order of the key's lowest row
  const int64_t n_tiles = (c.table + kSlotTile - 1) / kSlotTile;
  slot_count_kernel<<<(unsigned)n_tiles, kSlotThreads, 0, st>>>(W.T, c.table, W.fs, W.fd); count_launch();
  scan_exclusive(W.fs, W.os, n_tiles, st);
  scan_exclusive(W.fd, W.od, n_tiles, st);
  key_count_kernel<<<1, 1, 0, st>>>(W.fs, W.fd, W.os, W.od, n_tiles, c.keys, W.cnt, ctr); count_launch();
  slot_assign_kernel<<<(unsigned)n_tiles, kSlotThreads, 0, st>>>(W.T, c.table, W.os, W.od, W.cnt,
                                                                W.K.slot, c.keys); count_launch();
  TRY(cudaMemcpyAsync(ctr + kCtrKeys, W.cnt + kCntKeys, 8, cudaMemcpyDeviceToDevice, st));
  // candidates sorted by (key id, row) once
  int row_bits = 1, kid_bits = 1;
  while ((1ll << row_bits) < n) ++row_bits;
  while ((1ll << kid_bits) <= c.keys) ++kid_bits;  // all-ones id field >= c.keys
  cand_key_kernel<<<blocks_for(c.cand, 256, sm), 256, 0, st>>>(W.T, W.cand, ctr + kCtrCands, c.cand,
                                                              row_bits, c.keys); count_launch();
  // the candidates are in ascending row order (offsets per row), so a stable
  // sort on the key-id bits alone leaves each run in ray order
  radix_sort_pairs(reinterpret_cast<uint64_t*>(W.cand), nullptr, reinterpret_cast<uint64_t*>(W.cand2),
                   nullptr, c.cand, row_bits + kid_bits, st, row_bits, ctr + kCtrCands);
  const SortedCand SC{reinterpret_cast<const uint64_t*>(W.cand), ctr + kCtrCands, c.cand, row_bits};
  TRY(cudaMemsetAsync(W.K.cur, 0, c.keys * sizeof(uint32_t), st));
  TRY(cudaMemsetAsync(W.K.pos, 0, c.keys * sizeof(uint32_t), st));
  TRY(cudaMemsetAsync(W.K.end, 0, c.keys * sizeof(uint32_t), st));
  TRY(cudaMemsetAsync(W.K.tries, 0, c.keys * sizeof(uint32_t), st));
  TRY(cudaMemsetAsync(W.K.status, 0, c.keys * sizeof(uint32_t), st));
  run_start_kernel<<<blocks_for(c.cand, 256, sm), 256, 0, st>>>(SC, W.K, c.keys); count_launch();

  // validation order of the keys; key ids are dense in [0, keys): the sort
  // takes the live count from the device and leaves the rest alone
  const int nj = C.batch ? C.n_pairs : r->n_rx_phys;
  int jb = 0;
  while ((1 << jb) < nj) ++jb;
  const int mb = 3 * std::min(sc->grid_bits, 10);  // spread3 keeps 10 bits per axis
  const int fb_spec = std::min(12, mb);  // specular: cells of 16 voxels per axis
  unsigned long long* pair_keys = C.batch ? r->queue + 1 + 2 * C.n_pairs : nullptr;
  val_order_kernel<<<blocks_for(c.keys, 256, sm), 256, 0, st>>>(S, R, W.T, W.K, W.cnt, W.sk0, W.sv0,
                                                               jb, mb, fb_spec, pair_keys); count_launch();
  radix_sort_pairs(W.sk0, W.sv0, W.tk0, W.tv, c.keys, 1 + jb + mb, st, 0, W.cnt + kCntKeys);
  split_lists_kernel<<<blocks_for(c.keys, 256, sm), 256, 0, st>>>(W.sv0, c.keys, W.cnt, W.spec_list,
                                                                 W.diff_list); count_launch();

  // LOS paths first, then candidates in ray-id order until one validates
  los_kernel<<<(nj + kTraceThreads - 1) / kTraceThreads, kTraceThreads, 0, st>>>(
      S, C, r->rx, W.raw, ctr, c.paths); count_launch();
  if (r->p.diffraction && sc->n_edges > 0) {
    diffraction_kernel<<<blocks_for(sc->n_edges * nj, kTraceThreads, sm, 8), kTraceThreads, 0, st>>>(
        S, C, r->rx, sc->edges, sc->n_edges, W.raw, ctr, c.paths); count_launch();
  }
  if (r->ev[4]) TRY(cudaEventRecord(r->ev[4], st));
  ValArgs V{};
  V.T = W.T;
  V.K = W.K;
  V.R = R;
  V.rx = r->rx;
  V.ray_of_row = nullptr;
  V.paths = W.raw;
  V.path_cap = c.paths;
  V.SC = SC;
  V.pair_keys = pair_keys;
  V.pair_ready = C.batch ? r->stamps + 1 + C.n_pairs : nullptr;
  if (C.batch) {
    pair_nokey_stamp_kernel<<<(C.n_pairs + 255) / 256, 256, 0, st>>>(C.n_pairs, pair_keys, r->stamps); count_launch();
  }
  // specular keys: every candidate an item (one pass), then the lowest valid
  // rank per key; diffuse keys: each key walks its candidates in ray order,
  // on the context's second stream so that the two validations overlap on
  // the device (they touch disjoint keys; paths and counters are taken by
  // atomics and the paths are sorted afterwards)
  TRY(cudaMemsetAsync(W.cnt + kCntFetchS, 0, (kCntN - kCntFetchS) * sizeof(unsigned long long), st));
  TRY(cudaEventRecord(ctx->fork, st));
  TRY(cudaStreamWaitEvent(ctx->aux, ctx->fork, 0));
  validate_diffuse_kernel<<<blocks_for(c.keys, kTraceThreads, sm, 6), kTraceThreads, 0, ctx->aux>>>(
      S, C, V, W.diff_list, W.cnt + kCntDiff, W.cnt + kCntFetchD, ctr); count_launch();
  TRY(cudaEventRecord(ctx->join, ctx->aux));
  TRY(cudaMemsetAsync(W.spec_cnt, 0, c.keys * sizeof(uint32_t), st));
  TRY(cudaMemsetAsync(W.spec_cnt_t, 0, c.keys * sizeof(uint32_t), st));
  spec_count_kernel<<<blocks_for(c.keys, 256, sm), 256, 0, st>>>(W.K, W.spec_list, W.cnt + kCntSpec,
                                                                C.rep_tries, W.spec_cnt, W.spec_cnt_t,
                                                                W.spec_best, W.sw.hleft); count_launch();
  scan_exclusive(W.spec_cnt, W.spec_off, c.keys, st);
  scan_exclusive(W.spec_cnt_t, W.spec_off_t, c.keys, st);
  spec_expand_kernel<<<blocks_for(c.keys * 32, 256, sm), 256, 0, st>>>(
      W.K, W.spec_list, W.cnt + kCntSpec, W.spec_cnt, W.spec_off, W.spec_cnt_t, W.spec_off_t,
      W.items, c.cand, W.cnt + kCntItems); count_launch();
  // the items in one persistent pass; or, on request, in waves
  // (spec_wave_*), the candidates still in slots to their end, then
  // whatever items the waves left: the first list from its fetch counter
  // on, then the deferred one
  if (r->p.spec_waves == 1) {
    const SpecSlots& Q = W.sw;
    TRY(cudaMemsetAsync(Q.ctl, 0, Q.n * sizeof(int4), st));
    TRY(cudaMemsetAsync(Q.wc, 0, kWcN * sizeof(unsigned long long), st));
    const int adv = blocks_for(Q.n, kTraceThreads, sm, 16);
    for (int w = 0; w < kSpecWaves; ++w) {
      spec_wave_advance_kernel<<<adv, kTraceThreads, 0, st>>>(S, C, V, Q, W.items, W.cnt + kCntItems,
                                                              W.spec_best, W.cnt + kCntFetchS, ctr,
                                                              w); count_launch();
      spec_wave_cast_kernel<<<sm * 8, kTraceThreads, 0, st>>>(S, C, Q, W.cnt + kCntFetchS,
                                                             W.cnt + kCntItems, ctr, w); count_launch();
    }
    spec_resume_kernel<<<blocks_for(Q.n, kTraceThreads, sm, 5), kTraceThreads, 0, st>>>(
        S, C, V, Q, W.spec_best, ctr); count_launch();
    validate_specular_items_kernel<<<blocks_for(c.cand, kTraceThreads, sm, 5), kTraceThreads, 0, st>>>(
        S, C, V, W.items, W.cnt + kCntItems, W.spec_best, W.cnt + kCntFetchS, ctr); count_launch();
    validate_specular_items_kernel<<<blocks_for(c.cand, kTraceThreads, sm, 5), kTraceThreads, 0, st>>>(
        S, C, V, Q.defer, Q.wc + kWcDefer, W.spec_best, Q.wc + kWcDeferFetch, ctr); count_launch();
  } else {
    validate_specular_items_kernel<<<blocks_for(c.cand, kTraceThreads, sm, 5), kTraceThreads, 0, st>>>(
        S, C, V, W.items, W.cnt + kCntItems, W.spec_best, W.cnt + kCntFetchS, ctr); count_launch();
  }
  spec_finish_kernel<<<blocks_for(c.keys, kTraceThreads, sm, 8), kTraceThreads, 0, st>>>(
      S, C, V, W.spec_list, W.cnt + kCntSpec, W.spec_best, ctr); count_launch();
  TRY(cudaStreamWaitEvent(st, ctx->join, 0));
  if (r->ev[5]) TRY(cudaEventRecord(r->ev[5], st));
  if (r->p.keep_keys) {
    key_summary_kernel<<<blocks_for(c.keys, 256, sm), 256, 0, st>>>(
        W.cnt + kCntKeys, W.K, W.T, C.batch ? nullptr : r->ray_of_row, r->key_hi, r->key_lo,
        r->key_tried, r->key_rep); count_launch();
  }
  if (r->p.ray_labels) {
    // proposal labels: rays that are members of a validated specular key
    EmitArgs L{};
    L.T = W.T;
    L.key_status = W.K.status;
    L.labels = r->labels;
    emit_kernel<kModeLabel><<<blocks_for(n, 256, sm), 256, 0, st>>>(S, C, r->rx, R, r->vis, order, L,
                                                                    ctr); count_launch();
  }

  // deterministic order of the paths (padding sorts last), ranges, field;
  // the representative field also holds edge indices of diffracted paths
  int path_bits = row_bits;
  if (r->p.diffraction)
    while ((1ll << path_bits) < sc->n_edges) ++path_bits;
  path_sortkey_kernel<<<blocks_for(c.paths, 256, sm), 256, 0, st>>>(W.raw, ctr + kCtrPaths, c.paths,
                                                                   path_bits, W.psk, W.psi); count_launch();
  radix_sort_pairs(W.psk, W.psi, W.ptk, W.pti, c.paths, path_bits + 12, st, 0, ctr + kCtrPaths);
  path_gather_kernel<<<blocks_for(c.paths, 256, sm), 256, 0, st>>>(W.raw, W.psi, ctr + kCtrPaths,
                                                                  c.paths, (PathRec*)r->paths); count_launch();
  rx_range_kernel<<<(r->n_rx + 63) / 64, 64, 0, st>>>(W.psk, ctr + kCtrPaths, c.paths, r->n_rx,
                                                      path_bits + 4, r->rx_start_d, r->rx_count_d); count_launch();
  if (sc->have_materials) {
    field_kernel<<<blocks_for(c.paths, 256, sm), 256, 0, st>>>((const PathRec*)r->paths, ctr + kCtrPaths,
                                                              c.paths, sc->mat, r->p.freq, r->p.pol,
                                                              path_frame(r), r->path_a); count_launch();
    power_partial_kernel<<<dim3(kPowerChunks, r->n_rx), 256, 0, st>>>(r->path_a, r->rx_start_d,
                                                                     r->rx_count_d, r->power_part); count_launch();
    power_sum_kernel<<<(r->n_rx + 127) / 128, 128, 0, st>>>(r->power_part, r->n_rx, r->power); count_launch();
  }
  return NRT_OK;
}

// Counters back to the host after a (possibly replayed) simulation.
nrt_status finish_result(nrt_result* r) {
  nrt_scene* sc = r->scene;
  nrt_ctx* ctx = sc->ctx;
  cudaStream_t st = ctx->stream;
  unsigned long long hc[kCtrCount];
  if (!r->rx_count) r->rx_count = new int64_t[r->n_rx]();
  if (!r->rx_start) r->rx_start = new int64_t[r->n_rx]();
  TRY(cudaMemcpyAsync(hc, r->ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(r->rx_count, r->rx_count_d, r->n_rx * 8, cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(r->rx_start, r->rx_start_d, r->n_rx * 8, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  TRY(cudaGetLastError());
  r->n_paths = std::min<int64_t>((int64_t)hc[kCtrPaths], r->path_cap);
#ifdef NRT_CHECK_BOUNDS
  {
    unsigned long long w = 0;
    TRY(cudaMemcpyFromSymbol(&w, g_dbg_word, sizeof(w)));
    if (w) {
      ctx->last_error = "bounds check failed: kernel code " + std::to_string(w >> 48) +
                        " index " + std::to_string(w & 0xFFFFFFFFFFFFull);
      return NRT_ERR_OVERFLOW;
    }
  }
#endif
  r->field_done = sc->have_materials;
  nrt_counters& c = r->counters;
  c.rays = r->n_traced;
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
  c.diffuse_casts = (int64_t)hc[kCtrDiffCasts];
  c.diffraction_casts = (int64_t)hc[kCtrDfrCasts];
  c.pruned_legs = (int64_t)hc[kCtrPrunedLegs];
  c.spec_items = (int64_t)hc[kCtrSpecItems];
  c.spec_ended_without_cast = (int64_t)hc[kCtrSpecNoCast];
  c.spec_ended_at_first_leg = (int64_t)hc[kCtrSpecLeg1];
  if (c.error_flags & (kErrHashFull | kErrCandFull | kErrPathFull | kErrKeyFull)) {
    ctx->last_error = "device buffer overflow (flags " +
                      std::to_string(c.error_flags) + ")";
    return NRT_ERR_OVERFLOW;
  }
  if (c.error_flags & kErrStack) {
    ctx->last_error = "traversal stack overflow";
    return NRT_ERR_OVERFLOW;
  }
  if (c.error_flags & kErrRecheck) {
    ctx->last_error = "internal: a specular representative refined twice came out differently";
    return NRT_ERR_STATE;
  }
  return NRT_OK;
}

// Prologue shared by normal runs and graph capture: counters, visibility,
// hit records, trace.
nrt_status enqueue_trace(nrt_result* r, const SceneView& S, const SimConst& C,
                         const uint32_t* subset_d, const uint32_t* order, bool do_vis) {
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  const int sm = ctx->sm_count;
  const int64_t n = r->n_traced;
  TRY(cudaMemsetAsync(r->ctr, 0, kCtrCount * sizeof(unsigned long long), st));
  const float margin = 0.8660254037844386f * r->scene->params.rho + r->scene->params.r_p;
  if (do_vis && r->p.capture == NRT_CAPTURE_VIS) {
    const int64_t total = (int64_t)r->n_rx_phys * r->vis_words * 32;
    vis_kernel<<<blocks_for(total, kTraceThreads, sm), kTraceThreads, 0, st>>>(
        S, C, r->rx, r->scene->dps_recv, r->vis, r->ctr, margin); count_launch();
  }
  if (r->ev[1]) TRY(cudaEventRecord(r->ev[1], st));
  TRY(cudaMemsetAsync(r->rec_i, 0xFF, (size_t)r->n_seg * n * sizeof(int2), st));
  Records R{r->rec_q, r->rec_n, r->rec_d, r->rec_i, n};
  if (r->ev[2]) TRY(cudaEventRecord(r->ev[2], st));
  if (C.batch) {
    batch_stamp_init_kernel<<<(r->n_pairs + 255) / 256, 256, 0, st>>>(C, r->queue, r->stamps); count_launch();
  }
  if (C.batch && r->schedule == 1) {
    queue_init_kernel<<<(r->n_pairs + 255) / 256, 256, 0, st>>>(r->chunk_start, r->n_pairs, r->queue); count_launch();
    trace_persistent_kernel<<<sm * 8, kTraceThreads, 0, st>>>(S, C, order, R, r->chunk_start,
                                                              r->packet, r->queue, r->stamps, r->ctr); count_launch();
  } else {
    trace_kernel<<<blocks_for(n, kTraceThreads, sm, 8), kTraceThreads, 0, st>>>(
        S, C, subset_d, order, R, r->ctr + kCtrRayFetch, r->ctr,
        C.batch ? r->queue + 1 + r->n_pairs : nullptr, C.batch ? r->stamps + 1 : nullptr); count_launch();
  }
  if (r->ev[3]) TRY(cudaEventRecord(r->ev[3], st));
  return NRT_OK;
}

}  // namespace

// One simulation into r (scene, params, receivers and rows set).  Without a
// hint, the one host round trip sizes the candidate buffers and the hash
// table from an exact count, and everything after it is enqueued without
// synchronising.  With a hint (the capacities of an earlier run of the same
// shape, with headroom) nothing waits for the host: every device write is
// bounded by the capacities and an overflow is flagged, and run_trace redoes
// a run that overflowed its hint with exact sizes.
nrt_status run_trace_once(nrt_result* r, const uint32_t* subset_d, const Caps* hint) {
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
  for (int e = 0; e < 8; ++e)
    if (!r->ev[e]) TRY(cudaEventCreate(&r->ev[e]));
  TRY(cudaEventRecord(r->ev[0], st));
  Caps c0;
  nrt_status rc = alloc_result(r, c0, false);  // records, counters, visibility
  if (rc != NRT_OK) return rc;
  Work W;
  TRY(dbg_set_caps(-1, 0, 0, 0, n, r->n_rx, st));
  const uint32_t* order = nullptr;
  rc = make_order(r, C, subset_d, W, &order);
  if (rc != NRT_OK) return rc;
  rc = enqueue_trace(r, S, C, subset_d, order, !r->vis_shared);
  if (rc != NRT_OK) return rc;

  // candidate count per ray -> offsets and sizes (the one host round trip)
  TRY(dalloc(&W.cand_cnt, n, st));
  TRY(dalloc(&W.cand_off, n, st));
  Records R{r->rec_q, r->rec_n, r->rec_d, r->rec_i, n};
  EmitArgs A{};
  A.cand_cnt = W.cand_cnt;
  emit_kernel<kModeCount><<<blocks_for(n, 256, sm), 256, 0, st>>>(S, C, r->rx, R, r->vis, order, A, r->ctr); count_launch();
  scan_exclusive(W.cand_cnt, W.cand_off, n, st);
  for (int e = 0; e < 2; ++e)
    if (!r->ev_gap[e]) TRY(cudaEventCreate(&r->ev_gap[e]));
  Caps c;
  if (hint) {
    c = *hint;
    TRY(cudaEventRecord(r->ev_gap[0], st));
  } else {
  unsigned long long cnt2[2] = {0, 0};
  TRY(cudaMemcpyAsync(&cnt2[0], r->ctr + kCtrCands, 8, cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&cnt2[1], r->ctr + kCtrLeaders, 8, cudaMemcpyDeviceToHost, st));
  TRY(cudaEventRecord(r->ev_gap[0], st));
  TRY(cudaStreamSynchronize(st));
  if (r->p.cand_capacity > 0 && (int64_t)cnt2[0] > r->p.cand_capacity) {
    ctx->last_error = "more path candidates than cand_capacity";
    release_work(W, st);
    return NRT_ERR_OVERFLOW;
  }
  if (cnt2[0] >= 0xFFFFFFFFull) {
    ctx->last_error = "more than 2^32 path candidates";
    release_work(W, st);
    return NRT_ERR_OVERFLOW;
  }
  c.cand = std::max<int64_t>((int64_t)cnt2[0], 1);
  c.keys = std::max<int64_t>((int64_t)cnt2[1], 1);  // distinct keys <= per-warp distinct keys
  c.table = r->p.key_capacity;
  if (c.table <= 0) {
    c.table = 1 << 12;
    while (c.table < c.keys + c.keys / 2) c.table <<= 1;
  }
  if (c.table & (c.table - 1)) {
    ctx->last_error = "key_capacity must be a power of two";
    release_work(W, st);
    return NRT_ERR_ARG;
  }
  if (c.table > kMaxTable) {
    ctx->last_error = "more path keys than a 2^31-slot hash table holds";
    release_work(W, st);
    return NRT_ERR_OVERFLOW;
  }
  c.keys = std::min<int64_t>(c.keys, c.table);
  c.paths = c.keys + (C.batch ? r->n_pairs : r->n_rx_phys) + diffraction_slots(r);
  }
  rc = alloc_result(r, c, true);
  if (rc == NRT_OK) rc = alloc_work(ctx, W, c, n, st);
  TRY(dbg_set_caps(c.table, c.keys, c.cand, c.paths, n, r->n_rx, st));
  TRY(cudaEventRecord(r->ev_gap[1], st));
  if (rc == NRT_OK) rc = enqueue_rest(r, W, S, C, order);
  if (rc != NRT_OK) {
    release_work(W, st);
    return rc;
  }
  TRY(cudaEventRecord(r->ev[6], st));
  TRY(cudaEventRecord(r->ev[7], st));
  release_work(W, st);
  rc = finish_result(r);
  if (rc == NRT_OK && hint && r->counters.candidates > c.cand) {
    // (more candidates than the hint's capacity: flagged by the kernels too)
    ctx->last_error = "device buffer overflow (candidates over the hint)";
    rc = NRT_ERR_OVERFLOW;
  }
  return rc;
}

// Capacity hints per simulation shape (scene, rows, receivers, capture,
// depth, diffuse, diffraction, launch): the last exact run's counts + 25%.
std::vector<int64_t> hint_key(const nrt_result* r) {
  return {(int64_t)(intptr_t)r->scene, r->n_traced, r->n_rx, (int64_t)r->p.capture,
          (int64_t)r->p.max_depth, (int64_t)r->p.diffuse, (int64_t)r->p.diffraction,
          (int64_t)r->p.launch};
}

nrt_status run_trace(nrt_result* r, const uint32_t* subset_d) {
  nrt_ctx* ctx = r->scene->ctx;
  const bool hinted = !r->n_pairs && r->p.cand_capacity <= 0 && r->p.key_capacity <= 0;
  const std::vector<int64_t> key = hinted ? hint_key(r) : std::vector<int64_t>{};
  if (hinted) {
    auto it = ctx->caps_hint.find(key);
    if (it != ctx->caps_hint.end()) {
      Caps h;
      h.cand = it->second[0];
      h.keys = it->second[1];
      h.table = it->second[2];
      h.paths = it->second[3];
      const nrt_status rc = run_trace_once(r, subset_d, &h);
      if (rc != NRT_ERR_OVERFLOW) return rc;
      ctx->caps_hint.erase(key);  // outgrown: size exactly once more
    }
  }
  const nrt_status rc = run_trace_once(r, subset_d, nullptr);
  if (rc == NRT_OK && hinted) {
    const int64_t cand = r->counters.candidates + r->counters.candidates / 4 + 1024;
    const int64_t keys = r->counters.keys + r->counters.keys / 4 + 1024;
    int64_t table = 1 << 12;
    while (table < keys + keys / 2) table <<= 1;
    if (table <= kMaxTable && cand < 0xFFFFFFFFll) {
      const int64_t k = std::min<int64_t>(keys, table);
      const int64_t paths = k + r->n_rx_phys + diffraction_slots(r);
      ctx->caps_hint[key] = {cand, k, table, paths};
    }
  }
  return rc;
}

nrt_status run_field(nrt_result* r) {
  nrt_scene* sc = r->scene;
  nrt_ctx* ctx = sc->ctx;
  cudaStream_t st = ctx->stream;
  if (!sc->have_materials) {
    r->field_done = false;
    return NRT_OK;  // field computed once materials are set
  }
  unsigned long long* np = r->ctr + kCtrPaths;
  field_kernel<<<blocks_for(r->path_cap, 256, ctx->sm_count), 256, 0, st>>>(
      (const PathRec*)r->paths, np, r->path_cap, sc->mat, r->p.freq, r->p.pol, path_frame(r),
      r->path_a); count_launch();
  power_partial_kernel<<<dim3(kPowerChunks, r->n_rx), 256, 0, st>>>(r->path_a, r->rx_start_d,
                                                                   r->rx_count_d, r->power_part); count_launch();
  power_sum_kernel<<<(r->n_rx + 127) / 128, 128, 0, st>>>(r->power_part, r->n_rx, r->power); count_launch();
  TRY(cudaGetLastError());
  r->field_done = true;
  return NRT_OK;
}

// ---------------------------------------------------------------- batch graph
// A batch plan: run once to size every buffer (with 25% headroom), keep the
// buffers, and record the whole simulation -- trace as one persistent launch,
// candidates, dedup, validation, field -- into a CUDA graph.  A replay takes
// new transmitter positions and launches the graph; the visibility matrix of
// the fixed receiver is computed once.
nrt_status batch_graph_build(nrt_result* r) {
  nrt_scene* sc = r->scene;
  nrt_ctx* ctx = sc->ctx;
  cudaStream_t st = ctx->stream;
  const SceneView S = scene_view(sc);
  SimConst C = make_const(r);
  Caps c;
  const nrt_counters& m = r->counters;
  c.cand = std::max<int64_t>(m.candidates + m.candidates / 4 + 1024, 1);
  c.keys = std::max<int64_t>(m.keys + m.keys / 4 + 1024, 1);
  c.table = 1 << 12;
  while (c.table < 2 * c.keys) c.table <<= 1;
  if (c.table > kMaxTable) {
    ctx->last_error = "more path keys than a 2^31-slot hash table holds";
    return NRT_ERR_OVERFLOW;
  }
  c.paths = c.keys + r->n_pairs + diffraction_slots(r);
  // path buffers sized by the caps (the calibration run's paths are dropped)
  nrt_status rc = alloc_result(r, c, true);
  if (rc != NRT_OK) return rc;
  Work* W = new Work();
  r->work = W;
  const uint32_t* order = nullptr;
  rc = make_order(r, C, nullptr, *W, &order);
  if (rc != NRT_OK) return rc;
  rc = alloc_work(ctx, *W, c, r->n_traced, st);
  if (rc != NRT_OK) return rc;
  TRY(dbg_set_caps(c.table, c.keys, c.cand, c.paths, r->n_traced, r->n_rx, st));
  TRY(cudaStreamSynchronize(st));
  for (int e = 0; e < 8; ++e) {
    if (r->ev[e]) cudaEventDestroy(r->ev[e]);
    r->ev[e] = nullptr;
  }
  cudaGraph_t g;
  launch_counter() = 0;
  TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
#ifdef NRT_CHECK_BOUNDS
  debug_capture(true);
#endif
  rc = enqueue_trace(r, S, C, nullptr, order, false);
  Records R{r->rec_q, r->rec_n, r->rec_d, r->rec_i, r->n_traced};
  if (rc == NRT_OK) {
    EmitArgs A{};
    A.cand_cnt = W->cand_cnt;
    emit_kernel<kModeCount><<<blocks_for(r->n_traced, 256, ctx->sm_count), 256, 0, st>>>(S, C, r->rx, R, r->vis, order, A, r->ctr); count_launch();
    scan_exclusive(W->cand_cnt, W->cand_off, r->n_traced, st);
    rc = enqueue_rest(r, *W, S, C, order);
  }
  cudaError_t e2 = cudaStreamEndCapture(st, &g);
#ifdef NRT_CHECK_BOUNDS
  debug_capture(false);
#endif
  r->graph_launches = launch_counter();
  if (rc != NRT_OK) return rc;
  if (e2 != cudaSuccess) {
    ctx->last_error = std::string("graph capture: ") + cudaGetErrorString(e2);
    return NRT_ERR_CUDA;
  }
  cudaError_t e3 = cudaGraphInstantiate(&r->graph, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) {
    ctx->last_error = std::string("graph instantiate: ") + cudaGetErrorString(e3);
    return NRT_ERR_CUDA;
  }
  return NRT_OK;
}

nrt_status batch_graph_replay(nrt_result* r, const float* tx_host) {
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  if (!r->graph) {
    ctx->last_error = "no batch graph";
    return NRT_ERR_STATE;
  }
  if (tx_host) {
    std::vector<float4> t(r->n_pairs);
    for (int j = 0; j < r->n_pairs; ++j)
      t[j] = make_float4(tx_host[3 * j], tx_host[3 * j + 1], tx_host[3 * j + 2], 0.f);
    TRY(cudaMemcpyAsync(r->tx_pair, t.data(), r->n_pairs * sizeof(float4), cudaMemcpyHostToDevice, st));
  }
  launch_counter() = 0;
  cudaEvent_t e0, e1;
  TRY(cudaEventCreate(&e0));
  TRY(cudaEventCreate(&e1));
  TRY(cudaEventRecord(e0, st));
  TRY(cudaGraphLaunch(r->graph, st));
  TRY(cudaEventRecord(e1, st));
  TRY(cudaEventSynchronize(e1));
  cudaEventElapsedTime(&r->graph_ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  launch_counter() = r->graph_launches;
  return finish_result(r);
}

// The trace phase alone (no visibility), timed with events on the stream;
// used by the autotuner to compare packet sizes and schedules.
nrt_status run_trace_phase(nrt_result* r, float* ms) {
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  const SceneView S = scene_view(r->scene);
  SimConst C = make_const(r);
  Work W;
  const uint32_t* order = nullptr;
  nrt_status rc = make_order(r, C, r->ray_of_row, W, &order);
  if (rc != NRT_OK) return rc;
  cudaEvent_t saved[8];
  for (int e = 0; e < 8; ++e) {
    saved[e] = r->ev[e];
    r->ev[e] = nullptr;
  }
  cudaEvent_t e0, e1;
  TRY(cudaEventCreate(&e0));
  TRY(cudaEventCreate(&e1));
  TRY(cudaEventRecord(e0, st));
  rc = enqueue_trace(r, S, C, r->ray_of_row, order, false);
  TRY(cudaEventRecord(e1, st));
  TRY(cudaEventSynchronize(e1));
  cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int e = 0; e < 8; ++e) r->ev[e] = saved[e];
  release_work(W, st);
  return rc;
}

void free_work(nrt_result* r) {
  if (r->graph) cudaGraphExecDestroy(r->graph);
  r->graph = nullptr;
  if (r->work) {
    Work* W = (Work*)r->work;
    release_work(*W, r->scene->ctx->stream);
    delete W;
    r->work = nullptr;
  }
}

nrt_status run_backward(nrt_result* r, const float* dL_dP_h, float* g_eps, float* g_sig,
                        float* g_sca) {
  return adjoint_to_host(r, dL_dP_h, nullptr, g_eps, g_sig, g_sca);
}

// Material gradient sum_p Re(W_p da_p/dtheta) into host arrays: W_p from the
// per-RX dL/dP (host) or from per-path weights already on the device.
nrt_status adjoint_to_host(nrt_result* r, const float* dL_dP_h, const double2* wpath_d,
                           float* g_eps, float* g_sig, float* g_sca) {
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
  if (dL_dP_h) TRY(cudaMemcpyAsync(dldp, dL_dP_h, r->n_rx * 4, cudaMemcpyHostToDevice, st));
  else TRY(cudaMemsetAsync(dldp, 0, r->n_rx * 4, st));
  TRY(cudaMemsetAsync(partial, 0, nb * 3 * L * 8, st));
  if (np > 0)
    adjoint_kernel<<<(unsigned)nb, kAdjThreads, 0, st>>>((const PathRec*)r->paths, np, sc->mat,
                                                         r->p.freq, r->p.pol, path_frame(r), dldp,
                                                         wpath_d, L, partial); count_launch();
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
