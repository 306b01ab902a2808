// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/nrt.h"
#include "nrt_device.cuh"

struct nrt_ctx {
  int refs = 1;  // the caller's handle + one per live scene
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  int sm_count = 0;
  // launch order of the full Fibonacci launch, cached per ray count
  uint32_t* order = nullptr;
  int64_t order_n = 0;
  // polls of a bounded device wait before it gives up (0 = the default)
  int64_t wait_limit = 0;
  // second stream for overlapping work, forked from and joined into `stream`
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // capacity hints (candidates, keys, table slots, paths) per simulation shape
  std::map<std::vector<int64_t>, std::array<int64_t, 4>> caps_hint;
};

struct nrt_scene {
  int refs = 1;  // the caller's handle + one per live result
  nrt_ctx* ctx = nullptr;
  int64_t n = 0;
  int64_t n_dps = 0;
  nrt_scene_params params{};
  float bmin[3] = {0, 0, 0};
  int grid_bits = 0;  // Morton bits per axis
  // device arrays (owned)
  float4* disc_p = nullptr;
  float4* disc_n = nullptr;
  uint2* dps_range = nullptr;
  int32_t* dps_vox = nullptr;  // [n_dps][3]
  float4* dps_recv = nullptr;  // reception point (xyz)
  float4* dps_center = nullptr;  // local origin of the DPS's disc positions
  float4* label_box = nullptr;   // [65536][2]: box (lo, hi) of each surface label's discs
  float4* nodes = nullptr;     // 4-wide BVH: 8 float4 (128 B) per node
  int64_t n_nodes4 = 0;
  int root = 0;
  float build_ms = 0.0f;
  // materials
  int n_labels = 0;
  float* mat = nullptr;  // device [3][256]: eps_r, sigma, S
  bool have_materials = false;
  // edges (diffraction): 4 float4 per edge -- (a, m0 bits), (b, m1 bits), (n0, 0), (n1, 0)
  float4* edges = nullptr;
  int64_t n_edges = 0;
};

struct nrt_result {
  nrt_scene* scene = nullptr;
  nrt_trace_params p{};
  int n_rx = 0;        // receivers of the path keys and of the power (batch: pairs)
  int n_rx_phys = 0;   // physical receivers
  int n_pairs = 0;     // > 0: batch of TX-RX pairs
  int64_t n_traced = 0;  // rows (rays traced)
  int n_seg = 0;
  float tx[3] = {0, 0, 0};
  // device arrays
  float4* rx = nullptr;            // physical receivers
  uint32_t* ray_of_row = nullptr;  // nullptr: row == ray id
  float4* tx_pair = nullptr;       // batch: TX of each pair
  uint32_t* pair_start = nullptr;  // batch: first row of each pair [n_pairs + 1]
  int64_t* pair_rays = nullptr;    // batch: Fibonacci N of each pair
  uint32_t* chunk_start = nullptr; // batch: first work chunk of each pair [n_pairs + 1]
  // batch latency (ns, globaltimer): [0] trace start, [1 + j] pair j traced,
  // [1 + P + j] pair j's last key validated
  unsigned long long* stamps = nullptr;
  // batch: [0] work queue head, [1 + j] chunks left, [1 + P + j] rays left,
  // [1 + 2P + j] keys left of pair j
  unsigned long long* queue = nullptr;
  int packet = 64;     // rays per work item of the persistent trace
  int schedule = 1;    // 0 static grid-stride, 1 persistent work queue
  float4* rec_q = nullptr;   // [n_seg][n_traced]: q.xyz, segment length
  float4* rec_n = nullptr;   // normal.xyz, cos_in
  float4* rec_d = nullptr;   // outgoing direction.xyz, dps (bits)
  int2* rec_i = nullptr;     // point index (-1 miss), labels
  uint32_t* vis = nullptr;   // [n_rx_phys][vis_words]
  int64_t vis_words = 0;
  bool vis_shared = false;   // vis owned by a batch plan
  // paths (sorted)
  int64_t n_paths = 0;
  int64_t path_cap = 0;
  void* paths = nullptr;     // PathRec[path_cap]
  float2* path_a = nullptr;  // [path_cap]
  uint8_t* labels = nullptr;  // [n_traced] proposal labels (ray_labels)
  // per-key validation summaries (keep_keys), key_cap entries
  uint64_t* key_hi = nullptr;
  uint64_t* key_lo = nullptr;
  uint32_t* key_tried = nullptr;
  uint32_t* key_rep = nullptr;
  int64_t key_cap = 0;
  double* power = nullptr;   // [n_rx]
  double* power_part = nullptr;  // [n_rx][64] partial sums of the power reduction
  int64_t* rx_start_d = nullptr;  // [n_rx] device ranges of the sorted paths
  int64_t* rx_count_d = nullptr;
  int64_t* rx_count = nullptr;  // host copies
  int64_t* rx_start = nullptr;
  // counters
  unsigned long long* ctr = nullptr;  // device counters
  nrt_counters counters{};
  cudaEvent_t ev[8] = {};
  cudaEvent_t ev_gap[2] = {};  // around the host sizing round trip
  bool field_done = false;
  // graph mode: pipeline buffers and the instantiated graph, kept for replays
  void* work = nullptr;
  cudaGraphExec_t graph = nullptr;
  float graph_ms = 0.0f;
  int64_t graph_launches = 0;  // kernel nodes recorded into the graph
};

namespace nrt {

// counters slots in nrt_result::ctr
enum Ctr : int {
  kCtrSegments = 0,
  kCtrVisCasts,
  kCtrLosCasts,
  kCtrValCasts,
  kCtrDiffCasts,  // diffuse validation shadow casts (also in kCtrValCasts)
  kCtrCands,
  kCtrKeys,
  kCtrPaths,
  kCtrProbeMax,
  kCtrErr,
  kCtrKeysSpec,
  kCtrKeysDiff,
  kCtrPending,
  kCtrLeaders,
  kCtrCompact,
  kCtrDfrCasts,  // edge visibility casts (diffraction)
  kCtrRayFetch,  // trace: rays handed out to lanes
  kCtrPrunedLegs,  // specular refinement legs ended by the label-box test
  kCtrSpecItems,   // specular (key, candidate) items refined
  kCtrSpecNoCast,  // of which ended before any cast (side check, label box)
  kCtrSpecLeg1,    // of which ended at the first leg's cast
  kCtrCount
};

// Path record (device, 144 bytes)
struct alignas(16) PathRec {
  uint64_t hi, lo;
  uint32_t rep;   // representative row (LOS: kNone)
  uint32_t jtk;   // rx | type << 8 | k << 9
  float geo;
  float length;
  float cosv[5];
  uint32_t mats_lo, mats_hi;  // 5 material labels, one byte each
  float pts[15];
  float nd[3];    // diffuse: surface normal at the scatter point (facing the incoming ray)
  float pad[3];
};
static_assert(sizeof(PathRec) == 144, "PathRec layout");

// material label of interaction m of a path record
__device__ __forceinline__ int path_mat(const PathRec& P, int m) {
  const uint64_t mats = (uint64_t)P.mats_lo | ((uint64_t)P.mats_hi << 32);
  return (int)((mats >> (8 * m)) & 0xFF);
}

// Per-interaction factors of a path (the EM readings of the field: effective
// roughness R = sqrt(1 - S^2) on a specular reflection, S on the diffuse last
// interaction, times the Fresnel coefficient): c Gamma (scalar models: pol's
// coefficient; vector model: TE then TM) and, for the adjoint, c dGamma/deta
// and dc/dS Gamma.  mat holds [3][256] eps_r, sigma, S per label.  Shared by
// the field kernel and both adjoint kernels.
__device__ __forceinline__ void interaction_factors(const PathRec& p, int m, int k, int diffuse,
                                                    const float* __restrict__ mat, float freq,
                                                    int pol, float2* D, float2* dDe, float2* dDs) {
  const int l = path_mat(p, m);
  const float2 eta = permittivity(mat[l], mat[256 + l], freq);
  const float Sl = mat[512 + l];
  const bool last_d = diffuse && m == k - 1;
  const float R = sqrtf(fmaxf(0.0f, 1.0f - Sl * Sl));
  const float c = last_d ? Sl : R;
  const float dc = last_d ? 1.0f : (R > 0.0f ? -Sl / R : 0.0f);
  const int n = pol == 2 ? 2 : 1;
  for (int t = 0; t < n; ++t) {
    const int pp = pol == 2 ? t : pol;
    const float2 G = fresnel(eta, p.cosv[m], pp);
    D[t] = cscale(c, G);
    if (dDe) dDe[t] = cscale(c, dfresnel(eta, p.cosv[m], pp));
    if (dDs) dDs[t] = cscale(dc, G);
  }
}

void scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t st);
// n = capacity of the buffers (sets the grid); n_dev, if given, is the live
// count on the device (at most n): only the first *n_dev entries are sorted
// and the rest of keys/vals is left undefined
void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, int64_t n,
                      int bits, cudaStream_t st, int lo_bit = 0,
                      const unsigned long long* n_dev = nullptr);

SceneView scene_view(const nrt_scene* s);

// polls a bounded tensor-core wait makes before giving up (mlp.cu)
long long wait_limit(const nrt_ctx* ctx);

// drop one reference to a context (frees it with the last one)
void ctx_release(nrt_ctx* ctx);

// kernels launched on this host thread since the last reset
int64_t& launch_counter();
inline void count_launch_n(int64_t n = 1) { launch_counter() += n; }
#ifdef NRT_CHECK_BOUNDS
// debug builds: synchronise after every launch and report the first failing
// launch site on stderr
void debug_launch_check(const char* file, int line);
// stream capture in progress on this thread: skip the per-launch synchronisation
void debug_capture(bool on);
#define count_launch(...) (count_launch_n(__VA_ARGS__), debug_launch_check(__FILE__, __LINE__))
#else
#define count_launch(...) count_launch_n(__VA_ARGS__)
#endif

// scene.cu
nrt_status collapse_bvh4(nrt_scene* s, int64_t n_int, cudaStream_t st);
nrt_status build_scene(nrt_scene* s, const float* pos_d, const float* nrm_d, const uint16_t* surf_d,
                       const uint8_t* mat_d);
// trace.cu / paths.cu
nrt_status run_trace(nrt_result* r, const uint32_t* subset_d);
nrt_status batch_graph_build(nrt_result* r);
nrt_status run_trace_phase(nrt_result* r, float* ms);
nrt_status batch_graph_replay(nrt_result* r, const float* tx_host);
void free_work(nrt_result* r);
nrt_status run_field(nrt_result* r);
nrt_status run_backward(nrt_result* r, const float* dL_dP, float* g_eps, float* g_sig,
                        float* g_sca);
nrt_status adjoint_to_host(nrt_result* r, const float* dL_dP_h, const double2* wpath_d,
                           float* g_eps, float* g_sig, float* g_sca);

}  // namespace nrt

#define NRT_CUDA_TRY(ctx, expr)                                                   \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      (ctx)->last_error = std::string(#expr) + ": " + cudaGetErrorString(_e);     \
      return _e == cudaErrorMemoryAllocation ? NRT_ERR_OOM : NRT_ERR_CUDA;        \
    }                                                                             \
  } while (0)
