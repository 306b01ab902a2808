// nrt_backward_noalloc: the adjoint of the received power (the same result as
// nrt_backward) computed without allocating any device memory.
//
// Some callers cannot allocate: code that records work into a CUDA graph
// (cudaMalloc is not allowed while a stream is being captured), real-time
// loops that must not hit the allocator's device-wide synchronisation, and
// hosts whose framework owns every byte of device memory.  They pass device
// pointers for the input (dL/dP per receiver) and the output (the gradient),
// and the per-block partial sums of the reduction go to a fixed array that
// lives in the library's image on every GPU that loads it.
#include "nrt_internal.h"

namespace {

constexpr int kNaBlocks = 1024;     // fixed grid: paths are visited grid-stride
constexpr int kNaThreads = 256;
constexpr int kNaMaxLabels = 256;   // the largest label count accepted

}  // namespace

// Block partials [kNaBlocks][3][kNaMaxLabels] doubles: 6 MiB per device,
// held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_adjoint_scratch[kNaBlocks * 3 * kNaMaxLabels];

namespace {

using namespace nrt;

// The scratch array's device address, resolved once per device.  In host
// code g_adjoint_scratch names a host-side stand-in, never the device memory.
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};

// Per path: d|a|^2 / d(eps_r, sigma, S) of each interaction's label, scaled
// by 2 dL/dP_j and accumulated per block in shared memory.  The path count
// is read on the device (capped at the record capacity), so work recorded
// into a CUDA graph follows later traces of the same result.  Every block
// writes all 3 * n_labels of its partial slots, so nothing left by an
// earlier call is ever read.
__global__ void __launch_bounds__(kNaThreads)
    adjoint_noalloc_kernel(const PathRec* __restrict__ P, const unsigned long long* __restrict__ n_p,
                           int64_t cap, const float* __restrict__ mat, float freq, int pol,
                           const float* __restrict__ dLdP, int n_labels,
                           double* __restrict__ partial) {
  __shared__ double acc[3 * kNaMaxLabels];
  for (int i = threadIdx.x; i < 3 * n_labels; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const int64_t n = min((int64_t)*n_p, cap);
  const float ks = (float)(1.0 / (2.0 * 3.14159265358979323846 * kEps0)) / freq;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const PathRec p = P[i];
    const int k = (p.jtk >> 9) & 7;
    const int diffuse = (p.jtk >> 8) & 1;
    const int j = p.jtk & 0xFF;
    float2 fac[kMaxDepth], dfe[kMaxDepth], dfs[kMaxDepth];
    int labs[kMaxDepth];
    for (int m = 0; m < k; ++m) {
      labs[m] = path_mat(p, m);
      interaction_factors(p, m, k, diffuse, mat, freq, pol, &fac[m], &dfe[m], &dfs[m]);
    }
    float2 a = make_float2(p.geo, 0.0f);
    for (int m = 0; m < k; ++m) a = cmul(a, fac[m]);
    const float w = 2.0f * dLdP[j];
    const float2 ca = cconj(a);
    for (int m = 0; m < k; ++m) {
      float2 oth = make_float2(p.geo, 0.0f);
      for (int q = 0; q < k; ++q)
        if (q != m) oth = cmul(oth, fac[q]);
      const float2 de = cmul(ca, cmul(oth, dfe[m]));
      const float2 ds = cmul(ca, cmul(oth, dfs[m]));
      atomicAdd(&acc[labs[m]], (double)(w * de.x));
      atomicAdd(&acc[n_labels + labs[m]], (double)(w * de.y * ks));
      atomicAdd(&acc[2 * n_labels + labs[m]], (double)(w * ds.x));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * n_labels; i += blockDim.x)
    partial[(int64_t)blockIdx.x * 3 * kNaMaxLabels + i] = acc[i];
}

__global__ void adjoint_noalloc_reduce(const double* __restrict__ partial, int n_labels,
                                       float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n_labels) return;
  double s = 0.0;
  for (int b = 0; b < kNaBlocks; ++b) s += partial[(int64_t)b * 3 * kNaMaxLabels + t];
  out[t] = (float)s;
}

}  // namespace

extern "C" nrt_status nrt_backward_noalloc(nrt_result* r, const float* dL_dpower, float* grad) {
  if (!r || !dL_dpower || !grad) return NRT_ERR_ARG;
  nrt_scene* sc = r->scene;
  nrt_ctx* ctx = sc->ctx;
  if (!sc->have_materials) {
    ctx->last_error = "backward needs materials (nrt_set_materials)";
    return NRT_ERR_STATE;
  }
  if (r->p.pol == NRT_POL_VECTOR || r->p.diffraction) {
    ctx->last_error =
        "nrt_backward_noalloc supports the scalar polarisation models without diffraction only";
    return NRT_ERR_ARG;
  }
  const int L = sc->n_labels;
  if (L <= 0 || L > kNaMaxLabels) {
    ctx->last_error = "nrt_backward_noalloc accepts at most 256 material labels";
    return NRT_ERR_ARG;
  }
  if (ctx->device < 0 || ctx->device >= kMaxDevices) {
    ctx->last_error = "nrt_backward_noalloc supports device ordinals below 64";
    return NRT_ERR_ARG;
  }
  // the launches need the context's device current; the caller's current
  // device is put back before returning
  int prev = -1;
  NRT_CUDA_TRY(ctx, cudaGetDevice(&prev));
  if (prev != ctx->device) NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  nrt_status rc = NRT_OK;
  // one-time set-up per device (with that device current): the device
  // address of the scratch array
  double* scratch = g_scratch_addr[ctx->device];
  cudaError_t e = cudaSuccess;
  if (!scratch) {
    e = cudaGetSymbolAddress((void**)&scratch, g_adjoint_scratch);
    if (e == cudaSuccess) g_scratch_addr[ctx->device] = scratch;
  }
  if (e == cudaSuccess) {
    cudaStream_t st = ctx->stream;
    adjoint_noalloc_kernel<<<kNaBlocks, kNaThreads, 0, st>>>(
        (const PathRec*)r->paths, r->ctr + kCtrPaths, r->path_cap, sc->mat, r->p.freq, r->p.pol,
        dL_dpower, L, scratch);
    adjoint_noalloc_reduce<<<(3 * L + 127) / 128, 128, 0, st>>>(scratch, L, grad);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    ctx->last_error = std::string("nrt_backward_noalloc: ") + cudaGetErrorString(e);
    rc = NRT_ERR_CUDA;
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return rc;
}
