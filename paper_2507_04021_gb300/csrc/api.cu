// C ABI of libnrt (declarations and contracts in include/nrt.h).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "nrt_internal.h"

using namespace nrt;

namespace {

thread_local std::string g_err;

void free_dev(void* p) {
  if (p) cudaFree(p);
}

}  // namespace

// Handles are reference counted: a scene (or a proposal network) keeps its
// context alive and a result keeps its scene alive, so the *_free calls may
// come in any order.
void nrt::ctx_release(nrt_ctx* ctx) {
  if (--ctx->refs > 0) return;
  if (ctx->order) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->order);
  }
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->aux);
    cudaStreamDestroy(ctx->aux);
  }
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

namespace {

using nrt::ctx_release;

void scene_release(nrt_scene* s) {
  if (--s->refs > 0) return;
  cudaStreamSynchronize(s->ctx->stream);
  free_dev(s->disc_p);
  free_dev(s->disc_n);
  free_dev(s->dps_range);
  free_dev(s->dps_vox);
  free_dev(s->dps_recv);
  free_dev(s->dps_center);
  free_dev(s->label_box);
  free_dev(s->nodes);
  free_dev(s->mat);
  free_dev(s->edges);
  nrt_ctx* ctx = s->ctx;
  delete s;
  ctx_release(ctx);
}

__global__ void subset_check_kernel(const uint64_t* __restrict__ ids, int64_t n, int64_t n_rays,
                                    uint32_t* __restrict__ out, unsigned int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t v = ids[i];
    if ((int64_t)v >= n_rays || (i > 0 && ids[i - 1] == v)) atomicOr(bad, 1u);
    out[i] = (uint32_t)v;
  }
}

// Per-label materials from a device array [3][n_labels] into the scene's
// [3][256] table, each value brought into its range (eps_r >= 1, sigma >= 0,
// 0 <= S < 1; NaN goes to the lower bound); labels past n_labels get the
// host setter's defaults.  One block of 256 threads.
__global__ void materials_device_kernel(const float* __restrict__ in, int n_labels,
                                        float* __restrict__ mat) {
  const int l = threadIdx.x;
  float e = 1.0f, g = 0.0f, c = 0.0f;
  if (l < n_labels) {
    e = fmaxf(in[l], 1.0f);
    g = fmaxf(in[n_labels + l], 0.0f);
    c = fminf(fmaxf(in[2 * n_labels + l], 0.0f), 0.99999994f);
  }
  mat[l] = e;
  mat[256 + l] = g;
  mat[512 + l] = c;
}

__global__ void widen_kernel(const uint32_t* __restrict__ in, int64_t n, uint64_t* __restrict__ k,
                             uint32_t* __restrict__ v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    k[i] = in[i];
    v[i] = 0;
  }
}

}  // namespace

extern "C" {

const char* nrt_status_string(nrt_status s) {
  switch (s) {
    case NRT_OK: return "ok";
    case NRT_ERR_ARG: return "invalid argument";
    case NRT_ERR_CUDA: return "CUDA error";
    case NRT_ERR_OOM: return "out of device memory";
    case NRT_ERR_OVERFLOW: return "device buffer overflow";
    case NRT_ERR_TIMEOUT: return "device loop timeout";
    case NRT_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* nrt_last_error(const nrt_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_err.c_str();
}

void nrt_trace_params_default(nrt_trace_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->max_depth = 5;
  p->capture = NRT_CAPTURE_VIS;
  p->diffuse = 1;
  p->pol = NRT_POL_TE;
  p->kappa = 10;
  p->rep_tries = 0;
  p->record_hits = 1;
  p->n_rays = 1000000;
  p->r_rx = 0.1f;
  p->t_min = 1e-3f;
  p->t_a_deg = 1.0f;
  p->t_d = 0.01f;
  p->freq = 28e9f;
}

nrt_status nrt_create(nrt_ctx** out, int device, void* cuda_stream) {
  if (!out) return NRT_ERR_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    g_err = "no such CUDA device";
    return NRT_ERR_ARG;
  }
  nrt_ctx* c = new (std::nothrow) nrt_ctx();
  if (!c) return NRT_ERR_OOM;
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return NRT_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return NRT_ERR_CUDA;
    }
    c->own_stream = true;
  }
  // a second stream for work that may overlap on the device (the diffuse
  // and specular validations), joined back into the context stream by events
  if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return NRT_ERR_CUDA;
  }
  // keep freed stream-ordered memory cached in the pool between simulations
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  *out = c;
  return NRT_OK;
}

void nrt_destroy(nrt_ctx* ctx) {
  if (!ctx) return;
  ctx_release(ctx);
}

nrt_status nrt_set_wait_limit(nrt_ctx* ctx, int64_t polls) {
  if (!ctx || polls < 0) return NRT_ERR_ARG;
  ctx->wait_limit = polls;
  return NRT_OK;
}

nrt_status nrt_get_stream(const nrt_ctx* ctx, void** stream) {
  if (!ctx || !stream) return NRT_ERR_ARG;
  *stream = (void*)ctx->stream;
  return NRT_OK;
}

nrt_status nrt_sync(nrt_ctx* ctx) {
  if (!ctx) return NRT_ERR_ARG;
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return NRT_OK;
}

nrt_status nrt_scene_upload(nrt_ctx* ctx, const float* pos, const float* nrm,
                            const uint16_t* surf_label, const uint8_t* mat_label, int64_t n,
                            const nrt_scene_params* params, int inputs_on_device,
                            nrt_scene** out) {
  if (!ctx || !out || !params || !pos || !nrm || !surf_label || !mat_label) return NRT_ERR_ARG;
  if (n <= 0 || n >= (int64_t)1 << 31) {
    ctx->last_error = "point count must be in [1, 2^31)";
    return NRT_ERR_ARG;
  }
  if (!(params->rho > 0.f) || !(params->r_p > 0.f) || !(params->lambda_d > 0.f) ||
      !std::isfinite(params->rho) || !std::isfinite(params->r_p) ||
      !std::isfinite(params->lambda_d)) {
    ctx->last_error = "rho, r_p and lambda_d must be positive and finite";
    return NRT_ERR_ARG;
  }
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const float *pd = pos, *nd = nrm;
  const uint16_t* sd = surf_label;
  const uint8_t* md = mat_label;
  void* tmp = nullptr;
  if (!inputs_on_device) {
    const size_t bytes = n * (24 + 24 + 2 + 1) + 64;
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&tmp, bytes, st));
    char* b = (char*)tmp;
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(b, pos, n * 12, cudaMemcpyHostToDevice, st));
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(b + n * 12, nrm, n * 12, cudaMemcpyHostToDevice, st));
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(b + n * 24, surf_label, n * 2, cudaMemcpyHostToDevice, st));
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(b + n * 26, mat_label, n, cudaMemcpyHostToDevice, st));
    pd = (const float*)b;
    nd = (const float*)(b + n * 12);
    sd = (const uint16_t*)(b + n * 24);
    md = (const uint8_t*)(b + n * 26);
  }
  nrt_scene* s = new (std::nothrow) nrt_scene();
  if (!s) return NRT_ERR_OOM;
  s->ctx = ctx;
  ctx->refs++;
  s->n = n;
  s->params = *params;
  NRT_CUDA_TRY(ctx, cudaMalloc(&s->mat, 3 * 256 * sizeof(float)));
  nrt_status rc = build_scene(s, pd, nd, sd, md);
  if (tmp) cudaFreeAsync(tmp, st);
  if (rc != NRT_OK) {
    nrt_scene_free(s);
    return rc;
  }
  *out = s;
  return NRT_OK;
}

void nrt_scene_free(nrt_scene* s) {
  if (!s) return;
  scene_release(s);
}

nrt_status nrt_scene_info(const nrt_scene* s, int64_t* n_dps, float* bmin, float* build_ms) {
  if (!s) return NRT_ERR_ARG;
  if (n_dps) *n_dps = s->n_dps;
  if (bmin) memcpy(bmin, s->bmin, sizeof(s->bmin));
  if (build_ms) *build_ms = s->build_ms;
  return NRT_OK;
}

nrt_status nrt_scene_dps_read(const nrt_scene* s, int32_t* vox, int32_t* count, float* recv) {
  if (!s) return NRT_ERR_ARG;
  nrt_ctx* ctx = s->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t nd = s->n_dps;
  if (vox) NRT_CUDA_TRY(ctx, cudaMemcpyAsync(vox, s->dps_vox, nd * 12, cudaMemcpyDeviceToHost, st));
  std::vector<uint2> rg;
  std::vector<float4> rc;
  if (count) {
    rg.resize(nd);
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(rg.data(), s->dps_range, nd * 8, cudaMemcpyDeviceToHost, st));
  }
  if (recv) {
    rc.resize(nd);
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(rc.data(), s->dps_recv, nd * 16, cudaMemcpyDeviceToHost, st));
  }
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  for (int64_t d = 0; d < nd; ++d) {
    if (count) count[d] = (int32_t)rg[d].y;
    if (recv) {
      recv[3 * d] = rc[d].x;
      recv[3 * d + 1] = rc[d].y;
      recv[3 * d + 2] = rc[d].z;
    }
  }
  return NRT_OK;
}

nrt_status nrt_set_materials(nrt_scene* s, const float* eps_r, const float* sigma,
                             const float* scat, int n_labels) {
  if (!s || !eps_r || !sigma || !scat || n_labels <= 0 || n_labels > 256) return NRT_ERR_ARG;
  nrt_ctx* ctx = s->ctx;
  std::vector<float> h(3 * 256, 0.0f);
  for (int l = 0; l < 256; ++l) h[l] = 1.0f;
  for (int l = 0; l < n_labels; ++l) {
    if (!(eps_r[l] >= 1.0f) || !(sigma[l] >= 0.0f) || !(scat[l] >= 0.0f && scat[l] < 1.0f) ||
        !std::isfinite(eps_r[l]) || !std::isfinite(sigma[l])) {
      ctx->last_error = "material out of range (eps_r >= 1, sigma >= 0, 0 <= S < 1)";
      return NRT_ERR_ARG;
    }
    h[l] = eps_r[l];
    h[256 + l] = sigma[l];
    h[512 + l] = scat[l];
  }
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(s->mat, h.data(), h.size() * 4, cudaMemcpyHostToDevice,
                                    ctx->stream));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  s->n_labels = n_labels;
  s->have_materials = true;
  return NRT_OK;
}

nrt_status nrt_set_materials_device(nrt_scene* s, const float* mat, int n_labels) {
  if (!s || !mat || n_labels <= 0 || n_labels > 256) return NRT_ERR_ARG;
  nrt_ctx* ctx = s->ctx;
  int cur = 0;
  NRT_CUDA_TRY(ctx, cudaGetDevice(&cur));
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  materials_device_kernel<<<1, 256, 0, ctx->stream>>>(mat, n_labels, s->mat);
  const cudaError_t e = cudaGetLastError();
  cudaSetDevice(cur);
  NRT_CUDA_TRY(ctx, e);
  s->n_labels = n_labels;
  s->have_materials = true;
  return NRT_OK;
}

nrt_status nrt_scene_set_edges(nrt_scene* s, int64_t n_edges, const float* a, const float* b,
                               const float* n0, const float* n1, const uint8_t* m0,
                               const uint8_t* m1) {
  if (!s || n_edges < 0) return NRT_ERR_ARG;
  nrt_ctx* ctx = s->ctx;
  if (n_edges > 0 && (!a || !b || !n0 || !n1 || !m0 || !m1)) return NRT_ERR_ARG;
  if (n_edges > ((int64_t)1 << 24)) {
    ctx->last_error = "at most 2^24 edges";
    return NRT_ERR_ARG;
  }
  if (s->refs > 1) {
    ctx->last_error = "set the edges before tracing (results of this scene are alive)";
    return NRT_ERR_STATE;
  }
  std::vector<float4> h((size_t)4 * n_edges);
  for (int64_t e = 0; e < n_edges; ++e) {
    double v[4][3];
    const float* src[4] = {a + 3 * e, b + 3 * e, n0 + 3 * e, n1 + 3 * e};
    for (int q = 0; q < 4; ++q)
      for (int c = 0; c < 3; ++c) {
        if (!std::isfinite(src[q][c])) {
          ctx->last_error = "non-finite edge data";
          return NRT_ERR_ARG;
        }
        v[q][c] = src[q][c];
      }
    double ev[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
    const double len = std::sqrt(ev[0] * ev[0] + ev[1] * ev[1] + ev[2] * ev[2]);
    auto dot = [](const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    bool ok = len >= 1e-6;
    for (int q = 2; q < 4 && ok; ++q)
      ok = std::fabs(std::sqrt(dot(v[q], v[q])) - 1.0) <= 1e-3 &&
           std::fabs(dot(v[q], ev)) <= 1e-3 * len;
    if (ok) ok = std::fabs(dot(v[2], v[3])) <= 1.0 - 1e-6;
    if (!ok) {
      ctx->last_error = "edge " + std::to_string(e) +
                        ": short segment, or face normals not unit, not normal to the edge, or "
                        "not forming a wedge";
      return NRT_ERR_ARG;
    }
    float mb[2];  // material labels as raw bits in .w
    const int32_t mi[2] = {(int32_t)m0[e], (int32_t)m1[e]};
    memcpy(mb, mi, sizeof(mb));
    h[4 * e + 0] = make_float4(src[0][0], src[0][1], src[0][2], mb[0]);
    h[4 * e + 1] = make_float4(src[1][0], src[1][1], src[1][2], mb[1]);
    h[4 * e + 2] = make_float4(src[2][0], src[2][1], src[2][2], 0.0f);
    h[4 * e + 3] = make_float4(src[3][0], src[3][1], src[3][2], 0.0f);
  }
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  free_dev(s->edges);
  s->edges = nullptr;
  s->n_edges = 0;
  if (n_edges > 0) {
    NRT_CUDA_TRY(ctx, cudaMalloc(&s->edges, h.size() * sizeof(float4)));
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(s->edges, h.data(), h.size() * sizeof(float4),
                                      cudaMemcpyHostToDevice, ctx->stream));
    NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  s->n_edges = n_edges;
  return NRT_OK;
}

nrt_status nrt_trace(nrt_scene* s, const float* tx, const float* rx, int n_rx,
                     const nrt_trace_params* p_in, const uint32_t* ray_subset, int64_t n_subset,
                     int subset_on_device, nrt_result** out) {
  if (!s || !tx || !rx || !p_in || !out) return NRT_ERR_ARG;
  nrt_ctx* ctx = s->ctx;
  nrt_trace_params pl = *p_in;
  if (pl.launch == NRT_LAUNCH_DPS) {
    pl.n_rays = s->n_dps;  // one ray per DPS
  } else if (pl.launch != NRT_LAUNCH_FIB) {
    ctx->last_error = "unknown launch mode";
    return NRT_ERR_ARG;
  }
  const nrt_trace_params* p = &pl;
  if (n_rx <= 0 || n_rx > 256) {
    ctx->last_error = "n_rx must be in [1, 256]";
    return NRT_ERR_ARG;
  }
  if (p->max_depth < 1 || p->max_depth > kMaxDepth || p->n_rays <= 0 ||
      p->n_rays > (int64_t)0xFFFFFFFE || p->rep_tries < 0 || p->kappa < 0 ||
      !(p->freq > 0.f) || !(p->t_min >= 0.f) || (p->capture != 0 && p->capture != 1) ||
      p->pol < NRT_POL_TE || p->pol > NRT_POL_VECTOR || (p->diffraction != 0 && p->diffraction != 1) ||
      p->spec_waves < 0 || p->spec_waves > 2 || (p->capture == NRT_CAPTURE_SPHERE && p->diffuse)) {
    ctx->last_error = "invalid trace parameters";
    return NRT_ERR_ARG;
  }
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(tx[k])) return NRT_ERR_ARG;
  for (int k = 0; k < 3 * n_rx; ++k)
    if (!std::isfinite(rx[k])) return NRT_ERR_ARG;
  if (ray_subset && (n_subset <= 0 || n_subset > p->n_rays)) {
    ctx->last_error = "invalid ray subset size";
    return NRT_ERR_ARG;
  }
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  nrt_result* r = new (std::nothrow) nrt_result();
  if (!r) return NRT_ERR_OOM;
  r->scene = s;
  s->refs++;
  r->p = *p;
  r->n_rx = n_rx;
  r->n_rx_phys = n_rx;
  memcpy(r->tx, tx, sizeof(r->tx));
  std::vector<float4> rxh(n_rx);
  for (int j = 0; j < n_rx; ++j) rxh[j] = make_float4(rx[3 * j], rx[3 * j + 1], rx[3 * j + 2], 0.f);
  NRT_CUDA_TRY(ctx, cudaMalloc(&r->rx, n_rx * sizeof(float4)));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(r->rx, rxh.data(), n_rx * sizeof(float4),
                                    cudaMemcpyHostToDevice, st));
  if (ray_subset) {
    // rows are the subset in ascending ray-id order
    uint32_t* raw = nullptr;
    uint64_t *k = nullptr, *tk = nullptr;
    uint32_t *v = nullptr, *tv = nullptr;
    unsigned int* bad = nullptr;
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&raw, n_subset * 4, st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&k, n_subset * 8, st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&tk, n_subset * 8, st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&v, n_subset * 4, st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&tv, n_subset * 4, st));
    NRT_CUDA_TRY(ctx, cudaMallocAsync(&bad, 4, st));
    NRT_CUDA_TRY(ctx, cudaMemsetAsync(bad, 0, 4, st));
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(raw, ray_subset, n_subset * 4,
                                      subset_on_device ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice,
                                      st));
    const int g = (int)std::min<int64_t>((n_subset + 255) / 256, 4096);
    widen_kernel<<<g, 256, 0, st>>>(raw, n_subset, k, v);
    radix_sort_pairs(k, v, tk, tv, n_subset, 32, st);
    NRT_CUDA_TRY(ctx, cudaMalloc(&r->ray_of_row, n_subset * 4));
    subset_check_kernel<<<g, 256, 0, st>>>(k, n_subset, p->n_rays, r->ray_of_row, bad);
    unsigned int bh = 0;
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(&bh, bad, 4, cudaMemcpyDeviceToHost, st));
    NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    cudaFreeAsync(raw, st);
    cudaFreeAsync(k, st);
    cudaFreeAsync(tk, st);
    cudaFreeAsync(v, st);
    cudaFreeAsync(tv, st);
    cudaFreeAsync(bad, st);
    if (bh) {
      ctx->last_error = "ray subset has ids >= n_rays or duplicates";
      nrt_result_free(r);
      return NRT_ERR_ARG;
    }
    r->n_traced = n_subset;
  } else {
    r->n_traced = p->n_rays;
  }
  nrt_status rc = run_trace(r, r->ray_of_row);
  if (rc != NRT_OK) {
    nrt_result_free(r);
    return rc;
  }
  *out = r;
  return NRT_OK;
}

void nrt_result_free(nrt_result* r) {
  if (!r) return;
  cudaStreamSynchronize(r->scene->ctx->stream);
  free_work(r);
  free_dev(r->rx);
  free_dev(r->ray_of_row);
  free_dev(r->tx_pair);
  free_dev(r->pair_start);
  free_dev(r->pair_rays);
  free_dev(r->chunk_start);
  free_dev(r->stamps);
  free_dev(r->queue);
  cudaStream_t st = r->scene->ctx->stream;
  void* pool_ptrs[] = {r->rec_q, r->rec_n, r->rec_d, r->rec_i, r->vis, r->paths,
                       r->path_a, r->power, r->power_part, r->ctr, r->rx_start_d, r->rx_count_d, r->labels,
                       r->key_hi, r->key_lo, r->key_tried, r->key_rep};
  for (void* q : pool_ptrs)
    if (q) cudaFreeAsync(q, st);
  for (int e = 0; e < 8; ++e)
    if (r->ev[e]) cudaEventDestroy(r->ev[e]);
  for (int e = 0; e < 2; ++e)
    if (r->ev_gap[e]) cudaEventDestroy(r->ev_gap[e]);
  delete[] r->rx_count;
  delete[] r->rx_start;
  nrt_scene* s = r->scene;
  delete r;
  scene_release(s);
}

nrt_status nrt_result_counts(const nrt_result* r, int64_t* n_paths_per_rx, nrt_counters* c) {
  if (!r) return NRT_ERR_ARG;
  if (n_paths_per_rx)
    for (int j = 0; j < r->n_rx; ++j) n_paths_per_rx[j] = r->rx_count[j];
  if (c) *c = r->counters;
  return NRT_OK;
}

nrt_status nrt_result_times(const nrt_result* r, float* ms) {
  if (!r || !ms) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (!r->ev[7]) {  // graph replay: one device time for the whole simulation
    for (int k = 0; k < 8; ++k) ms[k] = 0.0f;
    ms[6] = r->graph_ms;
    return NRT_OK;
  }
  NRT_CUDA_TRY(ctx, cudaEventSynchronize(r->ev[7]));
  auto el = [&](int a, int b) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r->ev[a], r->ev[b]);
    return t;
  };
  ms[0] = el(0, 1);
  ms[1] = 0.0f;
  ms[2] = el(2, 3);
  ms[3] = el(3, 4);
  ms[4] = el(4, 5);
  ms[5] = el(5, 6);
  ms[6] = el(0, 7);
  ms[7] = 0.0f;
  if (r->ev_gap[0] && r->ev_gap[1]) cudaEventElapsedTime(&ms[7], r->ev_gap[0], r->ev_gap[1]);
  return NRT_OK;
}

nrt_status nrt_paths_read(const nrt_result* r, const nrt_path_view* v) {
  if (!r || !v) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  const int64_t np = r->n_paths;
  std::vector<PathRec> P(np);
  std::vector<float2> a(np);
  cudaStream_t st = ctx->stream;
  if (np > 0) {
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(P.data(), r->paths, np * sizeof(PathRec),
                                      cudaMemcpyDeviceToHost, st));
    if (r->field_done)
      NRT_CUDA_TRY(ctx, cudaMemcpyAsync(a.data(), r->path_a, np * sizeof(float2),
                                        cudaMemcpyDeviceToHost, st));
  }
  std::vector<uint32_t> rays, pstart;
  if (r->ray_of_row && np > 0) {
    rays.resize(r->n_traced);
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(rays.data(), r->ray_of_row, r->n_traced * 4,
                                      cudaMemcpyDeviceToHost, st));
  }
  if (r->n_pairs > 0) {
    pstart.resize(r->n_pairs + 1);
    NRT_CUDA_TRY(ctx, cudaMemcpyAsync(pstart.data(), r->pair_start, pstart.size() * 4,
                                      cudaMemcpyDeviceToHost, st));
  }
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  for (int64_t i = 0; i < np; ++i) {
    const PathRec& p = P[i];
    const int k = (p.jtk >> 9) & 7;
    if (v->key_hi) v->key_hi[i] = p.hi;
    if (v->key_lo) v->key_lo[i] = p.lo;
    const bool dfr = (p.jtk >> 12) & 1;  // diffracted: rep is the edge index
    uint32_t rep = p.rep;
    if (!dfr && rep != kNone && r->ray_of_row) rep = rays[rep];
    if (!dfr && rep != kNone && r->n_pairs > 0) rep -= pstart[p.jtk & 0xFF];  // ray id within its pair
    if (v->rep) v->rep[i] = rep;
    if (v->rx) v->rx[i] = (int32_t)(p.jtk & 0xFF);
    if (v->type) v->type[i] = dfr ? 2 : (int32_t)((p.jtk >> 8) & 1);
    if (v->k) v->k[i] = k;
    const uint64_t mats = (uint64_t)p.mats_lo | ((uint64_t)p.mats_hi << 32);
    const int nm = dfr ? 2 : k;  // material / cosine entries
    for (int m = 0; m < 5; ++m) {
      if (v->pts)
        for (int c = 0; c < 3; ++c) v->pts[15 * i + 3 * m + c] = m < k ? p.pts[3 * m + c] : 0.f;
      if (v->mats) v->mats[5 * i + m] = m < nm ? (uint8_t)((mats >> (8 * m)) & 0xFF) : 0;
      if (v->cos_theta) v->cos_theta[5 * i + m] = m < nm ? p.cosv[m] : 0.f;
    }
    if (v->geo) v->geo[i] = p.geo;
    if (v->tau) v->tau[i] = (float)((double)p.length / 299792458.0);
    if (v->normal)
      for (int c = 0; c < 3; ++c) v->normal[3 * i + c] = p.nd[c];
    if (v->a) {
      v->a[2 * i] = r->field_done ? a[i].x : 0.f;
      v->a[2 * i + 1] = r->field_done ? a[i].y : 0.f;
    }
  }
  return NRT_OK;
}

nrt_status nrt_keys_read(const nrt_result* r, uint64_t* key_hi, uint64_t* key_lo, uint32_t* tried,
                         uint32_t* rep) {
  if (!r || !key_hi || !key_lo || !tried || !rep) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (!r->key_hi) {
    ctx->last_error = "key summaries were not requested (trace parameter keep_keys)";
    return NRT_ERR_STATE;
  }
  const int64_t n = std::min<int64_t>(r->counters.keys, r->key_cap);
  cudaStream_t st = ctx->stream;
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(key_hi, r->key_hi, n * 8, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(key_lo, r->key_lo, n * 8, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(tried, r->key_tried, n * 4, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(rep, r->key_rep, n * 4, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return NRT_OK;
}

nrt_status nrt_ray_labels_read(const nrt_result* r, uint8_t* labels) {
  if (!r || !labels) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (!r->labels) {
    ctx->last_error = "ray labels were not requested (trace parameter ray_labels)";
    return NRT_ERR_STATE;
  }
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(labels, r->labels, r->n_traced, cudaMemcpyDeviceToHost,
                                    ctx->stream));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return NRT_OK;
}

nrt_status nrt_hits_read(const nrt_result* r, int32_t* idx, int32_t* dps, float* q, float* n,
                         float* t) {
  if (!r) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t rows = r->n_traced, S = r->n_seg, nrec = rows * S;
  std::vector<float4> hq(nrec), hn(nrec), hd(nrec);
  std::vector<int2> hi(nrec);
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(hq.data(), r->rec_q, nrec * 16, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(hn.data(), r->rec_n, nrec * 16, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(hd.data(), r->rec_d, nrec * 16, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(hi.data(), r->rec_i, nrec * 8, cudaMemcpyDeviceToHost, st));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  for (int64_t row = 0; row < rows; ++row) {
    bool dead = false;
    for (int64_t s = 0; s < S; ++s) {
      const int64_t a = s * rows + row, o = row * S + s;
      const bool hit = !dead && hi[a].x >= 0;
      if (!hit) dead = true;
      if (idx) idx[o] = hit ? hi[a].x : -1;
      int dv;
      memcpy(&dv, &hd[a].w, 4);
      if (dps) dps[o] = hit ? dv : -1;
      if (q) {
        q[3 * o] = hit ? hq[a].x : 0.f;
        q[3 * o + 1] = hit ? hq[a].y : 0.f;
        q[3 * o + 2] = hit ? hq[a].z : 0.f;
      }
      if (n) {
        n[3 * o] = hit ? hn[a].x : 0.f;
        n[3 * o + 1] = hit ? hn[a].y : 0.f;
        n[3 * o + 2] = hit ? hn[a].z : 0.f;
      }
      if (t) t[o] = hit ? hq[a].w : 0.f;
    }
  }
  return NRT_OK;
}

nrt_status nrt_vis_read(const nrt_result* r, uint32_t* bits) {
  if (!r || !bits) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (!r->vis) {
    ctx->last_error = "no visibility matrix (sphere capture)";
    return NRT_ERR_STATE;
  }
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(bits, r->vis, (size_t)r->n_rx * r->vis_words * 4,
                                    cudaMemcpyDeviceToHost, ctx->stream));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return NRT_OK;
}

nrt_status nrt_trace_batch(nrt_scene* s, const float* tx, const float* rx, const int64_t* budget,
                           int n_pairs, const nrt_trace_params* p, const nrt_batch_opts* opts,
                           nrt_result** out) {
  if (!s || !tx || !rx || !budget || !p || !out) return NRT_ERR_ARG;
  nrt_ctx* ctx = s->ctx;
  if (n_pairs < 1 || n_pairs > 256) {
    ctx->last_error = "n_pairs must be in [1, 256]";
    return NRT_ERR_ARG;
  }
  if (p->capture != NRT_CAPTURE_VIS || p->max_depth < 1 || p->max_depth > kMaxDepth ||
      p->rep_tries < 0 || p->kappa < 0 || !(p->freq > 0.f) ||
      p->pol < NRT_POL_TE || p->pol > NRT_POL_VECTOR ||
      (p->diffraction != 0 && p->diffraction != 1) || p->spec_waves < 0 || p->spec_waves > 2) {
    ctx->last_error = "invalid batch trace parameters (visibility capture required)";
    return NRT_ERR_ARG;
  }
  nrt_batch_opts o{64, 1, 0, 0};
  if (opts) o = *opts;
  if ((o.packet != 32 && o.packet != 64 && o.packet != 128) || (o.schedule != 0 && o.schedule != 1)) {
    ctx->last_error = "packet must be 32, 64 or 128 and schedule 0 or 1";
    return NRT_ERR_ARG;
  }
  int64_t total = 0, maxb = 0;
  std::vector<uint32_t> start(n_pairs + 1), cstart(n_pairs + 1);
  std::vector<float4> txp(n_pairs);
  for (int j = 0; j < n_pairs; ++j) {
    if (budget[j] < 1 || budget[j] >= ((int64_t)1 << 31)) {
      ctx->last_error = "ray budgets must be in [1, 2^31)";
      return NRT_ERR_ARG;
    }
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(tx[3 * j + k])) return NRT_ERR_ARG;
    start[j] = (uint32_t)total;
    cstart[j] = (uint32_t)(j == 0 ? 0 : cstart[j]);
    total += budget[j];
    maxb = std::max(maxb, budget[j]);
    txp[j] = make_float4(tx[3 * j], tx[3 * j + 1], tx[3 * j + 2], 0.f);
  }
  if (total >= ((int64_t)1 << 32) - 1) {
    ctx->last_error = "total rays of a batch must stay below 2^32";
    return NRT_ERR_ARG;
  }
  start[n_pairs] = (uint32_t)total;
  uint64_t ch = 0;
  for (int j = 0; j < n_pairs; ++j) {
    cstart[j] = (uint32_t)ch;
    ch += (uint64_t)((budget[j] + o.packet - 1) / o.packet);
  }
  cstart[n_pairs] = (uint32_t)ch;
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  nrt_result* r = new (std::nothrow) nrt_result();
  if (!r) return NRT_ERR_OOM;
  r->scene = s;
  s->refs++;
  if (p->launch != NRT_LAUNCH_FIB) {
    ctx->last_error = "batches use the Fibonacci launch";
    delete r;
    s->refs--;
    return NRT_ERR_ARG;
  }
  r->p = *p;
  r->p.n_rays = maxb;
  r->n_pairs = n_pairs;
  r->n_rx = n_pairs;
  r->n_rx_phys = 1;
  r->n_traced = total;
  r->packet = o.packet;
  r->schedule = o.schedule;
  memcpy(r->tx, tx, sizeof(r->tx));
  const float4 rxh = make_float4(rx[0], rx[1], rx[2], 0.f);
  nrt_status rc = NRT_OK;
  auto fail = [&](nrt_status e) {
    nrt_result_free(r);
    return e;
  };
  if (cudaMalloc(&r->rx, sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&r->tx_pair, n_pairs * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&r->pair_start, (n_pairs + 1) * 4) != cudaSuccess ||
      cudaMalloc(&r->pair_rays, n_pairs * 8) != cudaSuccess ||
      cudaMalloc(&r->chunk_start, (n_pairs + 1) * 4) != cudaSuccess ||
      cudaMalloc(&r->stamps, (2 * n_pairs + 1) * 8) != cudaSuccess ||
      cudaMalloc(&r->queue, (3 * n_pairs + 1) * 8) != cudaSuccess) {
    ctx->last_error = "device allocation failed";
    return fail(NRT_ERR_OOM);
  }
  cudaMemcpyAsync(r->rx, &rxh, sizeof(float4), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(r->tx_pair, txp.data(), n_pairs * sizeof(float4), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(r->pair_start, start.data(), (n_pairs + 1) * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(r->pair_rays, budget, n_pairs * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(r->chunk_start, cstart.data(), (n_pairs + 1) * 4, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(r->stamps, 0, (2 * n_pairs + 1) * 8, st);
  cudaMemsetAsync(r->queue, 0, (3 * n_pairs + 1) * 8, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(NRT_ERR_CUDA);
  rc = run_trace(r, nullptr);
  if (rc != NRT_OK) return fail(rc);
  if (o.use_graph) {
    r->vis_shared = true;  // the fixed RX's visibility matrix is kept, not recomputed
    rc = batch_graph_build(r);
    if (rc == NRT_OK) rc = batch_graph_replay(r, nullptr);
    if (rc != NRT_OK) return fail(rc);
  }
  *out = r;
  return NRT_OK;
}

nrt_status nrt_batch_replay(nrt_result* r, const float* tx) {
  if (!r) return NRT_ERR_ARG;
  if (!r->graph) {
    r->scene->ctx->last_error = "batch was not recorded into a graph (use_graph = 0)";
    return NRT_ERR_STATE;
  }
  return batch_graph_replay(r, tx);
}

nrt_status nrt_batch_times(const nrt_result* r, double* pair_ms, float* total_ms,
                           double* pair_paths_ms) {
  if (!r || r->n_pairs <= 0) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  const int P = r->n_pairs;
  std::vector<unsigned long long> t(2 * P + 1);
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(t.data(), r->stamps, t.size() * 8, cudaMemcpyDeviceToHost,
                                    ctx->stream));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  // a stamp that was never written (0, or before the start) reads as -1
  auto since = [&](unsigned long long v) {
    return v >= t[0] && v != 0ull ? (double)(v - t[0]) * 1e-6 : -1.0;
  };
  if (pair_ms)
    for (int j = 0; j < P; ++j) pair_ms[j] = since(t[1 + j]);
  if (pair_paths_ms)
    for (int j = 0; j < P; ++j) pair_paths_ms[j] = since(t[1 + P + j]);
  if (total_ms) {
    float ms[8];
    nrt_result_times(r, ms);
    *total_ms = ms[6];
  }
  return NRT_OK;
}

nrt_status nrt_autotune_batch(nrt_result* r, const int32_t* packets, const int32_t* schedules,
                              int n_cfg, int repeats, float* ms, int32_t* best) {
  if (!r || !packets || !schedules || !ms || n_cfg < 1 || r->n_pairs <= 0) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (r->graph) {
    ctx->last_error = "autotune a batch before recording it into a graph";
    return NRT_ERR_STATE;
  }
  const int keep_p = r->packet, keep_s = r->schedule;
  float best_ms = 1e30f;
  int best_i = 0;
  std::vector<uint32_t> cstart(r->n_pairs + 1);
  std::vector<uint32_t> start(r->n_pairs + 1);
  NRT_CUDA_TRY(ctx, cudaMemcpy(start.data(), r->pair_start, (r->n_pairs + 1) * 4,
                               cudaMemcpyDeviceToHost));
  for (int i = 0; i < n_cfg; ++i) {
    if ((packets[i] != 32 && packets[i] != 64 && packets[i] != 128) ||
        (schedules[i] != 0 && schedules[i] != 1))
      return NRT_ERR_ARG;
    uint64_t ch = 0;
    for (int j = 0; j < r->n_pairs; ++j) {
      cstart[j] = (uint32_t)ch;
      ch += (uint64_t)((start[j + 1] - start[j] + packets[i] - 1) / packets[i]);
    }
    cstart[r->n_pairs] = (uint32_t)ch;
    NRT_CUDA_TRY(ctx, cudaMemcpy(r->chunk_start, cstart.data(), cstart.size() * 4,
                                 cudaMemcpyHostToDevice));
    r->packet = packets[i];
    r->schedule = schedules[i];
    float t_min = 1e30f;
    for (int k = 0; k < std::max(repeats, 1); ++k) {
      float t = 0.f;
      nrt_status rc = run_trace_phase(r, &t);
      if (rc != NRT_OK) return rc;
      t_min = std::min(t_min, t);
    }
    ms[i] = t_min;
    if (t_min < best_ms) {
      best_ms = t_min;
      best_i = i;
    }
  }
  (void)keep_p;
  (void)keep_s;
  r->packet = packets[best_i];
  r->schedule = schedules[best_i];
  uint64_t ch = 0;
  for (int j = 0; j < r->n_pairs; ++j) {
    cstart[j] = (uint32_t)ch;
    ch += (uint64_t)((start[j + 1] - start[j] + r->packet - 1) / r->packet);
  }
  cstart[r->n_pairs] = (uint32_t)ch;
  NRT_CUDA_TRY(ctx, cudaMemcpy(r->chunk_start, cstart.data(), cstart.size() * 4,
                               cudaMemcpyHostToDevice));
  if (best) *best = best_i;
  return NRT_OK;
}

nrt_status nrt_field(nrt_result* r) {
  if (!r) return NRT_ERR_ARG;
  if (!r->scene->have_materials) {
    r->scene->ctx->last_error = "materials not set";
    return NRT_ERR_STATE;
  }
  return run_field(r);
}

nrt_status nrt_field_read(const nrt_result* r, float* power) {
  if (!r || !power) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (!r->field_done) {
    ctx->last_error = "field not computed (set materials, then nrt_field)";
    return NRT_ERR_STATE;
  }
  std::vector<double> h(r->n_rx);
  NRT_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), r->power, r->n_rx * 8, cudaMemcpyDeviceToHost,
                                    ctx->stream));
  NRT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  for (int j = 0; j < r->n_rx; ++j) power[j] = (float)h[j];
  return NRT_OK;
}

nrt_status nrt_field_read_device(const nrt_result* r, double* power) {
  if (!r || !power) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (!r->field_done) {
    ctx->last_error = "field not computed (set materials, then nrt_field)";
    return NRT_ERR_STATE;
  }
  int cur = 0;
  NRT_CUDA_TRY(ctx, cudaGetDevice(&cur));
  NRT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const cudaError_t e = cudaMemcpyAsync(power, r->power, (size_t)r->n_rx * sizeof(double),
                                        cudaMemcpyDeviceToDevice, ctx->stream);
  cudaSetDevice(cur);
  NRT_CUDA_TRY(ctx, e);
  return NRT_OK;
}

nrt_status nrt_backward(nrt_result* r, const float* dL_dpower, float* g_eps, float* g_sigma,
                        float* g_scat) {
  if (!r || !dL_dpower) return NRT_ERR_ARG;
  if (!r->scene->have_materials || !r->field_done) {
    r->scene->ctx->last_error = "backward needs materials and a computed field";
    return NRT_ERR_STATE;
  }
  return run_backward(r, dL_dpower, g_eps, g_sigma, g_scat);
}

}  // extern "C"
