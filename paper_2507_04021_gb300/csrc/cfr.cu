// Channel frequency response and the Eq. 5 loss (Sec. III-B).
//
// H_j(f_n) = sum over RX j's paths of a_p exp(-j 2 pi f_n tau_p) at N equally
// spaced frequencies f_n = f_c + (n - (N-1)/2) B/(N-1) around the centre
// frequency f_c at which the coefficients a_p are computed.  At 28 GHz a path
// accumulates ~1e3 cycles, so the phase is formed from the cycle count
// f_n tau_p in FP64, reduced to its fractional part exactly, and only then
// turned into a phasor (FP32 sincospi of a value in [-1, 1]); within a run of
// 16 frequencies the phasor advances by FP32 products with the per-path step,
// re-anchored from FP64 at every run.  The sums are FP64, in a fixed
// two-level order (the same result on every run).
//
// Eq. 5, L_j = |h_j - h^_j|^2 / |h^_j|^2 on the CIR h = IDFT(H), equals the
// same ratio on the CFR (Parseval), so it is evaluated on H; its material
// gradient is sum_p Re(W_p da_p/dtheta) with W_p = (2 w_j / |H^_j|^2) conj(g_p),
// g_p = sum_n (H_j(f_n) - H^_j(f_n)) exp(+j 2 pi f_n tau_p), contracted by the
// adjoint kernel.
#include <vector>

#include "nrt_internal.h"

namespace {

using namespace nrt;

constexpr int kCfrThreads = 256;
constexpr int kCfrGroup = 16;   // frequencies per block
constexpr int kCfrChunks = 64;  // blocks per (RX, frequency group)
constexpr double kC0 = 299792458.0;

// e^{-j 2 pi cyc} from a cycle count: exact FP64 reduction to [-1/2, 1/2]
__device__ __forceinline__ float2 phasor(double cyc) {
  const double fr = cyc - rint(cyc);
  float s, c;
  sincospif((float)(2.0 * fr), &s, &c);
  return make_float2(c, -s);
}

// Within a run of kCfrGroup frequencies the phasor advances by a fixed step
// e^{-j 2 pi df tau}; FP32 products drift by ~1e-6 rad over a run, and every
// run starts again from the exact FP64 cycle count.
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void tau_kernel(const PathRec* __restrict__ P, int64_t n, double* __restrict__ tau) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    tau[i] = (double)P[i].length / kC0;
}

__global__ void __launch_bounds__(kCfrThreads)
    cfr_partial_kernel(const float2* __restrict__ a, const double* __restrict__ tau,
                       const int64_t* __restrict__ start, const int64_t* __restrict__ count,
                       int n_freq, double f0, double df, double2* __restrict__ partial) {
  __shared__ double sh[kCfrThreads / 32][2];
  const int j = blockIdx.y, n0 = blockIdx.z * kCfrGroup;
  const int nf = min(kCfrGroup, n_freq - n0);
  const int64_t b = start[j], m = count[j];
  double re[kCfrGroup], im[kCfrGroup];
#pragma unroll
  for (int q = 0; q < kCfrGroup; ++q) re[q] = im[q] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 av = a[b + i];
    const double t = tau[b + i];
    float2 e = phasor((f0 + n0 * df) * t);
    const float2 step = phasor(df * t);
#pragma unroll
    for (int q = 0; q < kCfrGroup; ++q) {
      if (q >= nf) break;
      const float2 v = cmulf(av, e);
      re[q] += (double)v.x;
      im[q] += (double)v.y;
      e = cmulf(e, step);
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = 0; q < nf; ++q) {
    double x = re[q], y = im[q];
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
      y += __shfl_xor_sync(0xFFFFFFFFu, y, o);
    }
    __syncthreads();
    if (lane == 0) {
      sh[w][0] = x;
      sh[w][1] = y;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tx = 0.0, ty = 0.0;
      for (int k = 0; k < kCfrThreads / 32; ++k) {
        tx += sh[k][0];
        ty += sh[k][1];
      }
      partial[((int64_t)j * n_freq + n0 + q) * kCfrChunks + blockIdx.x] = make_double2(tx, ty);
    }
  }
}

__global__ void cfr_sum_kernel(const double2* __restrict__ partial, int64_t n, double2* __restrict__ H) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = 0.0, y = 0.0;
  for (int c = 0; c < kCfrChunks; ++c) {
    const double2 v = partial[i * kCfrChunks + c];
    x += v.x;
    y += v.y;
  }
  H[i] = make_double2(x, y);
}

// W_p = coef_j conj(g_p), g_p = sum_n dH_j(f_n) exp(+j 2 pi f_n tau_p)
__global__ void cfr_weight_kernel(const PathRec* __restrict__ P, const double* __restrict__ tau,
                                  int64_t n, const double2* __restrict__ dH,
                                  const double* __restrict__ coef, int n_freq, double f0, double df,
                                  double2* __restrict__ W) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = P[i].jtk & 0xFF;
    const double t = tau[i];
    const float2 step = phasor(df * t);
    double gx = 0.0, gy = 0.0;
    for (int q0 = 0; q0 < n_freq; q0 += kCfrGroup) {
      float2 e = phasor((f0 + q0 * df) * t);  // exp(-j ...); its conjugate is used
      float sx = 0.f, sy = 0.f;
      for (int q = q0; q < min(n_freq, q0 + kCfrGroup); ++q) {
        const double2 d = dH[(int64_t)j * n_freq + q];
        sx += (float)d.x * e.x + (float)d.y * e.y;
        sy += (float)d.y * e.x - (float)d.x * e.y;
        e = cmulf(e, step);
      }
      gx += (double)sx;
      gy += (double)sy;
    }
    W[i] = make_double2(coef[j] * gx, -coef[j] * gy);
  }
}

inline unsigned grid_for_n(int64_t n, int sm) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm * 16));
}

#define TRY(expr) NRT_CUDA_TRY(ctx, expr)

// H on the device (n_rx x n_freq double2) and tau per path
nrt_status cfr_device(nrt_result* r, double bandwidth, int n_freq, double2** H_out,
                      double** tau_out) {
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t np = r->n_paths;
  const double df = bandwidth / (n_freq - 1);
  const double f0 = (double)r->p.freq - 0.5 * (n_freq - 1) * df;
  double* tau = nullptr;
  double2 *partial = nullptr, *H = nullptr;
  TRY(cudaMallocAsync(&tau, std::max<int64_t>(np, 1) * 8, st));
  TRY(cudaMallocAsync(&partial, (size_t)r->n_rx * n_freq * kCfrChunks * sizeof(double2), st));
  TRY(cudaMallocAsync(&H, (size_t)r->n_rx * n_freq * sizeof(double2), st));
  TRY(cudaMemsetAsync(partial, 0, (size_t)r->n_rx * n_freq * kCfrChunks * sizeof(double2), st));
  if (np > 0) {
    tau_kernel<<<grid_for_n(np, ctx->sm_count), 256, 0, st>>>((const PathRec*)r->paths, np, tau);
    count_launch();
    const dim3 grid(kCfrChunks, r->n_rx, (n_freq + kCfrGroup - 1) / kCfrGroup);
    cfr_partial_kernel<<<grid, kCfrThreads, 0, st>>>(r->path_a, tau, r->rx_start_d, r->rx_count_d,
                                                     n_freq, f0, df, partial);
    count_launch();
  }
  const int64_t nh = (int64_t)r->n_rx * n_freq;
  cfr_sum_kernel<<<(unsigned)((nh + 127) / 128), 128, 0, st>>>(partial, nh, H);
  count_launch();
  cudaFreeAsync(partial, st);
  TRY(cudaGetLastError());
  *H_out = H;
  *tau_out = tau;
  return NRT_OK;
}

nrt_status check_cfr_args(nrt_result* r, double bandwidth, int n_freq) {
  if (!r) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  if (n_freq < 2 || n_freq > 65536 || !(bandwidth > 0.0)) {
    ctx->last_error = "CFR needs n_freq >= 2 and a positive bandwidth";
    return NRT_ERR_ARG;
  }
  if (!r->field_done) {
    ctx->last_error = "CFR needs the path coefficients (nrt_set_materials, nrt_field)";
    return NRT_ERR_STATE;
  }
  return NRT_OK;
}

}  // namespace

extern "C" {

nrt_status nrt_cfr(nrt_result* r, double bandwidth, int32_t n_freq, double* H_host) {
  nrt_status rc = check_cfr_args(r, bandwidth, n_freq);
  if (rc != NRT_OK) return rc;
  if (!H_host) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  double2* H = nullptr;
  double* tau = nullptr;
  rc = cfr_device(r, bandwidth, n_freq, &H, &tau);
  if (rc != NRT_OK) return rc;
  TRY(cudaMemcpyAsync(H_host, H, (size_t)r->n_rx * n_freq * sizeof(double2),
                      cudaMemcpyDeviceToHost, st));
  cudaFreeAsync(H, st);
  cudaFreeAsync(tau, st);
  TRY(cudaStreamSynchronize(st));
  return NRT_OK;
}

nrt_status nrt_cfr_backward(nrt_result* r, double bandwidth, int32_t n_freq,
                            const double* H_target, const float* rx_weight, double* loss,
                            float* g_eps, float* g_sig, float* g_sca) {
  nrt_status rc = check_cfr_args(r, bandwidth, n_freq);
  if (rc != NRT_OK) return rc;
  if (!H_target || !rx_weight) return NRT_ERR_ARG;
  nrt_ctx* ctx = r->scene->ctx;
  cudaStream_t st = ctx->stream;
  const int n_rx = r->n_rx;
  const int64_t nh = (int64_t)n_rx * n_freq;
  double2* H = nullptr;
  double* tau = nullptr;
  rc = cfr_device(r, bandwidth, n_freq, &H, &tau);
  if (rc != NRT_OK) return rc;
  std::vector<double> h(2 * nh);
  TRY(cudaMemcpyAsync(h.data(), H, nh * sizeof(double2), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  // per RX: the Eq. 5 ratio and the weight 2 w_j / |H^_j|^2 (host, n_rx x n_freq)
  std::vector<double> dh(2 * nh), coef(n_rx);
  for (int j = 0; j < n_rx; ++j) {
    double num = 0.0, den = 0.0;
    for (int q = 0; q < n_freq; ++q) {
      const int64_t i = (int64_t)j * n_freq + q;
      const double dx = h[2 * i] - H_target[2 * i], dy = h[2 * i + 1] - H_target[2 * i + 1];
      dh[2 * i] = dx;
      dh[2 * i + 1] = dy;
      num += dx * dx + dy * dy;
      den += H_target[2 * i] * H_target[2 * i] + H_target[2 * i + 1] * H_target[2 * i + 1];
    }
    if (loss) loss[j] = den > 0.0 ? num / den : 0.0;
    coef[j] = den > 0.0 ? 2.0 * (double)rx_weight[j] / den : 0.0;
  }
  double2 *dH = nullptr, *W = nullptr;
  double* cf = nullptr;
  const int64_t np = r->n_paths;
  TRY(cudaMallocAsync(&dH, nh * sizeof(double2), st));
  TRY(cudaMallocAsync(&cf, n_rx * sizeof(double), st));
  TRY(cudaMallocAsync(&W, std::max<int64_t>(np, 1) * sizeof(double2), st));
  TRY(cudaMemcpyAsync(dH, dh.data(), nh * sizeof(double2), cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(cf, coef.data(), n_rx * sizeof(double), cudaMemcpyHostToDevice, st));
  const double df = bandwidth / (n_freq - 1);
  const double f0 = (double)r->p.freq - 0.5 * (n_freq - 1) * df;
  if (np > 0) {
    cfr_weight_kernel<<<grid_for_n(np, ctx->sm_count), 256, 0, st>>>(
        (const PathRec*)r->paths, tau, np, dH, cf, n_freq, f0, df, W);
    count_launch();
  }
  rc = adjoint_to_host(r, nullptr, W, g_eps, g_sig, g_sca);
  cudaFreeAsync(H, st);
  cudaFreeAsync(tau, st);
  cudaFreeAsync(dH, st);
  cudaFreeAsync(cf, st);
  cudaFreeAsync(W, st);
  TRY(cudaStreamSynchronize(st));
  return rc;
}

}  // extern "C"
