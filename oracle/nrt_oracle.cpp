// FP64 CPU oracle for the point-cloud radio ray tracer.
//
// TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the benchmark's CPU
// baseline leg may load this library; the product path (the CUDA library and
// its Python binding) never does.  It shares no code, header, table or
// constant generator with the CUDA path: it is a plain, slow restatement of
// the method, step by step, in double precision.
//
// What it follows (Vaara et al., "Differentiable High-Performance Ray
// Tracing-Based Simulation of Radio Propagation with Point Clouds"):
//   Sec. II-A   voxelisation into discretised point sets (DPS), reception points
//   Sec. II-B   visibility from each RX to every DPS reception point; LOS casts;
//               rays launched once and reflected specularly at every hit
//   Sec. II-B-1 diffuse scattering only as the last interaction, validated by a
//               cast from the scatter point to the RX
//   Sec. II-B-2 specular refinement: path-length minimisation on infinite
//               planes (Eq. 1), then validation casts with the angle and plane
//               distance thresholds t_a, t_d and up to kappa retries (Table I)
//   Sec. II-B-4 duplicate removal by (interaction types, surface labels of the
//               closest points; voxel of a diffuse scatter point)
//   Sec. II-C   ray/disc intersection and the weighted average of Eq. 3 with
//               the weights of Eq. 4
// The EM formulas (the paper delegates them to an external library) are
// readings written from textbook physics: Fresnel coefficients with the
// ITU-R P.2040 complex permittivity, an effective-roughness reduction and a
// Lambertian diffuse lobe (Degli-Esposti 2007), free-space spreading and delay.
//
// Besides the values, the oracle reports where floating point could decide a
// discrete outcome differently in a lower-precision implementation ("ambiguous"
// decisions within a band delta of a threshold); tests compare only the
// decisions the oracle marks certain.
//
// Parity pins: see tests/test_oracle_*.py (closed forms, brute force vs grid,
// image-source enumeration in a shoebox room, finite differences).

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <set>
#include <tuple>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kInf = std::numeric_limits<double>::infinity();
const double kPi = 3.14159265358979323846;
const double kC0 = 299792458.0;         // speed of light, m/s
const double kEps0 = 8.8541878128e-12;  // vacuum permittivity, F/m

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return (1.0 / norm(a)) * a; }
inline double comp(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// Scene: points, voxels (DPS), reception points, and an acceleration grid.
// ---------------------------------------------------------------------------
struct Scene {
  int64_t n = 0;
  std::vector<V3> P, N;
  std::vector<int> surf, mat;
  std::vector<std::array<int, 3>> vox;  // voxel of each point
  std::vector<int> dps_of;              // DPS index of each point
  std::vector<std::array<int, 3>> dps_vox;
  std::vector<std::vector<int>> dps_pts;
  std::vector<V3> recv;                 // reception point = mean of the DPS's points
  std::vector<int> dps_morton;          // DPS of each rank in voxel Morton order
  double rho = 0, rp = 0, lambda_d = 0;
  float bmin_f[3] = {0, 0, 0};
  // acceleration grid (grid_cell <= 0 means brute force over all discs)
  bool brute = true;
  double g = 0, band_cap = 0;
  V3 gmin{0, 0, 0};
  int gd[3] = {0, 0, 0};
  std::vector<std::vector<int>> cells;
};

// Voxel index of a coordinate.  The voxel decides the DPS a point belongs to
// (Sec. II-A), an integer outcome, so it is taken in float32 -- the same
// precision as the kernel: floor(fl32(fl32(p - bmin) / rho)).
int voxel_f32(float p, float bmin, float rho) {
  volatile float d = p - bmin;
  volatile float s = d / rho;
  return (int)std::floor((float)s);
}

Scene* build_scene(const float* pos, const float* nrm, const uint16_t* surf, const uint8_t* mat,
                   int64_t n, double rho, double rp, double lambda_d, double grid_cell,
                   double band_cap) {
  Scene* S = new Scene();
  S->n = n;
  S->rho = rho;
  S->rp = rp;
  S->lambda_d = lambda_d;
  S->band_cap = band_cap;
  S->P.resize(n);
  S->N.resize(n);
  S->surf.resize(n);
  S->mat.resize(n);
  for (int k = 0; k < 3; ++k) S->bmin_f[k] = std::numeric_limits<float>::infinity();
  for (int64_t i = 0; i < n; ++i) {
    S->P[i] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    S->N[i] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
    S->surf[i] = surf[i];
    S->mat[i] = mat[i];
    for (int k = 0; k < 3; ++k) S->bmin_f[k] = std::min(S->bmin_f[k], pos[3 * i + k]);
  }
  // voxels and DPS (ordered by voxel coordinate, lexicographic)
  const float rho_f = (float)rho;
  S->vox.resize(n);
  std::map<std::array<int, 3>, int> index;
  for (int64_t i = 0; i < n; ++i) {
    std::array<int, 3> v;
    for (int k = 0; k < 3; ++k) v[k] = voxel_f32(pos[3 * i + k], S->bmin_f[k], rho_f);
    S->vox[i] = v;
    index.emplace(v, 0);
  }
  int next = 0;
  for (auto& kv : index) kv.second = next++;
  S->dps_vox.resize(next);
  S->dps_pts.resize(next);
  for (auto& kv : index) S->dps_vox[kv.second] = kv.first;
  S->dps_of.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    int d = index[S->vox[i]];
    S->dps_of[i] = d;
    S->dps_pts[d].push_back((int)i);
  }
  S->recv.resize(next);
  for (int d = 0; d < next; ++d) {
    V3 s{0, 0, 0};
    for (int i : S->dps_pts[d]) s = s + S->P[i];
    S->recv[d] = (1.0 / (double)S->dps_pts[d].size()) * s;
  }
  // DPS-directed launch order: voxel Morton code, x in the lowest bit
  {
    auto spread = [](uint64_t x) {
      uint64_t r = 0;
      for (int b = 0; b < 21; ++b) r |= ((x >> b) & 1ull) << (3 * b);
      return r;
    };
    std::vector<std::pair<uint64_t, int>> mk(next);
    for (int d = 0; d < next; ++d) {
      const auto& v = S->dps_vox[d];
      mk[d] = {spread((uint64_t)v[0]) | (spread((uint64_t)v[1]) << 1) | (spread((uint64_t)v[2]) << 2), d};
    }
    std::sort(mk.begin(), mk.end());
    S->dps_morton.resize(next);
    for (int d = 0; d < next; ++d) S->dps_morton[d] = mk[d].second;
  }
  // uniform grid: each disc listed in every cell overlapped by the cube of
  // half-size r_p + band_cap around its centre.
  if (grid_cell > 0 && n > 0) {
    S->brute = false;
    S->g = grid_cell;
    const double R = rp + band_cap + 1e-9;
    V3 lo{kInf, kInf, kInf}, hi{-kInf, -kInf, -kInf};
    for (int64_t i = 0; i < n; ++i) {
      lo = {std::min(lo.x, S->P[i].x), std::min(lo.y, S->P[i].y), std::min(lo.z, S->P[i].z)};
      hi = {std::max(hi.x, S->P[i].x), std::max(hi.y, S->P[i].y), std::max(hi.z, S->P[i].z)};
    }
    S->gmin = {lo.x - R, lo.y - R, lo.z - R};
    for (int k = 0; k < 3; ++k)
      S->gd[k] = (int)std::floor((comp(hi, k) + R - comp(S->gmin, k)) / grid_cell) + 1;
    S->cells.assign((size_t)S->gd[0] * S->gd[1] * S->gd[2], {});
    for (int64_t i = 0; i < n; ++i) {
      int a[3], b[3];
      for (int k = 0; k < 3; ++k) {
        a[k] = std::max(0, (int)std::floor((comp(S->P[i], k) - R - comp(S->gmin, k)) / grid_cell));
        b[k] = std::min(S->gd[k] - 1,
                        (int)std::floor((comp(S->P[i], k) + R - comp(S->gmin, k)) / grid_cell));
      }
      for (int z = a[2]; z <= b[2]; ++z)
        for (int y = a[1]; y <= b[1]; ++y)
          for (int x = a[0]; x <= b[0]; ++x)
            S->cells[((size_t)z * S->gd[1] + y) * S->gd[0] + x].push_back((int)i);
    }
  }
  return S;
}

// ---------------------------------------------------------------------------
// Ray/disc intersection and the closest hit (Sec. II-C, Eq. 3, Eq. 4).
// ---------------------------------------------------------------------------
struct DiscEval {
  bool ok;     // plane not parallel to the ray
  double t;    // ray parameter of the plane hit
  double r;    // distance of the plane hit from the disc centre
  double den;  // d . n_i
  V3 q;        // plane hit point q_i
};

inline DiscEval eval_disc(const Scene& S, int i, V3 o, V3 d) {
  DiscEval e;
  e.den = dot(d, S.N[i]);
  if (e.den == 0.0) {
    e.ok = false;
    e.t = e.r = 0.0;
    e.q = {0, 0, 0};
    return e;
  }
  e.ok = true;
  e.t = dot(S.P[i] - o, S.N[i]) / e.den;
  e.q = o + e.t * d;
  e.r = norm(e.q - S.P[i]);
  return e;
}

struct Hit {
  bool hit = false;
  double t = kInf;
  int idx = -1;   // point index of q_min
  int dps = -1;   // DPS of q_min
  V3 q{0, 0, 0};  // Eq. 3 weighted intersection
  V3 n{0, 0, 0};  // weighted normal, facing the incoming ray
  double cos_in = 0.0;
  bool amb = false;
};

struct CastCfg {
  double wjit = 0.0;    // shadow trajectories: relative jitter of the Eq. 4 weights
  int wseed = 0;
  double t_min = 1e-3;  // hits need t > t_min
  double delta = 0.0;   // ambiguity band (position units)
};

// Visit the discs that can matter for a cast on [t_lo, t_hi].  In brute
// force mode that is every disc; with the grid it is every disc listed in a
// cell the ray passes through, visited in order of t until `stop(t_enter)`.
template <class F, class Stop>
void for_candidate_discs(const Scene& S, V3 o, V3 d, double t_lo, double t_hi, F&& f, Stop&& stop) {
  if (S.brute) {
    for (int64_t i = 0; i < S.n; ++i) f((int)i);
    return;
  }
  // slab test against the grid box
  double t0 = t_lo, t1 = t_hi;
  double inv[3];
  for (int k = 0; k < 3; ++k) {
    double dk = comp(d, k), ok = comp(o, k);
    double lo = comp(S.gmin, k), hi = lo + S.gd[k] * S.g;
    if (dk == 0.0) {
      inv[k] = kInf;
      if (ok < lo || ok > hi) return;
      continue;
    }
    inv[k] = 1.0 / dk;
    double ta = (lo - ok) * inv[k], tb = (hi - ok) * inv[k];
    if (ta > tb) std::swap(ta, tb);
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
  }
  if (t0 > t1) return;
  V3 p = o + t0 * d;
  int c[3], step[3];
  double tnext[3];
  for (int k = 0; k < 3; ++k) {
    c[k] = (int)std::floor((comp(p, k) - comp(S.gmin, k)) / S.g);
    c[k] = std::min(std::max(c[k], 0), S.gd[k] - 1);
    double dk = comp(d, k);
    step[k] = dk > 0 ? 1 : (dk < 0 ? -1 : 0);
    if (step[k] == 0) {
      tnext[k] = kInf;
    } else {
      double bnd = comp(S.gmin, k) + (c[k] + (step[k] > 0 ? 1 : 0)) * S.g;
      tnext[k] = (bnd - comp(o, k)) * inv[k];
    }
  }
  for (;;) {
    const auto& cell = S.cells[((size_t)c[2] * S.gd[1] + c[1]) * S.gd[0] + c[0]];
    for (int i : cell) f(i);
    int k = 0;
    if (tnext[1] < tnext[k]) k = 1;
    if (tnext[2] < tnext[k]) k = 2;
    double tenter = tnext[k];
    if (tenter > t1 || stop(tenter)) return;
    c[k] += step[k];
    if (c[k] < 0 || c[k] >= S.gd[k]) return;
    double bnd = comp(S.gmin, k) + (c[k] + (step[k] > 0 ? 1 : 0)) * S.g;
    tnext[k] = (bnd - comp(o, k)) * inv[k];
  }
}

// Closest disc hit along o + t d (|d| = 1) with t in (t_min, t_max), ignoring
// the discs of DPS `skip`.  q_min is the hit with the smallest t; ties go to
// the smaller point index.  With `weighted`, the intersection point is the
// Eq. 3 average over the intersected discs of the DPS of q_min, with the Eq. 4
// weights exp(-|q_i - p_i|^2 / (2 r_p^2)) * exp(-lambda_d |q_i - q_min|), and
// the normal is the same weighted average of the disc normals, normalised and
// turned to face the incoming ray.
Hit cast(const Scene& S, V3 o, V3 d, int skip, double t_max, bool weighted, const CastCfg& cfg) {
  Hit h;
  const double rp = S.rp, cap = S.band_cap;
  struct Seen {
    int i;
    DiscEval e;
  };
  std::vector<Seen> seen;
  seen.reserve(256);
  double best_t = kInf;
  int best_i = -1;
  auto visit = [&](int i) {
    if (S.dps_of[i] == skip) return;
    DiscEval e = eval_disc(S, i, o, d);
    if (!e.ok) return;
    seen.push_back({i, e});
    if (e.t > cfg.t_min && e.t < t_max && e.r <= rp) {
      if (e.t < best_t || (e.t == best_t && i < best_i)) {
        best_t = e.t;
        best_i = i;
      }
    }
  };
  auto stop = [&](double tenter) {
    double lim = std::min(best_t, t_max);
    return tenter > lim + 2.0 * cap;
  };
  for_candidate_discs(S, o, d, cfg.t_min - cap, t_max + cap, visit, stop);

  auto band = [&](const DiscEval& e) {
    double b = cfg.delta / std::max(std::fabs(e.den), 1e-12);
    return std::min(b, cap);
  };
  const bool hit = best_i >= 0;
  double b_best = 0.0;
  DiscEval ebest{};
  if (hit) {
    for (const auto& s : seen)
      if (s.i == best_i) {
        ebest = s.e;
        break;
      }
    b_best = band(ebest);
  }
  // ambiguity: decisions a lower-precision implementation could take otherwise
  if (cfg.delta > 0) {
    const double t_lim = hit ? best_t : t_max;
    for (const auto& s : seen) {
      const DiscEval& e = s.e;
      double b = band(e);
      if (e.t < cfg.t_min - b) continue;
      if (e.t > t_lim + b + b_best) continue;
      bool near_or_in = e.r < rp + b;
      if (std::fabs(e.r - rp) < b) h.amb = true;                                  // disc edge
      if (near_or_in && std::fabs(e.t - cfg.t_min) < b) h.amb = true;            // t_min
      if (near_or_in && std::isfinite(t_max) && std::fabs(e.t - t_max) < b) h.amb = true;
      if (hit && s.i != best_i && near_or_in && e.t != best_t &&
          std::fabs(e.t - best_t) < b + b_best)
        h.amb = true;                                                             // depth tie
    }
  }
  if (!hit) return h;
  h.hit = true;
  h.t = best_t;
  h.idx = best_i;
  h.dps = S.dps_of[best_i];
  if (!weighted) return h;
  const V3 qmin = ebest.q;
  double sw = 0.0;
  V3 sq{0, 0, 0}, sn{0, 0, 0};
  for (int i : S.dps_pts[h.dps]) {
    DiscEval e = eval_disc(S, i, o, d);
    if (!e.ok) continue;
    double b = band(e);
    if (cfg.delta > 0 && e.t > cfg.t_min - b && std::fabs(e.r - rp) < b) h.amb = true;
    if (!(e.t > cfg.t_min && e.r <= rp)) continue;
    double w = std::exp(-e.r * e.r / (2.0 * rp * rp)) * std::exp(-S.lambda_d * norm(e.q - qmin));
    if (cfg.wjit != 0.0) {
      uint32_t hsh = (uint32_t)i * 2654435761u + (uint32_t)cfg.wseed * 40503u;
      w *= 1.0 + cfg.wjit * (((hsh >> 15) & 1u) ? 1.0 : -1.0);
    }
    sw += w;
    sq = sq + w * e.q;
    sn = sn + w * S.N[i];
  }
  h.q = (1.0 / sw) * sq;
  h.n = unit(sn);
  if (dot(h.n, d) > 0) h.n = -1.0 * h.n;
  h.cos_in = std::fabs(dot(d, h.n));
  return h;
}

// ---------------------------------------------------------------------------
// Launch directions: Fibonacci sphere with a 64-bit fixed-point golden angle.
//   z_i = 1 - (2i+1)/N,  r_i = sqrt(1 - z_i^2),
//   phi_i = 2 pi frac(i * G / 2^64),  G = round((2 - golden ratio) * 2^64).
// ---------------------------------------------------------------------------
const uint64_t kGolden64 = 0x61C8864680B583EBull;

V3 fib_dir(int64_t i, int64_t n) {
  double a = (2.0 * (double)i + 1.0) / (double)n;
  double z = 1.0 - a;
  double r = std::sqrt(std::max(0.0, a * (2.0 - a)));
  uint64_t u = (uint64_t)i * kGolden64;
  double phi = 2.0 * kPi * std::ldexp((double)u, -64);
  return {r * std::cos(phi), r * std::sin(phi), z};
}

// ---------------------------------------------------------------------------
// EM (readings; the paper leaves these to an external library).
// ---------------------------------------------------------------------------
typedef std::complex<double> cd;

// ITU-R P.2040 complex relative permittivity eta = eps_r - j sigma / (2 pi f eps0)
cd permittivity(double eps_r, double sigma, double f) {
  return cd(eps_r, -sigma / (2.0 * kPi * f * kEps0));
}

// Fresnel reflection coefficient; pol 0 = TE (perpendicular), 1 = TM (parallel)
cd fresnel(cd eta, double cos_t, int pol) {
  double sin2 = 1.0 - cos_t * cos_t;
  cd s = std::sqrt(eta - sin2);
  if (pol == 0) return (cos_t - s) / (cos_t + s);
  return (eta * cos_t - s) / (eta * cos_t + s);
}

cd dfresnel_deta(cd eta, double cos_t, int pol) {
  double sin2 = 1.0 - cos_t * cos_t;
  cd s = std::sqrt(eta - sin2);
  if (pol == 0) {
    cd den = cos_t + s;
    return -cos_t / (s * den * den);
  }
  cd den = eta * cos_t + s;
  return cos_t * (eta - 2.0 * sin2) / (s * den * den);
}

// ---------------------------------------------------------------------------
// Simulation (Sec. II-B): LOS, launch, bounce loop, capture, dedup, validation,
// refinement and field.
// ---------------------------------------------------------------------------
}  // namespace

extern "C" {

struct orc_params {
  int32_t max_depth;   // K, maximum number of interactions
  int32_t capture;     // 0 = RX sphere, 1 = visibility matrix
  int32_t diffuse;     // diffuse scattering as the last interaction
  int32_t pol;         // 0 TE, 1 TM
  int32_t kappa;       // refinement retries
  int32_t rep_tries;   // candidates tried per key, in ray order (0: all of them)
  int32_t validate;    // 0: stop after the trace (records only)
  int32_t n_threads;   // 0: OpenMP default
  int64_t n_rays;      // N of the Fibonacci launch
  double r_rx;         // RX sphere radius
  double t_min;        // minimum hit distance
  double delta;        // ambiguity band; 0 disables ambiguity tracking
  double t_a_deg;      // refinement angle threshold, degrees
  double t_d;          // refinement plane-distance threshold, m
  double freq;         // Hz
  int32_t launch;      // 0 Fibonacci sphere of n_rays, 1 one ray per DPS (Sec. II-B)
  int32_t diffraction; // 1: single-bounce edge diffraction (orc_sim_diffraction)
};

}  // extern "C"

namespace {

struct HitRec {
  int64_t idx = -1;
  int dps = -1;
  double t = 0, cos_in = 0;
  V3 q{0, 0, 0}, n{0, 0, 0};
  V3 dout{0, 0, 0};  // direction of the specular continuation
  bool amb = false;
};

struct Key {
  uint64_t hi = 0, lo = 0;
  bool operator<(const Key& o) const { return hi != o.hi ? hi < o.hi : lo < o.lo; }
  bool operator==(const Key& o) const { return hi == o.hi && lo == o.lo; }
};

// 128-bit path key: hi = [j:8 @56][diffuse:1 @55][k:3 @52][...], lo = labels.
// Specular: lo = l1 | l2<<16 | l3<<32 | l4<<48, hi[0:16] = l5.
// Diffuse:  lo = prefix labels l1..l(k-1), hi[0:48] = voxel x | y<<16 | z<<32.
Key make_key(int j, bool diffuse, int k, const int* labels, int n_labels, const int* voxel) {
  Key K;
  K.hi = ((uint64_t)(j & 0xFF) << 56) | ((uint64_t)(diffuse ? 1 : 0) << 55) |
         ((uint64_t)(k & 7) << 52);
  for (int m = 0; m < n_labels && m < 4; ++m) K.lo |= (uint64_t)(labels[m] & 0xFFFF) << (16 * m);
  if (!diffuse && n_labels >= 5) K.hi |= (uint64_t)(labels[4] & 0xFFFF);
  if (diffuse)
    K.hi |= (uint64_t)(voxel[0] & 0xFFFF) | ((uint64_t)(voxel[1] & 0xFFFF) << 16) |
            ((uint64_t)(voxel[2] & 0xFFFF) << 32);
  return K;
}

struct Cand {
  int64_t ray;
  bool certain;
};

struct PathOut {
  Key key;
  int j = 0, type = 0, k = 0;  // type 0 specular / LOS, 1 diffuse, 2 edge diffraction
  int64_t rep = -1;            // representative ray id (diffraction: edge index)
  V3 pts[5];
  V3 nd{0, 0, 0};  // diffuse paths: surface normal at the scatter point
  V3 e0{0, 0, 0}, e1{0, 0, 0}, en0{0, 0, 0}, en1{0, 0, 0};  // diffraction: the edge
  int mats[5] = {0, 0, 0, 0, 0};
  double cosv[5] = {0, 0, 0, 0, 0};
  double geo = 0, tau = 0, length = 0;
  bool certain = true;
  bool shadow_ok[2] = {false, false};
  std::shared_ptr<PathOut> shadow[2];
};

struct KeyOut {
  Key key;
  int j = 0, type = 0, k = 0;
  int64_t n_cand = 0;
  std::vector<int64_t> tried;
  std::vector<int> tried_valid, tried_amb;
  int64_t rep = -1;
  bool valid = false, certain = true;
  int path = -1;
};

struct Sim {
  const Scene* S = nullptr;
  orc_params p{};
  V3 tx{0, 0, 0};
  std::vector<V3> rx;
  int n_seg = 0;
  std::vector<int64_t> ray_ids;
  std::vector<HitRec> rec;     // [n_ray][n_seg]
  std::vector<HitRec> recp[2]; // shadow trajectories (perturbed launch), same layout
  std::vector<double> dq_sens, dn_sens;  // [n_ray][n_seg] shadow divergence
  std::vector<int> excl;       // first ambiguous hit (1-based), n_seg+1 = none
  std::vector<int> n_hits;
  // visibility bits, computed for the DPS the traced rays reach
  std::map<std::pair<int, int>, std::pair<bool, bool>> vis;  // (j, dps) -> (bit, amb)
  std::vector<KeyOut> keys;
  std::vector<PathOut> paths;
  std::vector<std::pair<bool, bool>> los;  // per RX (clear, amb)
  std::vector<double> power;
  // potential producers of keys under ambiguity
  std::map<std::pair<int, std::vector<int>>, int64_t> prefix_min;  // (e, labels 1..e-1)
  std::map<Key, std::vector<int64_t>> uncertain_cand;
  std::map<Key, std::vector<Cand>> cands;  // per key, in ray order
  std::vector<int64_t> ray_pos;  // ray id -> row, or -1
  mutable std::atomic<int64_t> val_casts{0}, vis_casts{0};
};

struct Validation {
  bool valid = false, amb = false;
  PathOut path;
};

double rx_margin(const Scene& S) { return std::sqrt(3.0) / 2.0 * S.rho + S.rp; }

// Visibility from RX j to the reception point of DPS D (Sec. II-B): cast from
// the RX toward the point; visible when nothing is hit before the reception
// point's voxel could begin (t < s - (sqrt(3)/2 rho + r_p)) or the first hit
// belongs to D itself.
std::pair<bool, bool> vis_cast(const Scene& S, V3 rxp, int D, const CastCfg& cfg) {
  V3 dv = S.recv[D] - rxp;
  double s = norm(dv);
  double t_max = s - rx_margin(S);
  if (t_max <= cfg.t_min) return {true, cfg.delta > 0 && t_max > cfg.t_min - cfg.delta};
  Hit h = cast(S, rxp, (1.0 / s) * dv, -1, t_max, false, cfg);
  bool bit = !h.hit || h.dps == D;
  return {bit, h.amb};
}

Validation validate_diffuse(const Sim& sim, const std::vector<HitRec>& rec, int64_t row, int k,
                            int j, const CastCfg& cfg) {
  const Scene& S = *sim.S;
  Validation v;
  const HitRec& hk = rec[row * sim.n_seg + (k - 1)];
  V3 u = sim.rx[j] - hk.q;
  double rs = norm(u);
  V3 w = (1.0 / rs) * u;
  double cs = dot(hk.n, w);
  if (cfg.delta > 0 && (std::fabs(cs) < 1e-5 || hk.cos_in < 1e-5)) v.amb = true;
  if (cs <= 0.0) return v;
  sim.val_casts++;
  Hit h = cast(S, hk.q, w, hk.dps, rs, false, cfg);
  if (h.amb) v.amb = true;
  if (h.hit) return v;
  v.valid = true;
  PathOut& P = v.path;
  P.type = 1;
  P.k = k;
  P.nd = hk.n;
  double ri = 0.0;
  for (int m = 0; m < k; ++m) {
    const HitRec& hm = rec[row * sim.n_seg + m];
    P.pts[m] = hm.q;
    P.mats[m] = S.mat[hm.idx];
    P.cosv[m] = hm.cos_in;
    ri += hm.t;
  }
  double lam = kC0 / sim.p.freq;
  P.geo = lam / (4.0 * kPi) * std::sqrt(S.rho * S.rho * hk.cos_in * cs / kPi) / (ri * rs);
  P.length = ri + rs;
  P.tau = P.length / kC0;
  return v;
}

// Specular refinement (Sec. II-B-2).  Phase 1: the minimiser of the path
// length of Eq. 1 over points on the infinite planes (q_m, n_m); each term is
// the norm of an affine function, so the minimiser with every reflection on
// the correct side is the image-method path, solved here exactly.  Phase 2:
// cast from I_{m-1} toward I_m; the interaction is valid when the hit lies on
// the key's surface with a normal within t_a and within t_d of the plane;
// otherwise the plane is replaced by the hit's and the solve retried, at most
// kappa times.  Finally the last leg I_k -> RX must be clear.
Validation validate_specular(const Sim& sim, const std::vector<HitRec>& rec, int64_t row, int k,
                             int j, const int* labels, const CastCfg& cfg) {
  const Scene& S = *sim.S;
  Validation v;
  V3 Pp[5], Pn[5];
  for (int m = 0; m < k; ++m) {
    const HitRec& hm = rec[row * sim.n_seg + m];
    Pp[m] = hm.q;
    Pn[m] = hm.n;
  }
  const V3 tx = sim.tx, rxp = sim.rx[j];
  const double cos_ta = std::cos(sim.p.t_a_deg * kPi / 180.0);
  const double ta = sim.p.t_a_deg * kPi / 180.0;
  for (int attempt = 0; attempt <= sim.p.kappa; ++attempt) {
    V3 img[6];
    img[0] = tx;
    for (int m = 0; m < k; ++m) img[m + 1] = img[m] - 2.0 * dot(img[m] - Pp[m], Pn[m]) * Pn[m];
    V3 I[7];
    I[0] = tx;
    I[k + 1] = rxp;
    V3 tgt = rxp;
    bool ok = true;
    for (int m = k; m >= 1; --m) {
      V3 dir = img[m] - tgt;
      double den = dot(dir, Pn[m - 1]);
      if (std::fabs(den) < 1e-300) {
        ok = false;
        break;
      }
      double u = dot(Pp[m - 1] - tgt, Pn[m - 1]) / den;
      I[m] = tgt + u * dir;
      tgt = I[m];
    }
    if (!ok) return v;
    for (int m = 1; m <= k; ++m) {
      double a = dot(I[m - 1] - I[m], Pn[m - 1]);
      double b = dot(I[m + 1] - I[m], Pn[m - 1]);
      if (cfg.delta > 0 && std::min(std::fabs(a), std::fabs(b)) < cfg.delta) v.amb = true;
      if (!(a * b > 0.0)) return v;
    }
    // phase 2: validation casts
    int prev_dps = -1;
    int fail_m = -1;
    Hit hv[5];
    bool dead = false;
    for (int m = 1; m <= k; ++m) {
      V3 seg = I[m] - I[m - 1];
      sim.val_casts++;
      Hit h = cast(S, I[m - 1], unit(seg), prev_dps, kInf, true, cfg);
      if (h.amb) v.amb = true;
      if (!h.hit || S.surf[h.idx] != labels[m - 1]) {
        dead = true;
        break;
      }
      double c = std::min(1.0, std::fabs(dot(Pn[m - 1], h.n)));
      double dist = std::fabs(dot(h.q - I[m], Pn[m - 1]));
      if (cfg.delta > 0) {
        if (std::fabs(std::acos(c) - ta) < 0.01 * ta) v.amb = true;
        if (std::fabs(dist - sim.p.t_d) < 0.01 * sim.p.t_d) v.amb = true;
      }
      hv[m - 1] = h;
      if (!(c >= cos_ta && dist <= sim.p.t_d)) {
        fail_m = m;
        break;
      }
      prev_dps = h.dps;
    }
    if (dead) return v;
    if (fail_m > 0) {
      if (attempt == sim.p.kappa) return v;
      Pp[fail_m - 1] = hv[fail_m - 1].q;
      Pn[fail_m - 1] = hv[fail_m - 1].n;
      continue;
    }
    // final leg to the RX
    V3 last = rxp - I[k];
    double s = norm(last);
    sim.val_casts++;
    Hit hf = cast(S, I[k], (1.0 / s) * last, prev_dps, s, false, cfg);
    if (hf.amb) v.amb = true;
    if (hf.hit) return v;
    v.valid = true;
    PathOut& P = v.path;
    P.type = 0;
    P.k = k;
    double len = 0.0;
    for (int m = 0; m <= k; ++m) len += norm(I[m + 1] - I[m]);
    for (int m = 1; m <= k; ++m) {
      P.pts[m - 1] = I[m];
      P.mats[m - 1] = S.mat[hv[m - 1].idx];
      P.cosv[m - 1] = std::fabs(dot(Pn[m - 1], unit(I[m] - I[m - 1])));
    }
    double lam = kC0 / sim.p.freq;
    P.length = len;
    P.geo = lam / (4.0 * kPi * len);
    P.tau = len / kC0;
    return v;
  }
  return v;
}

// One trajectory: the launch direction d0 reflected specularly at every hit.
void trace_one(Sim& sim, std::vector<HitRec>& rec, int64_t row, V3 d0, const CastCfg& cfg,
               int* excl, int* n_hits, V3 kick = V3{0, 0, 0}) {
  const Scene& S = *sim.S;
  V3 o = sim.tx, d = d0;
  int skip = -1;
  for (int k = 1; k <= sim.n_seg; ++k) {
    Hit h = cast(S, o, d, skip, kInf, true, cfg);
    HitRec& r = rec[row * sim.n_seg + (k - 1)];
    r.amb = h.amb;
    if (h.amb && excl && *excl > k) *excl = k;
    if (!h.hit) break;
    r.idx = h.idx;
    r.dps = h.dps;
    r.t = norm(h.q - o);  // length of the segment to the interaction point q
    r.q = h.q;
    r.n = h.n;
    r.cos_in = h.cos_in;
    if (n_hits) *n_hits = k;
    d = d - 2.0 * dot(d, h.n) * h.n;  // specular continuation
    r.dout = d;
    o = h.q + kick;  // shadows restart from a slightly displaced point
    skip = h.dps;
  }
}

// The nominal trajectory plus two shadows whose launch direction is turned by
// kShadowAngle about two axes orthogonal to it, whose every interaction
// point is displaced by kShadowKick before the next segment starts, and
// whose Eq. 4 weights are scaled by 1 +- kShadowJitter (sign from a hash of
// the point index).  Float32 coordinates of a 20 m scene carry ~2e-6 m of
// rounding per point and the weights inherit it; the shadows model both
// several times over and show how strongly they grow along the (chaotic)
// bounce sequence.  On a flat wall of identical normals the weight jitter
// moves nothing, as rounding does not either.  A hit whose shadows land on another disc or
// farther than delta from the nominal point is ambiguous, and the shadows'
// divergence sizes the comparison tolerances.
const double kShadowAngle = 1e-6;
const double kShadowKick = 1e-5;
const double kShadowJitter = 1e-3;

// Launch direction of ray rid: Fibonacci sphere, or (Sec. II-B) toward the
// reception point of the rid-th DPS in voxel Morton order.
V3 launch_dir(const Sim& sim, int64_t rid) {
  if (sim.p.launch == 1) return unit(sim.S->recv[sim.S->dps_morton[rid]] - sim.tx);
  return fib_dir(rid, sim.p.n_rays);
}

void trace_ray(Sim& sim, int64_t row, const CastCfg& cfg) {
  int64_t rid = sim.ray_ids[row];
  V3 d0 = launch_dir(sim, rid);
  sim.excl[row] = sim.n_seg + 1;
  sim.n_hits[row] = 0;
  trace_one(sim, sim.rec, row, d0, cfg, &sim.excl[row], &sim.n_hits[row]);
  if (cfg.delta <= 0) return;
  V3 a = std::fabs(d0.z) < 0.9 ? V3{0, 0, 1} : V3{1, 0, 0};
  V3 u = unit(V3{d0.y * a.z - d0.z * a.y, d0.z * a.x - d0.x * a.z, d0.x * a.y - d0.y * a.x});
  V3 w{d0.y * u.z - d0.z * u.y, d0.z * u.x - d0.x * u.z, d0.x * u.y - d0.y * u.x};
  for (int p = 0; p < 2; ++p) {
    CastCfg quiet = cfg;
    quiet.delta = 0.0;
    quiet.wjit = kShadowJitter;
    quiet.wseed = p + 1;
    V3 dp = unit(d0 + kShadowAngle * (p == 0 ? u : w));
    V3 kick = p == 0 ? V3{0.6, 0.48, 0.64} : V3{-0.48, 0.8, -0.36};  // unit, fixed
    trace_one(sim, sim.recp[p], row, dp, quiet, nullptr, nullptr, kShadowKick * kick);
  }
  for (int k = 1; k <= sim.n_seg; ++k) {
    const HitRec& h = sim.rec[row * sim.n_seg + (k - 1)];
    double dq = 0.0, dn = 0.0;
    bool split = false;
    for (int p = 0; p < 2; ++p) {
      const HitRec& g = sim.recp[p][row * sim.n_seg + (k - 1)];
      if (g.idx != h.idx) {
        split = true;
        continue;
      }
      if (h.idx < 0) continue;
      dq = std::max(dq, norm(g.q - h.q));
      dn = std::max(dn, norm(g.n - h.n));
    }
    sim.dq_sens[row * sim.n_seg + (k - 1)] = dq;
    sim.dn_sens[row * sim.n_seg + (k - 1)] = dn;
    if ((split || dq > cfg.delta) && sim.excl[row] > k) sim.excl[row] = k;
    if (h.idx < 0) break;
  }
}

int diffuse_voxel(const Scene& S, V3 q, int* v, double delta, bool* amb) {
  for (int k = 0; k < 3; ++k) {
    double s = (comp(q, k) - (double)S.bmin_f[k]) / S.rho;
    v[k] = (int)std::floor(s);
    double frac = s - std::floor(s);
    if (delta > 0 && std::min(frac, 1.0 - frac) * S.rho < delta) *amb = true;
  }
  return 0;
}

void run_sim(Sim& sim) {
  const Scene& S = *sim.S;
  CastCfg cfg;
  cfg.t_min = sim.p.t_min;
  cfg.delta = sim.p.delta;
  const int64_t n = (int64_t)sim.ray_ids.size();
  const int M = (int)sim.rx.size();
  const bool sphere = sim.p.capture == 0;
  sim.n_seg = sim.p.max_depth + (sphere ? 1 : 0);
  sim.rec.assign(n * sim.n_seg, HitRec());
  for (int p = 0; p < 2; ++p) sim.recp[p].assign(n * sim.n_seg, HitRec());
  sim.dq_sens.assign(n * sim.n_seg, 0.0);
  sim.dn_sens.assign(n * sim.n_seg, 0.0);
  sim.excl.assign(n, 0);
  sim.n_hits.assign(n, 0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < n; ++r) trace_ray(sim, r, cfg);

  // LOS (Sec. II-B): cast from the TX to every RX
  sim.los.assign(M, {false, false});
  for (int j = 0; j < M; ++j) {
    V3 dv = sim.rx[j] - sim.tx;
    double s = norm(dv);
    Hit h = cast(S, sim.tx, (1.0 / s) * dv, -1, s, false, cfg);
    sim.los[j] = {!h.hit, h.amb};
  }
  if (!sim.p.validate) return;

  // visibility matrix entries for the DPS reached
  if (!sphere) {
    std::set<int> reached;
    for (int64_t r = 0; r < n; ++r)
      for (int k = 1; k <= std::min(sim.n_hits[r], sim.p.max_depth); ++k)
        reached.insert(sim.rec[r * sim.n_seg + k - 1].dps);
    std::vector<std::pair<int, int>> pairs;
    for (int D : reached)
      for (int j = 0; j < M; ++j) pairs.push_back({j, D});
    std::vector<std::pair<bool, bool>> res(pairs.size());
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < (int64_t)pairs.size(); ++i)
      res[i] = vis_cast(S, sim.rx[pairs[i].first], pairs[i].second, cfg);
    for (size_t i = 0; i < pairs.size(); ++i) sim.vis[pairs[i]] = res[i];
    sim.vis_casts += (int64_t)pairs.size();
  }

  // candidates, in ray order
  std::map<Key, std::vector<Cand>>& cands = sim.cands;
  std::map<Key, std::tuple<int, int, int>> kinfo;  // j, type, k
  auto add_uncertain = [&](const Key& K, int64_t rid) { sim.uncertain_cand[K].push_back(rid); };
  for (int64_t r = 0; r < n; ++r) {
    const int64_t rid = sim.ray_ids[r];
    const int e = sim.excl[r];
    int labels[8];
    for (int m = 0; m < sim.n_hits[r]; ++m) labels[m] = S.surf[sim.rec[r * sim.n_seg + m].idx];
    if (e <= sim.n_seg) {
      std::vector<int> pre(labels, labels + std::min(e - 1, sim.n_hits[r]));
      auto key = std::make_pair(e, pre);
      auto it = sim.prefix_min.find(key);
      if (it == sim.prefix_min.end() || rid < it->second) sim.prefix_min[key] = rid;
    }
    if (sphere) {
      // segment s starts at hit s (s >= 1) and ends at hit s+1 (or runs to infinity)
      for (int s = 1; s <= std::min(sim.n_hits[r], sim.p.max_depth); ++s) {
        const HitRec& hs = sim.rec[r * sim.n_seg + s - 1];
        const HitRec& he = sim.rec[r * sim.n_seg + s];
        const V3 dseg = hs.dout;
        double t_end = (sim.n_hits[r] >= s + 1) ? he.t : kInf;
        for (int j = 0; j < M; ++j) {
          double ts = dot(sim.rx[j] - hs.q, dseg);
          ts = std::min(std::max(ts, 0.0), t_end);
          double dist = norm(hs.q + ts * dseg - sim.rx[j]);
          bool band = cfg.delta > 0 && std::fabs(dist - sim.p.r_rx) < cfg.delta;
          if (dist <= sim.p.r_rx || band) {
            Key K = make_key(j, false, s, labels, s, nullptr);
            bool certain = (s + 1 < e) && !band;
            if (dist <= sim.p.r_rx) {
              cands[K].push_back({rid, certain});
              kinfo[K] = {j, 0, s};
            }
            if (!certain) add_uncertain(K, rid);
          }
        }
      }
    } else {
      for (int k = 1; k <= std::min(sim.n_hits[r], sim.p.max_depth); ++k) {
        const HitRec& hk = sim.rec[r * sim.n_seg + k - 1];
        bool vamb = false;
        int vx[3];
        if (sim.p.diffuse) diffuse_voxel(S, hk.q, vx, cfg.delta, &vamb);
        for (int j = 0; j < M; ++j) {
          auto vb = sim.vis.at({j, hk.dps});
          if (!vb.first && !vb.second) continue;
          bool certain = (k < e) && !vb.second;
          Key Ks = make_key(j, false, k, labels, k, nullptr);
          if (vb.first) {
            cands[Ks].push_back({rid, certain});
            kinfo[Ks] = {j, 0, k};
          }
          if (!certain) add_uncertain(Ks, rid);
          if (sim.p.diffuse) {
            Key Kd = make_key(j, true, k, labels, k - 1, vx);
            bool dcert = certain && !vamb;
            if (vb.first) {
              cands[Kd].push_back({rid, dcert});
              kinfo[Kd] = {j, 1, k};
            }
            if (!dcert) {
              // the voxel may be taken on either side of a face closer than delta
              int alt[3][2], na[3];
              for (int a = 0; a < 3; ++a) {
                double s = (comp(hk.q, a) - (double)S.bmin_f[a]) / S.rho;
                double frac = s - std::floor(s);
                na[a] = 1;
                alt[a][0] = vx[a];
                if (cfg.delta > 0 && frac * S.rho < cfg.delta) alt[a][na[a]++] = vx[a] - 1;
                else if (cfg.delta > 0 && (1.0 - frac) * S.rho < cfg.delta) alt[a][na[a]++] = vx[a] + 1;
              }
              for (int a0 = 0; a0 < na[0]; ++a0)
                for (int a1 = 0; a1 < na[1]; ++a1)
                  for (int a2 = 0; a2 < na[2]; ++a2) {
                    int vv[3] = {alt[0][a0], alt[1][a1], alt[2][a2]};
                    add_uncertain(make_key(j, true, k, labels, k - 1, vv), rid);
                  }
            }
          }
        }
      }
    }
  }

  // per key: try the candidates in ray order until one validates -- all of
  // them (rep_tries = 0: every candidate is refined, Sec. II-B-2, and the
  // duplicates of a key are removed, Sec. II-B-4), or at most rep_tries
  std::vector<Key> klist;
  for (auto& kv : cands) {
    std::sort(kv.second.begin(), kv.second.end(),
              [](const Cand& a, const Cand& b) { return a.ray < b.ray; });
    klist.push_back(kv.first);
  }
  sim.keys.assign(klist.size(), KeyOut());
  std::vector<Validation> vout(klist.size());
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t qi = 0; qi < (int64_t)klist.size(); ++qi) {
    const Key& K = klist[qi];
    auto& cl = cands.at(K);
    KeyOut& ko = sim.keys[qi];
    ko.key = K;
    std::tie(ko.j, ko.type, ko.k) = kinfo.at(K);
    ko.n_cand = (int64_t)cl.size();
    int labels[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m < 4; ++m) labels[m] = (int)((K.lo >> (16 * m)) & 0xFFFF);
    labels[4] = (int)(K.hi & 0xFFFF);
    const int64_t ntry =
        sim.p.rep_tries > 0 ? std::min<int64_t>(cl.size(), sim.p.rep_tries) : (int64_t)cl.size();
    for (int64_t c = 0; c < ntry; ++c) {
      int64_t rid = cl[c].ray;
      int64_t row = sim.ray_pos[rid];
      Validation v = ko.type == 1 ? validate_diffuse(sim, sim.rec, row, ko.k, ko.j, cfg)
                                  : validate_specular(sim, sim.rec, row, ko.k, ko.j, labels, cfg);
      ko.tried.push_back(rid);
      ko.tried_valid.push_back(v.valid);
      ko.tried_amb.push_back(v.amb || !cl[c].certain);
      if (v.valid) {
        ko.valid = true;
        ko.rep = rid;
        vout[qi] = v;
        // the same candidate along the two shadow trajectories
        if (cfg.delta > 0) {
          for (int p = 0; p < 2; ++p) {
            CastCfg quiet = cfg;
            quiet.delta = 0.0;
            quiet.wjit = kShadowJitter;
            quiet.wseed = p + 1;
            Validation w = ko.type == 1
                               ? validate_diffuse(sim, sim.recp[p], row, ko.k, ko.j, quiet)
                               : validate_specular(sim, sim.recp[p], row, ko.k, ko.j, labels, quiet);
            vout[qi].path.shadow_ok[p] = w.valid;
            if (w.valid) vout[qi].path.shadow[p] = std::make_shared<PathOut>(w.path);
          }
        }
        break;
      }
    }
  }
  // a key's outcome is "tried-certain" when every candidate tried for it is a
  // certain candidate with an unambiguous validation
  for (size_t qi = 0; qi < klist.size(); ++qi) {
    KeyOut& ko = sim.keys[qi];
    bool certain = true;
    for (int a : ko.tried_amb)
      if (a) certain = false;
    ko.certain = certain;
    if (ko.valid) {
      PathOut P = vout[qi].path;
      P.key = ko.key;
      P.j = ko.j;
      P.rep = ko.rep;
      P.certain = certain;
      ko.path = (int)sim.paths.size();
      sim.paths.push_back(P);
    }
  }
  // LOS paths
  double lam = kC0 / sim.p.freq;
  for (int j = 0; j < M; ++j) {
    if (!sim.los[j].first) continue;
    PathOut P;
    P.key = make_key(j, false, 0, nullptr, 0, nullptr);
    P.j = j;
    P.type = 0;
    P.k = 0;
    P.rep = -1;
    double d = norm(sim.rx[j] - sim.tx);
    P.length = d;
    P.geo = lam / (4.0 * kPi * d);
    P.tau = d / kC0;
    P.certain = !sim.los[j].second;
    sim.paths.push_back(P);
  }
}

// ---------------------------------------------------------------------------
// Vector polarisation (pol = 2; a reading, the paper leaves the field model to
// an external library).  TX and RX are isotropic with vertical polarisation:
// the field leaves along d with unit vector theta^(d) of the spherical basis
// about +z, and is received with theta^(u), u the direction from the RX back
// along the arriving ray.  At an interaction with normal n, incoming d_i and
// outgoing d_o: s^ = unit(d_i x n), p^_in = s^ x d_i, p^_out = s^ x d_o; the
// s component is multiplied by c Gamma_TE and the p component by c Gamma_TM
// (c = R, or S at a diffuse last interaction, whose d_o points to the RX).
// A specular interaction's normal is unit(d_o - d_i).  In these bases a path
// is a = geo r^T D_k B_{k-1} ... B_1 D_1 e0: e0 the TX polarisation in the
// first incoming basis, B_m the real 2x2 change from the outgoing basis of
// interaction m to the incoming basis of m+1, D_m = diag(c Gamma_TE, c Gamma_TM),
// r the RX polarisation in the last outgoing basis.
// ---------------------------------------------------------------------------
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

V3 theta_hat(V3 d) {
  const double st = std::sqrt(d.x * d.x + d.y * d.y);
  if (st < 1e-12) return {1.0, 0.0, 0.0};  // along the z axis: x^ by convention
  return {d.z * d.x / st, d.z * d.y / st, -st};
}

struct Jones {
  int k = 0;
  double los = 0.0;       // k = 0: theta^(d) . theta^(-d)
  double e0[2] = {0, 0};
  double B[5][2][2] = {};
  double r[2] = {0, 0};
};

Jones make_jones(V3 tx, V3 rx, const V3* pts, int k, bool diffuse, V3 nd) {
  Jones J;
  J.k = k;
  V3 d[6];
  if (k == 0) {
    const V3 u = unit(rx - tx);
    J.los = dot(theta_hat(u), theta_hat((-1.0) * u));
    return J;
  }
  d[0] = unit(pts[0] - tx);
  for (int m = 1; m < k; ++m) d[m] = unit(pts[m] - pts[m - 1]);
  d[k] = unit(rx - pts[k - 1]);
  V3 sv[5], pin[5], pout[5];
  for (int m = 0; m < k; ++m) {
    const V3 n = (diffuse && m == k - 1) ? nd : unit(d[m + 1] - d[m]);
    V3 sx = cross(d[m], n);
    if (norm(sx) < 1e-12) sx = cross(d[m], std::fabs(d[m].z) < 0.9 ? V3{0, 0, 1} : V3{1, 0, 0});
    sv[m] = unit(sx);
    pin[m] = cross(sv[m], d[m]);
    pout[m] = cross(sv[m], d[m + 1]);
  }
  const V3 t0 = theta_hat(d[0]);
  J.e0[0] = dot(t0, sv[0]);
  J.e0[1] = dot(t0, pin[0]);
  for (int m = 0; m + 1 < k; ++m) {
    J.B[m][0][0] = dot(sv[m + 1], sv[m]);
    J.B[m][0][1] = dot(sv[m + 1], pout[m]);
    J.B[m][1][0] = dot(pin[m + 1], sv[m]);
    J.B[m][1][1] = dot(pin[m + 1], pout[m]);
  }
  const V3 tr = theta_hat((-1.0) * d[k]);
  J.r[0] = dot(tr, sv[k - 1]);
  J.r[1] = dot(tr, pout[k - 1]);
  return J;
}

// a / geo for diagonal factors D[m] = (c Gamma_TE, c Gamma_TM)
cd jones_amplitude(const Jones& J, const cd (*D)[2]) {
  if (J.k == 0) return cd(J.los, 0.0);
  cd v[2] = {J.e0[0], J.e0[1]};
  for (int m = 0; m < J.k; ++m) {
    v[0] *= D[m][0];
    v[1] *= D[m][1];
    if (m + 1 < J.k) {
      const cd a0 = J.B[m][0][0] * v[0] + J.B[m][0][1] * v[1];
      const cd a1 = J.B[m][1][0] * v[0] + J.B[m][1][1] * v[1];
      v[0] = a0;
      v[1] = a1;
    }
  }
  return J.r[0] * v[0] + J.r[1] * v[1];
}

// d(a/geo)/d(D[m][c]) for every interaction m and component c
void jones_partials(const Jones& J, const cd (*D)[2], cd (*dA)[2]) {
  cd fwd[5][2];  // field entering interaction m (its incoming basis)
  cd v[2] = {J.e0[0], J.e0[1]};
  for (int m = 0; m < J.k; ++m) {
    fwd[m][0] = v[0];
    fwd[m][1] = v[1];
    v[0] *= D[m][0];
    v[1] *= D[m][1];
    if (m + 1 < J.k) {
      const cd a0 = J.B[m][0][0] * v[0] + J.B[m][0][1] * v[1];
      const cd a1 = J.B[m][1][0] * v[0] + J.B[m][1][1] * v[1];
      v[0] = a0;
      v[1] = a1;
    }
  }
  cd w[2] = {J.r[0], J.r[1]};  // row vector after interaction m, in its outgoing basis
  for (int m = J.k - 1; m >= 0; --m) {
    dA[m][0] = w[0] * fwd[m][0];
    dA[m][1] = w[1] * fwd[m][1];
    // w <- w D_m B_{m-1}
    const cd u0 = w[0] * D[m][0], u1 = w[1] * D[m][1];
    if (m > 0) {
      w[0] = u0 * J.B[m - 1][0][0] + u1 * J.B[m - 1][1][0];
      w[1] = u0 * J.B[m - 1][0][1] + u1 * J.B[m - 1][1][1];
    }
  }
}

// ---------------------------------------------------------------------------
// Single-bounce edge diffraction (Sec. II-B-3).  An edge is a segment e0 -> e1
// with the outward normals n0, n1 of its two faces and their materials; the
// solid is the convex wedge {x : (x - D).n0 < 0 and (x - D).n1 < 0}.
//   Path: the point D of the edge line minimising |TX - D| + |D - RX| (the
//     path-length minimisation of the specular refinement, here in closed
//     form: unfold the two half-planes through the edge into one plane and
//     cross the edge with the straight line); kept when D lies strictly inside
//     the segment and TX and RX are both outside the wedge.
//   Visibility: from the TX and from the RX, a cast toward D with no hit
//     closer than rho (the voxel size) before D: the faces meeting at the
//     edge are crossed only at D itself.
//   Field (the paper leaves it to its EM library; a reading): the UTD wedge
//     coefficient of Kouyoumjian and Pathak (1974) with the face reflection
//     coefficients of Luebbers (1984) weighting the reflection-boundary terms,
//     for a spherical wave: a = lambda/(4 pi) D / sqrt(s s' (s + s')),
//     D = K [T1 + T2 + R0 T3 + Rn T4], K = -exp(-j pi/4) / (2 n sqrt(2 pi k) sin b0),
//     distance parameter L = s s' sin^2 b0 / (s + s').  R0 (Rn) is the
//     Fresnel coefficient of face 0 (n) at its true incidence cosine
//     sin b0 sin(phi') (sin b0 sin(n pi - phi)); soft coefficients (TE) for
//     pol 0, hard (TM) for pol 1, and for the vector model the edge-fixed
//     basis: a = geo (v_s D_s + v_h D_h), v_s = -(theta^_rx . b^)(theta^_tx . b^'),
//     v_h = -(theta^_rx . f^)(theta^_tx . f^'), with f^' = -unit(e x s'),
//     b^' = f^' x s', f^ = unit(e x s), b^ = f^ x s.
// ---------------------------------------------------------------------------
struct WedgeFrame {
  V3 e;          // unit edge direction
  double len;
  V3 n0, n1;     // face normals
  V3 t0;         // in face 0, normal to the edge, pointing away from it
  double nw;     // exterior angle / pi
};

WedgeFrame wedge_frame(V3 a, V3 b, V3 n0, V3 n1) {
  WedgeFrame W;
  const V3 ev = b - a;
  W.len = norm(ev);
  W.e = (1.0 / W.len) * ev;
  W.n0 = n0;
  W.n1 = n1;
  V3 t0 = unit(cross(n0, W.e));
  if (dot(t0, n1) > 0.0) t0 = (-1.0) * t0;
  V3 t1 = unit(cross(n1, W.e));
  if (dot(t1, n0) > 0.0) t1 = (-1.0) * t1;
  W.t0 = t0;
  W.nw = 2.0 - std::acos(std::max(-1.0, std::min(1.0, dot(t0, t1)))) / kPi;
  return W;
}

// angle of x about the edge through D, from face 0 through the exterior, in [0, 2 pi)
double wedge_angle(const WedgeFrame& W, V3 D, V3 x) {
  const V3 v = x - D;
  const V3 vp = v - dot(v, W.e) * W.e;
  double phi = std::atan2(dot(vp, W.n0), dot(vp, W.t0));
  if (phi < 0.0) phi += 2.0 * kPi;
  return phi;
}

// UTD transition function F(x) = 2j sqrt(x) exp(jx) int_{sqrt x}^inf exp(-j t^2) dt,
// x >= 0: the integral as (sqrt(pi)/2) exp(-j pi/4) minus int_0^{sqrt x} by
// composite 10-point Gauss-Legendre (panels of at most 0.05); for x > 60 the
// asymptotic series sum_n (-1)^n (2n-1)!! / (2jx)^n.
cd utd_F(double x) {
  if (x <= 0.0) return cd(0.0, 0.0);
  if (x > 60.0) {
    cd sum(1.0, 0.0), term(1.0, 0.0);
    for (int n = 1; n < 40; ++n) {
      term *= -(2.0 * n - 1.0) / (cd(0.0, 2.0 * x));
      sum += term;
      if (std::abs(term) < 1e-18) break;
    }
    return sum;
  }
  static double gx[10], gw[10];
  static bool init = false;
  if (!init) {  // Legendre nodes by Newton iteration on P_10
    for (int i = 0; i < 10; ++i) {
      double z = std::cos(kPi * (i + 0.75) / 10.5), pp = 0.0;
      for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= 10; ++j) {
          const double p3 = p2;
          p2 = p1;
          p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = 10.0 * (z * p1 - p2) / (z * z - 1.0);
        const double dz = p1 / pp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      gx[i] = z;
      gw[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
    init = true;
  }
  const double u = std::sqrt(x);
  const int np = std::max(1, (int)std::ceil(u / 0.05));
  const double h = u / np;
  cd acc(0.0, 0.0);
  for (int p = 0; p < np; ++p) {
    const double c = (p + 0.5) * h;
    for (int i = 0; i < 10; ++i) {
      const double t = c + 0.5 * h * gx[i];
      acc += (0.5 * h * gw[i]) * std::exp(cd(0.0, -t * t));
    }
  }
  const cd tail = 0.5 * std::sqrt(kPi) * std::exp(cd(0.0, -kPi / 4.0)) - acc;
  return cd(0.0, 2.0) * u * std::exp(cd(0.0, x)) * tail;
}

struct UtdTerms {
  cd t12, t3, t4;  // K (T1 + T2), K T3, K T4
};

UtdTerms utd_terms(double phi_in, double phi_out, double nw, double sinb, double L, double k) {
  const cd K = -std::exp(cd(0.0, -kPi / 4.0)) / (2.0 * nw * std::sqrt(2.0 * kPi * k) * sinb);
  auto a_pm = [&](double beta, int sgn) {
    const double N = std::round((beta + sgn * kPi) / (2.0 * kPi * nw));
    const double c = std::cos((2.0 * kPi * nw * N - beta) / 2.0);
    return 2.0 * c * c;
  };
  auto cot = [](double v) { return std::cos(v) / std::sin(v); };
  const double bm = phi_out - phi_in, bp = phi_out + phi_in;
  const cd T1 = cot((kPi + bm) / (2.0 * nw)) * utd_F(k * L * a_pm(bm, +1));
  const cd T2 = cot((kPi - bm) / (2.0 * nw)) * utd_F(k * L * a_pm(bm, -1));
  const cd T3 = cot((kPi - bp) / (2.0 * nw)) * utd_F(k * L * a_pm(bp, -1));
  const cd T4 = cot((kPi + bp) / (2.0 * nw)) * utd_F(k * L * a_pm(bp, +1));
  return {K * (T1 + T2), K * T3, K * T4};
}

// Geometry of the diffracted path TX -> D -> RX of one edge
struct DiffGeom {
  bool ok = false;
  V3 D{0, 0, 0};
  double tpar = 0;          // position of D along the edge
  double s_in = 0, s_out = 0, phi_in = 0, phi_out = 0, sinb = 0;
  double side_tx = 0, side_rx = 0;  // max signed distance to the two face planes
  double vs = 0, vh = 0;    // vector-model projections
};

DiffGeom diffraction_geometry(const WedgeFrame& W, V3 a, V3 tx, V3 rx) {
  DiffGeom G;
  const V3 wt = tx - a, wr = rx - a;
  const double at = dot(wt, W.e), ar = dot(wr, W.e);
  const double bt = norm(wt - at * W.e), br = norm(wr - ar * W.e);
  if (!(bt + br > 0.0)) return G;
  G.tpar = (at * br + ar * bt) / (bt + br);
  G.D = a + G.tpar * W.e;
  G.side_tx = std::max(dot(tx - G.D, W.n0), dot(tx - G.D, W.n1));
  G.side_rx = std::max(dot(rx - G.D, W.n0), dot(rx - G.D, W.n1));
  G.s_in = norm(G.D - tx);
  G.s_out = norm(rx - G.D);
  const V3 si = (1.0 / G.s_in) * (G.D - tx), so = (1.0 / G.s_out) * (rx - G.D);
  const double cb = dot(si, W.e);
  G.sinb = std::sqrt(std::max(0.0, 1.0 - cb * cb));
  G.phi_in = wedge_angle(W, G.D, tx);
  G.phi_out = wedge_angle(W, G.D, rx);
  const V3 fi = (-1.0) * unit(cross(W.e, si)), bi = cross(fi, si);
  const V3 fo = unit(cross(W.e, so)), bo = cross(fo, so);
  const V3 tht = theta_hat(si), thr = theta_hat((-1.0) * so);
  G.vs = -dot(thr, bo) * dot(tht, bi);
  G.vh = -dot(thr, fo) * dot(tht, fi);
  G.ok = G.tpar > 0.0 && G.tpar < W.len && G.side_tx > 0.0 && G.side_rx > 0.0 && G.sinb > 0.0;
  return G;
}

// a of a diffracted path and its derivatives w.r.t. the two face
// permittivities (d_eta[0] face 0, d_eta[1] face n)
cd diffraction_coefficient(const WedgeFrame& W, const DiffGeom& G, cd eta0, cd eta1, double freq,
                           int pol, cd* d_eta) {
  const double k = 2.0 * kPi * freq / kC0, lam = kC0 / freq;
  const double L = G.s_in * G.s_out * G.sinb * G.sinb / (G.s_in + G.s_out);
  const UtdTerms T = utd_terms(G.phi_in, G.phi_out, W.nw, G.sinb, L, k);
  const double geo = lam / (4.0 * kPi * std::sqrt(G.s_in * G.s_out * (G.s_in + G.s_out)));
  const double c0 = G.sinb * std::sin(G.phi_in), c1 = G.sinb * std::sin(W.nw * kPi - G.phi_out);
  cd a(0.0, 0.0), g0(0.0, 0.0), g1(0.0, 0.0);
  for (int t = 0; t < 2; ++t) {
    const double v = pol == 2 ? (t == 0 ? G.vs : G.vh) : (t == pol ? 1.0 : 0.0);
    if (v == 0.0) continue;
    const cd Dc = T.t12 + fresnel(eta0, c0, t) * T.t3 + fresnel(eta1, c1, t) * T.t4;
    a += v * Dc;
    g0 += v * dfresnel_deta(eta0, c0, t) * T.t3;
    g1 += v * dfresnel_deta(eta1, c1, t) * T.t4;
  }
  if (d_eta) {
    d_eta[0] = geo * g0;
    d_eta[1] = geo * g1;
  }
  return geo * a;
}

WedgeFrame path_wedge(const PathOut& P) { return wedge_frame(P.e0, P.e1, P.en0, P.en1); }

// a of a stored diffracted path for given TX and RX positions (ok = false
// when the edge gives no path there); its delay in *tau
cd diffracted_path_coefficient(const PathOut& P, V3 tx, V3 rx, const double* eps,
                               const double* sig, double freq, int pol, bool* ok, double* tau,
                               cd* d_eta) {
  const WedgeFrame W = path_wedge(P);
  const DiffGeom G = diffraction_geometry(W, P.e0, tx, rx);
  if (ok) *ok = G.ok;
  if (tau) *tau = (G.s_in + G.s_out) / kC0;
  return diffraction_coefficient(W, G, permittivity(eps[P.mats[0]], sig[P.mats[0]], freq),
                                 permittivity(eps[P.mats[1]], sig[P.mats[1]], freq), freq, pol,
                                 d_eta);
}

Jones path_jones(const Sim& sim, const PathOut& P) {
  return make_jones(sim.tx, sim.rx[P.j], P.pts, P.k, P.type == 1, P.nd);
}

cd path_coefficient(const Sim& sim, const PathOut& P, const double* eps, const double* sig,
                    const double* sca, double freq, int pol) {
  if (P.type == 2)
    return diffracted_path_coefficient(P, sim.tx, sim.rx[P.j], eps, sig, freq, pol, nullptr,
                                       nullptr, nullptr);
  if (pol == 2) {
    cd D[5][2];
    for (int m = 0; m < P.k; ++m) {
      const int l = P.mats[m];
      const cd eta = permittivity(eps[l], sig[l], freq);
      const bool last_diffuse = P.type == 1 && m == P.k - 1;
      const double c = last_diffuse ? sca[l] : std::sqrt(std::max(0.0, 1.0 - sca[l] * sca[l]));
      D[m][0] = c * fresnel(eta, P.cosv[m], 0);
      D[m][1] = c * fresnel(eta, P.cosv[m], 1);
    }
    return P.geo * jones_amplitude(path_jones(sim, P), D);
  }
  cd a(P.geo, 0.0);
  for (int m = 0; m < P.k; ++m) {
    int l = P.mats[m];
    cd G = fresnel(permittivity(eps[l], sig[l], freq), P.cosv[m], pol);
    bool last_diffuse = P.type == 1 && m == P.k - 1;
    double f = last_diffuse ? sca[l] : std::sqrt(std::max(0.0, 1.0 - sca[l] * sca[l]));
    a *= f * G;
  }
  return a;
}

}  // namespace

// ---------------------------------------------------------------------------
// C API (ctypes)
// ---------------------------------------------------------------------------
extern "C" {

void* orc_scene_create(const float* pos, const float* nrm, const uint16_t* surf,
                       const uint8_t* mat, int64_t n, double rho, double r_p, double lambda_d,
                       double grid_cell, double band_cap) {
  return build_scene(pos, nrm, surf, mat, n, rho, r_p, lambda_d, grid_cell, band_cap);
}

void orc_scene_destroy(void* s) { delete (Scene*)s; }

int64_t orc_scene_n_dps(void* s) { return (int64_t)((Scene*)s)->dps_pts.size(); }

void orc_scene_bmin(void* s, float* out) {
  for (int k = 0; k < 3; ++k) out[k] = ((Scene*)s)->bmin_f[k];
}

void orc_scene_dps(void* s, int32_t* vox, int32_t* count, double* recv) {
  Scene* S = (Scene*)s;
  for (size_t d = 0; d < S->dps_pts.size(); ++d) {
    for (int k = 0; k < 3; ++k) vox[3 * d + k] = S->dps_vox[d][k];
    count[d] = (int32_t)S->dps_pts[d].size();
    recv[3 * d] = S->recv[d].x;
    recv[3 * d + 1] = S->recv[d].y;
    recv[3 * d + 2] = S->recv[d].z;
  }
}

void orc_scene_point_dps(void* s, int32_t* out) {
  Scene* S = (Scene*)s;
  for (int64_t i = 0; i < S->n; ++i) out[i] = S->dps_of[i];
}

// One cast.  out: t, q[3], n[3], cos_in.  Returns 1 on a hit.
int orc_cast(void* s, const double* o, const double* d, int32_t skip_dps, double t_min,
             double t_max, double delta, int weighted, double* out, int64_t* idx, int32_t* dps,
             int32_t* amb) {
  Scene* S = (Scene*)s;
  CastCfg cfg;
  cfg.t_min = t_min;
  cfg.delta = delta;
  V3 dv = unit({d[0], d[1], d[2]});
  Hit h;  // a ray that is not finite hits nothing (and must not reach the grid walk)
  const double in[6] = {o[0], o[1], o[2], dv.x, dv.y, dv.z};
  bool finite = true;
  for (double v : in) finite = finite && std::isfinite(v);
  if (finite) h = cast(*S, {o[0], o[1], o[2]}, dv, skip_dps, t_max, weighted != 0, cfg);
  out[0] = h.t;
  out[1] = h.q.x; out[2] = h.q.y; out[3] = h.q.z;
  out[4] = h.n.x; out[5] = h.n.y; out[6] = h.n.z;
  out[7] = h.cos_in;
  *idx = h.idx;
  *dps = h.dps;
  *amb = h.amb ? 1 : 0;
  return h.hit ? 1 : 0;
}

// SDF intersection of the prior work (Eq. 2), for the ablation against the
// disc model.  The paper gives the Gaussian weight only; the rest is a
// reading.  Per DPS D: f_D(s) = sum_i w_i n_i.(s - p_i) / sum_i w_i with
// w_i = exp(-|p_i - s|^2 / (2 sigma^2)) over D's points, defined where
// sum_i w_i >= e^-2.  Along the ray, D is marched over the interval where the
// ray crosses the bounding box of its points grown by 2 sigma (clipped to
// (t_min, t_max)): samples t_k = t_in + k sigma / 2; the first k with both
// samples defined and f(t_k) > 0 >= f(t_k+1) brackets the surface (outside
// to inside), 20 bisection steps refine it and the hit is the midpoint.  Each
// DPS is marched over its whole interval (the grid and the bracket do not
// depend on other DPS).  The hit is the smallest t over all DPS (ties:
// smaller DPS index); its normal
// the normalised sum_i w_i n_i, turned to face the ray; its label the label of
// D's point nearest to the hit.  Ambiguous: a bracketing sample with |f| <
// delta, a weight sum within 1e-4 (relative) of the threshold, or two DPS hits
// within delta.
int orc_cast_sdf(void* s, const double* o_in, const double* d_in, double t_min, double t_max,
                 double sigma, double delta, double* out, int32_t* dps_out, int32_t* label_out,
                 int32_t* amb_out) {
  Scene* S = (Scene*)s;
  const V3 o{o_in[0], o_in[1], o_in[2]};
  const V3 d = unit({d_in[0], d_in[1], d_in[2]});
  if (!(std::isfinite(o.x) && std::isfinite(o.y) && std::isfinite(o.z) && std::isfinite(d.x) &&
        std::isfinite(d.y) && std::isfinite(d.z))) {
    *amb_out = 0;
    return 0;  // a ray that is not finite hits nothing
  }
  const double wmin = std::exp(-2.0), h = 0.5 * sigma, inv2s2 = 1.0 / (2.0 * sigma * sigma);
  double best = kInf;
  int best_D = -1;
  bool amb = false;
  std::vector<double> hits;  // t of every DPS hit, for the tie band
  auto eval = [&](const std::vector<int>& pts, V3 x, double* f, double* W) {
    double sw = 0.0, sf = 0.0;
    for (int i : pts) {
      const V3 v = x - S->P[i];
      const double w = std::exp(-dot(v, v) * inv2s2);
      sw += w;
      sf += w * dot(S->N[i], v);
    }
    *W = sw;
    *f = sw > 0.0 ? sf / sw : 0.0;
  };
  for (size_t D = 0; D < S->dps_pts.size(); ++D) {
    const std::vector<int>& pts = S->dps_pts[D];
    double lo[3] = {kInf, kInf, kInf}, hi[3] = {-kInf, -kInf, -kInf};
    for (int i : pts) {
      const double c[3] = {S->P[i].x, S->P[i].y, S->P[i].z};
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], c[a]);
        hi[a] = std::max(hi[a], c[a]);
      }
    }
    const double oc[3] = {o.x, o.y, o.z}, dc[3] = {d.x, d.y, d.z};
    double t0 = t_min, t1 = t_max;
    for (int a = 0; a < 3; ++a) {
      const double l = lo[a] - 2.0 * sigma, u = hi[a] + 2.0 * sigma;
      if (dc[a] == 0.0) {
        if (oc[a] < l || oc[a] > u) t0 = kInf;
        continue;
      }
      double ta = (l - oc[a]) / dc[a], tb = (u - oc[a]) / dc[a];
      if (ta > tb) std::swap(ta, tb);
      t0 = std::max(t0, ta);
      t1 = std::min(t1, tb);
    }
    if (!(t0 <= t1)) continue;
    double fa, Wa;
    eval(pts, o + t0 * d, &fa, &Wa);
    for (int k = 0;; ++k) {
      const double ta = t0 + k * h, tb = t0 + (k + 1) * h;
      // a bracket starting beyond the best hit (plus the tie band) cannot win
      if (tb > t1 || ta > best + delta) break;
      double fb, Wb;
      eval(pts, o + tb * d, &fb, &Wb);
      if (std::fabs(Wa - wmin) < 1e-4 * wmin || std::fabs(Wb - wmin) < 1e-4 * wmin) amb = true;
      const bool defined = Wa >= wmin && Wb >= wmin;
      if (defined && (std::fabs(fa) < delta || std::fabs(fb) < delta) && fa * fb <= delta * delta)
        amb = true;
      if (defined && fa > 0.0 && fb <= 0.0) {
        double l = ta, u = tb;
        for (int it = 0; it < 20; ++it) {
          const double m = 0.5 * (l + u);
          double fm, Wm;
          eval(pts, o + m * d, &fm, &Wm);
          if (fm > 0.0) l = m;
          else u = m;
        }
        const double t = 0.5 * (l + u);
        hits.push_back(t);
        if (t < best) {
          best = t;
          best_D = (int)D;
        }
        break;
      }
      fa = fb;
      Wa = Wb;
    }
  }
  for (double t : hits)
    if (t != best && std::fabs(t - best) < delta) amb = true;
  *amb_out = amb ? 1 : 0;
  if (best_D < 0) return 0;
  const V3 q = o + best * d;
  V3 sn{0, 0, 0};
  int lab = -1;
  double dmin = kInf;
  for (int i : S->dps_pts[best_D]) {
    const V3 v = q - S->P[i];
    const double w = std::exp(-dot(v, v) * inv2s2);
    sn = sn + w * S->N[i];
    const double dd = dot(v, v);
    if (dd < dmin || (dd == dmin && i < lab)) {
      dmin = dd;
      lab = i;
    }
  }
  V3 n = unit(sn);
  if (dot(n, d) > 0.0) n = (-1.0) * n;
  out[0] = best;
  out[1] = q.x; out[2] = q.y; out[3] = q.z;
  out[4] = n.x; out[5] = n.y; out[6] = n.z;
  *dps_out = best_D;
  *label_out = S->surf[lab] | (S->mat[lab] << 16);
  return 1;
}

void orc_fib_dirs(int64_t n, const int64_t* ids, int64_t m, double* out) {
  for (int64_t i = 0; i < m; ++i) {
    V3 d = fib_dir(ids[i], n);
    out[3 * i] = d.x;
    out[3 * i + 1] = d.y;
    out[3 * i + 2] = d.z;
  }
}

void* orc_sim_run(void* s, const double* tx, const double* rx, int n_rx, const orc_params* p,
                  const int64_t* ray_ids, int64_t n_ids) {
  Sim* sim = new Sim();
  sim->S = (Scene*)s;
  sim->p = *p;
#ifdef _OPENMP
  if (p->n_threads > 0) omp_set_num_threads(p->n_threads);
#endif
  sim->tx = {tx[0], tx[1], tx[2]};
  for (int j = 0; j < n_rx; ++j) sim->rx.push_back({rx[3 * j], rx[3 * j + 1], rx[3 * j + 2]});
  sim->ray_ids.assign(ray_ids, ray_ids + n_ids);
  sim->ray_pos.assign(p->n_rays, -1);
  for (int64_t i = 0; i < n_ids; ++i) sim->ray_pos[ray_ids[i]] = i;
  run_sim(*sim);
  return sim;
}

void orc_sim_destroy(void* s) { delete (Sim*)s; }

int orc_sim_n_seg(void* s) { return ((Sim*)s)->n_seg; }

// per-ray hit records [n_ids][n_seg]
void orc_sim_hits(void* s, int64_t* idx, int32_t* dps, double* t, double* q, double* nrm,
                  double* cos_in, int32_t* amb, int32_t* excl, int32_t* n_hits) {
  Sim* sim = (Sim*)s;
  int64_t n = (int64_t)sim->ray_ids.size();
  for (int64_t r = 0; r < n; ++r) {
    excl[r] = sim->excl[r];
    n_hits[r] = sim->n_hits[r];
    for (int k = 0; k < sim->n_seg; ++k) {
      const HitRec& h = sim->rec[r * sim->n_seg + k];
      int64_t o = r * sim->n_seg + k;
      idx[o] = h.idx;
      dps[o] = h.dps;
      t[o] = h.t;
      q[3 * o] = h.q.x; q[3 * o + 1] = h.q.y; q[3 * o + 2] = h.q.z;
      nrm[3 * o] = h.n.x; nrm[3 * o + 1] = h.n.y; nrm[3 * o + 2] = h.n.z;
      cos_in[o] = h.cos_in;
      amb[o] = h.amb;
    }
  }
}

void orc_sim_los(void* s, int32_t* clear, int32_t* amb) {
  Sim* sim = (Sim*)s;
  for (size_t j = 0; j < sim->los.size(); ++j) {
    clear[j] = sim->los[j].first;
    amb[j] = sim->los[j].second;
  }
}

int64_t orc_sim_n_vis(void* s) { return (int64_t)((Sim*)s)->vis.size(); }

void orc_sim_vis(void* s, int32_t* j, int32_t* dps, int32_t* bit, int32_t* amb) {
  Sim* sim = (Sim*)s;
  int64_t i = 0;
  for (auto& kv : sim->vis) {
    j[i] = kv.first.first;
    dps[i] = kv.first.second;
    bit[i] = kv.second.first;
    amb[i] = kv.second.second;
    ++i;
  }
}

// Visibility bits for explicit (rx, dps) pairs, without a simulation.
void orc_vis_pairs(void* s, const double* rx, const int32_t* j, const int32_t* dps, int64_t n,
                   double t_min, double delta, int32_t* bit, int32_t* amb) {
  Scene* S = (Scene*)s;
  CastCfg cfg;
  cfg.t_min = t_min;
  cfg.delta = delta;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    V3 r{rx[3 * j[i]], rx[3 * j[i] + 1], rx[3 * j[i] + 2]};
    auto v = vis_cast(*S, r, dps[i], cfg);
    bit[i] = v.first;
    amb[i] = v.second;
  }
}

int64_t orc_sim_n_keys(void* s) { return (int64_t)((Sim*)s)->keys.size(); }

void orc_sim_keys(void* s, uint64_t* hi, uint64_t* lo, int32_t* n_tried, int64_t* n_cand,
                  int64_t* rep, int32_t* valid, int32_t* certain, int32_t* path) {
  Sim* sim = (Sim*)s;
  for (size_t i = 0; i < sim->keys.size(); ++i) {
    const KeyOut& k = sim->keys[i];
    hi[i] = k.key.hi;
    lo[i] = k.key.lo;
    n_tried[i] = (int32_t)k.tried.size();
    n_cand[i] = k.n_cand;
    rep[i] = k.rep;
    valid[i] = k.valid;
    certain[i] = k.certain;
    path[i] = k.path;
  }
}

int64_t orc_sim_n_paths(void* s) { return (int64_t)((Sim*)s)->paths.size(); }

void orc_sim_paths(void* s, uint64_t* hi, uint64_t* lo, int32_t* j, int32_t* type, int32_t* k,
                   int64_t* rep, double* pts, int32_t* mats, double* cosv, double* geo,
                   double* tau, double* length, int32_t* certain) {
  Sim* sim = (Sim*)s;
  for (size_t i = 0; i < sim->paths.size(); ++i) {
    const PathOut& P = sim->paths[i];
    hi[i] = P.key.hi;
    lo[i] = P.key.lo;
    j[i] = P.j;
    type[i] = P.type;
    k[i] = P.k;
    rep[i] = P.rep;
    for (int m = 0; m < 5; ++m) {
      pts[15 * i + 3 * m] = P.pts[m].x;
      pts[15 * i + 3 * m + 1] = P.pts[m].y;
      pts[15 * i + 3 * m + 2] = P.pts[m].z;
      mats[5 * i + m] = P.mats[m];
      cosv[5 * i + m] = P.cosv[m];
    }
    geo[i] = P.geo;
    tau[i] = P.tau;
    length[i] = P.length;
    certain[i] = P.certain;
  }
}

// Single-bounce diffraction paths of every (edge, RX) pair, appended to the
// paths after the ray-traced ones (type 2, key hi = j << 56 | 1 << 52 |
// 1 << 51, lo = edge index, rep = edge index).  Edges as float32 arrays
// [n][3] (ends a, b; face normals n0, n1) and uint8 face materials.
// Ambiguous (not certain): D within delta of an edge end, TX or RX within
// delta of a face plane, or a visibility cast with an ambiguous decision.
void orc_sim_diffraction(void* s, int64_t n_edges, const float* ea, const float* eb,
                         const float* n0, const float* n1, const uint8_t* m0, const uint8_t* m1) {
  Sim* sim = (Sim*)s;
  const Scene& S = *sim->S;
  CastCfg cfg;
  cfg.t_min = sim->p.t_min;
  cfg.delta = sim->p.delta;
  const double lam = kC0 / sim->p.freq, dl = sim->p.delta;
  const int M = (int)sim->rx.size();
  auto v3 = [](const float* p, int64_t e) {
    return V3{(double)p[3 * e], (double)p[3 * e + 1], (double)p[3 * e + 2]};
  };
  std::vector<PathOut> out((size_t)n_edges * M);
  std::vector<char> keep((size_t)n_edges * M, 0), amb_q((size_t)n_edges * M, 0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n_edges * M; ++q) {
    const int64_t e = q / M;
    const int j = (int)(q % M);
    const V3 a = v3(ea, e), b = v3(eb, e);
    const WedgeFrame W = wedge_frame(a, b, v3(n0, e), v3(n1, e));
    const DiffGeom G = diffraction_geometry(W, a, sim->tx, sim->rx[j]);
    bool amb = dl > 0 && (std::fabs(G.tpar) < dl || std::fabs(G.tpar - W.len) < dl ||
                          std::fabs(G.side_tx) < dl || std::fabs(G.side_rx) < dl);
    amb_q[q] = amb;
    if (!G.ok) continue;
    bool vis = true;
    const V3 ends[2] = {sim->tx, sim->rx[j]};
    const double dist[2] = {G.s_in, G.s_out};
    for (int t = 0; t < 2 && vis; ++t) {
      const double tmax = dist[t] - S.rho;
      if (!(tmax > cfg.t_min)) continue;
      const Hit h = cast(S, ends[t], (1.0 / dist[t]) * (G.D - ends[t]), -1, tmax, false, cfg);
      sim->val_casts++;
      if (h.amb) amb = true;
      if (h.hit) vis = false;
    }
    amb_q[q] = amb;
    if (!vis) continue;
    PathOut& P = out[q];
    P.key.hi = ((uint64_t)(j & 0xFF) << 56) | (1ull << 52) | (1ull << 51);
    P.key.lo = (uint64_t)e;
    P.j = j;
    P.type = 2;
    P.k = 1;
    P.rep = e;
    P.pts[0] = G.D;
    P.mats[0] = m0[e];
    P.mats[1] = m1[e];
    P.cosv[0] = G.sinb * std::sin(G.phi_in);
    P.cosv[1] = G.sinb * std::sin(W.nw * kPi - G.phi_out);
    P.e0 = a;
    P.e1 = b;
    P.en0 = v3(n0, e);
    P.en1 = v3(n1, e);
    P.length = G.s_in + G.s_out;
    P.tau = P.length / kC0;
    P.geo = lam / (4.0 * kPi * std::sqrt(G.s_in * G.s_out * (G.s_in + G.s_out)));
    P.certain = !amb;
    keep[q] = 1;
  }
  for (size_t q = 0; q < out.size(); ++q) {
    if (keep[q]) sim->paths.push_back(out[q]);
    if (amb_q[q]) {  // either outcome possible under float rounding
      const int64_t e = (int64_t)q / M;
      const Key K{((uint64_t)((q % M) & 0xFF) << 56) | (1ull << 52) | (1ull << 51), (uint64_t)e};
      sim->uncertain_cand[K].push_back(e);
    }
  }
}

// UTD transition function F(x) (pins)
void orc_utd_F(double x, double* re, double* im) {
  const cd F = utd_F(x);
  *re = F.real();
  *im = F.imag();
}

// a of the diffracted path TX -> edge -> RX on explicit geometry (pins):
// edge ends a, b, face normals n0, n1, face permittivities eta0, eta1
// (re, im); returns 0 and leaves a untouched when the edge yields no path
int orc_diffraction_amplitude(const double* tx, const double* rx, const double* a,
                              const double* b, const double* n0, const double* n1,
                              const double* eta0, const double* eta1, double freq, int pol,
                              double* re, double* im) {
  auto v3 = [](const double* p) { return V3{p[0], p[1], p[2]}; };
  const WedgeFrame W = wedge_frame(v3(a), v3(b), v3(n0), v3(n1));
  const DiffGeom G = diffraction_geometry(W, v3(a), v3(tx), v3(rx));
  if (!G.ok) return 0;
  const cd A = diffraction_coefficient(W, G, cd(eta0[0], eta0[1]), cd(eta1[0], eta1[1]), freq,
                                       pol, nullptr);
  *re = A.real();
  *im = A.imag();
  return 1;
}

// Geometry of the diffracted path (pins): D, then s', s, phi', phi, n, sin b0
int orc_diffraction_geometry(const double* tx, const double* rx, const double* a, const double* b,
                             const double* n0, const double* n1, double* out) {
  auto v3 = [](const double* p) { return V3{p[0], p[1], p[2]}; };
  const WedgeFrame W = wedge_frame(v3(a), v3(b), v3(n0), v3(n1));
  const DiffGeom G = diffraction_geometry(W, v3(a), v3(tx), v3(rx));
  out[0] = G.D.x;
  out[1] = G.D.y;
  out[2] = G.D.z;
  out[3] = G.s_in;
  out[4] = G.s_out;
  out[5] = G.phi_in;
  out[6] = G.phi_out;
  out[7] = W.nw;
  out[8] = G.sinb;
  return G.ok ? 1 : 0;
}

// [n_paths][3] surface normal at the scatter point of each diffuse path,
// facing the incoming ray (0 for specular and LOS paths)
void orc_sim_path_normals(void* s, double* nd) {
  Sim* sim = (Sim*)s;
  for (size_t i = 0; i < sim->paths.size(); ++i) {
    const PathOut& P = sim->paths[i];
    nd[3 * i] = P.nd.x;
    nd[3 * i + 1] = P.nd.y;
    nd[3 * i + 2] = P.nd.z;
  }
}

// Candidate status of ray `rid` for key (hi, lo):
//   0 certainly not a candidate, 1 certainly a candidate, 2 uncertain (the ray
//   could produce the key under a decision the oracle marks ambiguous: a
//   visibility bit, a voxel face, a sphere boundary, or any hit from the
//   ray's first ambiguous hit on, given a matching label prefix).
int orc_sim_cand_status(void* s, uint64_t hi, uint64_t lo, int64_t rid) {
  Sim* sim = (Sim*)s;
  Key K{hi, lo};
  auto ct = sim->cands.find(K);
  if (ct != sim->cands.end())
    for (const Cand& c : ct->second)
      if (c.ray == rid) return c.certain ? 1 : 2;
  auto it = sim->uncertain_cand.find(K);
  if (it != sim->uncertain_cand.end())
    for (int64_t r : it->second)
      if (r == rid) return 2;
  if ((hi >> 51) & 1) return 0;  // a diffraction key: no ray candidates
  if (rid < 0 || rid >= (int64_t)sim->ray_pos.size()) return 0;
  int64_t row = sim->ray_pos[rid];
  if (row < 0) return 0;
  int e = sim->excl[row];
  int k = (int)((hi >> 52) & 7);
  int type = (int)((hi >> 55) & 1);
  int nlab = type == 1 ? k - 1 : k;
  int emax = sim->p.capture == 0 ? k + 1 : k;
  if (e > emax) return 0;
  int labels[5];
  for (int m = 0; m < 4; ++m) labels[m] = (int)((lo >> (16 * m)) & 0xFFFF);
  labels[4] = (int)(hi & 0xFFFF);
  for (int m = 0; m < std::min(e - 1, nlab); ++m) {
    if (m >= sim->n_hits[row]) return 0;
    if (sim->S->surf[sim->rec[row * sim->n_seg + m].idx] != labels[m]) return 0;
  }
  return 2;
}

int64_t orc_sim_n_tried(void* s) {
  Sim* sim = (Sim*)s;
  int64_t n = 0;
  for (const KeyOut& k : sim->keys) n += (int64_t)k.tried.size();
  return n;
}

// Flattened per-key lists of the candidates tried, in key order.
// Training labels of the launch proposal (an addition to the paper's
// method): a ray is labelled 1 when it is a candidate (member) of a valid
// specular key, whichever ray represents the key.  amb[row] = 1 when that
// could change under rounding: the ray's membership or the key's validity
// is uncertain and the ray is not certainly labelled 1 by another key.
void orc_sim_ray_labels(void* s, int32_t* label, int32_t* amb) {
  Sim* sim = (Sim*)s;
  const size_t n = sim->excl.size();
  for (size_t i = 0; i < n; ++i) label[i] = amb[i] = 0;
  auto row_of = [&](int64_t rid) -> int64_t {
    if (rid < 0 || rid >= (int64_t)sim->ray_pos.size()) return -1;
    return sim->ray_pos[rid];
  };
  for (const KeyOut& k : sim->keys) {
    if (k.type != 0 || k.k < 1) continue;  // specular keys (LOS has no member rays)
    auto ct = sim->cands.find(k.key);
    if (ct != sim->cands.end())
      for (const Cand& c : ct->second) {
        const int64_t row = row_of(c.ray);
        if (row < 0) continue;
        if (k.valid && k.certain && c.certain) label[row] = 1;
        else if (k.valid || !k.certain) amb[row] = 1;
      }
    auto ut = sim->uncertain_cand.find(k.key);
    if (ut != sim->uncertain_cand.end() && (k.valid || !k.certain))
      for (int64_t rid : ut->second) {
        const int64_t row = row_of(rid);
        if (row >= 0) amb[row] = 1;
      }
  }
  // uncertain candidates of keys the oracle never formed
  for (const auto& kv : sim->uncertain_cand) {
    if (((kv.first.hi >> 55) & 1) != 0) continue;
    bool known = false;
    for (const KeyOut& k : sim->keys)
      if (k.key.hi == kv.first.hi && k.key.lo == kv.first.lo) { known = true; break; }
    if (known) continue;
    for (int64_t rid : kv.second) {
      const int64_t row = row_of(rid);
      if (row >= 0) amb[row] = 1;
    }
  }
  for (size_t i = 0; i < n; ++i)
    if (label[i]) amb[i] = 0;
}

void orc_sim_tried(void* s, int64_t* ray, int32_t* valid, int32_t* amb) {
  Sim* sim = (Sim*)s;
  int64_t o = 0;
  for (const KeyOut& k : sim->keys)
    for (size_t i = 0; i < k.tried.size(); ++i, ++o) {
      ray[o] = k.tried[i];
      valid[o] = k.tried_valid[i];
      amb[o] = k.tried_amb[i];
    }
}

// Complex path coefficients (phase split: the propagation phase exp(-j 2 pi f tau)
// is not included) and per-RX received power P_j = sum |a|^2.
void orc_sim_field(void* s, const double* eps, const double* sig, const double* sca, double* a_re,
                   double* a_im, double* power, int n_rx) {
  Sim* sim = (Sim*)s;
  for (int j = 0; j < n_rx; ++j) power[j] = 0.0;
  for (size_t i = 0; i < sim->paths.size(); ++i) {
    cd a = path_coefficient(*sim, sim->paths[i], eps, sig, sca, sim->p.freq, sim->p.pol);
    a_re[i] = a.real();
    a_im[i] = a.imag();
    power[sim->paths[i].j] += std::norm(a);
  }
}

// Shadow sensitivity of each path: relative change of the coefficient and
// of the delay along the two shadow trajectories (-1 when a shadow does not
// validate: the path is fragile; 0 for LOS).
void orc_sim_path_sens(void* s, const double* eps, const double* sig, const double* sca,
                       double* a_sens, double* tau_sens) {
  Sim* sim = (Sim*)s;
  for (size_t i = 0; i < sim->paths.size(); ++i) {
    const PathOut& P = sim->paths[i];
    a_sens[i] = 0.0;
    tau_sens[i] = 0.0;
    if (P.k == 0) continue;
    cd a = path_coefficient(*sim, P, eps, sig, sca, sim->p.freq, sim->p.pol);
    if (P.type == 2) {
      // closed-form geometry: sensitivity to float32-sized moves of TX, RX
      // and the edge ends (-1 across a discontinuity: a shadow boundary)
      const double h = 4.0 * std::ldexp(1.0, -24);
      for (int q = 0; q < 12; ++q) {
        const V3 dir{q % 3 == 0 ? 1.0 : 0.0, q % 3 == 1 ? 1.0 : 0.0, q % 3 == 2 ? 1.0 : 0.0};
        const double sg = (q / 3) % 2 ? -1.0 : 1.0;
        V3 tx = sim->tx, rx = sim->rx[P.j];
        PathOut Q = P;
        if (q < 6) {
          tx = tx + (sg * h * std::max(1.0, norm(tx))) * dir;
        } else {
          rx = rx + (sg * h * std::max(1.0, norm(rx))) * dir;
          Q.e0 = Q.e0 + (sg * h * std::max(1.0, norm(Q.e0))) * dir;
          Q.e1 = Q.e1 - (sg * h * std::max(1.0, norm(Q.e1))) * dir;
        }
        bool ok = false;
        double tb = 0.0;
        const cd b = diffracted_path_coefficient(Q, tx, rx, eps, sig, sim->p.freq, sim->p.pol,
                                                 &ok, &tb, nullptr);
        const double rel = std::abs(b - a) / std::max(std::abs(a), 1e-300);
        if (!ok || rel > 0.25) {
          a_sens[i] = -1.0;
          tau_sens[i] = -1.0;
          break;
        }
        a_sens[i] = std::max(a_sens[i], rel);
        tau_sens[i] = std::max(tau_sens[i], std::fabs(tb - P.tau) / P.tau);
      }
      continue;
    }
    for (int p = 0; p < 2; ++p) {
      if (!P.shadow_ok[p] || !P.shadow[p]) {
        a_sens[i] = -1.0;
        tau_sens[i] = -1.0;
        break;
      }
      cd b = path_coefficient(*sim, *P.shadow[p], eps, sig, sca, sim->p.freq, sim->p.pol);
      a_sens[i] = std::max(a_sens[i], std::abs(b - a) / std::max(std::abs(a), 1e-300));
      tau_sens[i] = std::max(tau_sens[i], std::fabs(P.shadow[p]->tau - P.tau) / P.tau);
    }
  }
}

// Shadow divergence of the hit records [n_ray][n_seg].
void orc_sim_hit_sens(void* s, double* dq, double* dn) {
  Sim* sim = (Sim*)s;
  for (size_t i = 0; i < sim->dq_sens.size(); ++i) {
    dq[i] = sim->dq_sens[i];
    dn[i] = sim->dn_sens[i];
  }
}

// Analytic gradient of L with respect to (eps_r, sigma, S) per label, given
// dL/dP_j.  d|a|^2/dx = 2 Re(conj(a) da/dx); da/deta_l sums over the
// interactions with label l; deta/deps_r = 1, deta/dsigma = -j/(2 pi f eps0),
}  // extern "C"

namespace {

// material factors of a path: one per interaction, two (the faces) for a
// diffracted path
int n_factors(const PathOut& P) { return P.type == 2 ? 2 : P.k; }

// a and, per interaction m, da/deta_m and da/dS_m (the label's S) for the
// scalar model (pol 0 TE, 1 TM: product rule) and the vector model (pol 2:
// partials of the Jones product).  dR/dS = -S/R; the diffuse factor is S.
void path_derivs(const Sim& sim, const PathOut& P, const double* eps, const double* sig,
                 const double* sca, double f, int pol, cd* a_out, cd* da_deta, cd* da_dS) {
  if (P.type == 2) {  // diffraction: the two faces' reflection coefficients; no S
    *a_out = diffracted_path_coefficient(P, sim.tx, sim.rx[P.j], eps, sig, f, pol, nullptr,
                                         nullptr, da_deta);
    da_dS[0] = da_dS[1] = cd(0.0, 0.0);
    return;
  }
  cd G[5][2], dG[5][2];
  double c[5], dc[5];
  for (int m = 0; m < P.k; ++m) {
    const int l = P.mats[m];
    const cd eta = permittivity(eps[l], sig[l], f);
    for (int t = 0; t < 2; ++t) {
      const int pp = pol == 2 ? t : pol;
      G[m][t] = fresnel(eta, P.cosv[m], pp);
      dG[m][t] = dfresnel_deta(eta, P.cosv[m], pp);
    }
    const bool last_diffuse = P.type == 1 && m == P.k - 1;
    const double R = std::sqrt(std::max(0.0, 1.0 - sca[l] * sca[l]));
    c[m] = last_diffuse ? sca[l] : R;
    dc[m] = last_diffuse ? 1.0 : (R > 0.0 ? -sca[l] / R : 0.0);
  }
  if (pol == 2) {
    cd D[5][2], dA[5][2];
    for (int m = 0; m < P.k; ++m)
      for (int t = 0; t < 2; ++t) D[m][t] = c[m] * G[m][t];
    const Jones J = path_jones(sim, P);
    *a_out = P.geo * jones_amplitude(J, D);
    jones_partials(J, D, dA);
    for (int m = 0; m < P.k; ++m) {
      da_deta[m] = P.geo * (dA[m][0] * (c[m] * dG[m][0]) + dA[m][1] * (c[m] * dG[m][1]));
      da_dS[m] = P.geo * (dA[m][0] * (dc[m] * G[m][0]) + dA[m][1] * (dc[m] * G[m][1]));
    }
    return;
  }
  cd fac[5];
  for (int m = 0; m < P.k; ++m) fac[m] = c[m] * G[m][0];
  cd a(P.geo, 0.0);
  for (int m = 0; m < P.k; ++m) a *= fac[m];
  *a_out = a;
  for (int m = 0; m < P.k; ++m) {
    cd others(P.geo, 0.0);
    for (int q = 0; q < P.k; ++q)
      if (q != m) others *= fac[q];
    da_deta[m] = others * (c[m] * dG[m][0]);
    da_dS[m] = others * (dc[m] * G[m][0]);
  }
}

}  // namespace

extern "C" {

// Complex derivatives of every path coefficient (phase split, Sec. II-B
// readings) with respect to the per-label (eps_r, sigma, S): out[p][t][l] for
// t = 0 eps_r, 1 sigma, 2 S, as (re, im) pairs, before they are contracted
// with a loss.
void orc_sim_path_grads(void* s, const double* eps, const double* sig, const double* sca,
                        int n_labels, double* out) {
  Sim* sim = (Sim*)s;
  const double f = sim->p.freq;
  const cd deta_dsig(0.0, -1.0 / (2.0 * kPi * f * kEps0));
  const size_t per = (size_t)3 * n_labels * 2;
  for (size_t i = 0; i < sim->paths.size(); ++i) {
    double* o = out + i * per;
    for (size_t q = 0; q < per; ++q) o[q] = 0.0;
    const PathOut& P = sim->paths[i];
    cd a, de[5], dS[5];
    path_derivs(*sim, P, eps, sig, sca, f, sim->p.pol, &a, de, dS);
    for (int m = 0; m < n_factors(P); ++m) {
      const int l = P.mats[m];
      const cd v[3] = {de[m], de[m] * deta_dsig, dS[m]};
      for (int t = 0; t < 3; ++t) {
        o[(t * n_labels + l) * 2] += v[t].real();
        o[(t * n_labels + l) * 2 + 1] += v[t].imag();
      }
    }
  }
}

// Gradient of a loss of the received powers: d|a|^2/dx = 2 Re(conj(a) da/dx),
// weighted by dL/dP_j of the path's receiver.
void orc_sim_backward(void* s, const double* eps, const double* sig, const double* sca,
                      const double* dL_dP, double* g_eps, double* g_sig, double* g_sca,
                      int n_labels) {
  Sim* sim = (Sim*)s;
  const double f = sim->p.freq;
  for (int l = 0; l < n_labels; ++l) g_eps[l] = g_sig[l] = g_sca[l] = 0.0;
  const cd deta_dsig(0.0, -1.0 / (2.0 * kPi * f * kEps0));
  for (const PathOut& P : sim->paths) {
    cd a, de[5], dS[5];
    path_derivs(*sim, P, eps, sig, sca, f, sim->p.pol, &a, de, dS);
    const double w = dL_dP[P.j] * 2.0;
    for (int m = 0; m < n_factors(P); ++m) {
      const int l = P.mats[m];
      g_eps[l] += w * (std::conj(a) * de[m]).real();
      g_sig[l] += w * (std::conj(a) * de[m] * deta_dsig).real();
      g_sca[l] += w * (std::conj(a) * dS[m]).real();
    }
  }
}

// Algorithmic disc reads of a cast: the discs of every DPS (other than the
// skipped one) whose r_p-inflated box the segment [t_min, t_end] enters.
static int64_t discs_entered(const Scene& S, V3 o, V3 d, int skip, double t_min, double t_end) {
  int64_t cnt = 0;
  for (size_t D = 0; D < S.dps_pts.size(); ++D) {
    if ((int)D == skip) continue;
    V3 lo{kInf, kInf, kInf}, hi{-kInf, -kInf, -kInf};
    for (int i : S.dps_pts[D]) {
      lo = {std::min(lo.x, S.P[i].x), std::min(lo.y, S.P[i].y), std::min(lo.z, S.P[i].z)};
      hi = {std::max(hi.x, S.P[i].x), std::max(hi.y, S.P[i].y), std::max(hi.z, S.P[i].z)};
    }
    double t0 = t_min, t1 = t_end;
    bool miss = false;
    for (int k = 0; k < 3 && !miss; ++k) {
      double a = comp(lo, k) - S.rp, b = comp(hi, k) + S.rp, ok = comp(o, k), dk = comp(d, k);
      if (dk == 0.0) {
        if (ok < a || ok > b) miss = true;
        continue;
      }
      double ta = (a - ok) / dk, tb = (b - ok) / dk;
      if (ta > tb) std::swap(ta, tb);
      t0 = std::max(t0, ta);
      t1 = std::min(t1, tb);
    }
    if (!miss && t0 <= t1) cnt += (int64_t)S.dps_pts[D].size();
  }
  return cnt;
}

// Per ray and cast of a simulation: discs entered before the hit (or, after
// a miss, along the whole ray); -1 for casts not made.
void orc_sim_disc_counts(void* s, int64_t* out) {
  Sim* sim = (Sim*)s;
  const Scene& S = *sim->S;
  const int64_t n = (int64_t)sim->ray_ids.size();
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t r = 0; r < n; ++r) {
    V3 o = sim->tx, d = launch_dir(*sim, sim->ray_ids[r]);
    int skip = -1;
    for (int k = 0; k < sim->n_seg; ++k) {
      int64_t& dst = out[r * sim->n_seg + k];
      if (k > sim->n_hits[r]) {
        dst = -1;
        continue;
      }
      const HitRec& h = sim->rec[r * sim->n_seg + k];
      const bool hit = k < sim->n_hits[r];
      dst = discs_entered(S, o, d, skip, sim->p.t_min, hit ? h.t : 1e30);
      if (!hit) continue;
      o = h.q;
      d = h.dout;
      skip = h.dps;
    }
  }
}

// The same count for the diffuse validation shadow casts (scatter point of a
// tried candidate -> RX, skipping the scatter DPS, Sec. II-B-1): every
// `stride`-th tried candidate of the diffuse keys, in key order.  *n_casts
// receives the number of casts counted, *sum their discs.
void orc_sim_shadow_disc_counts(void* s, int64_t stride, int64_t* sum, int64_t* n_casts) {
  Sim* sim = (Sim*)s;
  const Scene& S = *sim->S;
  CastCfg cfg;
  cfg.t_min = sim->p.t_min;
  std::vector<std::pair<int64_t, int>> items;  // (row, key index)
  int64_t idx = 0;
  for (size_t ki = 0; ki < sim->keys.size(); ++ki) {
    const KeyOut& k = sim->keys[ki];
    if (k.type != 1) continue;
    for (int64_t rid : k.tried) {
      if (idx++ % stride) continue;
      const int64_t row = (rid >= 0 && rid < (int64_t)sim->ray_pos.size()) ? sim->ray_pos[rid] : -1;
      if (row >= 0) items.push_back({row, (int)ki});
    }
  }
  int64_t tot = 0, cnt = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : tot, cnt)
  for (int64_t i = 0; i < (int64_t)items.size(); ++i) {
    const KeyOut& k = sim->keys[items[i].second];
    const HitRec& hk = sim->rec[items[i].first * sim->n_seg + (k.k - 1)];
    const V3 u = sim->rx[k.j] - hk.q;
    const double rs = norm(u);
    const V3 w = (1.0 / rs) * u;
    if (dot(hk.n, w) <= 0.0) continue;  // no cast
    const Hit h = cast(S, hk.q, w, hk.dps, rs, false, cfg);
    tot += discs_entered(S, hk.q, w, hk.dps, sim->p.t_min, h.hit ? h.t : rs);
    ++cnt;
  }
  *sum = tot;
  *n_casts = cnt;
}

// The same count for visibility casts (RX j -> reception point of DPS D).
void orc_vis_disc_counts(void* s, const double* rx, const int32_t* j, const int32_t* dps,
                         int64_t n, double t_min, int64_t* out) {
  Scene* S = (Scene*)s;
  CastCfg cfg;
  cfg.t_min = t_min;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    V3 r{rx[3 * j[i]], rx[3 * j[i] + 1], rx[3 * j[i] + 2]};
    V3 v = S->recv[dps[i]] - r;
    double sl = norm(v);
    double t_max = sl - rx_margin(*S);
    if (t_max <= t_min) {
      out[i] = 0;
      continue;
    }
    V3 d = (1.0 / sl) * v;
    Hit h = cast(*S, r, d, -1, t_max, false, cfg);
    out[i] = discs_entered(*S, r, d, -1, t_min, h.hit ? h.t : t_max);
  }
}

// Vector-polarisation coefficient / geo of a path given explicitly: TX, RX,
// k interaction points (pts[3k]), diffuse flag with the scatter normal nd,
// and the diagonal factors D (c Gamma_TE, c Gamma_TM per interaction, as
// re/im pairs [k][2][2]).  For closed-form pins of the vector model.
void orc_jones_amplitude(const double* tx, const double* rx, const double* pts, int k, int diffuse,
                         const double* nd, const double* D, double* re, double* im) {
  V3 p[5];
  for (int m = 0; m < k; ++m) p[m] = {pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]};
  const Jones J = make_jones({tx[0], tx[1], tx[2]}, {rx[0], rx[1], rx[2]}, p, k, diffuse != 0,
                             {nd[0], nd[1], nd[2]});
  cd DD[5][2];
  for (int m = 0; m < k; ++m)
    for (int t = 0; t < 2; ++t) DD[m][t] = cd(D[(m * 2 + t) * 2], D[(m * 2 + t) * 2 + 1]);
  const cd a = jones_amplitude(J, DD);
  *re = a.real();
  *im = a.imag();
}

// Standalone EM helpers for closed-form pins.
void orc_fresnel(double eps_r, double sigma, double freq, double cos_t, int pol, double* re,
                 double* im) {
  cd G = fresnel(permittivity(eps_r, sigma, freq), cos_t, pol);
  *re = G.real();
  *im = G.imag();
}

void orc_dfresnel(double eta_re, double eta_im, double cos_t, int pol, double* re, double* im) {
  cd G = dfresnel_deta(cd(eta_re, eta_im), cos_t, pol);
  *re = G.real();
  *im = G.imag();
}

void orc_fresnel_eta(double eta_re, double eta_im, double cos_t, int pol, double* re, double* im) {
  cd G = fresnel(cd(eta_re, eta_im), cos_t, pol);
  *re = G.real();
  *im = G.imag();
}

// Casts made: [0] trace segments, [1] visibility, [2] validation, [3] LOS.
void orc_sim_cast_counts(void* s, int64_t* out) {
  Sim* sim = (Sim*)s;
  int64_t segs = 0;
  for (size_t r = 0; r < sim->ray_ids.size(); ++r)
    segs += std::min(sim->n_hits[r] + 1, sim->n_seg);
  out[0] = segs;
  out[1] = sim->vis_casts.load();
  out[2] = sim->val_casts.load();
  out[3] = (int64_t)sim->rx.size();
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
