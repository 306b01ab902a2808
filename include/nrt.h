/*
 * nrt.h -- C ABI of the GB300 point-cloud radio ray tracer (libnrt.so).
 *
 * The library implements the path computation of Vaara et al.,
 * "Differentiable High-Performance Ray Tracing-Based Simulation of Radio
 * Propagation with Point Clouds" (arXiv 2507.04021), as CUDA kernels for
 * sm_103a, plus the EM field of each path and its adjoint.
 *
 * Conventions (every entry point):
 *   - Plain pointers and sizes only.  "host" buffers live in host memory,
 *     "device" buffers in device memory of the context's device.
 *   - The caller owns every input array; the library copies what it keeps.
 *   - The library owns nrt_ctx / nrt_scene / nrt_result until the matching
 *     *_free / nrt_destroy call.  Handles are reference counted: a scene keeps
 *     its context alive and a result keeps its scene alive, so the free calls
 *     may come in any order (the memory goes with the last one).
 *   - Work is enqueued on the context's CUDA stream.  Calls that return
 *     host data (*_read, nrt_result_counts) synchronise that stream.
 *   - No C++ exception crosses the ABI.  On error nothing is written to the
 *     outputs and nrt_last_error() describes the failure.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef NRT_H_
#define NRT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nrt_ctx nrt_ctx;
typedef struct nrt_scene nrt_scene;
typedef struct nrt_result nrt_result;

typedef enum {
  NRT_OK = 0,
  NRT_ERR_ARG = 1,       /* invalid argument (NaN input, zero normal, bad size, ...) */
  NRT_ERR_CUDA = 2,      /* a CUDA runtime call failed */
  NRT_ERR_OOM = 3,       /* device allocation failed */
  NRT_ERR_OVERFLOW = 4,  /* a fixed-capacity buffer (hash table, candidates) overflowed */
  NRT_ERR_TIMEOUT = 5,   /* a bounded device loop gave up (watchdog) */
  NRT_ERR_STATE = 6      /* call out of order (e.g. backward without a field) */
} nrt_status;

/* Scene parameters (Table I of the paper: rho = 0.0625, r_p = 0.015,
 * lambda_d = 100). */
typedef struct {
  float rho;       /* voxel size of the discretised point sets (DPS), m (Sec. II-A) */
  float r_p;       /* disc radius, m (Sec. II-C) */
  float lambda_d;  /* depth attenuation of Eq. 4, 1/m */
} nrt_scene_params;

enum { NRT_CAPTURE_SPHERE = 0, NRT_CAPTURE_VIS = 1 };
enum { NRT_POL_TE = 0, NRT_POL_TM = 1, NRT_POL_VECTOR = 2 };
enum { NRT_LAUNCH_FIB = 0, NRT_LAUNCH_DPS = 1 };

/* Trace parameters.  nrt_trace_params_default() fills the paper's values
 * (Table I: kappa = 10, t_a = 1 degree, t_d = 0.01 m). */
typedef struct {
  int32_t max_depth;    /* K: maximum number of interactions (<= 5) */
  int32_t capture;      /* NRT_CAPTURE_SPHERE (RX sphere of radius r_rx) or
                           NRT_CAPTURE_VIS (visibility matrix, Sec. II-B) */
  int32_t diffuse;      /* 1: diffuse scattering as the last interaction (Sec. II-B-1) */
  int32_t pol;          /* NRT_POL_TE or NRT_POL_TM: scalar Fresnel model, every
                           interaction reflects with that coefficient.
                           NRT_POL_VECTOR: vertically polarised isotropic TX and RX
                           (theta^ of the spherical basis about +z); at each
                           interaction the component across the plane of
                           incidence takes Gamma_TE and the one in it Gamma_TM,
                           with the basis rotations between interactions (the
                           paper delegates the field model to an EM library,
                           Sec. II-B; this is the vector reading of it) */
  int32_t kappa;        /* refinement retries (Sec. II-B-2) */
  int32_t rep_tries;    /* 0 (default): every candidate of a path key is refined and
                           validated and the lowest valid ray id represents the key
                           (the paper refines all candidates, Sec. II-B-2, then
                           removes duplicates, Sec. II-B-4); > 0: at most that many
                           candidates per key, in ray-id order (a cap that changes
                           the result) */
  int32_t record_hits;  /* 1: keep per-ray hit records readable by nrt_hits_read */
  int32_t ray_labels;   /* 1: per-ray proposal labels, readable by nrt_ray_labels_read */
  int64_t n_rays;       /* N of the Fibonacci-sphere launch */
  float r_rx;           /* RX sphere radius, m (sphere capture) */
  float t_min;          /* minimum hit distance, m (default 1e-3) */
  float t_a_deg;        /* refinement angle threshold, degrees */
  float t_d;            /* refinement plane-distance threshold, m */
  float freq;           /* carrier frequency, Hz */
  int32_t keep_keys;    /* 1: keep per-key validation summaries, readable by nrt_keys_read */
  int64_t key_capacity;   /* hash-table slots (power of two, at most 2^31; 0 = automatic) */
  int64_t cand_capacity;  /* candidate buffer entries (0 = automatic) */
  int32_t launch;       /* NRT_LAUNCH_FIB: Fibonacci sphere of n_rays rays;
                           NRT_LAUNCH_DPS: one ray per DPS toward its reception
                           point (Sec. II-B), ray i = the i-th DPS in voxel Morton
                           order, n_rays taken as the scene's DPS count */
  int32_t diffraction;  /* 1: single-bounce diffraction on the scene's edges
                           (Sec. II-B-3, nrt_scene_set_edges): one candidate per
                           (edge, RX), kept when its point lies inside the edge,
                           TX and RX lie outside the wedge and both see it */
  int32_t spec_waves;   /* schedule of the specular refinement (Sec. II-B-2):
                           0 (default) or 2: one persistent pass in which a lane
                           refines a candidate from start to end; 1: waves of up
                           to 2^22 candidates held in device memory, each leg
                           cast by a lean kernel (experimental: the same paths
                           on most office workloads tested, but the wave cast
                           kernel and the refinement round the Eq. 4 normal of
                           a cast differently in rare cases, and a representative
                           chosen by the waves can then fail the re-refinement
                           check, NRT_ERR_STATE) */
} nrt_trace_params;

/* Per-simulation counters (nrt_result_counts). */
typedef struct {
  int64_t rays;              /* rays launched */
  int64_t segments;          /* primary ray segments cast (trace) */
  int64_t vis_casts;         /* visibility-matrix casts */
  int64_t los_casts;         /* TX -> RX casts */
  int64_t validation_casts;  /* refinement, diffuse and final-leg casts */
  int64_t candidates;        /* path candidates emitted */
  int64_t keys;              /* distinct path keys */
  int64_t paths;             /* valid paths (including LOS) */
  int64_t n_dps;             /* DPS in the scene */
  int64_t hash_probes_max;   /* longest hash probe sequence seen */
  int64_t error_flags;       /* device error bits, 0 = none: 1 traversal stack
                                would overflow (tree deeper than the stack);
                                2 hash probe limit reached; 4 candidate buffer
                                full; 8 more distinct keys than the key
                                capacity; 16 path buffer full (any of these
                                makes the call return NRT_ERR_OVERFLOW); 32 an
                                internal consistency check failed (a path
                                refined twice came out differently:
                                NRT_ERR_STATE). */
  int64_t kernel_launches;   /* library kernels launched by the call */
  int64_t diffuse_casts;     /* of validation_casts: diffuse shadow casts (Sec. II-B-1) */
  int64_t diffraction_casts; /* edge visibility casts (Sec. II-B-3) */
  int64_t pruned_legs;       /* specular refinement legs ended without a cast: the
                                leg's ray cannot enter the box of the key's surface
                                label there, so its closest hit is another surface */
  int64_t spec_items;        /* specular (key, candidate) pairs refined (Sec. II-B-2) */
  int64_t spec_ended_without_cast;  /* of which ended before any cast */
  int64_t spec_ended_at_first_leg;  /* of which ended at the first leg's cast */
  int64_t reserved[1];
} nrt_counters;

/* Path view for nrt_paths_read: caller-allocated arrays of n_paths entries
 * (n_paths from nrt_result_counts).  Any pointer may be NULL to skip it.
 * Paths are ordered by (rx, type, interactions, representative ray id);
 * diffracted paths (type 2) come last for their RX, by edge index.
 * A diffracted path has k = 1, pts[0] = the diffraction point, rep = the
 * edge index, mats[0..1] = the materials of faces 0 and n, cos_theta[0..1]
 * = the incidence cosines on those faces; its key is
 * hi = rx << 56 | 1 << 52 | 1 << 51, lo = edge index. */
typedef struct {
  uint64_t* key_hi;  /* 128-bit path key, see nrt_trace */
  uint64_t* key_lo;
  uint32_t* rep;     /* representative ray id (0xFFFFFFFF for LOS) */
  int32_t* rx;       /* RX index */
  int32_t* type;     /* 0 specular / LOS, 1 diffuse last interaction, 2 edge diffraction */
  int32_t* k;        /* number of interactions (0 = LOS) */
  float* pts;        /* [n][5][3] interaction points */
  uint8_t* mats;     /* [n][5] material labels of the interactions */
  float* cos_theta;  /* [n][5] cosine of the incidence angle at each interaction */
  float* geo;        /* material-independent amplitude factor */
  float* tau;        /* delay, s */
  float* a;          /* [n][2] complex path coefficient (real, imag), without the
                        propagation phase exp(-j 2 pi f tau) */
  float* normal;     /* [n][3] surface normal at the scatter point of a diffuse
                        path, facing the incoming ray (0 for specular / LOS) */
} nrt_path_view;

/* Status text for a status code (static storage). */
const char* nrt_status_string(nrt_status s);

/* Last error message of this context ("" if none). */
const char* nrt_last_error(const nrt_ctx* ctx);

/* Create a context on CUDA device `device` working on `cuda_stream`
 * (a cudaStream_t; NULL = the context creates its own stream).
 * Errors: NRT_ERR_ARG (bad device), NRT_ERR_CUDA. */
nrt_status nrt_create(nrt_ctx** out, int device, void* cuda_stream);
void nrt_destroy(nrt_ctx* ctx);

/* Synchronise the context stream. */
nrt_status nrt_sync(nrt_ctx* ctx);

/* The context's CUDA stream (cudaStream_t) into *stream: the stream every
 * call enqueues its work on. */
nrt_status nrt_get_stream(const nrt_ctx* ctx, void** stream);

/* Measured L2 read bandwidth (the ceiling of the L2 roofline reported beside
 * the HBM one for the traversal kernels; not part of the paper): a device
 * buffer of `bytes` (in [2^20, 2^30], well under the 129 MB L2 for the L2
 * figure) is filled, read once to warm the cache, then read `reps` times
 * (1..1000) with 16-byte loads that bypass L1; *gbs (host) = bytes x reps /
 * CUDA-event time, in GB/s.  Allocates and frees its buffer; synchronises.
 * Errors: NRT_ERR_ARG, NRT_ERR_OOM, NRT_ERR_CUDA. */
nrt_status nrt_measure_l2(nrt_ctx* ctx, int64_t bytes, int32_t reps, float* gbs);

/* Watchdog of the bounded device waits (the tensor-core kernels' mbarrier
 * waits for their MMAs: nrt_gemm_bf16, nrt_mlp_score, nrt_mlp_train): a wait
 * makes at most `polls` non-blocking polls (0 restores the default: 2^22
 * potentially blocking polls), then the kernel records a timeout, waits with
 * the default limit for its own MMAs in flight, frees its tensor memory and
 * returns; the call reports NRT_ERR_TIMEOUT (nrt_mlp_score, which does not
 * synchronise, leaves it to the next nrt_mlp_train) and the context stays
 * usable.  Not part of the paper: a
 * failure-detection control (a small limit makes a wait run out on purpose).
 * Errors: NRT_ERR_ARG for polls < 0. */
nrt_status nrt_set_wait_limit(nrt_ctx* ctx, int64_t polls);

/* Fill the paper's default trace parameters. */
void nrt_trace_params_default(nrt_trace_params* p);

/* Upload an augmented point cloud (Sec. II: position p_i, normal n, surface
 * label l_s, material label l_m) and build the ray-traceable scene
 * (Sec. II-A): voxels of size rho; each DPS is the point set of one voxel with
 * an AABB inflated by r_p and a reception point at the mean position.
 *   pos, nrm   : float [n][3] (host, or device if inputs_on_device); nrm unit
 *   surf_label : uint16 [n];  mat_label : uint8 [n]
 * The DPS are ordered along a Morton curve and a bounding-volume hierarchy
 * is built over their AABBs on the device.
 * Errors: NRT_ERR_ARG for n <= 0, NaN/inf positions, zero normals,
 * non-positive rho / r_p / lambda_d, or a scene more than 2^21 voxels wide. */
nrt_status nrt_scene_upload(nrt_ctx* ctx, const float* pos, const float* nrm,
                            const uint16_t* surf_label, const uint8_t* mat_label, int64_t n,
                            const nrt_scene_params* params, int inputs_on_device,
                            nrt_scene** out);
void nrt_scene_free(nrt_scene* scene);

/* Scene summary: number of DPS, voxel-grid origin bmin (float[3]) and the
 * device time of the build (ms).  Any output may be NULL. */
nrt_status nrt_scene_info(const nrt_scene* scene, int64_t* n_dps, float* bmin, float* build_ms);

/* Read the DPS in library order: voxel coordinates int32[n_dps][3], point
 * count int32[n_dps], reception point float[n_dps][3].  Host outputs. */
nrt_status nrt_scene_dps_read(const nrt_scene* scene, int32_t* vox, int32_t* count,
                              float* recv);

/* Per-label materials: relative permittivity eps_r, conductivity sigma (S/m)
 * and scattering coefficient S (ITU-R P.2040 convention for the complex
 * permittivity eta = eps_r - j sigma / (2 pi f eps0)).  Host arrays of
 * n_labels (<= 256) entries.  Errors: NRT_ERR_ARG for eps_r < 1, sigma < 0,
 * S outside [0, 1). */
nrt_status nrt_set_materials(nrt_scene* scene, const float* eps_r, const float* sigma,
                             const float* scat, int n_labels);

/* Same materials from DEVICE memory, for a learning loop whose parameters
 * live on the GPU (Sec. III-B learns eps_r, sigma and S per label by gradient
 * descent): mat is a device float[3][n_labels] -- eps_r, then sigma, then S,
 * each n_labels (<= 256) long, read by a kernel enqueued on the context
 * stream (the call does not synchronise; mat must stay valid until that
 * kernel has run).  Values cannot be checked on the host without a copy, so
 * the kernel brings each into its range instead: eps_r = max(eps_r, 1),
 * sigma = max(sigma, 0), S clamped to [0, 1 - 2^-24]; NaN goes to the lower
 * bound.  The call makes the context's device current for its launch and
 * restores the caller's current device.  Errors: NRT_ERR_ARG for NULL mat or
 * n_labels outside [1, 256]; NRT_ERR_CUDA. */
nrt_status nrt_set_materials_device(nrt_scene* scene, const float* mat, int n_labels);

/* Edges of the augmented point cloud (Sec. II, used by the diffraction of
 * Sec. II-B-3): host arrays of n_edges entries -- segment ends a, b
 * (float[3] each), the outward unit normals n0, n1 of the two faces meeting
 * there (float[3] each; the solid is the convex wedge behind both faces) and
 * their material labels m0, m1.  Copied to the device; replaces any earlier
 * set (n_edges = 0 clears it).  The diffraction coefficient (the paper leaves
 * it to its EM library) is the UTD wedge coefficient of Kouyoumjian and
 * Pathak with Luebbers' face reflection coefficients; see nrt_trace.
 * Errors: NRT_ERR_ARG for non-finite values, a segment shorter than 1e-6 m,
 * normals not unit (1e-3) or not normal to the edge (1e-3), faces that do not
 * form a wedge (|n0 . n1| > 1 - 1e-6), n_edges > 2^24; NRT_ERR_STATE while a
 * result of this scene is alive (its batch plan may read the edges). */
nrt_status nrt_scene_set_edges(nrt_scene* scene, int64_t n_edges, const float* a, const float* b,
                               const float* n0, const float* n1, const uint8_t* m0,
                               const uint8_t* m1);

/* Intersection models for nrt_cast. */
enum { NRT_ISECT_DISC = 0, NRT_ISECT_SDF = 1 };

typedef struct {
  int32_t model;  /* NRT_ISECT_DISC: the paper's model (Sec. II-C) -- ray/disc
                     intersections of the DPS of the closest disc, the Eq. 3
                     point with the Eq. 4 weights, the weighted normal;
                     NRT_ISECT_SDF: the SDF of the prior work (Eq. 2), kept for
                     the ablation: per DPS the Eq. 2-weighted mean of the points'
                     tangent-plane distances (defined where the weight sum is
                     >= e^-2), marched in steps of sigma/2 over the ray's crossing
                     of the points' box grown by 2 sigma, the first
                     outside-to-inside sign change refined by 20 bisections */
  float sigma;    /* SDF: Gaussian width of Eq. 2, m, in (0, 1) */
  float t_min;    /* hits need t > t_min (>= 0) */
  float t_max;    /* and t < t_max (INFINITY for no bound) */
} nrt_cast_params;

/* Closest hits of n arbitrary rays against the scene.  o, d: device
 * float[n][3] (d need not be unit; it is normalised).  Outputs, device,
 * caller-allocated, any may be NULL: t float[n] (ray parameter of the hit
 * point along unit d; +inf on a miss), normal float[n][3] (facing the ray; 0
 * on a miss), dps int32[n] (-1 on a miss), labels uint32[n] (surface |
 * material << 16 of the closest disc, or of the hit DPS's point nearest to
 * the SDF hit).  Enqueued on the context stream; synchronises to read the
 * traversal status.  Errors: NRT_ERR_ARG (NULL rays, n > 2^31, unknown
 * model, sigma outside (0, 1) for the SDF, not 0 <= t_min < t_max),
 * NRT_ERR_OVERFLOW (traversal stack overflow), NRT_ERR_CUDA. */
nrt_status nrt_cast(nrt_scene* scene, const float* o, const float* d, int64_t n,
                    const nrt_cast_params* params, float* t, float* normal, int32_t* dps,
                    uint32_t* labels);

/* One simulation for one TX (Sec. II-B):
 *   LOS casts TX -> every RX; Fibonacci launch of n_rays directions (or the
 *   subset `ray_subset` of their ids); every interaction continues as a
 *   specular reflection up to max_depth; path candidates from the RX sphere
 *   or the RX -> DPS visibility matrix; duplicates removed by a 128-bit key
 *   of (RX, type, interactions, surface labels[, scatter voxel]); the
 *   lowest-ray-id candidate that validates represents a key (diffuse: a
 *   cast scatter point -> RX; specular: image-method refinement on the
 *   interaction planes, Eq. 1, validated by casts with thresholds t_a, t_d
 *   and up to kappa retries); with `diffraction`, one single-bounce
 *   diffracted path per (edge, RX) that passes its checks (Sec. II-B-3);
 *   then the field of every path (`pol`).
 *   tx : host float[3];  rx : host float[n_rx][3] (n_rx <= 256)
 *   ray_subset : NULL, or uint32[n_subset] ray ids < n_rays (host, or device
 *                when subset_on_device)
 * Key layout: hi = [rx:8 @56][diffuse:1 @55][k:3 @52][low 52 bits]; specular:
 * lo = l1 | l2<<16 | l3<<32 | l4<<48, hi low 16 bits = l5; diffuse: lo =
 * labels of the k-1 specular interactions, hi low 48 bits = scatter voxel
 * x | y<<16 | z<<32 (each taken modulo 2^16); diffracted: hi = rx << 56 |
 * 1 << 52 | 1 << 51, lo = edge index.  The outputs do not depend on the order
 * in which the GPU hands rays and keys to its lanes: the same inputs give
 * bit-identical paths (the counter of validation casts, a measure of work,
 * may differ slightly: a candidate stops once its key has a lower valid
 * rank).  Buffer sizing: with key_capacity and cand_capacity at 0, the first
 * simulation of a shape (scene, rays, receivers, capture, depth, diffuse,
 * diffraction, launch) on a context sizes the candidate and key buffers from
 * an exact count (one host round trip); later ones reuse that run's counts
 * plus 25% and enqueue everything at once, and a run that outgrows them is
 * redone with exact sizes inside the same call, with the same result.
 * Errors: NRT_ERR_ARG, NRT_ERR_OOM, NRT_ERR_OVERFLOW (hash table or candidate
 * buffer too small: raise key_capacity / cand_capacity), NRT_ERR_CUDA. */
nrt_status nrt_trace(nrt_scene* scene, const float* tx, const float* rx, int n_rx,
                     const nrt_trace_params* params, const uint32_t* ray_subset,
                     int64_t n_subset, int subset_on_device, nrt_result** out);
void nrt_result_free(nrt_result* result);

/* Counters and per-RX path counts (host int64[n_rx], may be NULL). */
nrt_status nrt_result_counts(const nrt_result* result, int64_t* n_paths_per_rx,
                             nrt_counters* counters);

/* Device times of the simulation phases in ms: [0] visibility (with the
 * launch order and buffer set-up before it), [1] unused (0), [2] trace,
 * [3] candidates + dedup + LOS, [4] validation/refinement, [5] field,
 * [6] total, [7] the part of [3] the device spends waiting for the host to
 * size the candidate and key buffers from the counted candidates (the one
 * host round trip of a simulation).  Host float[8]. */
nrt_status nrt_result_times(const nrt_result* result, float* ms);

/* Read all paths into caller-allocated host arrays. */
nrt_status nrt_paths_read(const nrt_result* result, const nrt_path_view* view);

/* Per-ray hit records (requires record_hits): host arrays [n_traced][S]
 * with S = max_depth (+1 for sphere capture); rays in launch order (ray ids
 * 0..n_rays-1, or the subset order).  idx = point index of q_min (-1 after a
 * miss), dps = library DPS index, q = Eq. 3 point, n = weighted normal
 * facing the incoming ray, t = segment length.  Any pointer may be NULL. */
nrt_status nrt_hits_read(const nrt_result* result, int32_t* idx, int32_t* dps, float* q,
                         float* n, float* t);

/* Visibility matrix bits (capture = VIS): host uint32[n_rx][(n_dps+31)/32],
 * bit d of row j = DPS d visible from RX j. */
nrt_status nrt_vis_read(const nrt_result* result, uint32_t* bits);

/* Recompute the field of the stored paths with the scene's current materials
 * (geometry does not depend on materials).  Enqueued on the context stream. */
nrt_status nrt_field(nrt_result* result);

/* Received power per RX, P_j = sum over paths of |a|^2 (host float[n_rx]):
 * the incoherent sum of the path coefficients (the paper hands its paths to
 * an EM library for the field, Sec. II; its learning experiment, Sec. III-B,
 * reads the channel from the same per-path coefficients -- see nrt_cfr for
 * the coherent CFR).  Errors: NRT_ERR_STATE before the field was computed. */
nrt_status nrt_field_read(const nrt_result* result, float* power_per_rx);

/* Received power per RX into DEVICE memory: power is a device double[n_rx]
 * (the FP64 sums of nrt_field_read before their rounding to float), copied
 * on the context stream without synchronising, so that a learning loop
 * (Sec. III-B) can form its loss on the GPU.  The call makes the context's
 * device current for the copy and restores the caller's current device.
 * Errors: NRT_ERR_ARG for NULL;
 * NRT_ERR_STATE before the field was computed; NRT_ERR_CUDA. */
nrt_status nrt_field_read_device(const nrt_result* result, double* power);

/* Adjoint of the received power (the differentiable electromagnetic
 * computation used to learn per-label relative permittivity, conductivity and
 * scattering coefficient, Sec. III-B): given dL/dP_j (host float[n_rx]), the
 * gradient of L with respect to each label's eps_r, sigma and S (host
 * float[n_labels] each), recomputed from the stored interaction sequences
 * (material labels and incidence cosines) rather than from stored
 * intermediates.  Errors: NRT_ERR_STATE before nrt_set_materials. */
nrt_status nrt_backward(nrt_result* result, const float* dL_dpower, float* g_eps, float* g_sigma,
                        float* g_scat);

/* ---------------------------------------------------------------- batches
 * Many TX-RX pairs in one simulation: the robot-trajectory workload (a TX
 * moving along a path, one fixed RX, an uneven ray budget per position).
 * Pair j launches its own Fibonacci set of budget[j] rays from tx[j]; the
 * path keys carry j in their RX field, so paths, counts, power, field and
 * adjoint are per pair (pass n_rx = n_pairs-sized arrays to the readout
 * calls).  The trace runs as ONE persistent launch whose warps pull work items
 * of `packet` rays from a queue, so uneven budgets balance themselves; the
 * visibility matrix of the fixed RX is computed once. */
typedef struct {
  int32_t packet;     /* rays per work item of the persistent trace: 32, 64 or 128 */
  int32_t schedule;   /* 0 static grid-stride, 1 persistent work queue */
  int32_t use_graph;  /* 1: record the whole simulation into a CUDA graph; the
                         result then serves nrt_batch_replay */
  int32_t reserved;
} nrt_batch_opts;

/* tx: host float[n_pairs][3]; rx: host float[3] (the fixed receiver);
 * budget: host int64[n_pairs], each in [1, 2^31); n_pairs in [1, 256];
 * params->capture must be NRT_CAPTURE_VIS (params->n_rays is ignored).
 * With use_graph the call runs once to size every buffer (25% headroom),
 * records the simulation into a CUDA graph and replays it once.
 * Errors: NRT_ERR_ARG, NRT_ERR_OOM, NRT_ERR_OVERFLOW, NRT_ERR_CUDA. */
nrt_status nrt_trace_batch(nrt_scene* scene, const float* tx, const float* rx,
                           const int64_t* budget, int n_pairs, const nrt_trace_params* params,
                           const nrt_batch_opts* opts, nrt_result** out);

/* Replay the recorded graph with new TX positions (host float[n_pairs][3], or
 * NULL to keep them); the budgets and the RX are those of the recording.
 * The result's paths/counts/power are replaced.  Errors: NRT_ERR_STATE
 * without use_graph; NRT_ERR_OVERFLOW when a replay needs more than the
 * recorded capacities (rebuild the batch). */
nrt_status nrt_batch_replay(nrt_result* result, const float* tx);

/* Per-pair latency of the last batch run, from device timestamps (globaltimer)
 * taken from the start of the trace: pair_ms[j] = the moment pair j's last
 * ray was traced (either schedule); pair_paths_ms[j] = the moment pair j's
 * last path key finished validation, i.e. its path set is known (its field
 * follows in one pass over all paths, done at total_ms).  host double[n_pairs]
 * each, any may be NULL; -1 for a stamp that was not written.  total_ms =
 * device time of the whole simulation (graph replay or normal run). */
nrt_status nrt_batch_times(const nrt_result* result, double* pair_ms, float* total_ms,
                           double* pair_paths_ms);

/* Autotuner: time the batch trace phase for each (packet, schedule) pair
 * (host int32[n_cfg] each; `repeats` timed runs, the minimum kept) into
 * host float ms[n_cfg]; the fastest configuration is stored in the result
 * (used by later replays only after a rebuild) and returned in *best. */
nrt_status nrt_autotune_batch(nrt_result* result, const int32_t* packets, const int32_t* schedules,
                              int n_cfg, int repeats, float* ms, int32_t* best);

/* Same gradient as nrt_backward, computed without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate -- work recorded into a CUDA graph (no cudaMalloc during
 * stream capture), real-time loops that must avoid the allocator's
 * device-wide synchronisation, hosts whose framework owns all device memory.
 *   dL_dpower : device float[n_rx]  (input)
 *   grad      : device float[3 * n_labels]: d/d eps_r, then d/d sigma, then
 *               d/d S, each n_labels long (output, caller-allocated)
 * The reduction's partial sums use a fixed 6 MiB array inside the library
 * (1024 blocks x 3 x 256 doubles) that every GPU loading the library keeps
 * until the process exits.  The first call on a device resolves that array's
 * device address (cudaGetSymbolAddress with the device current); make that
 * first call before any stream capture.  All calls share the array: calls
 * whose kernels overlap on the GPU (several streams or contexts at once)
 * race on it.  Each call writes every partial it reads, so no state carries
 * over between calls.  The kernel reads the result's path count on the
 * device, so a call recorded into a CUDA graph follows later traces of the
 * same result (nrt_batch_replay).  Work is enqueued on the context stream;
 * the call does not synchronise.  The call makes the context's device
 * current for its launches and restores the caller's current device.
 * Errors: NRT_ERR_ARG for NULL pointers, more than 256 labels or a result
 * traced with NRT_POL_VECTOR or with diffraction (scalar reflection and
 * scattering models only); NRT_ERR_STATE before
 * nrt_set_materials; NRT_ERR_CUDA. */
nrt_status nrt_backward_noalloc(nrt_result* result, const float* dL_dpower, float* grad);

/* Channel frequency response (Sec. III-B): for every receiver j and
 * f_n = f_c + (n - (N-1)/2) B/(N-1), n = 0..N-1, with f_c the simulation's
 * frequency (the path coefficients are taken there),
 *   H_j(f_n) = sum over RX j's paths of a_p exp(-j 2 pi f_n tau_p),
 * summed in FP64 (phase from the FP64 cycle count).  The CIR is its inverse
 * DFT.  H: host double[n_rx][n_freq][2] (re, im).  Needs the field
 * (materials set).  Synchronises.  Errors: NRT_ERR_ARG (n_freq < 2,
 * bandwidth <= 0), NRT_ERR_STATE (no materials). */
nrt_status nrt_cfr(nrt_result* result, double bandwidth, int32_t n_freq, double* H);

/* Eq. 5 loss per receiver, L_j = |h_j - h^_j|^2 / |h^_j|^2 on the CIR (equal
 * to the same ratio on the CFR by Parseval), and the gradient of
 * sum_j w_j L_j with respect to the per-label eps_r, sigma, S.
 *   H_target : host double[n_rx][n_freq][2], the target CFR (same grid)
 *   rx_weight: host float[n_rx] (0 leaves a receiver out)
 *   loss     : host double[n_rx] or NULL
 *   g_*      : host float[n_labels] each, or NULL
 * Synchronises.  Errors as nrt_cfr. */
nrt_status nrt_cfr_backward(nrt_result* result, double bandwidth, int32_t n_freq,
                            const double* H_target, const float* rx_weight, double* loss,
                            float* g_eps, float* g_sig, float* g_sca);

/* Per-key validation summary of a simulation run with keep_keys = 1 (used to
 * merge ray-range shards into the single-run result, Sec. II-B's lowest valid
 * ray per key): for each of the result's keys (nrt_result_counts' keys),
 * host arrays key_hi/key_lo (uint64), tried (uint32: candidates validated,
 * in ray-id order, the valid one included) and rep (uint32: ray id of the
 * validated candidate, 0xFFFFFFFF when the key found no valid candidate).
 * Errors: NRT_ERR_STATE when not requested. */
nrt_status nrt_keys_read(const nrt_result* result, uint64_t* key_hi, uint64_t* key_lo,
                         uint32_t* tried, uint32_t* rep);

/* ------------------------------------------------------------------ ray-range shards
 * One simulation split across GPUs by ray range (rays are independent until
 * duplicate paths are removed, Sec. II-B-4): every rank traces its range
 * (ray_subset), exports its paths to device buffers, the ranks all-gather
 * them, and nrt_shard_merge keeps per key the entry of the lowest shard in
 * ray-range order -- the key's lowest valid ray id, so the merged paths and
 * per-RX power equal one simulation of the whole launch.
 *
 * nrt_paths_export: the result's paths (nrt_result_counts' paths, in
 * nrt_paths_read order) into caller-allocated DEVICE arrays, any may be NULL:
 * key words, the representative ray id (0 for LOS and diffracted paths, which
 * have none and are the same on every shard) and |a|^2 (double; needs the
 * field).  Enqueued on the context stream.  Errors: NRT_ERR_STATE for power
 * without a field. */
nrt_status nrt_paths_export(const nrt_result* result, uint64_t* key_hi, uint64_t* key_lo,
                            uint32_t* rep, double* power);

/* Merge of n shard entries (DEVICE arrays): key_hi/key_lo, shard index
 * (ray-range order), rep (0xFFFFFFFF = the shard found no valid candidate),
 * tried (candidates the shard tried for the key, the valid one included; NULL
 * = exported valid paths, no try budget) and rep_tries (0 = no cap; > 0 =
 * the budget carried from shard to shard in ray order, with tried given).
 * win[i] (device uint8) = 1 when entry i represents its key; with power
 * (device double per entry, |a|^2) and power_out (device double[n_rx]), the
 * per-RX received power of the merged paths (RX = key_hi >> 56).  Allocates
 * scratch on the context stream; does not synchronise.  Errors: NRT_ERR_ARG. */
nrt_status nrt_shard_merge(nrt_ctx* ctx, int64_t n, const uint64_t* key_hi, const uint64_t* key_lo,
                           const uint32_t* shard, const uint32_t* tried, const uint32_t* rep,
                           int32_t rep_tries, const double* power, int32_t n_rx, uint8_t* win,
                           double* power_out);

/* ------------------------------------------------------------------ learned launch proposal
 * Not part of the paper, which traces a fixed Fibonacci launch (Sec. II-B):
 * a small network scores launch directions by the probability that the ray
 * is a member of a valid specular path key, and a Gumbel-top-k draw over
 * its logits picks the rays to trace (as a ray subset of the same launch).
 *
 * Training labels: with trace parameter ray_labels = 1, a simulation marks
 * each traced ray 1 when it is a candidate (member) of a valid specular key,
 * whichever ray represents the key.  host uint8_t labels[n_rows], rows in
 * ascending ray-id order.  Errors: NRT_ERR_STATE when not requested. */
nrt_status nrt_ray_labels_read(const nrt_result* result, uint8_t* labels);

/* The network: features = sin and cos of pi 2^k v_c for the 6 coordinates
 * v = (float32 launch direction, (tx - box centre) / box half-size) and
 * k = 0..7 (96 inputs, column (c * 8 + k) * 2 + {0 sin, 1 cos}); layers
 * 96 -> 128 -> 128 -> 128 (ReLU) -> 1 logit.  Weights and activations are
 * BF16, contractions accumulate in FP32 on the tensor cores, biases and the
 * master parameters are FP32.  Packed parameter order (float32):
 * W1[128][96], b1[128], W2[128][128], b2[128], W3[128][128], b3[128],
 * w4[128], b4[1]: 45,569 values. */
typedef struct nrt_mlp nrt_mlp;

typedef struct {
  float lr, beta1, beta2, eps; /* Adam (Kingma and Ba) with bias correction */
  float pos_weight;            /* weight of positive labels in the cross-entropy */
  int32_t batch;               /* samples per step, a positive multiple of 128 */
} nrt_mlp_train_opts;

/* params: host float[n_params] (n_params must be 45,569); box_min/box_max:
 * host float[3], the scene box used to normalise the TX; n_rays: N of the
 * Fibonacci launch whose directions are scored.  The network lives on the
 * context's device; Adam state starts at zero. */
nrt_status nrt_mlp_create(nrt_ctx* ctx, const float* params, int64_t n_params,
                          const float* box_min, const float* box_max, int64_t n_rays,
                          nrt_mlp** out);
void nrt_mlp_free(nrt_mlp* mlp);
/* host float[45569]: the FP32 master parameters / the gradient of the last step */
nrt_status nrt_mlp_params_read(const nrt_mlp* mlp, float* params);
nrt_status nrt_mlp_grads_read(const nrt_mlp* mlp, float* grads);
/* Checkpoint and resume of training (not part of the paper): the FP32 master
 * parameters, Adam's first and second moments (host float[45569] each) and
 * the number of Adam steps taken (their bias correction).  Writing restores
 * all of it and the BF16 weight copies, so training continues exactly as it
 * would have without the interruption.  Both synchronise.  Errors:
 * NRT_ERR_ARG for NULL pointers, a negative step, non-finite values or a
 * negative second moment. */
nrt_status nrt_mlp_state_read(const nrt_mlp* mlp, float* params, float* adam_m, float* adam_v,
                              int64_t* step);
nrt_status nrt_mlp_state_write(nrt_mlp* mlp, const float* params, const float* adam_m,
                               const float* adam_v, int64_t step);

/* BF16 input features of launch rays ray_ids (device uint32[n]; NULL: rays
 * 0..n-1) from TX tx (host float[3]) into device uint16_t[n][96] (bfloat16
 * bits).  Asynchronous on the context stream. */
nrt_status nrt_mlp_features(nrt_mlp* mlp, const float* tx, const uint32_t* ray_ids, int64_t n,
                            uint16_t* out);

/* Logits of launch rays ray_ids (device uint32[n] or NULL) from TX tx (host
 * float[3]) into device float[n].  Asynchronous on the context stream.  The
 * first call allocates and fills a table of the launch's directions (16 B
 * per ray, for launches of at most 2^26 rays; the network frees it), which
 * later calls read instead of recomputing each direction. */
nrt_status nrt_mlp_score(nrt_mlp* mlp, const float* tx, const uint32_t* ray_ids, int64_t n,
                         float* logits);

/* n_steps Adam steps of the mean weighted binary cross-entropy on device
 * samples: tx_table float[n_tx][3], tx_index int32[n], ray_id uint32[n],
 * label float[n] in {0, 1}; step s uses the `batch` samples at positions
 * start + s batch, ... (mod n) of `order` (device uint32[n] permutation, or
 * NULL for 0..n-1).  loss: host float[n_steps] (mean loss of each step) or
 * NULL.  Synchronises.  Errors: NRT_ERR_ARG; NRT_ERR_TIMEOUT if a tensor-core
 * wait ran out (the step's results are then invalid). */
nrt_status nrt_mlp_train(nrt_mlp* mlp, const float* tx_table, int32_t n_tx,
                         const int32_t* tx_index, const uint32_t* ray_id, const float* label,
                         int64_t n, const uint32_t* order, int64_t start, int32_t n_steps,
                         const nrt_mlp_train_opts* opts, float* loss);

/* Launch selection: the k_top largest keys fl32(logit_i + fl32(g_i)), g_i
 * standard Gumbel noise from a SplitMix64 counter generator (stream `seed`,
 * counter i), ties to the smaller index; plus one uniform index in each of
 * k_uniform equal strata of [0, n) (counters n + s).  The union, unique and
 * ascending, goes to device uint32 ids[] (capacity k_top + k_uniform);
 * *n_ids (host) receives its size.  logits: device float[n].  Synchronises. */
nrt_status nrt_propose(nrt_ctx* ctx, const float* logits, int64_t n, int64_t k_top,
                       int64_t k_uniform, uint64_t seed, uint32_t* ids, int64_t* n_ids);

/* The tensor-core contraction behind the network: C[M][N] (+)= A[M][K] B[N][K]^T,
 * A and B bfloat16 bits in K-major rows (device, 16-byte aligned, lda/ldb
 * multiples of 8), C float (device, ldc a multiple of 4).  N a multiple of
 * 16 in [16, 256]; K a multiple of 8.  accumulate = 1 adds into C; k_split > 0
 * splits K across thread blocks (implies adding into C).  Synchronises.
 * Errors: NRT_ERR_ARG on shapes or alignment; NRT_ERR_TIMEOUT. */
nrt_status nrt_gemm_bf16(nrt_ctx* ctx, const uint16_t* A, int64_t lda, const uint16_t* B,
                         int64_t ldb, float* C, int64_t ldc, int64_t M, int32_t N, int64_t K,
                         int32_t accumulate, int64_t k_split);

#ifdef __cplusplus
}
#endif

#endif /* NRT_H_ */
