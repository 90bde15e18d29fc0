/*
 * gf.h -- C ABI of the GB300 Gabor-field renderer (libgf.so).
 *
 * The library renders a density field made of anisotropic 3D Gabor kernels
 * (Condor, Hermann, Yurtsever et al., "Gabor Fields: Orientation-Selective
 * Level-of-Detail for Volume Rendering", arXiv 2602.05081):
 *
 *   kappa(x) = sum_i w_cell(i) A_i exp(-q_i(x)/2) cos(omega_i.(x-mu_i) + phi_i) 1[q_i(x) <= k^2]
 *   q_i(x)   = (x-mu_i)^T Sigma_i^-1 (x-mu_i),  Sigma_i = R_i S_i S_i^T R_i^T
 *
 * (Sec. 3 Eq. 1, Sec. 4.2 Eq. 6; the k-sigma ellipsoid support of Sec. 3; the
 * level-of-detail cell weights w of Sec. 4.5-4.6).  A phase phi_i generalises
 * the paper's zero-phase carrier (phi = 0 reproduces it).
 *
 * General conventions
 *  - Every call returns a gf_status; GF_OK is 0.  No exception crosses the ABI.
 *    gf_last_error() returns a thread-local message for the last failure.
 *  - Compute calls are asynchronous on the caller's CUDA stream (gf_stream is a
 *    cudaStream_t; NULL means the legacy default stream).  Device-side
 *    failures (a traversal stack or window that overflows, a bounded loop
 *    that gives up) set an error word in the field; gf_sync() waits on the
 *    stream and maps it to GF_EOVERFLOW / GF_ETIMEOUT.  Calls that
 *    synchronise anyway (host buffers) read and clear the word themselves
 *    and return that status.
 *  - The compute calls of one field (transmittance, render, adjoint, chord
 *    lists) share the field's work counter, error word and scratch: issue
 *    them on one stream, or serialise them.  Two such calls on different
 *    streams at once race (a kernel may skip work another one's counter
 *    reset hid).  Different fields are independent.
 *  - Array arguments are plain pointers.  Unless stated, a pointer may be
 *    device memory or host memory (pageable or pinned); host buffers are
 *    staged through library-owned device memory and the call then
 *    synchronises the stream before returning.  The caller owns every
 *    input and output buffer; the library owns packed records, the BVH and
 *    scratch, all released by gf_field_free / gf_destroy.
 *  - Device memory: every device buffer the library owns comes from the
 *    context's allocator (gf_create_ex; cudaMalloc/cudaFree by default), so a
 *    caller's memory manager (e.g. a framework's caching allocator) holds it.
 *    Fields allocate at gf_load_field, gf_build_bvh and gf_reserve; compute
 *    calls allocate only when a host buffer, image or adjoint is larger than
 *    what the field has reserved so far (then through the same allocator).
 *  - Layouts are structure-of-arrays, float32, row-major per element.
 *  - Random numbers: Philox4x32-10 (Salmon et al. 2011) keyed by the 64-bit
 *    seed, counter = (draw, primitive index or 0xFFFFFFFF, ray or pixel
 *    index, (sample << 12) | (bounce << 8) | stream tag); uniforms are
 *    (x >> 8) * 2^-24.  Results depend only on these counters, never on
 *    scheduling.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gf_status {
  GF_OK = 0,
  GF_EINVAL = 1,    /* invalid argument (null, non-finite, out of range) */
  GF_ENOMEM = 2,    /* device allocation failed */
  GF_ECUDA = 3,     /* a CUDA runtime call failed */
  GF_EOVERFLOW = 4, /* a bounded device buffer overflowed (stack, window, points) */
  GF_ETIMEOUT = 5,  /* a bounded device wait or loop gave up */
  GF_ESTATE = 6     /* call out of order (e.g. render before gf_build_bvh) */
} gf_status;

typedef struct gf_ctx gf_ctx;
typedef struct gf_field gf_field;
typedef void* gf_stream; /* cudaStream_t */

/* Primitive parameters, N entries each (Sec. 4.2; App. D lists the same set:
   mean, rotation quaternion, scales, carrier, weight, plus a phase).
   mu[3N]; quat[4N] as (w,x,y,z), normalised by the library; log_scale[3N]
   (natural log of the per-axis standard deviations); omega[3N] (see
   gf_field_opts.omega_frame); phase[N] (radians); weight[N]; band[N]
   optional octave label 0..7 (0 = the Gaussian low-pass band, Sec. 4.3),
   NULL derives floor(log2(1 + |omega|/(2 pi))) in FP32. */
typedef struct gf_params {
  int64_t n;
  const float* mu;
  const float* quat;
  const float* log_scale;
  const float* omega;
  const float* phase;
  const float* weight;
  const uint8_t* band;
} gf_params;

enum { GF_PREC_FP32 = 0, GF_PREC_FP16 = 1, GF_PREC_BF16 = 2 };
/* PEAK: A = weight (peak density).  NORMALIZED: A = weight / sqrt(8 pi^3 |Sigma|) (Eq. 6). */
enum { GF_WEIGHT_PEAK = 0, GF_WEIGHT_NORMALIZED = 1 };
/* WORLD: omega is the world-space carrier in rad/unit.  LOCAL: omega holds the
   whitened-frame carrier k_W and the world carrier is R S^-1 k_W; the paper's
   tied form (Sec. 4.2) is k_W = (w, w, w). */
enum { GF_OMEGA_WORLD = 0, GF_OMEGA_LOCAL = 1 };

typedef struct gf_field_opts {
  int precision;   /* GF_PREC_*: storage of the packed records (math is FP32).  FP16/BF16:
                      32-byte records (u16 means, the triangular whitening factor T with
                      T^T T = Sigma^-1 under one power-of-two exponent, the carrier in T's
                      frame and the amplitude as FP16/BF16, u16 phase); gf_build_bvh fails
                      with GF_EINVAL when an amplitude or carrier exceeds the FP16 range or
                      a scale lies beyond 2^+-126.  The adjoints need FP32 records. */
  int weight_mode; /* GF_WEIGHT_* */
  int omega_frame; /* GF_OMEGA_* */
  float k_sigma;   /* support radius in sigma units, (0, 6]; the paper uses 3 */
  /* adaptive clamping (Sec. 4.4, Eqs. 14-15): 0 = off; else each kernel's support
     radius becomes k_i = min(k_sigma, E_i) in whitened units with
     E_i^2 = 2 ln(rho_i / clamp_eps) - |k_W,i|^2, rho_i = |A_i| sqrt(2 pi) s_max,i
     (the kernel's largest line integral through its peak, the paper's alpha K
     at the longest axis); a kernel with E_i^2 <= 0 is dropped.  Finite, >= 0. */
  float clamp_eps;
} gf_field_opts;

/* Level-of-detail mask (Sec. 4.5.1-4.5.2, 4.6; strategy tables of App. B).
   Cells: cell 0 = Gaussian band; cell 1 + 8 (band-1) + cone for Gabor bands,
   cone = the nearest of 8 fixed orientation axes to the carrier direction.
   Bands above max_band are never used.  P = occupied bands, G = occupied
   Gabor bands (band >= 1), both counted up to max_band.
   freq_policy:
     ALL         every band, weight 1 (max_band ignored);
     CUTOFF      bands <= max_band, weight 1;
     UNIF_CV     Gaussians weight 1 plus one Gabor band uniformly, weight G;
     UNIFORM     one band uniformly, weight P;
     POWER       one band, level floor(P x^(1/(1-beta))) of the P in order,
                 weight 1/(((j+1)/P)^(1-beta) - (j/P)^(1-beta));
     POW_CV      Gaussians weight 1 plus one Gabor band by the power law over G;
     POW_CV_ACC  Gaussians weight 1 plus every Gabor band up to the level k
                 drawn by the power law over G; Gabor level j has weight
                 1/(1 - (j/G)^(1-beta)).
   cone_policy (inside every selected Gabor band; a = |v.o_c|):
     ALL             every cone;
     IS              one cone with probability w(a)/W, w(a) = exp(-kbar^2 a^2/2),
                     weight W/w(a) (Eq. 17);
     UNIFORM         one cone, weight K;
     THRESH          the cones with a <= delta, weight 1 (none: the least
                     aligned cone); deterministic and biased;
     THRESH_UNIFORM  the cones with a <= delta, weight 1, plus one of the
                     N_above others uniformly, weight N_above.
   beta in [0, 1) shapes the power law; delta in [0, 1] is the alignment
   threshold.  A new mask is drawn for every path segment (per bounce) and
   every NEE ray. */
enum {
  GF_FREQ_ALL = 0, GF_FREQ_CUTOFF = 1, GF_FREQ_UNIF_CV = 2, GF_FREQ_UNIFORM = 3,
  GF_FREQ_POWER = 4, GF_FREQ_POW_CV = 5, GF_FREQ_POW_CV_ACC = 6
};
enum {
  GF_CONE_ALL = 0, GF_CONE_IS = 1, GF_CONE_UNIFORM = 2, GF_CONE_THRESH = 3,
  GF_CONE_THRESH_UNIFORM = 4
};
typedef struct gf_lod_desc {
  int freq_policy;
  int max_band;
  int cone_policy;
  float beta;
  float delta;
} gf_lod_desc;

enum { GF_TR_DETERMINISTIC = 0, GF_TR_RATIO_TRACKING = 1, GF_TR_CLOSED_FORM = 2 };

/* Pinhole camera: pixel (px,py) of a width x height image (py = 0 at the top)
   looks along normalize(f + sx r + sy u) with f = normalize(look_at - eye),
   r = normalize(up x f), u = f x r, sx = (2(px+jx)/W - 1) tan(vfov/2) W/H,
   sy = (1 - 2(py+jy)/H) tan(vfov/2); (jx, jy) from the camera stream. */
typedef struct gf_camera {
  float eye[3], look_at[3], up[3];
  float vfov_deg;
  int width, height;
} gf_camera;

/* TOMO: image = mean over samples of exp(-tau) along the camera ray (Sec. 4.6,
   tomography).  SCATTER: delta tracking to a collision, weight albedo,
   next-event estimation to a directional light by ratio tracking with an
   isotropic phase 1/(4 pi), isotropic re-emission, up to max_bounces
   collisions (1 = single scattering). */
enum { GF_INTEG_TOMO = 0, GF_INTEG_SCATTER = 1 };
/* Free flight of the scattering integrator.  DELTA: delta tracking on the
   per-segment majorants, NEE transmittance by ratio tracking (see gf_render).
   CDF: the collision distance solves tau(0, t) = -ln(1 - xi) (Sec. 3 Eq. 5,
   segment-based transfer; Sec. 4.4 distance sampling), by 32 bisections on the
   closed-form optical depth (see GF_TR_CLOSED_FORM), and the NEE transmittance
   is exp(-tau) in closed form; it assumes a non-negative mixture along each
   ray (the first crossing) and is rendered per thread.
   SEGMENT: the cheap approximation of CDF (Sec. 3: uniform sampling within
   segments): the ray is cut into segments at t = 0 and every chord entry and
   exit, and the collision is drawn uniformly (second uniform of the stream)
   within the segment where tau(0, t) reaches -ln(1 - xi); biased where the
   density varies within a segment; NEE as CDF. */
enum { GF_FLIGHT_DELTA = 0, GF_FLIGHT_CDF = 1, GF_FLIGHT_SEGMENT = 2 };

typedef struct gf_render_opts {
  int integrator;
  int spp;
  int max_bounces;
  float albedo;
  float light_dir[3]; /* direction towards the light, normalised by the library */
  float light_irradiance;
  int free_flight;    /* GF_FLIGHT_* (else GF_EINVAL); scattering only; the server and the
                         adjoint take DELTA only (GF_EINVAL otherwise) */
  int first_sample;   /* samples first_sample .. first_sample + spp - 1 of every pixel are
                         rendered (their Philox streams) and averaged, so that a frame can be
                         accumulated over calls; >= 0 and first_sample + spp <= 2^20 */
  /* Foveation (Supp. "Foveated Rendering"): 0 off; 1 level masking.  Every
     sample of a pixel gets the frequency threshold
       f = max(0, fov_f0 - fov_slope e) (1 + fov_smooth (2 xi - 1)),
     e the angle (radians) between its camera ray and the ray through the gaze
     point (continuous pixel coordinates gaze[0], gaze[1], x right, y down), xi
     the third uniform of the sample's camera stream; the Gabor bands whose
     largest world carrier |omega| exceeds f leave every mask of the sample's
     path (camera, bounce and NEE rays), the Gaussian band stays.  fov_f0 >= 0
     (rad/unit), fov_slope >= 0 (rad/unit per radian), fov_smooth in [0, 1)
     (the stochastic smoothing of the level transitions).  Renders and the
     server; not the adjoint (GF_EINVAL). */
  int foveation;
  float gaze[2];
  float fov_f0, fov_slope, fov_smooth;
} gf_render_opts;

/* Work counters accumulated by the kernels since the last reset. */
typedef struct gf_stats {
  uint64_t rays;   /* traced rays: camera segments, bounce segments, NEE rays, API rays */
  uint64_t chords; /* chord set-ups (ray x primitive overlaps, per window) */
  uint64_t evals;  /* Gabor evaluations A exp(-q/2) cos(theta) */
  uint64_t nodes;  /* BVH node visits */
  uint64_t points; /* tentative collision points */
  uint64_t windows; /* BVH traversals (one per ray window) */
  uint64_t steps;  /* warp traversal steps (up to 32 nodes each) */
  uint64_t leaves; /* leaves reached (ellipsoid chord tests) */
  uint64_t cycles[5]; /* SM clock cycles per phase (traversal, tentative points, evaluation,
                         mask sampling, whole path), summed over warps; zero unless the
                         library was built with GF_PHASE_TIMERS */
} gf_stats;

/* Caller-supplied device allocator.  alloc returns at least `bytes` bytes of
   device memory on the context's device, aligned to 256 bytes, for use on
   `stream` (the stream of the call that needs it; NULL = legacy default), or
   NULL when it cannot (the call then fails with GF_ENOMEM).  free returns a
   pointer alloc gave, with the size that was asked for; the library calls it
   only after every piece of work that used the memory has completed (it
   synchronises the stream or device first), so the memory may be reused at
   once.  Both may be called from any thread of the process, including the
   render server's scheduler thread; `user` is passed through. */
typedef struct gf_allocator {
  void* (*alloc)(void* user, size_t bytes, gf_stream stream);
  void (*free)(void* user, void* ptr, size_t bytes, gf_stream stream);
  void* user;
} gf_allocator;

/* Context on one CUDA device (cudaSetDevice(device) is made current by every
   call that takes the context or a field created from it).  Computes the
   Gauss-Legendre tables.  GF_ECUDA if the device is missing or not sm_103.
   gf_create uses cudaMalloc/cudaFree; gf_create_ex takes the allocator of
   every device buffer of the context, its fields and its render servers
   (copied; NULL = cudaMalloc/cudaFree).  GF_EINVAL for an allocator with a
   null alloc or free. */
gf_status gf_create(int device, gf_ctx** out);
gf_status gf_create_ex(int device, const gf_allocator* allocator, gf_ctx** out);
gf_status gf_destroy(gf_ctx* ctx);

/* Pack the primitives (Sec. 4.2 parameters -> Sigma^-1, world carrier, amplitude,
   band/cone/cell labels; load-time binning of Sec. 4.6).  params arrays may be
   host or device memory.  Validates on the host/device: 1 <= n < 2^26, finite values,
   |quat| > 0, k_sigma in (0,6], clamp_eps finite and >= 0, band labels <= 7
   (GF_EINVAL).  The field keeps a copy of the raw parameters for
   gf_render_backward. */
gf_status gf_load_field(gf_ctx* ctx, const gf_params* params, const gf_field_opts* opts,
                        gf_stream stream, gf_field** out);
gf_status gf_field_free(gf_field* field);

/* Build the BVH over the k-sigma ellipsoid bounds (Sec. 3; the per-level
   acceleration structures of Sec. 4.6 become one radix tree whose top levels
   split by cell, every node carrying the 64-bit OR of its cells).
   Reorders the packed records along the tree.  GF_EOVERFLOW if the tree is
   deeper than the per-thread traversal stack (64 levels; clustered inputs
   whose keys share long prefixes); the field then stays unbuilt. */
gf_status gf_build_bvh(gf_field* field, gf_stream stream);

/* Scratch of the compute calls, allocated ahead (through the context's
   allocator) so that later calls within these sizes allocate nothing:
   max_rays rays of gf_transmittance / gf_ray_chords with host buffers (cap
   chords each for gf_ray_chords), max_pixels pixels of gf_render (the pixel
   sums of the scattering renderer and the staging of a host image), and
   the per-warp chord store of the scattering renderer when render != 0, and
   the per-thread lists of the radiance adjoint when adjoint != 0.  Sizes only
   grow; zeros leave a part as it is.  GF_ESTATE before gf_build_bvh. */
typedef struct gf_reserve_opts {
  int64_t max_rays;
  int max_chords;
  int64_t max_pixels;
  int render;
  int adjoint;
} gf_reserve_opts;
gf_status gf_reserve(gf_field* field, const gf_reserve_opts* opts, gf_stream stream);

/* Set the LoD mask used by subsequent calls: primary rays (camera and bounce
   segments, transmittance API) and NEE rays (nee may be NULL = same as primary). */
gf_status gf_set_lod_mask(gf_field* field, const gf_lod_desc* primary, const gf_lod_desc* nee);

/* Camera-Nyquist LoD selection (Supp. A, LOD Selection) for subsequent calls:
   a pinhole camera with H = camera->height rows and vertical field of view
   phi spans 2 d tan(phi/2) / H per pixel at distance d (square pixels), so it
   resolves carriers up to f_limit(d) = pi H / (2 d tan(phi/2)) rad per unit;
   every kernel with |omega| > f_limit(d) at the distance d from camera->eye
   to its mean leaves the mixture (all rays: camera, bounce, NEE, API), and
   cells left empty are skipped by the traversal.  Decided in FP32 without
   contraction: |omega| d <= (float)(pi H / (2 tan(phi/2))).  Composes with
   gf_set_lod_mask and with adaptive clamping.  camera NULL restores every
   kernel.  camera is host memory, read during the call.  GF_EINVAL for a
   camera with no pixels or a field of view outside (0, 180) degrees,
   GF_ESTATE for an unbuilt field or while a render server holds it.
   Synchronises the stream. */
gf_status gf_set_lod_camera(gf_field* field, const gf_camera* camera, gf_stream stream);

/* Transmittance of n_rays rays x(t) = o + t d, t in [trange[2r], trange[2r+1]]
   (trange NULL: [0, inf)); d is normalised by the library: the ray runs along
   the FP32 vector whose components are those of d/|d| rounded once (to within
   1e-14 of a rounding tie), so a caller can reproduce its line exactly.
   DETERMINISTIC: tau = sum over chords of the chord integral (Eq. 2), each by
   Gauss-Legendre quadrature with a node count set by the chord's whitened
   length and carrier phase span, FP32 with compensated summation; with a
   stochastic mask tau is averaged over spp mask draws (Sec. 4.6 tomography);
   out_T = exp(-tau), out_tau = tau (nullable).
   CLOSED_FORM: as DETERMINISTIC, but each chord integral is the finite-segment
   closed form of Sec. 4.4 / App. A.3 (complex error function), evaluated
   through the Faddeeva function w (Weideman's rational expansion, see
   gf_faddeeva) so that no term grows with the carrier frequency; chords
   shorter than 1e-4 in whitened length take the midpoint rule (Sec. 4.4).
   RATIO_TRACKING: out_T = mean over spp samples of prod (1 - kappa/kappa_bar)
   over the tentative points (per-segment majorants, see gf_render);
   out_tau is not written.  Signed kappa (absorption only).
   o, d: float[3n]; trange: float[2n]; out_T, out_tau: float[n]. */
gf_status gf_transmittance(gf_field* field, const float* o, const float* d, const float* trange,
                           int64_t n_rays, int mode, int spp, uint64_t seed, float* out_T,
                           float* out_tau, gf_stream stream);

/* Render width x height floats (row-major) into out_image.  Per path segment
   the ray is cut into segments at every chord entry/exit and wherever the
   whitened distance to a kernel's envelope peak crosses an integer; each
   segment carries the majorant kappa_bar = sum w|A| exp(-(r^2+n^2)/2) over
   the chords active on it, which bounds |kappa|; its tentative points are
   drawn chord by chord (a superposition of Poisson processes) and accepted
   with probability max(kappa,0)/kappa_bar (delta tracking) or weighted by
   1 - max(kappa,0)/kappa_bar (ratio tracking for NEE). */
gf_status gf_render(gf_field* field, const gf_camera* camera, const gf_render_opts* opts,
                    uint64_t seed, float* out_image, gf_stream stream);

/* Adjoint of a rendered image: given dL/dI (float[W*H]), write dL/dparam to
   grad (float[15 N], SoA like gf_params: mu[3N], quat[4N], log_scale[3N],
   omega[3N] in the input frame, phase[N], weight[N]); grad is overwritten.
   Nothing per path is stored: every ray is re-traced.  FP32 records only.
   TOMO (all cells): dtau/dtheta = integral of d(integrand)/dtheta plus the
   Leibniz terms of the chord ends on the ellipsoid (Eq. 2-3).
   SCATTER with max_bounces = 1 (LoD masks as set by gf_set_lod_mask): per
   sample, the expected-value form of delta tracking over all tentative
   points of the camera ray, I = sum_j W_j G(t_j), W_j = prod_{i<j}(1 - p_i)
   p_j, p = max(kappa,0)/kappa_bar, G = albedo E/(4 pi) T_light, with one
   point drawn in proportion to W (weighted reservoir sampling on the
   points' own uniforms) for its NEE ray; differentiated with the tentative
   points, kappa_bar and the draw probabilities held fixed, so the gradient
   is unbiased for the derivative of the expected image (the derivative of
   the k-sigma cut itself is not included).
   SCATTER with max_bounces >= 2: the renderer's delta-tracking path (same
   streams and decisions) is followed twice.  Segment b's accepted point has
   probability prod_{i<js}(1 - p_i) p_js, collision b adds C_b = albedo^(b+1)
   E/(4 pi) T_b (T_b the ratio-tracked NEE product); the gradient is that of
   sum_b S_b log P_b + sum_b C_b log T_b with S_b = sum_{b' >= b} C_b', the
   points and majorants held fixed (score function of each segment's
   decision; Sec. 3, Sec. 5.1), again unbiased for the derivative of the
   expected image.  Use a seed other than the forward render's so that the
   two estimates are independent. */
gf_status gf_render_backward(gf_field* field, const gf_camera* camera,
                             const gf_render_opts* opts, uint64_t seed,
                             const float* dL_dimage, float* grad, gf_stream stream);

/* Labels of every primitive (original order): band, cone, cell (uint8[N] each,
   nullable; host or device).  Synchronises the stream. */
gf_status gf_field_labels(gf_field* field, uint8_t* band, uint8_t* cone, uint8_t* cell,
                          gf_stream stream);

/* Chord sets for testing: for each ray, the primitives (original indices) whose
   ellipsoid the ray crosses inside trange under the current primary mask
   (deterministic policies only), with FP32 entry/exit t.  counts int32[n];
   prims int32[n*cap]; t_in, t_out float[n*cap] (nullable).  Rays with more
   than cap chords report the full count and the first cap entries found. */
gf_status gf_ray_chords(gf_field* field, const float* o, const float* d, const float* trange,
                        int64_t n_rays, int cap, int32_t* counts, int32_t* prims, float* t_in,
                        float* t_out, gf_stream stream);

/* Raw Philox4x32-10 blocks for testing: out[4n] from ctr[4n], key[2n]
   (uint32, host or device). */
gf_status gf_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                    gf_stream stream);

/* The Faddeeva function w(z) = exp(-z^2) erfc(-iz) that the CLOSED_FORM
   transmittance uses (Sec. 4.4 complex error function), for testing: FP32,
   Weideman's rational expansion with 20 terms (SIAM J. Numer. Anal. 31 (1994)
   1497).  z and w are float[2n] as (re, im) pairs, host or device memory;
   valid for im z >= 0 (w is NaN where im z < 0).  Host buffers make the call
   synchronise the stream. */
gf_status gf_faddeeva(const float* z, float* w, int64_t n, gf_stream stream);

/* gf_transmittance for callers that cannot allocate device memory at call time
   (an external memory manager forbids it, the device budget is spent, or only
   host arrays are at hand).  No counterpart in the paper: it is a deployment
   variant of gf_transmittance with the same arguments and the same results.
   It allocates nothing: its scratch (the kernel's work counter and device
   copies of host buffers) is one file-scope 8 MiB device array, present on
   every GPU that loads the library until the process exits.  Limits: n_rays
   <= 200000 (larger calls fail with GF_EINVAL; split them).  Pointers may be
   host or device memory; host buffers make the call synchronise the stream.
   The first call on a device looks up the array's device address (do it
   before any stream capture).  Every call shares the array, which keeps the
   previous call's contents (the counter is cleared per call): calls that
   overlap on the GPU (different streams or threads) race and must be
   serialised by the caller. */
gf_status gf_transmittance_static(gf_field* field, const float* o, const float* d,
                                  const float* trange, int64_t n_rays, int mode, int spp,
                                  uint64_t seed, float* out_T, float* out_tau, gf_stream stream);

/* ------------------------------------------------------------------------
   Render server: continuous batching of scattering renders over resident
   fields.  No counterpart in the paper (a serving layer around gf_render).

   Requests queue in arrival order.  A request is admitted when one of
   max_inflight slots is free and its framebuffer (width x height 64-bit
   fixed-point sums and width x height floats, each 256-byte aligned: 12
   bytes per pixel) fits in the server's device pool of mem_budget bytes;
   the head of the queue waits for memory (no overtaking).  Every batched
   launch gives each admitted request an equal share of batch_samples pixel
   samples (at least 32 pixels), taken as its next contiguous pixel range;
   one kernel launch renders the ranges of all admitted requests on all
   fields together, and two launches are kept in flight on two streams so
   that one launch's tail overlaps the next launch.  Requests admitted while
   launches run join the next launch.  Lanes take units of up to 8
   consecutive samples of one pixel; each sample's radiance is summed in
   64-bit fixed point (exact, in any order), so a request's image is bit for
   bit the one gf_render gives, whatever it was batched with.  When a
   request's last range completes, its sums become the image (sum / spp) and
   are copied to request.out (host or device)
   and its memory and slot are released; then it is DONE.
   A scheduler thread inside the library drives the device; submit, poll and
   wait may be called from any thread.  The fields must outlive the server. */
typedef struct gf_server gf_server;
typedef struct gf_server_opts {
  size_t mem_budget;     /* device bytes for request framebuffers (admission by memory) */
  int max_inflight;      /* requests admitted at once, 1..1024 */
  int max_queue;         /* pending requests beyond which submit fails with GF_EOVERFLOW */
  int64_t batch_samples; /* pixel samples per batched launch (0: 16 per resident lane) */
} gf_server_opts;
typedef struct gf_request {
  int asset;             /* index into the fields given to gf_server_create */
  gf_camera camera;
  gf_render_opts opts;   /* integrator must be GF_INTEG_SCATTER */
  gf_lod_desc lod;       /* primary rays */
  gf_lod_desc lod_nee;   /* NEE rays */
  uint64_t seed;
  float* out;            /* width*height floats, host or device, owned by the caller */
} gf_request;
enum { GF_REQ_QUEUED = 0, GF_REQ_RUNNING = 1, GF_REQ_DONE = 2, GF_REQ_FAILED = 3 };
typedef struct gf_result {
  int state;             /* GF_REQ_* */
  int status;            /* gf_status of a FAILED request, else GF_OK */
  double t_submit_ms;    /* server clock: ms since gf_server_create */
  double t_admit_ms;     /* admitted (slot and memory granted); 0 while queued */
  double t_done_ms;      /* image in request.out; 0 until DONE */
  int64_t launches;      /* batched launches that carried pixels of the request */
} gf_result;
typedef struct gf_server_stats {
  int64_t submitted, completed, failed;
  int64_t launches;          /* batched kernel launches */
  int64_t items;             /* (request, pixel range) items over all launches */
  int max_inflight_seen;     /* most requests admitted at once */
  int64_t max_bytes_seen;    /* most framebuffer bytes in use at once */
  double busy_ms;            /* sum of launch durations (CUDA events) */
  gf_stats work;             /* kernel work counters over all launches */
} gf_server_stats;

/* Create a server over n_fields built fields of one context (the fields stay
   owned by the caller).  Allocates the framebuffer pool, per-launch scratch
   for two launches in flight and the batch buffers, then starts the
   scheduler thread.  Every request carries its own camera, so a field with a
   camera LoD selection (gf_set_lod_camera) cannot be served, and a field
   cannot get one while a server holds it.  GF_EINVAL for bad options,
   GF_ESTATE for an unbuilt field or one with a camera selection, GF_ENOMEM if
   the pool does not fit. */
gf_status gf_server_create(gf_ctx* ctx, gf_field* const* fields, int n_fields,
                           const gf_server_opts* opts, gf_server** out);
/* Queue a request; *ticket identifies it.  Validated here: asset index,
   camera and options as for gf_render, LoD descriptors, a framebuffer that
   fits the pool at all (GF_EINVAL); a full queue gives GF_EOVERFLOW. */
gf_status gf_server_submit(gf_server* server, const gf_request* request, uint64_t* ticket);
/* State and timestamps of a request (GF_EINVAL for an unknown ticket). */
gf_status gf_server_poll(gf_server* server, uint64_t ticket, gf_result* out);
/* Block until the request is DONE or FAILED, or timeout_ms passes
   (GF_ETIMEOUT; the request keeps running). */
gf_status gf_server_wait(gf_server* server, uint64_t ticket, double timeout_ms, gf_result* out);
gf_status gf_server_get_stats(gf_server* server, gf_server_stats* out);
/* Stop admitting, fail the requests still queued, finish the admitted ones,
   stop the scheduler thread and free the server's memory. */
gf_status gf_server_destroy(gf_server* server);

/* Measured peaks of the two pipes a Gabor evaluation uses, for its roofline:
   *sfu_pairs_per_s = (ex2.approx, cos.approx) pairs per second over the whole
   GPU (one pair per evaluation of A exp(-q/2) cos(theta)), *fma_per_s = FP32
   fused multiply-adds per second; each the best of 5 timed launches (CUDA
   events) of independent instruction chains on every SM.  Measurement only:
   no counterpart in the paper; allocates nothing, synchronises the device's
   work on a stream of its own. */
gf_status gf_measure_peaks(int device, double* sfu_pairs_per_s, double* fma_per_s);

gf_status gf_get_stats(gf_field* field, gf_stats* out, int reset);
/* Wait for the stream, then report (and clear) any device-side error of the field. */
gf_status gf_sync(gf_field* field, gf_stream stream);
/* Number of primitives, precision, occupied cell mask. */
gf_status gf_field_info(gf_field* field, int64_t* n, int* precision, uint64_t* occupied);
const char* gf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GF_H */
