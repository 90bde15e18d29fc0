/*
 * gf_oracle.h -- plain FP64 CPU oracle for the Gabor-field rendering path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py load this code.
 * It shares no code, header, table or constant generator with the CUDA
 * library: everything here is written from the paper's definitions
 * (arXiv 2602.05081, "Gabor Fields") and is slow on purpose.
 *
 * Conventions (identical meaning to the CUDA library, independent code):
 *   primitive i: mean mu, rotation R (unit quaternion w,x,y,z), scales
 *   s = exp(log_scale), Sigma = R S S^T R^T (Sec. 4.2), carrier omega
 *   (world rad/unit, or the whitened-frame vector k_W with
 *   omega = R S^-1 k_W when omega_frame == 1, the tied form of Sec. 4.2 being
 *   k_W = (w,w,w)), phase phi, amplitude A = weight (peak mode) or
 *   weight / sqrt(8 pi^3 |Sigma|) (normalised mode, Eq. 6).
 *   kernel: A exp(-q/2) cos(omega.(x-mu) + phi) 1[q <= k^2],
 *   q = (x-mu)^T Sigma^-1 (x-mu)  (Eq. 6 with the k-sigma support of Sec. 3).
 *
 * Multiple scattering (max_bounces >= 2) is pinned at two bounces: the
 * second-bounce radiance of a pixel on one Gaussian equals the nested
 * quadrature of the path integral (collision on the camera ray, isotropic
 * direction, collision on the second leg, NEE), with closed-form
 * transmittances; later bounces repeat the same loop step.  Its adjoint is
 * pinned the same way: the two-bounce gradient equals the central finite
 * differences of that quadrature.
 */
#ifndef GF_ORACLE_H
#define GF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox stream tags: the fourth counter word is (sample<<12)|(bounce<<8)|tag. */
#define OR_TAG_CAMERA 1u
#define OR_TAG_MASK 2u
#define OR_TAG_TRACK 3u
#define OR_TAG_NEE 4u
#define OR_TAG_NEE_MASK 5u
#define OR_TAG_SCATTER 6u

typedef struct {
  int64_t n;
  const float *mu, *quat, *log_scale, *omega, *phase, *weight; /* host arrays */
  const uint8_t *band; /* nullable: derived from |omega| when NULL */
  int weight_mode;     /* 0 peak amplitude, 1 normalised (Eq. 6) */
  int omega_frame;     /* 0 world, 1 whitened frame (k_W) */
  double k_sigma;      /* support radius in sigma units (3 in the paper) */
  double clamp_eps;    /* adaptive clamping (Sec. 4.4, Eqs. 14-15); 0 = off */
} or_field_desc;

typedef struct {
  int freq_policy; /* 0 all, 1 cutoff, 2 uniform + control variate, 3 uniform,
                      4 power law, 5 power law + control variate,
                      6 power law + control variate, accumulating */
  int max_band;    /* bands above this are never used (cutoff / sampled modes) */
  int cone_policy; /* 0 all, 1 importance w(a)=exp(-kbar^2 a^2/2), 2 uniform,
                      3 threshold culling, 4 threshold + uniform */
  float beta;      /* power-law shape, [0, 1) */
  float delta;     /* alignment threshold on a = |v . o|, [0, 1] */
} or_lod;

typedef struct {
  float eye[3], look_at[3], up[3];
  float vfov_deg;
  int width, height;
} or_camera;

typedef struct {
  int integrator;   /* 0 tomography (mean over samples of exp(-tau)), 1 scattering */
  int spp;
  int max_bounces;  /* collisions per path; 1 = single scattering */
  float albedo;
  float light_dir[3]; /* direction towards the light */
  float light_irradiance;
  int free_flight;    /* 0 delta tracking (NEE by ratio tracking); 1 inversion of the
                         optical-depth CDF by bisection (NEE transmittance exp(-tau));
                         2 uniform sampling within the crossing segment (NEE as 1) */
  int foveation;      /* 1: per-sample band cutoff by eccentricity (Supp., Foveated
                         Rendering): f = max(0, f0 - slope e) (1 + smooth (2 xi - 1)), e the
                         angle between the camera ray and the ray through the gaze pixel
                         coordinates, xi the camera stream's third uniform; Gabor bands whose
                         largest |omega| exceeds f leave every mask of the path */
  float gaze[2];
  float fov_f0, fov_slope, fov_smooth;
} or_render_opts;

typedef struct or_field or_field;

or_field* or_field_create(const or_field_desc* desc);

/* support radius of primitive i in sigma (whitened) units: k_sigma, or its
   adaptive extent when clamp_eps > 0 (0 = the primitive is dropped, by the
   clamp or by the camera selection below) */
double or_field_extent(const or_field* f, int64_t i);

/* camera-Nyquist LoD selection (Supp. A, LOD Selection): a pinhole camera
   with H rows and vertical field of view phi spans 2 d tan(phi/2) / H per
   pixel at distance d (the same along both image axes: square pixels), so
   the finest carrier it resolves there is f_limit(d) = pi H / (2 d tan(phi/2))
   rad per unit.  Every kernel whose |omega| exceeds f_limit at the distance d
   from the eye to its mean is removed from the mixture until the next call.
   The decision is taken in FP32 without contraction:
   |omega| d <= (float)(pi H / (2 tan(phi/2))).  cam == NULL keeps all. */
void or_field_set_camera_lod(or_field* f, const or_camera* cam);
void or_field_free(or_field* f);
int64_t or_field_size(const or_field* f);
/* per-primitive labels (band, cone, cell) and per-cell mean |k_W| */
void or_field_labels(const or_field* f, uint8_t* band, uint8_t* cone, uint8_t* cell);
void or_field_cells(const or_field* f, uint64_t* occupied, double* kbar64);
/* derived per-primitive quantities: Sigma^-1 (9, row major), omega (3), A */
void or_field_prim(const or_field* f, int64_t i, double* sinv9, double* omega3, double* amp);

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* one LoD mask draw (Sec. 4.5, App. B tables): mask bits and per-cell weights */
void or_sample_mask(const or_field* f, const or_lod* lod, const double v[3], uint64_t seed,
                    uint32_t ray, uint32_t sample, uint32_t bounce, uint32_t tag,
                    uint64_t* mask, double* w64);

/* density kappa(x) (Eq. 1) under a mask (w64 == NULL: all cells weight 1) */
double or_density(const or_field* f, const double x[3], uint64_t mask, const double* w64);

/* chord of primitive i on ray o + t v (v normalised here), clipped to [tmin,tmax]:
   returns 1 and lo/hi if non-empty */
int or_chord(const or_field* f, int64_t i, const double o[3], const double v[3], double tmin,
             double tmax, double* lo, double* hi);

/* integral of primitive i over its chord on the ray (Eq. 2 with alpha folded in A) */
double or_chord_integral(const or_field* f, int64_t i, const double o[3], const double v[3],
                         double tmin, double tmax);

/* tentative points of primitive i's chord (superposition sampler); returns the count
   (may exceed cap: only the first cap are written) */
int or_chord_points(const or_field* f, int64_t i, const double o[3], const double v[3], double tmin,
                    double tmax, double weight, uint64_t seed, uint32_t ray, uint32_t word,
                    double* t_out, double* uacc_out, int cap);

/* majorant kappa_bar(t) on a ray under mask (per-segment majorant, see the .c file) */
double or_majorant(const or_field* f, const double o[3], const double v[3], double tmin,
                   double tmax, double t, uint64_t mask, const double* w64);

/* transmittance of n rays (float inputs as the CUDA library receives them).
   mode 0: deterministic quadrature of tau (averaged over spp mask draws), T = exp(-tau)
   mode 1: ratio tracking, T = mean over spp of prod(1 - kappa/kappa_bar)      */
void or_transmittance(const or_field* f, const or_lod* lod, const float* o, const float* d,
                      const float* trange, int64_t n_rays, int mode, int spp, uint64_t seed,
                      double* T, double* tau, int n_threads);

/* free flight by inversion of the optical-depth CDF (Sec. 3 Eq. 5, segment-based
   transfer; Sec. 4.4 distance sampling): with xi the first uniform of the
   (seed, ray, word) stream, the distance t solves tau(tmin, t) = -ln(1 - xi),
   found by 60 bisections of [tmin, last chord exit]; returns 0 (escape) when
   the whole ray's tau does not reach the target.  The density must be
   non-negative along the ray for t to be the first crossing. */
int or_cdf_flight(const or_field* f, const double o[3], const double v[3], double tmin,
                  double tmax, uint64_t mask, const double* w64, uint64_t seed, uint32_t ray,
                  uint32_t word, double* t_hit);

/* free flight by uniform sampling within the crossing segment (Sec. 3: the cheap
   approximation of the inversion): segments are cut at tmin and at every chord
   entry and exit; the first segment [e_{k-1}, e_k] with tau(tmin, e_k) >= the
   target -ln(1 - xi) holds the collision e_{k-1} + u (e_k - e_{k-1}), xi and u
   the first two uniforms of the (seed, ray, word) stream.  Returns 0 when the
   whole ray's tau does not reach the target. */
int or_segment_flight(const or_field* f, const double o[3], const double v[3], double tmin,
                      double tmax, uint64_t mask, const double* w64, uint64_t seed,
                      uint32_t ray, uint32_t word, double* t_hit);

/* delta tracking along one ray: returns 1 and the collision t, or 0 if the ray escapes */
int or_delta_track(const or_field* f, const double o[3], const double v[3], double tmin,
                   double tmax, uint64_t mask, const double* w64, uint64_t seed, uint32_t ray,
                   uint32_t word, double* t_hit);

/* render a crop [x0,x0+w) x [y0,y0+h) of the image (row-major, w*h doubles) */
void or_render(const or_field* f, const or_lod* lod, const or_lod* lod_nee,
               const or_camera* cam, const or_render_opts* ro, uint64_t seed, int x0, int y0,
               int w, int h, double* out, int n_threads);

/* per-pixel sample values of a crop: out has w*h*spp doubles (pixel-major) */
void or_render_samples(const or_field* f, const or_lod* lod, const or_lod* lod_nee,
                       const or_camera* cam, const or_render_opts* ro, uint64_t seed, int x0,
                       int y0, int w, int h, double* out, int n_threads);

/* rays traced by or_render / or_render_samples since the last reset */
long long or_rays_traced(int reset);

/* camera ray of pixel (px,py), sample s */
void or_camera_ray(const or_camera* cam, uint64_t seed, int px, int py, int s, double o[3],
                   double v[3]);

/* tomography loss and its gradient w.r.t. the 15 parameters of every primitive:
   image I = mean_s exp(-tau_s) over jittered pinhole rays, L = sum (I - target)^2;
   grad layout (SoA, like the inputs): mu[3N], quat[4N], log_scale[3N], omega[3N],
   phase[N], weight[N].  Returns L. */
double or_tomo_loss_grad(const or_field_desc* desc, const or_camera* cam, int spp, uint64_t seed,
                         const float* target, double* grad, int n_threads);
/* tomography image only (same estimator, deterministic quadrature, all cells) */
/* radiance adjoint.  max_bounces 1 (single scattering): expected-value
   estimator over all tentative points of the ray, one NEE point drawn in
   proportion to its weight.  max_bounces >= 2: the delta-tracking path of
   the renderer (same streams and decisions), differentiated through the
   probability of each segment's accepted point and each NEE product.  Both
   hold the points, the majorant and the draw probabilities fixed (see the
   .c file).  Per ray (or pixel) the mean of spp samples goes to value/image;
   grad (15 N, SoA as the inputs) receives sum dLdI[r] / spp * d sample /
   d theta.  Rays: o, v double[3 n]. */
void or_radiance_grad_rays(const or_field_desc* desc, const or_lod* lod, const or_lod* lod_nee,
                           const or_render_opts* ro, const double* o, const double* v,
                           int64_t n_rays, int spp, uint64_t seed, const double* dLdI,
                           double* value, double* grad, int n_threads);
void or_radiance_grad_image(const or_field_desc* desc, const or_lod* lod, const or_lod* lod_nee,
                            const or_camera* cam, const or_render_opts* ro, uint64_t seed,
                            const double* dLdI, double* image, double* grad, int n_threads);

void or_tomo_image(const or_field_desc* desc, const or_camera* cam, int spp, uint64_t seed,
                   double* image, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
