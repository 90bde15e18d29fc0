/*
 * gf_oracle.c -- plain FP64 CPU oracle for the Gabor-field rendering path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by the smoke check and by the
 * CPU-baseline leg of the benchmark, never by the product path.  Nothing here
 * is shared with the CUDA library.  Every function states the passage of
 * arXiv 2602.05081 ("Gabor Fields") it follows; where the paper is silent the
 * reading is named in the comment.
 *
 * Pinned by tests/test_oracle_pins.py: closed-form line integrals (App. A.4,
 * Sec. 4.4 whitened form, real erf for zero frequency), brute-force chord
 * sampling, invariants (all-bands mask, band sums, phase shift by pi,
 * rotation), the Philox known-answer vectors, estimator expectations (ratio
 * tracking, delta tracking CDF, masked optical depth, the Jensen bias of
 * Sec. 4.5.3) and central finite differences for the gradient.
 */
#include "gf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_NO_PRIM 0xFFFFFFFFu
#define OR_MAX_CELLS 64
#define OR_N_CONES 8

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the       */
/* multiply-xor round function, key bumped by the Weyl constants between     */
/* rounds.  Written from the published definition.                            */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* stream layout: key = seed; counter = (draw, primitive, ray, word) */
static void rng4(uint64_t seed, uint32_t draw, uint32_t prim, uint32_t ray, uint32_t word,
                 uint32_t x[4]) {
  uint32_t c[4] = {draw, prim, ray, word};
  uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(c, k, x);
}
static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
static uint32_t stream_word(uint32_t sample, uint32_t bounce, uint32_t tag) {
  return (sample << 12) | ((bounce & 15u) << 8) | (tag & 255u);
}

/* ------------------------------------------------------------------------ */
/* primitives                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
  double mu[3];
  double R[3][3];  /* columns are the principal axes */
  double s[3];
  double sinv[3][3]; /* Sigma^-1 = R S^-2 R^T */
  double omega[3];   /* world-space carrier, rad per unit length */
  double kw[3];      /* whitened-frame carrier k_W = S R^T omega */
  double phi, A;
  double k;          /* support radius in whitened units (k_sigma or adaptive; 0 = removed) */
  double k_own;      /* the radius before any camera selection */
  int band, cone, cell;
} or_prim;

struct or_field {
  int64_t n;
  or_prim* p;
  double k;
  uint64_t occupied;
  double kbar[OR_MAX_CELLS];
  double axes[OR_N_CONES][3];
  double band_wmax[8]; /* largest world carrier |omega| per band (foveation) */
};

int64_t or_field_size(const or_field* f) { return f->n; }

double or_field_extent(const or_field* f, int64_t i) { return f->p[i].k; }

void or_field_set_camera_lod(or_field* f, const or_camera* cam) {
  if (!cam) {
    for (int64_t i = 0; i < f->n; ++i) f->p[i].k = f->p[i].k_own;
    return;
  }
  const double th = tan(0.5 * (double)cam->vfov_deg * OR_PI / 180.0);
  const float c = (float)(OR_PI * (double)cam->height / (2.0 * th));
  for (int64_t i = 0; i < f->n; ++i) {
    or_prim* P = &f->p[i];
    float ox = (float)P->omega[0], oy = (float)P->omega[1], oz = (float)P->omega[2];
    float wn = sqrtf((ox * ox + oy * oy) + oz * oz);
    float dx = (float)P->mu[0] - cam->eye[0], dy = (float)P->mu[1] - cam->eye[1],
          dz = (float)P->mu[2] - cam->eye[2];
    float d = sqrtf((dx * dx + dy * dy) + dz * dz);
    P->k = (wn * d <= c) ? P->k_own : 0.0;
  }
}

/* cone axes on the upper hemisphere, Fibonacci spiral (reading of the
   unspecified orientation bins of Sec. 4.5.2) */
static void cone_axes(double ax[OR_N_CONES][3]) {
  for (int k = 0; k < OR_N_CONES; ++k) {
    double z = 1.0 - (k + 0.5) / OR_N_CONES;
    double r = sqrt(1.0 - z * z);
    double ph = k * OR_PI * (3.0 - sqrt(5.0));
    ax[k][0] = r * cos(ph);
    ax[k][1] = r * sin(ph);
    ax[k][2] = z;
  }
}

/* rotation matrix of the unit quaternion (w,x,y,z) (Sec. 4.2, Sigma = R S S^T R^T) */
static void quat_to_R(const double q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

/* band: octave label given by the caller, else floor(log2(1 + f)) with f the
   carrier frequency in cycles per unit (decided in FP32, like the kernel) */
static int band_from_omega(const double om[3]) {
  float wx = (float)om[0], wy = (float)om[1], wz = (float)om[2];
  float n2 = (wx * wx + wy * wy) + wz * wz;
  float fr = sqrtf(n2) / 6.28318530717958647692f;
  float onef = 1.0f + fr;
  int b = 0;
  for (int j = 1; j <= 7; ++j)
    if (onef >= (float)(1 << j)) b = j;
  return b;
}

/* orientation bin: the axis of largest |omega . o_k| (Sec. 4.5.2 binning by
   modulation orientation), ties to the lowest k, decided in FP32 */
static int cone_from_omega(const double om[3], double ax[OR_N_CONES][3]) {
  float wx = (float)om[0], wy = (float)om[1], wz = (float)om[2];
  int best = 0;
  float bv = -1.0f;
  for (int k = 0; k < OR_N_CONES; ++k) {
    float ox = (float)ax[k][0], oy = (float)ax[k][1], oz = (float)ax[k][2];
    float t0 = wx * ox;
    float t1 = wy * oy;
    float t2 = wz * oz;
    float d = fabsf((t0 + t1) + t2);
    if (d > bv) { bv = d; best = k; }
  }
  return best;
}

or_field* or_field_create(const or_field_desc* D) {
  or_field* f = (or_field*)calloc(1, sizeof(or_field));
  f->n = D->n;
  f->k = D->k_sigma;
  f->p = (or_prim*)calloc((size_t)(D->n > 0 ? D->n : 1), sizeof(or_prim));
  cone_axes(f->axes);
  double ksum[OR_MAX_CELLS] = {0};
  double kcnt[OR_MAX_CELLS] = {0};
  for (int64_t i = 0; i < D->n; ++i) {
    or_prim* P = &f->p[i];
    double q[4];
    double qn = 0;
    for (int j = 0; j < 4; ++j) { q[j] = D->quat[4 * i + j]; qn += q[j] * q[j]; }
    qn = sqrt(qn);
    for (int j = 0; j < 4; ++j) q[j] /= qn;
    quat_to_R(q, P->R);
    for (int j = 0; j < 3; ++j) {
      P->mu[j] = D->mu[3 * i + j];
      P->s[j] = exp((double)D->log_scale[3 * i + j]);
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double acc = 0;
        for (int j = 0; j < 3; ++j) acc += P->R[a][j] * P->R[b][j] / (P->s[j] * P->s[j]);
        P->sinv[a][b] = acc;
      }
    double in[3] = {D->omega[3 * i], D->omega[3 * i + 1], D->omega[3 * i + 2]};
    if (D->omega_frame == 1) {
      /* tied / local form: omega = R S^-1 k_W (Sec. 4.2, App. A) */
      for (int a = 0; a < 3; ++a) {
        double acc = 0;
        for (int j = 0; j < 3; ++j) acc += P->R[a][j] * in[j] / P->s[j];
        P->omega[a] = acc;
      }
      for (int j = 0; j < 3; ++j) P->kw[j] = in[j];
    } else {
      for (int a = 0; a < 3; ++a) P->omega[a] = in[a];
      /* k_W = S R^T omega: the carrier seen in the whitened frame */
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int a = 0; a < 3; ++a) acc += P->R[a][j] * in[a];
        P->kw[j] = P->s[j] * acc;
      }
    }
    P->phi = D->phase[i];
    double alpha = D->weight[i];
    if (D->weight_mode == 1)
      P->A = alpha / (pow(2.0 * OR_PI, 1.5) * P->s[0] * P->s[1] * P->s[2]);
    else
      P->A = alpha;
    P->band = D->band ? (int)D->band[i] : band_from_omega(P->omega);
    if (P->band > 7) P->band = 7;
    P->cone = P->band == 0 ? 0 : cone_from_omega(P->omega, f->axes);
    P->cell = P->band == 0 ? 0 : 1 + OR_N_CONES * (P->band - 1) + P->cone;
    f->occupied |= 1ull << P->cell;
    double kw2 = P->kw[0] * P->kw[0] + P->kw[1] * P->kw[1] + P->kw[2] * P->kw[2];
    ksum[P->cell] += sqrt(kw2);
    kcnt[P->cell] += 1;
    /* adaptive clamping (Sec. 4.4, Eqs. 14-15): along a ray through the peak the
       kernel integrates to at most rho = |A| sqrt(2 pi) s_max (the longest axis);
       the extent E where rho exp(-(E^2 + |k_W|^2)/2) falls to clamp_eps bounds
       the support, never beyond k_sigma; E^2 <= 0 drops the kernel */
    P->k = D->k_sigma;
    if (D->clamp_eps > 0) {
      double smax = fmax(fmax(P->s[0], P->s[1]), P->s[2]);
      double rho = fabs(P->A) * sqrt(2.0 * OR_PI) * smax;
      double e2 = 2.0 * log(rho / D->clamp_eps) - kw2;
      P->k = e2 <= 0 ? 0.0 : fmin(D->k_sigma, sqrt(e2));
    }
    P->k_own = P->k;
    double wn = sqrt(P->omega[0] * P->omega[0] + P->omega[1] * P->omega[1] + P->omega[2] * P->omega[2]);
    if (wn > f->band_wmax[P->band]) f->band_wmax[P->band] = wn;
  }
  for (int c = 0; c < OR_MAX_CELLS; ++c) f->kbar[c] = kcnt[c] > 0 ? ksum[c] / kcnt[c] : 0.0;
  return f;
}

void or_field_free(or_field* f) {
  if (!f) return;
  free(f->p);
  free(f);
}

void or_field_labels(const or_field* f, uint8_t* band, uint8_t* cone, uint8_t* cell) {
  for (int64_t i = 0; i < f->n; ++i) {
    if (band) band[i] = (uint8_t)f->p[i].band;
    if (cone) cone[i] = (uint8_t)f->p[i].cone;
    if (cell) cell[i] = (uint8_t)f->p[i].cell;
  }
}

void or_field_cells(const or_field* f, uint64_t* occupied, double* kbar64) {
  if (occupied) *occupied = f->occupied;
  if (kbar64) memcpy(kbar64, f->kbar, sizeof(f->kbar));
}

void or_field_prim(const or_field* f, int64_t i, double* sinv9, double* omega3, double* amp) {
  const or_prim* P = &f->p[i];
  if (sinv9)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) sinv9[3 * a + b] = P->sinv[a][b];
  if (omega3)
    for (int a = 0; a < 3; ++a) omega3[a] = P->omega[a];
  if (amp) *amp = P->A;
}

/* ------------------------------------------------------------------------ */
/* LoD mask (Sec. 4.5.1, 4.5.2, 4.6; App. B strategy tables)                 */
/* Cells: cell 0 is the Gaussian low-pass band (no orientation), cell        */
/* 1 + 8 (band-1) + cone for Gabor bands 1..7.  A ray uses a primitive iff   */
/* its cell bit is set (the visibility-mask test of Sec. 4.6), and scales it */
/* by the cell's reciprocal-probability weight.                               */
/* ------------------------------------------------------------------------ */
static uint64_t band_cells(const or_field* f, int b) {
  if (b == 0) return f->occupied & 1ull;
  uint64_t m = 0;
  for (int c = 0; c < OR_N_CONES; ++c) m |= 1ull << (1 + OR_N_CONES * (b - 1) + c);
  return m & f->occupied;
}

/* power-law level choice over n levels (App. B frequency table): the level is
   floor(n x^(1/(1-beta))), x uniform, i.e. level j when
   (j/n)^(1-beta) <= x < ((j+1)/n)^(1-beta); the thresholds are compared in
   FP32, as the kernel does */
static int power_level(double x, int n, double beta) {
  float e = (float)(1.0 - beta);
  int j = 0;
  while (j + 1 < n && (float)x >= powf((float)(j + 1) / (float)n, e)) ++j;
  return j;
}
/* probability of power-law level j out of n: ((j+1)/n)^(1-beta) - (j/n)^(1-beta) */
static double power_prob(int j, int n, double beta) {
  return pow((double)(j + 1) / n, 1.0 - beta) - pow((double)j / n, 1.0 - beta);
}

void or_sample_mask(const or_field* f, const or_lod* L, const double v[3], uint64_t seed,
                    uint32_t ray, uint32_t sample, uint32_t bounce, uint32_t tag,
                    uint64_t* mask_out, double* w64) {
  uint32_t word = stream_word(sample, bounce, tag);
  double bw[8] = {0};
  int sel[8] = {0};
  int maxb = L->freq_policy == 0 ? 7 : L->max_band;
  int occ[8], nocc = 0, gab[8], ngab = 0;
  for (int b = 0; b <= 7 && b <= maxb; ++b)
    if (band_cells(f, b)) {
      occ[nocc++] = b;
      if (b > 0) gab[ngab++] = b;
    }
  uint32_t x[4];
  rng4(seed, 0, OR_NO_PRIM, ray, word, x);
  uint32_t x24 = x[0] >> 8;
  const double beta = L->beta;
  if (L->freq_policy == 0 || L->freq_policy == 1) {
    for (int j = 0; j < nocc; ++j) { sel[occ[j]] = 1; bw[occ[j]] = 1.0; }
  } else if (L->freq_policy == 2) {
    /* Uniform + control variate: Gaussians always (weight 1), one Gabor band
       uniformly with weight P-1 (App. B, frequency table) */
    if (band_cells(f, 0)) { sel[0] = 1; bw[0] = 1.0; }
    if (ngab > 0) {
      int j = (int)(((uint64_t)x24 * (uint64_t)ngab) >> 24);
      sel[gab[j]] = 1;
      bw[gab[j]] = (double)ngab;
    }
  } else if (L->freq_policy == 3) {
    /* Uniform: one level out of P with weight P */
    if (nocc > 0) {
      int j = (int)(((uint64_t)x24 * (uint64_t)nocc) >> 24);
      sel[occ[j]] = 1;
      bw[occ[j]] = (double)nocc;
    }
  } else if (L->freq_policy == 4) {
    /* Power law over all P levels, weight 1 / P(level) */
    if (nocc > 0) {
      int j = power_level(u01(x[0]), nocc, beta);
      sel[occ[j]] = 1;
      bw[occ[j]] = 1.0 / power_prob(j, nocc, beta);
    }
  } else {
    /* control variate: Gaussians always, weight 1; power law over the G Gabor
       levels: one level (5), or every level up to the drawn one (6, level j
       kept with probability 1 - (j/G)^(1-beta)) */
    if (band_cells(f, 0)) { sel[0] = 1; bw[0] = 1.0; }
    if (ngab > 0) {
      int k = power_level(u01(x[0]), ngab, beta);
      if (L->freq_policy == 5) {
        sel[gab[k]] = 1;
        bw[gab[k]] = 1.0 / power_prob(k, ngab, beta);
      } else {
        for (int j = 0; j <= k; ++j) {
          sel[gab[j]] = 1;
          bw[gab[j]] = 1.0 / (1.0 - pow((double)j / ngab, 1.0 - beta));
        }
      }
    }
  }
  uint64_t mask = 0;
  for (int c = 0; c < OR_MAX_CELLS; ++c) w64[c] = 0.0;
  for (int b = 0; b <= 7; ++b) {
    if (!sel[b]) continue;
    uint64_t cells = band_cells(f, b);
    if (b == 0 || L->cone_policy == 0) {
      mask |= cells;
      for (int c = 0; c < OR_MAX_CELLS; ++c)
        if (cells >> c & 1ull) w64[c] = bw[b];
      continue;
    }
    int cc[OR_N_CONES], nc = 0;
    for (int k = 0; k < OR_N_CONES; ++k) {
      int c = 1 + OR_N_CONES * (b - 1) + k;
      if (cells >> c & 1ull) cc[nc++] = c;
    }
    uint32_t y[4];
    rng4(seed, (uint32_t)(1 + b), OR_NO_PRIM, ray, word, y);
    if (L->cone_policy == 2) {
      /* Uniform orientation bin, weight K (App. B, orientation table) */
      int j = (int)(((uint64_t)(y[0] >> 8) * (uint64_t)nc) >> 24);
      mask |= 1ull << cc[j];
      w64[cc[j]] = bw[b] * nc;
    } else if (L->cone_policy == 3 || L->cone_policy == 4) {
      /* alignment a = |v . o| decided in FP32 against delta: threshold culling
         keeps the bins with a <= delta (weight 1; if none, the least aligned
         bin, the one of largest contribution); threshold + uniform keeps them
         and draws one of the N_above others uniformly, weight N_above */
      int above[OR_N_CONES], na = 0, best = -1;
      float abest = 2.0f;
      for (int j = 0; j < nc; ++j) {
        int k = (cc[j] - 1) % OR_N_CONES;
        float a = fabsf((float)v[0] * (float)f->axes[k][0] + (float)v[1] * (float)f->axes[k][1] +
                        (float)v[2] * (float)f->axes[k][2]);
        if (a < abest) { abest = a; best = cc[j]; }
        if (a <= L->delta) {
          mask |= 1ull << cc[j];
          w64[cc[j]] = bw[b];
        } else {
          above[na++] = cc[j];
        }
      }
      if (L->cone_policy == 3) {
        if (na == nc && best >= 0) {
          mask |= 1ull << best;
          w64[best] = bw[b];
        }
      } else if (na > 0) {
        int j = (int)(((uint64_t)(y[0] >> 8) * (uint64_t)na) >> 24);
        mask |= 1ull << above[j];
        w64[above[j]] = bw[b] * na;
      }
    } else {
      /* Importance sampling: p_i = w_i / W, weight W / w_i with
         w(a) = exp(-kbar^2 a^2 / 2), a = |v . o_i| (Eq. 17, App. B) */
      double wc[OR_N_CONES], W = 0;
      for (int j = 0; j < nc; ++j) {
        int k = (cc[j] - 1) % OR_N_CONES;
        double a = fabs(v[0] * f->axes[k][0] + v[1] * f->axes[k][1] + v[2] * f->axes[k][2]);
        double kb = f->kbar[cc[j]];
        wc[j] = exp(-0.5 * kb * kb * a * a);
        W += wc[j];
      }
      double target = u01(y[0]) * W, acc = 0;
      int pick = nc - 1;
      for (int j = 0; j < nc; ++j) {
        acc += wc[j];
        if (target < acc) { pick = j; break; }
      }
      mask |= 1ull << cc[pick];
      w64[cc[pick]] = bw[b] * W / wc[pick];
    }
  }
  *mask_out = mask;
}

/* ------------------------------------------------------------------------ */
/* density and chords                                                        */
/* ------------------------------------------------------------------------ */
/* kernel value at x (Eq. 6 with amplitude A, phase phi and the k-sigma
   support of Sec. 3), evaluated directly in 3D */
static double prim_value(const or_prim* P, const double x[3], double k) {
  double y[3] = {x[0] - P->mu[0], x[1] - P->mu[1], x[2] - P->mu[2]};
  double q = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) q += y[a] * P->sinv[a][b] * y[b];
  if (q > k * k) return 0.0;
  double th = P->omega[0] * y[0] + P->omega[1] * y[1] + P->omega[2] * y[2] + P->phi;
  return P->A * exp(-0.5 * q) * cos(th);
}

double or_density(const or_field* f, const double x[3], uint64_t mask, const double* w64) {
  double acc = 0;
  for (int64_t i = 0; i < f->n; ++i) {
    const or_prim* P = &f->p[i];
    if (!(mask >> P->cell & 1ull)) continue;
    double w = w64 ? w64[P->cell] : 1.0;
    acc += w * prim_value(P, x, P->k);
  }
  return acc;
}

/* along a ray x(t) = o + t v: q(t) = a t^2 + 2 beta t + gamma with
   a = v^T Sigma^-1 v, beta = v^T Sigma^-1 d, gamma = d^T Sigma^-1 d, d = o - mu
   (App. A.1).  t* = -beta/a minimises q; r2 = q(t*) is evaluated at the
   closest point to avoid cancellation. */
typedef struct {
  int has;
  double lo, hi;      /* clipped chord */
  double a, tstar, r2, hw;
} or_chord_t;

static or_chord_t chord_of(const or_prim* P, const double o[3], const double v[3], double k,
                           double tmin, double tmax) {
  or_chord_t c;
  memset(&c, 0, sizeof(c));
  double d[3] = {o[0] - P->mu[0], o[1] - P->mu[1], o[2] - P->mu[2]};
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = P->sinv[a][0] * v[0] + P->sinv[a][1] * v[1] + P->sinv[a][2] * v[2];
  double a = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
  double beta = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
  double ts = -beta / a;
  double p[3] = {d[0] + ts * v[0], d[1] + ts * v[1], d[2] + ts * v[2]};
  double r2 = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r2 += p[i] * P->sinv[i][j] * p[j];
  c.a = a;
  c.tstar = ts;
  c.r2 = r2;
  if (!(r2 < k * k)) return c;
  c.hw = sqrt((k * k - r2) / a);
  c.lo = fmax(ts - c.hw, tmin);
  c.hi = fmin(ts + c.hw, tmax);
  c.has = c.lo < c.hi;
  return c;
}

static void normalise(const double in[3], double out[3]) {
  double n = sqrt(in[0] * in[0] + in[1] * in[1] + in[2] * in[2]);
  out[0] = in[0] / n; out[1] = in[1] / n; out[2] = in[2] / n;
}

/* The direction of a caller's ray: the unit vector of the FP32 input d, rounded
   to FP32.  This is the input rounding of the library's boundary (its rays are
   FP32 unit vectors), applied here so that both sides trace the same line; the
   rounding of a direction moves a point at distance t by ~6e-8 t, which a
   carrier of ~1e3 rad/unit turns into phase errors of ~1e-4 rad. */
static void api_direction(const float d[3], double v[3]) {
  double dd[3] = {d[0], d[1], d[2]};
  normalise(dd, v);
  for (int k = 0; k < 3; ++k) v[k] = (double)(float)v[k];
}

int or_chord(const or_field* f, int64_t i, const double o[3], const double v_in[3], double tmin,
             double tmax, double* lo, double* hi) {
  double v[3];
  normalise(v_in, v);
  or_chord_t c = chord_of(&f->p[i], o, v, f->p[i].k, tmin, tmax);
  if (lo) *lo = c.lo;
  if (hi) *hi = c.hi;
  return c.has;
}

/* ------------------------------------------------------------------------ */
/* quadrature: composite Gauss-Legendre, 20 nodes per panel; panels keep the  */
/* whitened length <= 1/2 and the carrier phase change <= 2 rad, where the    */
/* 20-node rule is exact to rounding for this integrand.                      */
/* ------------------------------------------------------------------------ */
#define OR_GL_N 20
static double g_glx[OR_GL_N], g_glw[OR_GL_N];
static int g_gl_ready = 0;

/* nodes and weights: Newton iteration on the Legendre recurrence */
static void gl_init(void) {
  if (g_gl_ready) return;
  int n = OR_GL_N;
  for (int i = 0; i < n; ++i) {
    double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double z1 = z;
      z = z1 - p1 / pp;
      if (fabs(z - z1) < 1e-16) break;
    }
    g_glx[i] = z;
    g_glw[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
  g_gl_ready = 1;
}

static int n_panels(const or_prim* P, const or_chord_t* c, const double v[3]) {
  double len = c->hi - c->lo;
  double ls = sqrt(c->a) * len;
  double B = fabs(P->omega[0] * v[0] + P->omega[1] * v[1] + P->omega[2] * v[2]);
  double np = fmax(fmax(ls / 0.5, B * len / 2.0), 1.0);
  return (int)ceil(np);
}

/* tau_i = A int_chord exp(-q/2) cos(theta) dt (Eq. 2) */
static double chord_integral(const or_prim* P, const or_chord_t* c, const double o[3],
                             const double v[3], double k) {
  if (!c->has) return 0.0;
  int np = n_panels(P, c, v);
  double h = (c->hi - c->lo) / np, acc = 0;
  for (int p = 0; p < np; ++p) {
    double a = c->lo + p * h, m = a + 0.5 * h, part = 0;
    for (int j = 0; j < OR_GL_N; ++j) {
      double t = m + 0.5 * h * g_glx[j];
      double x[3] = {o[0] + t * v[0], o[1] + t * v[1], o[2] + t * v[2]};
      double y[3] = {x[0] - P->mu[0], x[1] - P->mu[1], x[2] - P->mu[2]};
      double q = 0;
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) q += y[r] * P->sinv[r][s] * y[s];
      double th = P->omega[0] * y[0] + P->omega[1] * y[1] + P->omega[2] * y[2] + P->phi;
      part += g_glw[j] * exp(-0.5 * q) * cos(th);
    }
    acc += 0.5 * h * part;
  }
  (void)k;
  return P->A * acc;
}

double or_chord_integral(const or_field* f, int64_t i, const double o[3], const double v_in[3],
                         double tmin, double tmax) {
  gl_init();
  double v[3];
  normalise(v_in, v);
  or_chord_t c = chord_of(&f->p[i], o, v, f->p[i].k, tmin, tmax);
  return chord_integral(&f->p[i], &c, o, v, f->p[i].k);
}

/* ------------------------------------------------------------------------ */
/* per-segment majorant and tentative points                                  */
/*                                                                            */
/* The ray is cut at the entry/exit points of every chord (the segments of    */
/* Sec. 3, Eq. 4) and, inside each chord, where the whitened distance to the   */
/* envelope peak s = sqrt(a)|t - t*| crosses an integer.  On each resulting   */
/* segment the majorant is constant:                                          */
/*   kappa_bar = sum over active chords of w |A| exp(-(r2 + n^2)/2),          */
/*   n = floor(s) on that piece,                                              */
/* which bounds |kappa| because |cos| <= 1 and exp(-s^2/2) <= exp(-n^2/2).    */
/* Its Poisson process of tentative points is the superposition of one        */
/* process per chord (rate w|A|exp(-(r2+n^2)/2) piecewise along the chord),   */
/* so each chord draws its own points from its own Philox stream: counter =   */
/* (draw, primitive index, ray, word); per point x[0] gives the exponential   */
/* step and x[1] the acceptance uniform.                                      */
/* ------------------------------------------------------------------------ */
static double piece_rate(double wA, double r2, int n) { return wA * exp(-0.5 * (r2 + (double)n * n)); }

static int chord_points(const or_chord_t* c, double wA, double k, uint64_t seed, uint32_t prim,
                        uint32_t ray, uint32_t word, double* ts, double* ua, int cap) {
  if (!c->has || !(wA > 0)) return 0;
  double sa = sqrt(c->a);
  double smax = sqrt(k * k - c->r2);
  int J = 0;
  while ((double)(J + 1) < smax) ++J;  /* interior boundaries at t* +- j/sqrt(a), j=1..J */
  double bnd[32];
  int pn[33];
  int nb = 0;
  if (J > 15) J = 15;
  for (int j = J; j >= 1; --j) bnd[nb++] = c->tstar - j / sa;
  for (int j = 1; j <= J; ++j) bnd[nb++] = c->tstar + j / sa;
  /* piece p lies left of bnd[p]; pieces 0..J-1 carry n = J..1, piece J carries 0 */
  for (int p = 0; p <= nb; ++p) pn[p] = p < J ? J - p : p - J;
  double t = c->lo;
  int p = 0;
  while (p < nb && bnd[p] <= t) ++p;
  int count = 0;
  uint32_t draw = 0;
  for (int guard = 0; guard < (1 << 20); ++guard) {
    uint32_t x[4];
    rng4(seed, draw++, prim, ray, word, x);
    double z = -log1p(-u01(x[0]));
    double uacc = u01(x[1]);
    for (;;) {
      double end = p < nb ? fmin(bnd[p], c->hi) : c->hi;
      double lam = piece_rate(wA, c->r2, pn[p]);
      double capz = lam * (end - t);
      if (z < capz) {
        t += z / lam;
        if (count < cap) { ts[count] = t; ua[count] = uacc; }
        ++count;
        break;
      }
      z -= capz;
      t = end;
      if (t >= c->hi) return count;
      ++p;
    }
  }
  return count;
}

int or_chord_points(const or_field* f, int64_t i, const double o[3], const double v_in[3],
                    double tmin, double tmax, double weight, uint64_t seed, uint32_t ray,
                    uint32_t word, double* t_out, double* uacc_out, int cap) {
  double v[3];
  normalise(v_in, v);
  or_chord_t c = chord_of(&f->p[i], o, v, f->p[i].k, tmin, tmax);
  return chord_points(&c, weight * fabs(f->p[i].A), f->p[i].k, seed, (uint32_t)i, ray, word, t_out,
                      uacc_out, cap);
}

static double chord_bound(const or_chord_t* c, double wA, double t) {
  if (!c->has || t < c->lo || t > c->hi) return 0.0;
  double s = sqrt(c->a) * fabs(t - c->tstar);
  int n = (int)floor(s);
  return piece_rate(wA, c->r2, n);
}

double or_majorant(const or_field* f, const double o[3], const double v_in[3], double tmin,
                   double tmax, double t, uint64_t mask, const double* w64) {
  double v[3];
  normalise(v_in, v);
  double acc = 0;
  for (int64_t i = 0; i < f->n; ++i) {
    const or_prim* P = &f->p[i];
    if (!(mask >> P->cell & 1ull)) continue;
    double w = w64 ? w64[P->cell] : 1.0;
    or_chord_t c = chord_of(P, o, v, P->k, tmin, tmax);
    acc += chord_bound(&c, w * fabs(P->A), t);
  }
  return acc;
}

/* ------------------------------------------------------------------------ */
/* per-ray work: all chords of all N primitives (no acceleration structure)  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t prim;
  double w;
  or_chord_t c;
} or_hit;

typedef struct {
  double t, ua;
} or_pt;

static int cmp_pt(const void* A, const void* B) {
  double a = ((const or_pt*)A)->t, b = ((const or_pt*)B)->t;
  return (a > b) - (a < b);
}

static int collect_hits(const or_field* f, const double o[3], const double v[3], double tmin,
                        double tmax, uint64_t mask, const double* w64, or_hit** out) {
  int cap = 64, n = 0;
  or_hit* h = (or_hit*)malloc(sizeof(or_hit) * cap);
  for (int64_t i = 0; i < f->n; ++i) {
    const or_prim* P = &f->p[i];
    if (!(mask >> P->cell & 1ull)) continue;
    double w = w64 ? w64[P->cell] : 1.0;
    if (!(w > 0)) continue;
    or_chord_t c = chord_of(P, o, v, P->k, tmin, tmax);
    if (!c.has) continue;
    if (n == cap) { cap *= 2; h = (or_hit*)realloc(h, sizeof(or_hit) * cap); }
    h[n].prim = i; h[n].w = w; h[n].c = c;
    ++n;
  }
  *out = h;
  return n;
}

static int gather_points(const or_field* f, const or_hit* h, int nh, uint64_t seed, uint32_t ray,
                         uint32_t word, or_pt** out) {
  int cap = 256, n = 0;
  or_pt* pts = (or_pt*)malloc(sizeof(or_pt) * cap);
  double tb[4096], ub[4096];
  for (int j = 0; j < nh; ++j) {
    const or_prim* P = &f->p[h[j].prim];
    int m = chord_points(&h[j].c, h[j].w * fabs(P->A), P->k, seed, (uint32_t)h[j].prim, ray, word,
                         tb, ub, 4096);
    if (m > 4096) m = 4096;
    for (int q = 0; q < m; ++q) {
      if (n == cap) { cap *= 2; pts = (or_pt*)realloc(pts, sizeof(or_pt) * cap); }
      pts[n].t = tb[q]; pts[n].ua = ub[q];
      ++n;
    }
  }
  *out = pts;
  return n;
}

/* kappa and kappa_bar at a point of the ray, over the chords hit */
static void eval_point(const or_field* f, const or_hit* h, int nh, const double o[3],
                       const double v[3], double t, double* kap, double* kbar) {
  double x[3] = {o[0] + t * v[0], o[1] + t * v[1], o[2] + t * v[2]};
  double k = 0, kb = 0;
  for (int j = 0; j < nh; ++j) {
    if (t < h[j].c.lo || t > h[j].c.hi) continue;
    const or_prim* P = &f->p[h[j].prim];
    k += h[j].w * prim_value(P, x, P->k);
    kb += chord_bound(&h[j].c, h[j].w * fabs(P->A), t);
  }
  *kap = k;
  *kbar = kb;
}

/* ratio tracking (Novak et al. 2014; Sec. 5.1 uses it for reference
   tomography): T = prod over tentative points of (1 - kappa/kappa_bar).
   clamp_neg selects the extinction max(kappa, 0) of scattering media. */
static double ratio_track(const or_field* f, const double o[3], const double v[3], double tmin,
                          double tmax, uint64_t mask, const double* w64, uint64_t seed,
                          uint32_t ray, uint32_t word, int clamp_neg) {
  or_hit* h;
  int nh = collect_hits(f, o, v, tmin, tmax, mask, w64, &h);
  or_pt* pts;
  int np = gather_points(f, h, nh, seed, ray, word, &pts);
  double T = 1.0;
  for (int j = 0; j < np; ++j) {
    double kap, kb;
    eval_point(f, h, nh, o, v, pts[j].t, &kap, &kb);
    if (clamp_neg && kap < 0) kap = 0;
    if (kb > 0) T *= 1.0 - kap / kb;
  }
  free(h);
  free(pts);
  return T;
}

/* delta tracking (Woodcock): first tentative point, in t order, accepted with
   probability max(kappa,0)/kappa_bar */
int or_delta_track(const or_field* f, const double o[3], const double v_in[3], double tmin,
                   double tmax, uint64_t mask, const double* w64, uint64_t seed, uint32_t ray,
                   uint32_t word, double* t_hit) {
  double v[3];
  normalise(v_in, v);
  or_hit* h;
  int nh = collect_hits(f, o, v, tmin, tmax, mask, w64, &h);
  or_pt* pts;
  int np = gather_points(f, h, nh, seed, ray, word, &pts);
  qsort(pts, (size_t)np, sizeof(or_pt), cmp_pt);
  int hit = 0;
  for (int j = 0; j < np; ++j) {
    double kap, kb;
    eval_point(f, h, nh, o, v, pts[j].t, &kap, &kb);
    double kp = kap > 0 ? kap : 0;
    if (pts[j].ua * kb < kp) {
      *t_hit = pts[j].t;
      hit = 1;
      break;
    }
  }
  free(h);
  free(pts);
  return hit;
}

static double det_tau(const or_field* f, const double o[3], const double v[3], double tmin,
                      double tmax, uint64_t mask, const double* w64) {
  double acc = 0;
  for (int64_t i = 0; i < f->n; ++i) {
    const or_prim* P = &f->p[i];
    if (!(mask >> P->cell & 1ull)) continue;
    double w = w64 ? w64[P->cell] : 1.0;
    if (!(w > 0)) continue;
    or_chord_t c = chord_of(P, o, v, P->k, tmin, tmax);
    if (!c.has) continue;
    acc += w * chord_integral(P, &c, o, v, P->k);
  }
  return acc;
}

int or_cdf_flight(const or_field* f, const double o[3], const double v_in[3], double tmin,
                  double tmax, uint64_t mask, const double* w64, uint64_t seed, uint32_t ray,
                  uint32_t word, double* t_hit) {
  gl_init();
  double v[3];
  normalise(v_in, v);
  uint32_t x[4];
  rng4(seed, 0, OR_NO_PRIM, ray, word, x);
  const double target = -log(1.0 - u01(x[0]));
  /* the optical depth stops growing at the last chord exit */
  double tend = tmin;
  for (int64_t i = 0; i < f->n; ++i) {
    const or_prim* P = &f->p[i];
    if (!(mask >> P->cell & 1ull)) continue;
    if (w64 && !(w64[P->cell] > 0)) continue;
    or_chord_t c = chord_of(P, o, v, P->k, tmin, tmax);
    if (c.has && c.hi > tend) tend = c.hi;
  }
  if (!(tend > tmin) || det_tau(f, o, v, tmin, tend, mask, w64) < target) return 0;
  double lo = tmin, hi = tend;
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (det_tau(f, o, v, tmin, mid, mask, w64) < target) lo = mid;
    else hi = mid;
  }
  *t_hit = 0.5 * (lo + hi);
  return 1;
}

/* Free flight by uniform sampling within the crossing segment (Sec. 3,
   segment-based transfer: uniform sampling within segments as the cheap
   approximation of the CDF inversion; Sec. 4.4 distance sampling).  The ray is
   cut into segments at tmin and at every chord entry and exit; with xi the
   first uniform of the segment's tracking stream and target -ln(1 - xi), the
   crossing segment [e_{k-1}, e_k] is the first whose end reaches
   tau(tmin, e_k) >= target, and the collision is e_{k-1} + u (e_k - e_{k-1})
   with u the stream's second uniform.  Returns 0 when the ray's whole optical
   depth stays below the target. */
static int cmp_dbl(const void* A, const void* B) {
  double a = *(const double*)A, b = *(const double*)B;
  return (a > b) - (a < b);
}

int or_segment_flight(const or_field* f, const double o[3], const double v_in[3], double tmin,
                      double tmax, uint64_t mask, const double* w64, uint64_t seed, uint32_t ray,
                      uint32_t word, double* t_hit) {
  gl_init();
  double v[3];
  normalise(v_in, v);
  uint32_t x[4];
  rng4(seed, 0, OR_NO_PRIM, ray, word, x);
  const double target = -log(1.0 - u01(x[0]));
  or_hit* h;
  int nh = collect_hits(f, o, v, tmin, tmax, mask, w64, &h);
  double* ev = (double*)malloc(sizeof(double) * (size_t)(2 * nh + 1));
  int ne = 0;
  ev[ne++] = tmin;
  for (int j = 0; j < nh; ++j) {
    ev[ne++] = h[j].c.lo;
    ev[ne++] = h[j].c.hi;
  }
  free(h);
  qsort(ev, (size_t)ne, sizeof(double), cmp_dbl);
  int hit = 0;
  for (int k = 1; k < ne && !hit; ++k) {
    if (!(ev[k] > ev[k - 1])) continue;
    if (det_tau(f, o, v, tmin, ev[k], mask, w64) >= target) {
      *t_hit = ev[k - 1] + u01(x[1]) * (ev[k] - ev[k - 1]);
      hit = 1;
    }
  }
  free(ev);
  return hit;
}

static int nthreads_of(int n) {
#ifdef _OPENMP
  return n > 0 ? n : omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void or_transmittance(const or_field* f, const or_lod* lod, const float* o, const float* d,
                      const float* trange, int64_t n_rays, int mode, int spp, uint64_t seed,
                      double* T, double* tau, int n_threads) {
  gl_init();
  int nt = nthreads_of(n_threads);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int64_t r = 0; r < n_rays; ++r) {
    double oo[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
    double v[3];
    api_direction(d + 3 * r, v);
    double tmin = trange ? trange[2 * r] : 0.0;
    double tmax = trange ? trange[2 * r + 1] : INFINITY;
    double acc = 0;
    for (int s = 0; s < spp; ++s) {
      uint64_t mask;
      double w64[OR_MAX_CELLS];
      or_sample_mask(f, lod, v, seed, (uint32_t)r, (uint32_t)s, 0, OR_TAG_MASK, &mask, w64);
      if (mode == 0)
        acc += det_tau(f, oo, v, tmin, tmax, mask, w64);
      else
        acc += ratio_track(f, oo, v, tmin, tmax, mask, w64, seed, (uint32_t)r,
                           stream_word((uint32_t)s, 0, OR_TAG_TRACK), 0);
    }
    acc /= spp;
    if (mode == 0) {
      if (tau) tau[r] = acc;
      T[r] = exp(-acc);
    } else {
      T[r] = acc;
      if (tau) tau[r] = acc > 0 ? -log(acc) : INFINITY;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* camera and path tracing                                                   */
/* ------------------------------------------------------------------------ */
/* pinhole camera: jitter inside the pixel from the camera stream, draw 0 */
void or_camera_ray(const or_camera* C, uint64_t seed, int px, int py, int s, double o[3],
                   double v[3]) {
  double eye[3] = {C->eye[0], C->eye[1], C->eye[2]};
  double fw[3] = {C->look_at[0] - eye[0], C->look_at[1] - eye[1], C->look_at[2] - eye[2]};
  normalise(fw, fw);
  double up[3] = {C->up[0], C->up[1], C->up[2]};
  double rt[3] = {up[1] * fw[2] - up[2] * fw[1], up[2] * fw[0] - up[0] * fw[2],
                  up[0] * fw[1] - up[1] * fw[0]};
  normalise(rt, rt);
  double uv[3] = {fw[1] * rt[2] - fw[2] * rt[1], fw[2] * rt[0] - fw[0] * rt[2],
                  fw[0] * rt[1] - fw[1] * rt[0]};
  uint32_t x[4];
  uint32_t pix = (uint32_t)py * (uint32_t)C->width + (uint32_t)px;
  rng4(seed, 0, OR_NO_PRIM, pix, stream_word((uint32_t)s, 0, OR_TAG_CAMERA), x);
  double jx = u01(x[0]), jy = u01(x[1]);
  double th = tan(0.5 * (double)C->vfov_deg * OR_PI / 180.0);
  double asp = (double)C->width / (double)C->height;
  double sx = (2.0 * (px + jx) / C->width - 1.0) * th * asp;
  double sy = (1.0 - 2.0 * (py + jy) / C->height) * th;
  double dd[3] = {fw[0] + sx * rt[0] + sy * uv[0], fw[1] + sx * rt[1] + sy * uv[1],
                  fw[2] + sx * rt[2] + sy * uv[2]};
  normalise(dd, v);
  o[0] = eye[0]; o[1] = eye[1]; o[2] = eye[2];
}

/* one path sample.  Tomography: exp(-tau) along the camera ray.  Scattering:
   delta tracking to a collision, weight albedo, next-event estimation to the
   directional light by ratio tracking, isotropic phase 1/(4 pi), then an
   isotropic new direction; the LoD mask is redrawn at every bounce
   (Sec. 4.5, per path segment; Sec. 4.6 pipeline steps 1-6). */
/* traced rays (camera, bounce and NEE segments) since the last reset */
static long long g_rays = 0;
long long or_rays_traced(int reset) {
  long long r;
#pragma omp atomic read
  r = g_rays;
  if (reset) {
#pragma omp atomic write
    g_rays = 0;
  }
  return r;
}
static void count_ray(void) {
#pragma omp atomic
  g_rays += 1;
}

/* Foveation (Supp., Foveated Rendering): the cells a sample's path keeps.  The
   frequency threshold falls linearly with the eccentricity e of the camera ray
   v (its angle to the ray through the gaze point), f = max(0, f0 - slope e),
   perturbed per sample by the third uniform of the camera stream (stochastic
   smoothing); Gabor bands whose largest carrier exceeds f leave, the Gaussian
   band stays. */
static uint64_t fov_cells(const or_field* f, const or_camera* C, const or_render_opts* ro,
                          const double v[3], uint64_t seed, uint32_t pix, uint32_t s) {
  if (!ro->foveation) return ~0ull;
  double eye[3] = {C->eye[0], C->eye[1], C->eye[2]};
  double fw[3] = {C->look_at[0] - eye[0], C->look_at[1] - eye[1], C->look_at[2] - eye[2]};
  normalise(fw, fw);
  double up[3] = {C->up[0], C->up[1], C->up[2]};
  double rt[3] = {up[1] * fw[2] - up[2] * fw[1], up[2] * fw[0] - up[0] * fw[2],
                  up[0] * fw[1] - up[1] * fw[0]};
  normalise(rt, rt);
  double uv[3] = {fw[1] * rt[2] - fw[2] * rt[1], fw[2] * rt[0] - fw[0] * rt[2],
                  fw[0] * rt[1] - fw[1] * rt[0]};
  double th = tan(0.5 * (double)C->vfov_deg * OR_PI / 180.0);
  double asp = (double)C->width / (double)C->height;
  double sx = (2.0 * ro->gaze[0] / C->width - 1.0) * th * asp;
  double sy = (1.0 - 2.0 * ro->gaze[1] / C->height) * th;
  double g[3] = {fw[0] + sx * rt[0] + sy * uv[0], fw[1] + sx * rt[1] + sy * uv[1],
                 fw[2] + sx * rt[2] + sy * uv[2]};
  normalise(g, g);
  double c = v[0] * g[0] + v[1] * g[1] + v[2] * g[2];
  c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
  double thr = ro->fov_f0 - ro->fov_slope * acos(c);
  if (thr < 0) thr = 0;
  if (ro->fov_smooth > 0) {
    uint32_t x[4];
    rng4(seed, 0, OR_NO_PRIM, pix, stream_word(s, 0, OR_TAG_CAMERA), x);
    thr *= 1.0 + ro->fov_smooth * (2.0 * u01(x[2]) - 1.0);
  }
  uint64_t m = 1ull;
  for (int b = 1; b < 8; ++b)
    if (f->band_wmax[b] <= thr) m |= 0xFFull << (1 + OR_N_CONES * (b - 1));
  return m;
}

static double path_sample(const or_field* f, const or_lod* lod, const or_lod* lodn,
                          const or_camera* C, const or_render_opts* ro, uint64_t seed, int px,
                          int py, int s) {
  double o[3], v[3];
  or_camera_ray(C, seed, px, py, s, o, v);
  uint32_t pix = (uint32_t)py * (uint32_t)C->width + (uint32_t)px;
  const uint64_t allow = fov_cells(f, C, ro, v, seed, pix, (uint32_t)s);
  if (ro->integrator == 0) {
    uint64_t mask;
    double w64[OR_MAX_CELLS];
    or_sample_mask(f, lod, v, seed, pix, (uint32_t)s, 0, OR_TAG_MASK, &mask, w64);
    mask &= allow;
    count_ray();
    return exp(-det_tau(f, o, v, 0.0, INFINITY, mask, w64));
  }
  double l[3] = {ro->light_dir[0], ro->light_dir[1], ro->light_dir[2]};
  normalise(l, l);
  double thr = 1.0, L = 0.0;
  for (int b = 0; b < ro->max_bounces; ++b) {
    uint64_t mask;
    double w64[OR_MAX_CELLS];
    or_sample_mask(f, lod, v, seed, pix, (uint32_t)s, (uint32_t)b, OR_TAG_MASK, &mask, w64);
    mask &= allow;
    double th;
    count_ray();
    const uint32_t tw = stream_word((uint32_t)s, (uint32_t)b, OR_TAG_TRACK);
    if (ro->free_flight == 2
            ? !or_segment_flight(f, o, v, 0.0, INFINITY, mask, w64, seed, pix, tw, &th)
        : ro->free_flight ? !or_cdf_flight(f, o, v, 0.0, INFINITY, mask, w64, seed, pix, tw, &th)
                          : !or_delta_track(f, o, v, 0.0, INFINITY, mask, w64, seed, pix, tw, &th))
      break;
    double x[3] = {o[0] + th * v[0], o[1] + th * v[1], o[2] + th * v[2]};
    thr *= ro->albedo;
    uint64_t nmask;
    double nw[OR_MAX_CELLS];
    or_sample_mask(f, lodn, l, seed, pix, (uint32_t)s, (uint32_t)b, OR_TAG_NEE_MASK, &nmask, nw);
    nmask &= allow;
    count_ray();
    double Tl = ro->free_flight
                    ? exp(-det_tau(f, x, l, 0.0, INFINITY, nmask, nw))
                    : ratio_track(f, x, l, 0.0, INFINITY, nmask, nw, seed, pix,
                                  stream_word((uint32_t)s, (uint32_t)b, OR_TAG_NEE), 1);
    L += thr * ro->light_irradiance * Tl / (4.0 * OR_PI);
    uint32_t y[4];
    rng4(seed, 0, OR_NO_PRIM, pix, stream_word((uint32_t)s, (uint32_t)b, OR_TAG_SCATTER), y);
    double z = 1.0 - 2.0 * u01(y[0]);
    double rr = sqrt(fmax(0.0, 1.0 - z * z));
    double ph = 2.0 * OR_PI * u01(y[1]);
    v[0] = rr * cos(ph); v[1] = rr * sin(ph); v[2] = z;
    o[0] = x[0]; o[1] = x[1]; o[2] = x[2];
  }
  return L;
}

void or_render_samples(const or_field* f, const or_lod* lod, const or_lod* lodn,
                       const or_camera* C, const or_render_opts* ro, uint64_t seed, int x0,
                       int y0, int w, int h, double* out, int n_threads) {
  gl_init();
  int nt = nthreads_of(n_threads);
  (void)nt;
  int64_t total = (int64_t)w * h * ro->spp;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t idx = 0; idx < total; ++idx) {
    int s = (int)(idx % ro->spp);
    int64_t pi = idx / ro->spp;
    int px = x0 + (int)(pi % w), py = y0 + (int)(pi / w);
    out[idx] = path_sample(f, lod, lodn, C, ro, seed, px, py, s);
  }
}

void or_render(const or_field* f, const or_lod* lod, const or_lod* lodn, const or_camera* C,
               const or_render_opts* ro, uint64_t seed, int x0, int y0, int w, int h,
               double* out, int n_threads) {
  int64_t total = (int64_t)w * h * ro->spp;
  double* smp = (double*)malloc(sizeof(double) * (size_t)(total > 0 ? total : 1));
  or_render_samples(f, lod, lodn, C, ro, seed, x0, y0, w, h, smp, n_threads);
  for (int64_t p = 0; p < (int64_t)w * h; ++p) {
    double acc = 0;
    for (int s = 0; s < ro->spp; ++s) acc += smp[p * ro->spp + s];
    out[p] = acc / ro->spp;
  }
  free(smp);
}

/* ------------------------------------------------------------------------ */
/* tomography gradient (adjoint of Eq. 2-3 under L2 loss)                    */
/*                                                                            */
/* d tau / d theta = int_chord d g/d theta dt + g(hi) d hi/d theta            */
/*                   - g(lo) d lo/d theta   (Leibniz; an endpoint on the      */
/*                   ellipsoid moves with q(t) = k^2: dt/dtheta =             */
/*                   -(dq/dtheta)/(dq/dt)).                                   */
/* Parameters: mu(3), raw quaternion(4, normalised inside), log scale(3),     */
/* omega(3, in the input frame), phase(1), weight(1).                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  double mu[3], q[4], qn, qh[4], ls[3], s[3], R[3][3], dR[4][3][3];
  double omega_in[3], omega[3], phi, weight, A;
  int frame, wmode;
} or_gprim;

/* derivative of R(qhat) w.r.t. the raw quaternion, through qhat = q/|q| */
static void gprim_init(or_gprim* G, const or_field_desc* D, int64_t i) {
  double qn = 0;
  for (int j = 0; j < 4; ++j) { G->q[j] = D->quat[4 * i + j]; qn += G->q[j] * G->q[j]; }
  G->qn = sqrt(qn);
  for (int j = 0; j < 4; ++j) G->qh[j] = G->q[j] / G->qn;
  quat_to_R(G->qh, G->R);
  double w = G->qh[0], x = G->qh[1], y = G->qh[2], z = G->qh[3];
  /* dR/d(qhat_j) */
  double dRh[4][3][3] = {
      {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}},
      {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}},
      {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}},
      {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}}};
  /* d qhat_j / d q_m = (delta_jm - qhat_j qhat_m) / |q| */
  for (int m = 0; m < 4; ++m)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double acc = 0;
        for (int j = 0; j < 4; ++j)
          acc += dRh[j][a][b] * (((j == m) ? 1.0 : 0.0) - G->qh[j] * G->qh[m]) / G->qn;
        G->dR[m][a][b] = acc;
      }
  for (int j = 0; j < 3; ++j) {
    G->mu[j] = D->mu[3 * i + j];
    G->ls[j] = D->log_scale[3 * i + j];
    G->s[j] = exp(G->ls[j]);
    G->omega_in[j] = D->omega[3 * i + j];
  }
  G->frame = D->omega_frame;
  G->wmode = D->weight_mode;
  if (G->frame == 1) {
    for (int a = 0; a < 3; ++a) {
      double acc = 0;
      for (int j = 0; j < 3; ++j) acc += G->R[a][j] * G->omega_in[j] / G->s[j];
      G->omega[a] = acc;
    }
  } else {
    for (int a = 0; a < 3; ++a) G->omega[a] = G->omega_in[a];
  }
  G->phi = D->phase[i];
  G->weight = D->weight[i];
  G->A = G->wmode == 1 ? G->weight / (pow(2.0 * OR_PI, 1.5) * G->s[0] * G->s[1] * G->s[2])
                       : G->weight;
}

/* at a point y = x - mu: value g, dq/dparam (14 slots, mu..log_scale used),
   dtheta/dparam, and dA/dparam */
typedef struct {
  double g, env, c, sn, q;
  double dq[15], dth[15], dA[15];
} or_gpoint;

static void gpoint(const or_gprim* G, const double y[3], or_gpoint* P) {
  memset(P, 0, sizeof(*P));
  double z[3];
  for (int j = 0; j < 3; ++j) z[j] = G->R[0][j] * y[0] + G->R[1][j] * y[1] + G->R[2][j] * y[2];
  double q = 0;
  for (int j = 0; j < 3; ++j) q += z[j] * z[j] / (G->s[j] * G->s[j]);
  double th = G->omega[0] * y[0] + G->omega[1] * y[1] + G->omega[2] * y[2] + G->phi;
  P->q = q;
  P->env = exp(-0.5 * q);
  P->c = cos(th);
  P->sn = sin(th);
  P->g = G->A * P->env * P->c;
  /* mu: dq/dmu = -2 Sigma^-1 y ; dtheta/dmu = -omega */
  for (int a = 0; a < 3; ++a) {
    double acc = 0;
    for (int j = 0; j < 3; ++j) acc += G->R[a][j] * z[j] / (G->s[j] * G->s[j]);
    P->dq[a] = -2.0 * acc;
    P->dth[a] = -G->omega[a];
  }
  /* quaternion: q = sum_j (R^T y)_j^2 / s_j^2 */
  for (int m = 0; m < 4; ++m) {
    double dqm = 0, dthm = 0;
    for (int j = 0; j < 3; ++j) {
      double dz = G->dR[m][0][j] * y[0] + G->dR[m][1][j] * y[1] + G->dR[m][2][j] * y[2];
      dqm += 2.0 * z[j] * dz / (G->s[j] * G->s[j]);
      if (G->frame == 1) dthm += G->omega_in[j] / G->s[j] * dz;
    }
    P->dq[3 + m] = dqm;
    P->dth[3 + m] = dthm;
  }
  /* log scale */
  for (int j = 0; j < 3; ++j) {
    P->dq[7 + j] = -2.0 * z[j] * z[j] / (G->s[j] * G->s[j]);
    if (G->frame == 1) P->dth[7 + j] = -G->omega_in[j] * z[j] / G->s[j];
    if (G->wmode == 1) P->dA[7 + j] = -G->A;
  }
  /* omega in the input frame */
  for (int j = 0; j < 3; ++j) P->dth[10 + j] = G->frame == 1 ? z[j] / G->s[j] : y[j];
  P->dth[13] = 1.0;
  P->dA[14] = G->wmode == 1 ? G->A / G->weight : 1.0;
  if (G->wmode == 0) P->dA[14] = 1.0;
}

/* dtau/dparam for one chord; returns tau_i */
static double chord_grad(const or_gprim* G, const or_prim* Pr, const or_chord_t* c,
                         const double o[3], const double v[3], double tmin, double tmax,
                         double k, double* dtau) {
  for (int j = 0; j < 15; ++j) dtau[j] = 0;
  if (!c->has) return 0.0;
  int np = n_panels(Pr, c, v);
  double h = (c->hi - c->lo) / np, tau = 0;
  for (int p = 0; p < np; ++p) {
    double m = c->lo + (p + 0.5) * h;
    for (int j = 0; j < OR_GL_N; ++j) {
      double t = m + 0.5 * h * g_glx[j], wq = 0.5 * h * g_glw[j];
      double y[3] = {o[0] + t * v[0] - G->mu[0], o[1] + t * v[1] - G->mu[1],
                     o[2] + t * v[2] - G->mu[2]};
      or_gpoint P;
      gpoint(G, y, &P);
      tau += wq * P.g;
      for (int r = 0; r < 15; ++r) {
        double d = G->A * P.env * (-0.5 * P.dq[r] * P.c - P.sn * P.dth[r]) + P.dA[r] * P.env * P.c;
        dtau[r] += wq * d;
      }
    }
  }
  /* Leibniz terms at ends that lie on the ellipsoid (not on tmin/tmax) */
  double ends[2] = {c->lo, c->hi};
  double sgn[2] = {-1.0, 1.0};
  for (int e = 0; e < 2; ++e) {
    double t = ends[e];
    int on_ellipsoid = (e == 0) ? (c->tstar - c->hw > tmin) : (c->tstar + c->hw < tmax);
    if (!on_ellipsoid) continue;
    double y[3] = {o[0] + t * v[0] - G->mu[0], o[1] + t * v[1] - G->mu[1],
                   o[2] + t * v[2] - G->mu[2]};
    or_gpoint P;
    gpoint(G, y, &P);
    /* dq/dt = 2 v^T Sigma^-1 y = -v . dq/dmu */
    double dqdt = -(v[0] * P.dq[0] + v[1] * P.dq[1] + v[2] * P.dq[2]);
    for (int r = 0; r < 10; ++r) dtau[r] += sgn[e] * P.g * (-P.dq[r] / dqdt);
  }
  (void)k;
  return tau;
}

static or_field* field_of(const or_field_desc* D) { return or_field_create(D); }

void or_tomo_image(const or_field_desc* D, const or_camera* C, int spp, uint64_t seed,
                   double* image, int n_threads) {
  gl_init();
  or_field* f = field_of(D);
  or_lod all = {0, 7, 0};
  or_render_opts ro;
  memset(&ro, 0, sizeof(ro));
  ro.integrator = 0;
  ro.spp = spp;
  or_render(f, &all, &all, C, &ro, seed, 0, 0, C->width, C->height, image, n_threads);
  or_field_free(f);
}

double or_tomo_loss_grad(const or_field_desc* D, const or_camera* C, int spp, uint64_t seed,
                         const float* target, double* grad, int n_threads) {
  gl_init();
  or_field* f = field_of(D);
  int64_t N = D->n;
  int W = C->width, H = C->height;
  int nt = nthreads_of(n_threads);
  double* img = (double*)calloc((size_t)W * H, sizeof(double));
  /* forward */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t p = 0; p < (int64_t)W * H; ++p) {
    int px = (int)(p % W), py = (int)(p / W);
    double acc = 0;
    for (int s = 0; s < spp; ++s) {
      double o[3], v[3];
      or_camera_ray(C, seed, px, py, s, o, v);
      acc += exp(-det_tau(f, o, v, 0.0, INFINITY, ~0ull, NULL));
    }
    img[p] = acc / spp;
  }
  double L = 0;
  for (int64_t p = 0; p < (int64_t)W * H; ++p) {
    double r = img[p] - target[p];
    L += r * r;
  }
  /* backward: dL/dtau_{p,s} = -2 (I_p - target_p) exp(-tau_{p,s}) / spp */
  or_gprim* G = (or_gprim*)malloc(sizeof(or_gprim) * (size_t)(N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i) gprim_init(&G[i], D, i);
  double* g15 = (double*)calloc((size_t)N * 15, sizeof(double));
  for (int64_t p = 0; p < (int64_t)W * H; ++p) {
    int px = (int)(p % W), py = (int)(p / W);
    for (int s = 0; s < spp; ++s) {
      double o[3], v[3];
      or_camera_ray(C, seed, px, py, s, o, v);
      double tau = det_tau(f, o, v, 0.0, INFINITY, ~0ull, NULL);
      double dLdtau = -2.0 * (img[p] - target[p]) * exp(-tau) / spp;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
      for (int64_t i = 0; i < N; ++i) {
        or_chord_t c = chord_of(&f->p[i], o, v, f->p[i].k, 0.0, INFINITY);
        if (!c.has) continue;
        double dt[15];
        chord_grad(&G[i], &f->p[i], &c, o, v, 0.0, INFINITY, f->p[i].k, dt);
        for (int r = 0; r < 15; ++r) g15[i * 15 + r] += dLdtau * dt[r];
      }
    }
  }
  /* SoA output: mu[3N], quat[4N], log_scale[3N], omega[3N], phase[N], weight[N] */
  for (int64_t i = 0; i < N; ++i) {
    for (int j = 0; j < 3; ++j) grad[3 * i + j] = g15[i * 15 + j];
    for (int j = 0; j < 4; ++j) grad[3 * N + 4 * i + j] = g15[i * 15 + 3 + j];
    for (int j = 0; j < 3; ++j) grad[7 * N + 3 * i + j] = g15[i * 15 + 7 + j];
    for (int j = 0; j < 3; ++j) grad[10 * N + 3 * i + j] = g15[i * 15 + 10 + j];
    grad[13 * N + i] = g15[i * 15 + 13];
    grad[14 * N + i] = g15[i * 15 + 14];
  }
  free(g15);
  free(G);
  free(img);
  or_field_free(f);
  return L;
}

/* ------------------------------------------------------------------------ */
/* single-scattering radiance adjoint                                        */
/*                                                                            */
/* Free flight by delta tracking has the same mean as the expected-value     */
/* estimator over ALL tentative points t_j of the ray (rate kappa_bar):      */
/*   I = sum_j W_j G(t_j),  W_j = prod_{i<j} (1 - p_i) p_j,                   */
/*   p_j = max(kappa_j, 0) / kappa_bar_j,  G = albedo E/(4 pi) T_light,       */
/* because the points before t form a Poisson process independent of the    */
/* point at t (Campbell's formula gives int T kappa+ G dt).  One point js is */
/* drawn with probability W_j / sum W by weighted reservoir sampling in t    */
/* order (point j replaces the candidate when u_j S_j < W_j, S_j the running */
/* sum of W and u_j the point's own second uniform), and its NEE             */
/* transmittance is ratio tracked, so a sample is sum W * G(t_js).  The      */
/* derivative is taken with                                                 */
/* the tentative points, kappa_bar and the draw probabilities held fixed    */
/* (each keeps the estimator's mean equal to I for nearby parameters), so   */
/* only kappa_j and the NEE kappa_k vary:                                   */
/*   d sample / d p_i  = (sum W / W_js) G dW_js/dp_i,                       */
/*   d sample / d q_k  = sum W  albedo E/(4 pi) (-prod_{m != k} (1 - q_m)),  */
/*   d p / d theta     = 1[kappa > 0] d kappa/d theta / kappa_bar,           */
/* with d kappa/d theta summed over the kernels covering the point.  The    */
/* k-sigma cut contributes no term (the derivative of the truncated field   */
/* is taken where it is smooth).                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
  double t, ua, kap, kb;
} or_rpt;

static int cmp_rpt(const void* A, const void* B) {
  double a = ((const or_rpt*)A)->t, b = ((const or_rpt*)B)->t;
  return (a > b) - (a < b);
}

/* all tentative points of a ray, sorted, with kappa and kappa_bar */
static int ray_points(const or_field* f, const double o[3], const double v[3], uint64_t mask,
                      const double* w64, uint64_t seed, uint32_t ray, uint32_t word,
                      or_hit** hits, int* nhits, or_rpt** out) {
  int nh = collect_hits(f, o, v, 0.0, INFINITY, mask, w64, hits);
  or_pt* pts;
  int np = gather_points(f, *hits, nh, seed, ray, word, &pts);
  or_rpt* r = (or_rpt*)malloc(sizeof(or_rpt) * (size_t)(np > 0 ? np : 1));
  for (int j = 0; j < np; ++j) {
    r[j].t = pts[j].t;
    r[j].ua = pts[j].ua;
    eval_point(f, *hits, nh, o, v, pts[j].t, &r[j].kap, &r[j].kb);
  }
  free(pts);
  qsort(r, (size_t)np, sizeof(or_rpt), cmp_rpt);
  *nhits = nh;
  *out = r;
  return np;
}

/* add coef * d kappa(x(t)) / d theta to the 15 N gradient */
static void add_dkappa(const or_field* f, const or_gprim* G, const or_hit* h, int nh,
                       const double o[3], const double v[3], double t, double coef,
                       double* g15) {
  if (coef == 0.0) return;
  for (int j = 0; j < nh; ++j) {
    if (t < h[j].c.lo || t > h[j].c.hi) continue;
    const or_gprim* Gi = &G[h[j].prim];
    double y[3] = {o[0] + t * v[0] - Gi->mu[0], o[1] + t * v[1] - Gi->mu[1],
                   o[2] + t * v[2] - Gi->mu[2]};
    or_gpoint P;
    gpoint(Gi, y, &P);
    if (P.q > f->p[h[j].prim].k * f->p[h[j].prim].k) continue;
    double cw = coef * h[j].w;
    for (int r = 0; r < 15; ++r) {
      double d = Gi->A * P.env * (-0.5 * P.dq[r] * P.c - P.sn * P.dth[r]) + P.dA[r] * P.env * P.c;
      g15[h[j].prim * 15 + r] += cw * d;
    }
  }
}

static double path_grad_sample(const or_field* f, const or_gprim* G, const or_lod* lod,
                               const or_lod* lodn, const or_render_opts* ro, const double o0[3],
                               const double v0[3], uint64_t seed, uint32_t ray, uint32_t s,
                               double dLdI, double* g15);

/* one sample of the estimator along o + t v; adds dLdI * d sample/d theta
   to g15 and returns the sample (max_bounces >= 2: path_grad_sample) */
static double radiance_grad_sample(const or_field* f, const or_gprim* G, const or_lod* lod,
                                   const or_lod* lodn, const or_render_opts* ro,
                                   const double o[3], const double v[3], uint64_t seed,
                                   uint32_t ray, uint32_t s, double dLdI, double* g15) {
  if (ro->max_bounces >= 2)
    return path_grad_sample(f, G, lod, lodn, ro, o, v, seed, ray, s, dLdI, g15);
  double l[3] = {ro->light_dir[0], ro->light_dir[1], ro->light_dir[2]};
  normalise(l, l);
  uint64_t mask;
  double w64[OR_MAX_CELLS];
  or_sample_mask(f, lod, v, seed, ray, s, 0, OR_TAG_MASK, &mask, w64);
  or_hit* h;
  int nh;
  or_rpt* pt;
  int np = ray_points(f, o, v, mask, w64, seed, ray, stream_word(s, 0, OR_TAG_TRACK), &h, &nh, &pt);
  double* p = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
  double* W = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
  double P = 1.0, SW = 0.0;
  for (int j = 0; j < np; ++j) {
    double kp = pt[j].kap > 0 ? pt[j].kap : 0.0;
    p[j] = pt[j].kb > 0 ? kp / pt[j].kb : 0.0;
    W[j] = P * p[j];
    SW += W[j];
    P *= 1.0 - p[j];
  }
  double value = 0.0;
  int js = -1;
  {
    double S = 0.0;
    for (int j = 0; j < np; ++j) {
      S += W[j];
      if (W[j] > 0.0 && pt[j].ua * S < W[j]) js = j;
    }
  }
  if (SW > 0.0 && js >= 0) {
    double x[3] = {o[0] + pt[js].t * v[0], o[1] + pt[js].t * v[1], o[2] + pt[js].t * v[2]};
    /* NEE by ratio tracking from x_js */
    uint64_t nmask;
    double nw[OR_MAX_CELLS];
    or_sample_mask(f, lodn, l, seed, ray, s, 0, OR_TAG_NEE_MASK, &nmask, nw);
    or_hit* hl;
    int nhl;
    or_rpt* ql;
    int nq = ray_points(f, x, l, nmask, nw, seed, ray, stream_word(s, 0, OR_TAG_NEE), &hl, &nhl, &ql);
    double* q = (double*)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1));
    double Tl = 1.0;
    for (int k = 0; k < nq; ++k) {
      double kp = ql[k].kap > 0 ? ql[k].kap : 0.0;
      q[k] = ql[k].kb > 0 ? kp / ql[k].kb : 0.0;
      Tl *= 1.0 - q[k];
    }
    const double E = ro->albedo * ro->light_irradiance / (4.0 * OR_PI);
    double Gv = E * Tl;
    value = SW * Gv;
    if (dLdI != 0.0) {
      /* camera points i <= js: d sample/d p_i = (SW / W_js) G dW_js/dp_i */
      for (int i = 0; i <= js; ++i) {
        if (!(pt[i].kap > 0) || !(pt[i].kb > 0)) continue;
        double dW;
        if (i == js) {
          dW = 1.0;
          for (int m = 0; m < js; ++m) dW *= 1.0 - p[m];
        } else {
          dW = -p[js];
          for (int m = 0; m < js; ++m)
            if (m != i) dW *= 1.0 - p[m];
        }
        double coef = dLdI * SW / W[js] * Gv * dW / pt[i].kb;
        add_dkappa(f, G, h, nh, o, v, pt[i].t, coef, g15);
      }
      /* NEE points: d sample/d q_k = -SW E prod_{m != k} (1 - q_m) */
      for (int k = 0; k < nq; ++k) {
        if (!(ql[k].kap > 0) || !(ql[k].kb > 0)) continue;
        double pr = 1.0;
        for (int m = 0; m < nq; ++m)
          if (m != k) pr *= 1.0 - q[m];
        double coef = -dLdI * SW * E * pr / ql[k].kb;
        add_dkappa(f, G, hl, nhl, x, l, ql[k].t, coef, g15);
      }
    }
    free(q);
    free(ql);
    free(hl);
  }
  free(p);
  free(W);
  free(pt);
  free(h);
  return value;
}

/* ------------------------------------------------------------------------ */
/* multiple-scattering radiance adjoint (max_bounces >= 2)                   */
/*                                                                            */
/* A path of delta tracking (Sec. 3) chooses, on segment b, the collision at */
/* its first accepted tentative point js_b (probability                      */
/* P_b = prod_{i<js} (1 - p_i) p_js, p = max(kappa,0)/kappa_bar), or escapes */
/* (prod over all points of 1 - p_i).  At the collision x_{b+1}: throughput  */
/* thr_b = albedo^(b+1), NEE by ratio tracking T_b = prod_k (1 - q_k), so    */
/* the sample is L = sum_b C_b, C_b = thr_b E/(4 pi) T_b.  C_b depends on the */
/* segments 0..b and on NEE b.  With the tentative points and kappa_bar held */
/* fixed (as for single scattering), the derivative of the expected sample  */
/* is the expectation of                                                    */
/*   sum_b S_b d log P_b + sum_b C_b d log T_b,   S_b = sum_{b' >= b} C_b',   */
/*   d log P_b = sum_{i<js} -dp_i/(1 - p_i) + dp_js/p_js,                    */
/*   d T_b     = -sum_k dq_k prod_{m != k} (1 - q_m),                        */
/* dp = 1[kappa > 0] d kappa / kappa_bar; an escaping segment has S = 0.     */
/* The path, its masks, points and decisions are those of path_sample.       */
/* ------------------------------------------------------------------------ */
#define OR_MAX_SEG 16
static double path_grad_sample(const or_field* f, const or_gprim* G, const or_lod* lod,
                               const or_lod* lodn, const or_render_opts* ro, const double o0[3],
                               const double v0[3], uint64_t seed, uint32_t ray, uint32_t s,
                               double dLdI, double* g15) {
  double l[3] = {ro->light_dir[0], ro->light_dir[1], ro->light_dir[2]};
  normalise(l, l);
  const double E0 = ro->light_irradiance / (4.0 * OR_PI);
  double o[3] = {o0[0], o0[1], o0[2]}, v[3] = {v0[0], v0[1], v0[2]};
  /* per collision segment: its ray, accepted point, NEE origin and C_b, thr_b */
  double so[OR_MAX_SEG][3], sv[OR_MAX_SEG][3], sx[OR_MAX_SEG][3], C[OR_MAX_SEG], thrs[OR_MAX_SEG];
  int js[OR_MAX_SEG];
  int nseg = 0;
  double thr = 1.0, L = 0.0;
  for (int b = 0; b < ro->max_bounces && b < OR_MAX_SEG; ++b) {
    uint64_t mask;
    double w64[OR_MAX_CELLS];
    or_sample_mask(f, lod, v, seed, ray, s, (uint32_t)b, OR_TAG_MASK, &mask, w64);
    or_hit* h;
    int nh;
    or_rpt* pt;
    int np = ray_points(f, o, v, mask, w64, seed, ray, stream_word(s, (uint32_t)b, OR_TAG_TRACK),
                        &h, &nh, &pt);
    int acc = -1;
    for (int j = 0; j < np && acc < 0; ++j) {
      double kp = pt[j].kap > 0 ? pt[j].kap : 0.0;
      if (pt[j].ua * pt[j].kb < kp) acc = j;
    }
    double th = acc >= 0 ? pt[acc].t : 0.0;
    free(pt);
    free(h);
    if (acc < 0) break; /* escapes: no contribution depends on this segment */
    double x[3] = {o[0] + th * v[0], o[1] + th * v[1], o[2] + th * v[2]};
    thr *= ro->albedo;
    uint64_t nmask;
    double nw[OR_MAX_CELLS];
    or_sample_mask(f, lodn, l, seed, ray, s, (uint32_t)b, OR_TAG_NEE_MASK, &nmask, nw);
    double Tl = ratio_track(f, x, l, 0.0, INFINITY, nmask, nw, seed, ray,
                            stream_word(s, (uint32_t)b, OR_TAG_NEE), 1);
    for (int k = 0; k < 3; ++k) {
      so[nseg][k] = o[k];
      sv[nseg][k] = v[k];
      sx[nseg][k] = x[k];
    }
    js[nseg] = acc;
    thrs[nseg] = thr;
    C[nseg] = thr * E0 * Tl;
    L += C[nseg];
    ++nseg;
    uint32_t y[4];
    rng4(seed, 0, OR_NO_PRIM, ray, stream_word(s, (uint32_t)b, OR_TAG_SCATTER), y);
    double z = 1.0 - 2.0 * u01(y[0]);
    double rr = sqrt(fmax(0.0, 1.0 - z * z));
    double ph = 2.0 * OR_PI * u01(y[1]);
    v[0] = rr * cos(ph); v[1] = rr * sin(ph); v[2] = z;
    for (int k = 0; k < 3; ++k) o[k] = x[k];
  }
  if (dLdI == 0.0 || nseg == 0) return L;
  double S = 0.0;
  for (int b = nseg - 1; b >= 0; --b) {
    S += C[b];
    /* segment b: the tracking points up to the accepted one */
    uint64_t mask;
    double w64[OR_MAX_CELLS];
    or_sample_mask(f, lod, sv[b], seed, ray, s, (uint32_t)b, OR_TAG_MASK, &mask, w64);
    or_hit* h;
    int nh;
    or_rpt* pt;
    ray_points(f, so[b], sv[b], mask, w64, seed, ray, stream_word(s, (uint32_t)b, OR_TAG_TRACK), &h,
               &nh, &pt);
    for (int i = 0; i <= js[b]; ++i) {
      if (!(pt[i].kap > 0) || !(pt[i].kb > 0)) continue;
      const double p = pt[i].kap / pt[i].kb;
      const double coef = i == js[b] ? S / p : -S / (1.0 - p);
      add_dkappa(f, G, h, nh, so[b], sv[b], pt[i].t, dLdI * coef / pt[i].kb, g15);
    }
    free(pt);
    free(h);
    /* NEE b: d C_b = -thr_b E0 sum_k dq_k prod_{m != k} (1 - q_m) */
    uint64_t nmask;
    double nw[OR_MAX_CELLS];
    or_sample_mask(f, lodn, l, seed, ray, s, (uint32_t)b, OR_TAG_NEE_MASK, &nmask, nw);
    or_hit* hl;
    int nhl;
    or_rpt* ql;
    int nq = ray_points(f, sx[b], l, nmask, nw, seed, ray, stream_word(s, (uint32_t)b, OR_TAG_NEE),
                        &hl, &nhl, &ql);
    for (int k = 0; k < nq; ++k) {
      if (!(ql[k].kap > 0) || !(ql[k].kb > 0)) continue;
      double pr = 1.0;
      for (int m = 0; m < nq; ++m) {
        if (m == k) continue;
        double kp = ql[m].kap > 0 ? ql[m].kap : 0.0;
        if (ql[m].kb > 0) pr *= 1.0 - kp / ql[m].kb;
      }
      add_dkappa(f, G, hl, nhl, sx[b], l, ql[k].t, -dLdI * thrs[b] * E0 * pr / ql[k].kb, g15);
    }
    free(ql);
    free(hl);
  }
  return L;
}

static void soa_grad(const double* g15, int64_t N, double* grad) {
  for (int64_t i = 0; i < N; ++i) {
    for (int j = 0; j < 3; ++j) grad[3 * i + j] = g15[i * 15 + j];
    for (int j = 0; j < 4; ++j) grad[3 * N + 4 * i + j] = g15[i * 15 + 3 + j];
    for (int j = 0; j < 3; ++j) grad[7 * N + 3 * i + j] = g15[i * 15 + 7 + j];
    for (int j = 0; j < 3; ++j) grad[10 * N + 3 * i + j] = g15[i * 15 + 10 + j];
    grad[13 * N + i] = g15[i * 15 + 13];
    grad[14 * N + i] = g15[i * 15 + 14];
  }
}

void or_radiance_grad_rays(const or_field_desc* D, const or_lod* lod, const or_lod* lodn,
                           const or_render_opts* ro, const double* o, const double* v_in,
                           int64_t n_rays, int spp, uint64_t seed, const double* dLdI,
                           double* value, double* grad, int n_threads) {
  gl_init();
  or_field* f = field_of(D);
  int64_t N = D->n;
  or_gprim* G = (or_gprim*)malloc(sizeof(or_gprim) * (size_t)(N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i) gprim_init(&G[i], D, i);
  int nt = nthreads_of(n_threads);
  (void)nt;
  double* g15 = (double*)calloc((size_t)N * 15, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    double* loc = (double*)calloc((size_t)N * 15, sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_rays; ++r) {
      double v[3];
      normalise(v_in + 3 * r, v);
      double acc = 0;
      for (int s = 0; s < spp; ++s)
        acc += radiance_grad_sample(f, G, lod, lodn, ro, o + 3 * r, v, seed, (uint32_t)r,
                                    (uint32_t)s, dLdI ? dLdI[r] / spp : 0.0, loc);
      if (value) value[r] = acc / spp;
    }
#pragma omp critical
    for (int64_t k = 0; k < N * 15; ++k) g15[k] += loc[k];
    free(loc);
  }
  if (grad) soa_grad(g15, N, grad);
  free(g15);
  free(G);
  or_field_free(f);
}

void or_radiance_grad_image(const or_field_desc* D, const or_lod* lod, const or_lod* lodn,
                            const or_camera* C, const or_render_opts* ro, uint64_t seed,
                            const double* dLdI, double* image, double* grad, int n_threads) {
  gl_init();
  or_field* f = field_of(D);
  int64_t N = D->n;
  or_gprim* G = (or_gprim*)malloc(sizeof(or_gprim) * (size_t)(N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i) gprim_init(&G[i], D, i);
  int nt = nthreads_of(n_threads);
  (void)nt;
  int64_t npix = (int64_t)C->width * C->height;
  double* g15 = (double*)calloc((size_t)N * 15, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    double* loc = (double*)calloc((size_t)N * 15, sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int64_t pix = 0; pix < npix; ++pix) {
      int px = (int)(pix % C->width), py = (int)(pix / C->width);
      double acc = 0;
      for (int s = 0; s < ro->spp; ++s) {
        double o[3], v[3];
        or_camera_ray(C, seed, px, py, s, o, v);
        acc += radiance_grad_sample(f, G, lod, lodn, ro, o, v, seed, (uint32_t)pix, (uint32_t)s,
                                    dLdI ? dLdI[pix] / ro->spp : 0.0, loc);
      }
      if (image) image[pix] = acc / ro->spp;
    }
#pragma omp critical
    for (int64_t k = 0; k < N * 15; ++k) g15[k] += loc[k];
    free(loc);
  }
  if (grad) soa_grad(g15, N, grad);
  free(g15);
  free(G);
  or_field_free(f);
}
