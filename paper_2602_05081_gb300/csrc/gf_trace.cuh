// gf_trace.cuh -- per-ray work shared by the render, transmittance and server
// kernels: LoD mask sampling, deterministic optical depth (Gauss-Legendre and
// closed-form chord integrals), tentative points, ratio and delta tracking,
// CDF-inversion free flight, path samples.  One thread owns one ray (or one
// pixel's paths); a warp advances 32 rays, or 32/G rays with G lanes each.
#pragma once
#include "../../include/gf.h"
#include "gf_device.cuh"

namespace gf {

// Gauss-Legendre rules: n in {8,12,16,20,24,32,48,64}, flattened
constexpr int kNumRules = 8;
constexpr int kGLTotal = 8 + 12 + 16 + 20 + 24 + 32 + 48 + 64;
__host__ __device__ constexpr int gl_n(int r) {
  return r == 0 ? 8 : r == 1 ? 12 : r == 2 ? 16 : r == 3 ? 20 : r == 4 ? 24 : r == 5 ? 32 : r == 6 ? 48 : 64;
}
__host__ __device__ constexpr int gl_off(int r) {
  return r == 0 ? 0 : gl_off(r - 1) + gl_n(r - 1);
}
// node count from the chord's whitened length plus half its carrier phase span
// (radians): the smallest rule whose error stays below 1e-8 of the envelope
// integral for Gaussian x cosine integrands of that size
__device__ __forceinline__ int gl_rule(float m) {
  return m < 2.f ? 0 : m < 6.f ? 1 : m < 10.f ? 2 : m < 18.f ? 3 : m < 24.f ? 4 : m < 40.f ? 5 : m < 56.f ? 6 : 7;
}

// tentative points held per thread per window
constexpr int kPts = 8;

// Work counters, per thread; flush sums them over the warp.
constexpr int kNumStats = 16;
enum : int {
  ST_RAYS = 0, ST_CHORDS, ST_EVALS, ST_NODES, ST_POINTS, ST_WINDOWS, ST_STEPS, ST_LEAVES,
  ST_CYC_TRAV, ST_CYC_GEN, ST_CYC_EVAL, ST_CYC_MASK, ST_CYC_TOTAL
};
struct Counters {
  unsigned long long rays = 0, chords = 0, evals = 0, nodes = 0, points = 0, windows = 0,
                     steps = 0, leaves = 0;
  unsigned long long cyc[5] = {0, 0, 0, 0, 0};  // pass 1, pass 2, (unused), mask, whole path
};

#ifdef GF_PHASE_TIMERS
#define GF_TIC(v) long long v = clock64()
#define GF_TOC(cnt, k, v) (cnt).cyc[k] += (unsigned long long)(clock64() - (v))
#else
#define GF_TIC(v)
#define GF_TOC(cnt, k, v)
#endif

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}
// counters -> global stats; called by all 32 lanes of the warp
__device__ __forceinline__ void flush_counters(const DevField& F, Counters& c, uint32_t lane) {
  unsigned long long v[8] = {c.rays, c.chords, c.evals, c.nodes, c.points, c.windows, c.steps,
                             c.leaves};
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = warp_sum_u64(v[k]);
#ifdef GF_PHASE_TIMERS
  unsigned long long y[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) y[k] = warp_sum_u64(c.cyc[k]);
#endif
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) atomicAdd(F.stats + k, v[k]);
#ifdef GF_PHASE_TIMERS
#pragma unroll
    for (int k = 0; k < 5; ++k) atomicAdd(F.stats + ST_CYC_TRAV + k, y[k]);
#endif
  }
  c = Counters();
}

// ---------------------------------------------------------------------------
// LoD mask (Sec. 4.5.1, 4.5.2, 4.6; App. B strategy tables).  Within a band
// either every occupied cone is selected with one weight or exactly one cone
// is, so a mask is its cell bits plus one weight per band.
// ---------------------------------------------------------------------------
// A drawn mask: cell bits, the weight of each band, and per band one cone
// whose weight is the band's times a factor (threshold + uniform draws one
// bin above the threshold with weight N_above): byte b of cx is
// cone | factor << 3, 0 for none.
struct Mask {
  unsigned long long bits;
  float bw[8];
  uint32_t cx[2] = {0u, 0u};  // no cone with an extra factor unless a draw sets one
};

__device__ __forceinline__ float cone_factor(const uint32_t cx[2], uint32_t cell, int b) {
  const uint32_t e = (cx[b >> 2] >> (8 * (b & 3))) & 0xFFu;
  return (e != 0u && ((cell - 1u) & 7u) == (e & 7u)) ? (float)(e >> 3) : 1.f;
}

__device__ __forceinline__ float mask_weight(const Mask& m, uint32_t cell) {
  if (!(m.bits >> cell & 1ull)) return 0.f;
  const int b = cell == 0 ? 0 : (int)((cell - 1u) >> 3) + 1;
  float w = m.bw[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) w = (b == k) ? m.bw[k] : w;
  return b == 0 ? w : w * cone_factor(m.cx, cell, b);
}

__device__ __forceinline__ unsigned band_cells8(unsigned long long occ, int b) {
  return b == 0 ? (unsigned)(occ & 1ull) : (unsigned)((occ >> (1 + kCones * (b - 1))) & 0xFFull);
}
// position of the (j+1)-th set bit of m (m has more than j set bits)
__device__ __forceinline__ int nth_bit(unsigned m, int j) { return (int)__fns(m, 0, j + 1); }

__host__ __device__ __forceinline__ bool lod_is_deterministic(const LodDev& L) {
  return (L.freq_policy == 0 || L.freq_policy == 1) && (L.cone_policy == 0 || L.cone_policy == 3);
}

// power-law level out of n (App. B): level j when (j/n)^(1-beta) <= x < ((j+1)/n)^(1-beta)
__device__ __forceinline__ int power_level(float x, int n, float beta) {
  const float e = 1.0f - beta;
  int j = 0;
  for (int k = 1; k < n; ++k) j += x >= powf((float)k / (float)n, e) ? 1 : 0;
  return j;
}
__device__ __forceinline__ float power_prob(int j, int n, float beta) {
  const float e = 1.0f - beta;
  return powf((float)(j + 1) / (float)n, e) - powf((float)j / (float)n, e);
}

// EXT = false compiles the ALL / CUTOFF / UNIF_CV / UNIFORM bands and ALL / IS /
// UNIFORM cones only; EXT = true adds the power-law and threshold strategies
template <bool EXT>
__device__ __forceinline__ Mask sample_mask_impl(const DevField& F, const LodDev& L, float3 v,
                                                 uint64_t seed, uint32_t ray, uint32_t sample,
                                                 uint32_t bounce, uint32_t tag) {
  Mask M;
  M.bits = 0;
  M.cx[0] = 0u;
  M.cx[1] = 0u;
  const int maxb = L.freq_policy == 0 ? 7 : L.max_band;
  unsigned occ = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b)
    if (b <= maxb && band_cells8(F.occupied, b)) occ |= 1u << b;
  float bw[8];
  unsigned sel = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) bw[b] = 0.f;
  const uint32_t word = stream_word(sample, bounce, tag);
  if (L.freq_policy == 0 || L.freq_policy == 1) {
    sel = occ;
#pragma unroll
    for (int b = 0; b < 8; ++b) bw[b] = 1.f;
  } else {
    const uint32_t x24 = rng4(seed, 0, kNoPrim, ray, word).x >> 8;
    int pickb = -1;
    float wb = 0.f;
    if (L.freq_policy == 2) {
      // Gaussians always (weight 1) + one Gabor band uniformly (weight P-1)
      if (occ & 1u) {
        sel |= 1u;
        bw[0] = 1.f;
      }
      const unsigned gab = occ & ~1u;
      const int G = __popc(gab);
      if (G > 0) {
        pickb = nth_bit(gab, (int)(((unsigned long long)x24 * (unsigned)G) >> 24));
        wb = (float)G;
      }
    } else if (L.freq_policy == 3) {
      // one band out of P uniformly (weight P)
      const int Q = __popc(occ);
      if (Q > 0) {
        pickb = nth_bit(occ, (int)(((unsigned long long)x24 * (unsigned)Q) >> 24));
        wb = (float)Q;
      }
    } else if (EXT && L.freq_policy == 4) {
      // power law over the P levels, weight 1/P(level)
      const int Q = __popc(occ);
      if (Q > 0) {
        const int j = power_level(u01(x24 << 8), Q, L.beta);
        pickb = nth_bit(occ, j);
        wb = 1.0f / power_prob(j, Q, L.beta);
      }
    } else if (EXT) {
      // Gaussians always (weight 1); power law over the G Gabor levels: one (5),
      // or every level up to the drawn one, level j with weight 1/(1 - (j/G)^(1-beta)) (6)
      if (occ & 1u) {
        sel |= 1u;
        bw[0] = 1.f;
      }
      const unsigned gab = occ & ~1u;
      const int G = __popc(gab);
      if (G > 0) {
        const int k = power_level(u01(x24 << 8), G, L.beta);
        if (L.freq_policy == 5) {
          pickb = nth_bit(gab, k);
          wb = 1.0f / power_prob(k, G, L.beta);
        } else {
          for (int j = 0; j <= k; ++j) {
            const int b = nth_bit(gab, j);
            sel |= 1u << b;
            const float wj = 1.0f / (1.0f - powf((float)j / (float)G, 1.0f - L.beta));
#pragma unroll
            for (int q = 0; q < 8; ++q) bw[q] = (q == b) ? wj : bw[q];
          }
        }
      }
    }
    if (pickb >= 0) {
      sel |= 1u << pickb;
#pragma unroll
      for (int b = 0; b < 8; ++b) bw[b] = (b == pickb) ? wb : bw[b];
    }
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    M.bw[b] = bw[b];
    if (!(sel >> b & 1u)) continue;
    const unsigned cells = band_cells8(F.occupied, b);
    if (b == 0) {
      M.bits |= (unsigned long long)cells;
      continue;
    }
    if (L.cone_policy == 0) {
      M.bits |= (unsigned long long)cells << (1 + kCones * (b - 1));
      continue;
    }
    const uint32_t y = rng4(seed, (uint32_t)(1 + b), kNoPrim, ray, word).x;
    const int nc = __popc(cells);
    int k;
    float cf;
    if (EXT && (L.cone_policy == 3 || L.cone_policy == 4)) {
      // alignment a = |v . o| against delta (FP32): threshold culling keeps the
      // bins with a <= delta, weight 1 (none: the least aligned bin);
      // threshold + uniform keeps them and draws one of the N_above others,
      // weight N_above
      unsigned below = 0u, above = 0u;
      int best = 0;
      float abest = 2.f;
#pragma unroll
      for (int c = 0; c < kCones; ++c) {
        if (!(cells >> c & 1u)) continue;
        // no contraction: the same float operations as the oracle's decision
        const float a = fabsf(__fadd_rn(__fadd_rn(__fmul_rn(v.x, F.axes[c][0]), __fmul_rn(v.y, F.axes[c][1])),
                                        __fmul_rn(v.z, F.axes[c][2])));
        if (a < abest) {
          abest = a;
          best = c;
        }
        if (a <= L.delta) below |= 1u << c;
        else above |= 1u << c;
      }
      if (L.cone_policy == 3) {
        if (below == 0u) below = 1u << best;
      } else if (above != 0u) {
        const int na = __popc(above);
        const int c = nth_bit(above, (int)(((unsigned long long)(y >> 8) * (unsigned)na) >> 24));
        below |= 1u << c;
        M.cx[b >> 2] |= ((uint32_t)c | ((uint32_t)na << 3)) << (8 * (b & 3));
      }
      M.bw[b] = bw[b];
      M.bits |= (unsigned long long)below << (1 + kCones * (b - 1));
      continue;
    }
    if (L.cone_policy == 2) {
      // one cone uniformly, weight K
      k = nth_bit(cells, (int)(((unsigned long long)(y >> 8) * (unsigned)nc) >> 24));
      cf = (float)nc;
    } else {
      // importance sampling: p = w(a)/W with w(a) = exp(-kbar^2 a^2 / 2), weight W/w(a)
      float wc[kCones], W = 0.f;
#pragma unroll
      for (int c = 0; c < kCones; ++c) {
        wc[c] = 0.f;
        if (cells >> c & 1u) {
          const float a = fabsf(v.x * F.axes[c][0] + v.y * F.axes[c][1] + v.z * F.axes[c][2]);
          const float kb = F.kbar[1 + kCones * (b - 1) + c];
          wc[c] = expf(-0.5f * kb * kb * a * a);
          W += wc[c];
        }
      }
      const float target = u01(y) * W;
      float acc = 0.f, wk = 0.f;
      k = -1;
      int last = 0;
      float wlast = 0.f;
#pragma unroll
      for (int c = 0; c < kCones; ++c) {
        if (cells >> c & 1u) {
          last = c;
          wlast = wc[c];
          acc += wc[c];
          if (k < 0 && target < acc) {
            k = c;
            wk = wc[c];
          }
        }
      }
      if (k < 0) {
        k = last;
        wk = wlast;
      }
      cf = W / wk;
    }
    M.bw[b] = bw[b] * cf;
    M.bits |= 1ull << (1 + kCones * (b - 1) + k);
  }
  M.bits &= F.cells_on;  // cells the camera selection emptied are not traversed
  return M;
}

// The strategies that draw (or test alignments) run in a call of their own:
// inlined at every mask site of the scattering renderer they made its loop
// too large for the instruction cache (at 8 bounces with Uniform + CV bands
// and importance-sampled cones, 932 -> 777 ms per 1024x1024 8-spp launch).
// The extended strategies keep a copy without the common ones' registers.
static __device__ __noinline__ Mask sample_mask_call(const DevField& F, const LodDev& L, float3 v,
                                                     uint64_t seed, uint32_t ray, uint32_t sample,
                                                     uint32_t bounce, uint32_t tag) {
  if (L.freq_policy >= 4 || L.cone_policy >= 3)
    return sample_mask_impl<true>(F, L, v, seed, ray, sample, bounce, tag);
  return sample_mask_impl<false>(F, L, v, seed, ray, sample, bounce, tag);
}

// Band cutoffs with every cone (ALL / CUTOFF x ALL) draw nothing: the occupied
// cells of the bands up to the cutoff, weight 1, inline.
__device__ __forceinline__ Mask sample_mask(const DevField& F, const LodDev& L, float3 v,
                                            uint64_t seed, uint32_t ray, uint32_t sample,
                                            uint32_t bounce, uint32_t tag) {
  if ((L.freq_policy == 0 || L.freq_policy == 1) && L.cone_policy == 0) {
    Mask M;
    const int maxb = L.freq_policy == 0 ? 7 : L.max_band;
    const unsigned long long keep = maxb >= 7 ? ~0ull : (1ull << (1 + kCones * maxb)) - 1ull;
    M.bits = F.occupied & keep & F.cells_on;
#pragma unroll
    for (int b = 0; b < 8; ++b) M.bw[b] = 1.f;
    M.cx[0] = 0u;
    M.cx[1] = 0u;
    return M;
  }
  return sample_mask_call(F, L, v, seed, ray, sample, bounce, tag);
}

// ---------------------------------------------------------------------------
// deterministic optical depth along one ray (Eq. 2-3): every chord is
// integrated by Gauss-Legendre as soon as its leaf is reached; FP32 with an
// accurate cosine, Neumaier compensation across chords.
// ---------------------------------------------------------------------------
struct SpanTest {
  float t0, t1;
  __device__ __forceinline__ bool operator()(float tn, float tf) const {
    return fmaxf(tn, t0) <= fminf(tf, t1);
  }
};

__device__ __forceinline__ void gl_pick(int r, int& n, int& off) {
  n = gl_n(7);
  off = gl_off(7);
#pragma unroll
  for (int q = 6; q >= 0; --q)
    if (r <= q) {
      n = gl_n(q);
      off = gl_off(q);
    }
}

struct DetLeaf {
  const DevField* F;
  const Mask* M;
  float3 o, v;
  float tmin, tmax;
  const float* glx;
  const float* glw;
  float s = 0.f, c = 0.f;
  unsigned long long nch = 0, nev = 0;
  // lane `sub` of `group` lanes takes the Gauss-Legendre nodes sub, sub + group, ...
  // (the transmittance kernel splits a ray's tree instead and passes 0 and 1)
  int sub = 0, group = 1;
  __device__ __forceinline__ void operator()(int j) {
    const Mask& Mk = *M;
    Chord ch;
    float w;
    if (!prim_chord(*F, j, o, v, tmin, tmax, [&](uint32_t c) { return mask_weight(Mk, c); }, w, ch))
      return;
    ++nch;
    const float len = ch.dtout - ch.dtin;
    int n, off;
    gl_pick(gl_rule(sqrtf(ch.a) * len + 0.5f * fabsf(ch.B) * len), n, off);
    const float mid = 0.5f * (ch.dtin + ch.dtout), hl = 0.5f * len;
    const float y2 = -0.5f * kLog2e * ch.a, y1 = -kLog2e * ch.b, y0 = -0.5f * kLog2e * ch.g;
    const float scale = w * ch.absA * hl;
    // every node's term goes into the ray's compensated sum (the node sums of
    // a chord can cancel as much as the chords of a ray)
    for (int k = sub; k < n; k += group) {
      const float dt = fmaf(hl, glx[off + k], mid);
      const float y = fmaf(fmaf(y2, dt, y1), dt, y0);
      neumaier_add(s, c, scale * glw[off + k] * ex2f(y) * cosf(fmaf(ch.B, dt, ch.delta)));
    }
    nev += (unsigned long long)((n - sub + group - 1) / group);
  }
};

__device__ __forceinline__ float det_tau(const DevField& F, const Mask& M, float3 o, float3 v,
                                         float tmin, float tmax, const float* glx,
                                         const float* glw, Counters& cnt, int sub = 0,
                                         int group = 1) {
  const float3 inv = safe_inv(v);
  float t0, t1;
  if (M.bits == 0ull || !scene_span(F, o, inv, tmin, tmax, t0, t1)) return 0.f;
  DetLeaf leaf;
  leaf.sub = 0;
  leaf.group = 1;
  leaf.F = &F;
  leaf.M = &M;
  leaf.o = o;
  leaf.v = v;
  leaf.tmin = tmin;
  leaf.tmax = tmax;
  leaf.glx = glx;
  leaf.glw = glw;
  SpanTest test{t0, t1};
  // the lanes of a group walk disjoint subtrees of the same ray
  unsigned long long nodes = 0, leaves = 0;
  traverse_from(F, group_start(F, sub, group), o, inv, M.bits, test, leaf, nodes, leaves);
  cnt.nodes += nodes;
  cnt.leaves += leaves;
  if (sub == 0) cnt.windows += 1;
  cnt.chords += leaf.nch;
  cnt.evals += leaf.nev;
  return __fadd_rn(leaf.s, leaf.c);
}

// ---------------------------------------------------------------------------
// closed-form chord integrals (Sec. 4.4, App. A.3)
//
// The integral of |A| exp(-q/2) cos(theta) over a chord, written with the
// Faddeeva function w so that no term grows with the carrier frequency.  With
// u = dt - dts (envelope peak at dts), s = sqrt(a/2), x = s u, beta = B/(2s)
// and delta' = B dts + delta the carrier phase at the peak:
//   int = |A| e^(-qmin/2) sqrt(pi)/(2s) Re{e^(i delta') [F(x0) - F(x1)]},
//   F(x) = e^(-beta^2) erfc(x - i beta).
// From erfc(y) = e^(-y^2) w(iy), erfc(y) = 2 - erfc(-y) and w(-conj z) = conj w(z):
//   e^(-qmin/2) Re{e^(i delta') F(x)}
//     = e^(-q/2) Re{e^(i theta) w(beta + i|x|)}                         x >= 0
//     = 2 e^(-qmin/2 - beta^2) cos(delta')
//       - e^(-q/2) Re{e^(i theta) conj w(beta + i|x|)}                   x < 0
// where q = qmin + 2 x^2 and theta = B dt + delta belong to the end point, so
// w is only taken in the upper half plane.  A chord shorter than 1e-4 in
// whitened length takes the midpoint rule (Sec. 4.4).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float closed_end(const Weideman& W, float x, float beta, float qmin,
                                            float theta) {
  const float2 w = faddeeva_w(W, beta, fabsf(x));
  float sn, cs;
  sincosf(theta, &sn, &cs);
  const float e = ex2f(-0.5f * kLog2e * fmaf(2.0f * x, x, qmin));
  return x >= 0.0f ? e * fmaf(cs, w.x, -sn * w.y) : -e * fmaf(cs, w.x, sn * w.y);
}

__device__ __forceinline__ float chord_closed(const Weideman& W, const Chord& ch) {
  const float len = ch.dtout - ch.dtin;
  const float ra = sqrtf(ch.a);
  if (ra * len < 1e-4f) {
    const float m = 0.5f * (ch.dtin + ch.dtout);
    const float q = fmaf(fmaf(ch.a, m, 2.0f * ch.b), m, ch.g);
    return ch.absA * len * ex2f(-0.5f * kLog2e * q) * cosf(fmaf(ch.B, m, ch.delta));
  }
  const float s = 0.70710678118654752f * ra;
  const float beta = ch.B / (2.0f * s);
  const float x0 = s * (ch.dtin - ch.dts), x1 = s * (ch.dtout - ch.dts);
  float acc = closed_end(W, x0, beta, ch.qmin, fmaf(ch.B, ch.dtin, ch.delta)) -
              closed_end(W, x1, beta, ch.qmin, fmaf(ch.B, ch.dtout, ch.delta));
  if (x0 < 0.0f && x1 >= 0.0f)  // the chord holds the peak: the full-line term
    acc += 2.0f * ex2f(-kLog2e * fmaf(beta, beta, 0.5f * ch.qmin)) *
           cosf(fmaf(ch.B, ch.dts, ch.delta));
  return ch.absA * (0.88622692545275801f / s) * acc;  // sqrt(pi)/2 / s
}

struct ClosedLeaf {
  const DevField* F;
  const Mask* M;
  float3 o, v;
  float tmin, tmax;
  float s = 0.f, c = 0.f;
  float tend = -INFINITY;  // the last chord exit
  unsigned long long nch = 0;
  __device__ __forceinline__ void operator()(int j) {
    const Mask& Mk = *M;
    Chord ch;
    float w;
    if (!prim_chord(*F, j, o, v, tmin, tmax, [&](uint32_t c) { return mask_weight(Mk, c); }, w, ch))
      return;
    ++nch;
    tend = fmaxf(tend, ch.tc + ch.dtout);
    neumaier_add(s, c, w * chord_closed(F->wd, ch));
  }
};

__device__ __forceinline__ float closed_tau(const DevField& F, const Mask& M, float3 o, float3 v,
                                            float tmin, float tmax, Counters& cnt, int sub = 0,
                                            int group = 1, float* tend = nullptr) {
  const float3 inv = safe_inv(v);
  float t0, t1;
  if (tend) *tend = -INFINITY;
  if (M.bits == 0ull || !scene_span(F, o, inv, tmin, tmax, t0, t1)) return 0.f;
  ClosedLeaf leaf;
  leaf.F = &F;
  leaf.M = &M;
  leaf.o = o;
  leaf.v = v;
  leaf.tmin = tmin;
  leaf.tmax = tmax;
  SpanTest test{t0, t1};
  // the lanes of a group walk disjoint subtrees of the same ray
  unsigned long long nodes = 0, leaves = 0;
  traverse_from(F, group_start(F, sub, group), o, inv, M.bits, test, leaf, nodes, leaves);
  cnt.nodes += nodes;
  cnt.leaves += leaves;
  if (sub == 0) cnt.windows += 1;
  cnt.chords += leaf.nch;
  if (tend) *tend = leaf.tend;
  return __fadd_rn(leaf.s, leaf.c);
}

// Free flight by inversion of the optical-depth CDF (Sec. 3 Eq. 5, segment-based
// transfer; Sec. 4.4 distance sampling): with xi the first uniform of the
// segment's tracking stream, the distance solves tau(0, t) = -ln(1 - xi),
// found by 32 bisections of [0, last chord exit] on the closed-form optical
// depth (one windowed traversal each).  Returns false when the whole ray's
// optical depth does not reach the target.  The first crossing needs a
// non-negative density along the ray.
__device__ __forceinline__ bool cdf_flight(const DevField& F, const Mask& M, float3 o, float3 v,
                                           uint64_t seed, uint32_t ray, uint32_t word, float& th,
                                           Counters& cnt) {
  const uint4 y = rng4(seed, 0, kNoPrim, ray, word);
  const float target = -log1pf(-u01(y.x));
  float tend;
  const float total = closed_tau(F, M, o, v, 0.f, INFINITY, cnt, 0, 1, &tend);
  if (!(tend > 0.f) || total < target) return false;
  float lo = 0.f, hi = tend;
  for (int it = 0; it < 32; ++it) {
    const float mid = 0.5f * (lo + hi);
    if (closed_tau(F, M, o, v, 0.f, mid, cnt) < target) lo = mid;
    else hi = mid;
  }
  th = 0.5f * (lo + hi);
  return true;
}

// Free flight by uniform sampling within the crossing segment (Sec. 3: the
// cheap approximation of the CDF inversion; Sec. 4.4 distance sampling).  The
// ray is cut into segments at t = 0 and at every chord entry and exit; the
// segment [e_a, e_b] in which tau(0, t) reaches the target -ln(1 - xi) holds
// the collision e_a + u (e_b - e_a), xi and u the first two uniforms of the
// segment's tracking stream.  The crossing segment is found by bisection on t
// that stops once no chord end lies inside the bracket: every step is one
// traversal giving tau(0, mid), the chord ends inside both halves of the
// bracket and the nearest ends around them.
struct SegLeaf {
  const DevField* F;
  const Mask* M;
  float3 o, v;
  float lo, mid, hi;  // the bracket and its midpoint
  float s = 0.f, c = 0.f;  // tau(0, mid), compensated
  int n_left = 0, n_right = 0;  // chord ends in (lo, mid) and in (mid, hi)
  float below_lo = 0.f, below_mid = 0.f;             // largest end <= lo, <= mid (or 0)
  float above_mid = INFINITY, above_hi = INFINITY;   // smallest end >= mid, >= hi
  __device__ __forceinline__ void end(float e) {
    n_left += (e > lo && e < mid) ? 1 : 0;
    n_right += (e > mid && e < hi) ? 1 : 0;
    if (e <= lo) below_lo = fmaxf(below_lo, e);
    if (e <= mid) below_mid = fmaxf(below_mid, e);
    if (e >= mid) above_mid = fminf(above_mid, e);
    if (e >= hi) above_hi = fminf(above_hi, e);
  }
  __device__ __forceinline__ void operator()(int j) {
    const Mask& Mk = *M;
    Chord ch;
    float w;
    if (!prim_chord(*F, j, o, v, 0.f, INFINITY, [&](uint32_t cc) { return mask_weight(Mk, cc); }, w,
                    ch))
      return;
    end(ch.tc + ch.dtin);
    end(ch.tc + ch.dtout);
    if (ch.tc + ch.dtin >= mid) return;
    // the chord's part in [0, mid]
    if (ch.tc + ch.dtout > mid) ch.dtout = mid - ch.tc;
    neumaier_add(s, c, w * chord_closed(F->wd, ch));
  }
};

__device__ __forceinline__ bool segment_flight(const DevField& F, const Mask& M, float3 o, float3 v,
                                               uint64_t seed, uint32_t ray, uint32_t word,
                                               float& th, Counters& cnt) {
  const uint4 y = rng4(seed, 0, kNoPrim, ray, word);
  const float target = -log1pf(-u01(y.x));
  float tend;
  const float total = closed_tau(F, M, o, v, 0.f, INFINITY, cnt, 0, 1, &tend);
  if (!(tend > 0.f) || total < target) return false;
  const float3 inv = safe_inv(v);
  float t0, t1;
  if (!scene_span(F, o, inv, 0.f, INFINITY, t0, t1)) return false;
  float lo = 0.f, hi = tend;
  float ea = 0.f, eb = tend;
  for (int it = 0; it < 48; ++it) {
    SegLeaf leaf;
    leaf.F = &F;
    leaf.M = &M;
    leaf.o = o;
    leaf.v = v;
    leaf.lo = lo;
    leaf.hi = hi;
    leaf.mid = 0.5f * (lo + hi);
    SpanTest test{t0, t1};
    unsigned long long nodes = 0, leaves = 0;
    traverse_ray(F, o, inv, M.bits, test, leaf, nodes, leaves);
    cnt.nodes += nodes;
    cnt.leaves += leaves;
    cnt.windows += 1;
    const bool right = __fadd_rn(leaf.s, leaf.c) < target;
    if (right) {
      lo = leaf.mid;
      ea = leaf.below_mid;
      eb = leaf.above_hi;
      if (leaf.n_right == 0) break;
    } else {
      hi = leaf.mid;
      ea = leaf.below_lo;
      eb = leaf.above_mid;
      if (leaf.n_left == 0) break;
    }
    if (!(hi > lo)) break;
  }
  if (!(eb < INFINITY)) eb = tend;
  th = ea + u01(y.y) * (eb - ea);
  return true;
}

// ---------------------------------------------------------------------------
// Tracking.  The majorant is constant on every segment between consecutive
// chord ends and whitened-distance integers: kappa_bar = sum over the active
// chords of w|A| exp(-(r^2 + n^2)/2), n = floor(sqrt(a)|t - t*|).  Its
// Poisson process of tentative points is drawn chord by chord (superposition),
// each chord from its own Philox stream (counter = draw, primitive, ray, word;
// x.x -> exponential step, x.y -> acceptance uniform).
//
// Window by window, pass 1 traverses the ray and keeps the kPts smallest-t
// points beyond the window start in registers, pruning boxes that start past
// the current kPts-th point; pass 2 traverses only boxes containing one of
// those points and sums kappa and kappa_bar there.  The estimate depends only
// on the chords and their streams, never on the windows.
// ---------------------------------------------------------------------------
struct PointBuf {
  float t[kPts], u[kPts];
};

// The tentative points of one chord under the per-segment majorant (Sec. 3;
// R2/R3): rate h exp(-n^2/2) on the chord's whitened-distance pieces n, drawn
// from the chord's own Philox stream from its entry on.  emit(t, u) receives
// each point, in order along the chord, with its acceptance uniform, and
// returns false to end the walk.
template <class Emit>
__device__ __forceinline__ void chord_points(const DevField& F, const Chord& ch, float h,
                                             uint64_t seed, uint32_t ray, uint32_t word,
                                             const float* env, Emit emit) {
  const float sa = sqrtf(ch.a), invs = 1.0f / sa, dts = ch.dts, dtout = ch.dtout;
  int J = (int)ceilf(sa * ch.hw) - 1;
  J = J < 0 ? 0 : (J > 6 ? 6 : J);
  float dt = ch.dtin;
  int p = 0;
  while (p < 2 * J) {
    const float bp = p < J ? dts - (float)(J - p) * invs : dts + (float)(p - J + 1) * invs;
    if (bp <= dt) ++p;
    else break;
  }
  for (uint32_t draw = 0; draw < (1u << 16); ++draw) {
    const uint4 x = rng4(seed, draw, ch.orig, ray, word);
    float z = -__logf(1.0f - u01(x.x));
    bool more = false;
    for (int q = 0; q < 2 * J + 2; ++q) {
      const float bp = p < J ? dts - (float)(J - p) * invs : dts + (float)(p - J + 1) * invs;
      const float end = p < 2 * J ? fminf(bp, dtout) : dtout;
      const int nn = p < J ? J - p : p - J;
      const float lam = h * env[nn];
      const float capz = lam * (end - dt);
      if (z < capz) {
        dt += z / lam;
        more = true;
        break;
      }
      z -= capz;
      dt = end;
      if (dt >= dtout) return;
      ++p;
    }
    if (!more) return;
    if (!emit(ch.tc + dt, u01(x.y))) return;
  }
  set_err(F, ERR_GUARD);
}

struct CollectLeaf {
  const DevField* F;
  const Mask* M;
  float3 o, v;
  float tmin, tmax;
  float ta;     // window start: points must be > ta (>= ta in the first window)
  bool first;
  float bound;  // points beyond are not needed: min(t1, kPts-th point so far)
  PointBuf* B;
  uint64_t seed;
  uint32_t ray, word;
  const float* env;
  unsigned long long nch = 0;
  __device__ __forceinline__ void insert(float t, float u) {
#pragma unroll
    for (int i = 0; i < kPts; ++i) {
      const bool sw = t < B->t[i];
      const float tt = B->t[i], uu = B->u[i];
      B->t[i] = sw ? t : tt;
      B->u[i] = sw ? u : uu;
      t = sw ? tt : t;
      u = sw ? uu : u;
    }
    bound = fminf(bound, B->t[kPts - 1]);
  }
  __device__ void operator()(int j) {
    const Mask& Mk = *M;
    Chord ch;
    float w;
    if (!prim_chord(*F, j, o, v, tmin, tmax, [&](uint32_t c) { return mask_weight(Mk, c); }, w, ch))
      return;
    if (!(ch.tc + ch.dtin <= bound && ch.tc + ch.dtout >= ta)) return;
    ++nch;
    const float h = w * ch.absA * expf(-0.5f * ch.qmin);
    chord_points(*F, ch, h, seed, ray, word, env, [&](float t, float u) {
      if (t > bound) return false;
      if (first ? t >= ta : t > ta) insert(t, u);
      return true;
    });
  }
};

struct CollectTest {
  const float* ta;
  const float* bound;
  __device__ __forceinline__ bool operator()(float tn, float tf) const {
    return fmaxf(tn, *ta) <= fminf(tf, *bound);
  }
};

struct PointTest {
  const PointBuf* B;
  int n;
  __device__ __forceinline__ bool operator()(float tn, float tf) const {
    bool hit = false;
#pragma unroll
    for (int i = 0; i < kPts; ++i) hit |= (i < n) && B->t[i] >= tn && B->t[i] <= tf;
    return hit;
  }
};

struct AccumLeaf {
  const DevField* F;
  const Mask* M;
  float3 o, v;
  float tmin, tmax;
  const PointBuf* B;
  int n;
  const float* env;
  float kap[kPts], kb[kPts];
  unsigned long long nev = 0;
  __device__ void operator()(int j) {
    const Mask& Mk = *M;
    Chord ch;
    float w;
    if (!prim_chord(*F, j, o, v, tmin, tmax, [&](uint32_t c) { return mask_weight(Mk, c); }, w, ch))
      return;
    const float tin = ch.tc + ch.dtin, tout = ch.tc + ch.dtout;
    const float wa = w * ch.absA;
    const float y2 = -0.5f * kLog2e * ch.a, y1 = -kLog2e * ch.b;
    const float y0 = fmaf(-0.5f * kLog2e, ch.g, log2f(wa));
    const float h = wa * expf(-0.5f * ch.qmin);
    const float sa = sqrtf(ch.a);
#pragma unroll
    for (int i = 0; i < kPts; ++i) {
      const float t = B->t[i];
      if (i < n && t >= tin && t <= tout) {
        const float dt = t - ch.tc;
        const float y = fmaf(fmaf(y2, dt, y1), dt, y0);
        kap[i] = fmaf(ex2f(y), cosf_fast(fmaf(ch.B, dt, ch.delta)), kap[i]);
        int m = (int)(fabsf(dt - ch.dts) * sa);
        m = m > 7 ? 7 : m;
        kb[i] = fmaf(h, env[m], kb[i]);
        ++nev;
      }
    }
  }
};

// Ratio tracking (DELTA = false): returns prod (1 - kappa/kappa_bar).
// Delta tracking (DELTA = true): returns 1 and *t_hit at the first accepted
// point (probability max(kappa,0)/kappa_bar), else 0.
template <bool DELTA>
__device__ float track(const DevField& F, const Mask& M, float3 o, float3 v, float tmin,
                       float tmax, bool clamp_neg, uint64_t seed, uint32_t ray, uint32_t word,
                       const float* env, Counters& cnt, float* t_hit) {
  const unsigned am = __activemask();
  const float3 inv = safe_inv(v);
  float t0 = 0.f, t1 = 0.f;
  float Tr = 1.f, hit = 0.f;
  // `more`: this lane still has windows to process; all lanes that entered
  // iterate together until none has
  bool more = M.bits != 0ull && scene_span(F, o, inv, tmin, tmax, t0, t1);
  float ta = t0;
  bool first = true;
  for (int guard = 0; guard < (1 << 16); ++guard) {
    if (!__any_sync(am, more)) break;
    if (!more) continue;
    PointBuf B;
#pragma unroll
    for (int i = 0; i < kPts; ++i) {
      B.t[i] = INFINITY;
      B.u[i] = 0.f;
    }
    GF_TIC(c0);
    CollectLeaf cl;
    cl.F = &F;
    cl.M = &M;
    cl.o = o;
    cl.v = v;
    cl.tmin = tmin;
    cl.tmax = tmax;
    cl.ta = ta;
    cl.first = first;
    cl.bound = t1;
    cl.B = &B;
    cl.seed = seed;
    cl.ray = ray;
    cl.word = word;
    cl.env = env;
    CollectTest ctest{&cl.ta, &cl.bound};
    traverse_ray(F, o, inv, M.bits, ctest, cl, cnt.nodes, cnt.leaves);
    GF_TOC(cnt, 0, c0);
    cnt.windows += 1;
    cnt.chords += cl.nch;
    int n = 0;
#pragma unroll
    for (int i = 0; i < kPts; ++i) n += B.t[i] < INFINITY ? 1 : 0;
    cnt.points += (unsigned long long)n;
    if (n == 0) {
      more = false;
      continue;
    }
    GF_TIC(c1);
    AccumLeaf al;
    al.F = &F;
    al.M = &M;
    al.o = o;
    al.v = v;
    al.tmin = tmin;
    al.tmax = tmax;
    al.B = &B;
    al.n = n;
    al.env = env;
#pragma unroll
    for (int i = 0; i < kPts; ++i) {
      al.kap[i] = 0.f;
      al.kb[i] = 0.f;
    }
    PointTest ptest{&B, n};
    traverse_ray(F, o, inv, M.bits, ptest, al, cnt.nodes, cnt.leaves);
    GF_TOC(cnt, 1, c1);
    cnt.windows += 1;
    cnt.evals += al.nev;
    if (DELTA) {
      bool found = false;
#pragma unroll
      for (int i = 0; i < kPts; ++i) {
        if (!found && i < n && B.u[i] * al.kb[i] < fmaxf(al.kap[i], 0.f)) {
          *t_hit = B.t[i];
          found = true;
        }
      }
      if (found) {
        hit = 1.f;
        more = false;
        continue;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kPts; ++i) {
        if (i < n && al.kb[i] > 0.f) {
          const float k = clamp_neg ? fmaxf(al.kap[i], 0.f) : al.kap[i];
          Tr *= 1.f - k / al.kb[i];
        }
      }
    }
    if (n < kPts) {  // every point of the ray has been used
      more = false;
      continue;
    }
    ta = B.t[kPts - 1];
    first = false;
  }
  return DELTA ? hit : Tr;
}

// ---------------------------------------------------------------------------
// camera and path samples
// ---------------------------------------------------------------------------
struct CamDev {
  float3 eye, fw, rt, up;
  float tanh, aspect;
  int W, H;
};

__device__ __forceinline__ float3 normalize3(float3 a) {
  const float n = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
  return make_float3(a.x / n, a.y / n, a.z / n);
}

__device__ __forceinline__ void camera_ray(const CamDev& C, uint64_t seed, int px, int py, int s,
                                           float3& o, float3& v) {
  const uint32_t pix = (uint32_t)py * (uint32_t)C.W + (uint32_t)px;
  const uint4 x = rng4(seed, 0, kNoPrim, pix, stream_word((uint32_t)s, 0, TAG_CAMERA));
  const float jx = u01(x.x), jy = u01(x.y);
  const float sx = (2.0f * ((float)px + jx) / (float)C.W - 1.0f) * C.tanh * C.aspect;
  const float sy = (1.0f - 2.0f * ((float)py + jy) / (float)C.H) * C.tanh;
  const float3 d = make_float3(C.fw.x + sx * C.rt.x + sy * C.up.x, C.fw.y + sx * C.rt.y + sy * C.up.y,
                               C.fw.z + sx * C.rt.z + sy * C.up.z);
  v = normalize3(d);
  o = C.eye;
}

struct PathParams {
  CamDev cam;
  int integrator, spp, max_bounces;
  int free_flight;  // GF_FLIGHT_DELTA, GF_FLIGHT_CDF or GF_FLIGHT_SEGMENT
  int s0;           // first sample index (samples s0 .. s0 + spp - 1)
  int fov;          // foveation: 1 = per-sample band cutoff by eccentricity
  float3 gaze;      // unit direction of the ray through the gaze point
  float fov_f0, fov_slope, fov_smooth;
  float albedo, irradiance;
  float3 light;
  uint64_t seed;
  LodDev lod, lod_nee;
};

// Foveation (Supp. "Foveated Rendering"): the cells a sample's path keeps.
// The threshold falls linearly with the eccentricity e of the camera ray v,
// f = max(0, f0 - slope e), and is perturbed per sample by the third uniform
// of the camera stream (stochastic smoothing of the level transitions); the
// Gabor bands whose largest carrier exceeds f leave, the Gaussian band stays.
__device__ __forceinline__ unsigned long long fov_cells(const DevField& F, const PathParams& P,
                                                        float3 v, uint32_t pix, uint32_t s) {
  if (!P.fov) return ~0ull;
  const float c = fminf(1.f, fmaxf(-1.f, v.x * P.gaze.x + v.y * P.gaze.y + v.z * P.gaze.z));
  float f = fmaxf(0.f, P.fov_f0 - P.fov_slope * acosf(c));
  if (P.fov_smooth > 0.f) {
    const uint4 x = rng4(P.seed, 0, kNoPrim, pix, stream_word(s, 0, TAG_CAMERA));
    f *= 1.f + P.fov_smooth * (2.f * u01(x.z) - 1.f);
  }
  unsigned long long m = 1ull;
#pragma unroll
  for (int b = 1; b < 8; ++b)
    if (F.band_wmax[b] <= f) m |= 0xFFull << (1 + kCones * (b - 1));
  return m;
}

// One sample of pixel (px, py): tomography exp(-tau) or scattering radiance.
// Called by all lanes of a warp together (inactive lanes with active = false):
// every phase (camera tracking, NEE, scattering) runs with the lanes that need
// it converged, and the lanes regroup after each phase.
// FF selects the free flight at compile time (GF_FLIGHT_DELTA, GF_FLIGHT_CDF or
// GF_FLIGHT_SEGMENT), so that each kernel carries only the stack of the path it runs.
template <int FF>
static __device__ float path_sample(const DevField& F, const PathParams& P, bool active, int px,
                                    int py, int s, const float* glx, const float* glw,
                                    const float* env, Counters& cnt) {
  float3 o = make_float3(0.f, 0.f, 0.f), v = make_float3(0.f, 0.f, 1.f);
  if (active) camera_ray(P.cam, P.seed, px, py, s, o, v);
  const uint32_t pix = (uint32_t)py * (uint32_t)P.cam.W + (uint32_t)px;
  const unsigned long long allow = fov_cells(F, P, v, pix, (uint32_t)s);
  if (P.integrator == 0) {
    float T = 0.f;
    if (active) {
      Mask m = sample_mask(F, P.lod, v, P.seed, pix, (uint32_t)s, 0, TAG_MASK);
      m.bits &= allow;
      cnt.rays += 1;
      T = expf(-det_tau(F, m, o, v, 0.f, INFINITY, glx, glw, cnt));
    }
    __syncwarp();
    return T;
  }
  float thr = 1.f, Lsum = 0.f;
  bool alive = active;
  GF_TIC(ct);
  for (int b = 0; b < P.max_bounces; ++b) {
    float th = 0.f, hit = 0.f;
    if (alive) {
      GF_TIC(cm);
      Mask m = sample_mask(F, P.lod, v, P.seed, pix, (uint32_t)s, (uint32_t)b, TAG_MASK);
      m.bits &= allow;
      GF_TOC(cnt, 3, cm);
      cnt.rays += 1;
      const uint32_t tw = stream_word((uint32_t)s, (uint32_t)b, TAG_TRACK);
      if constexpr (FF == GF_FLIGHT_CDF)
        hit = cdf_flight(F, m, o, v, P.seed, pix, tw, th, cnt) ? 1.f : 0.f;
      else if constexpr (FF == GF_FLIGHT_SEGMENT)
        hit = segment_flight(F, m, o, v, P.seed, pix, tw, th, cnt) ? 1.f : 0.f;
      else
        hit = track<true>(F, m, o, v, 0.f, INFINITY, true, P.seed, pix, tw, env, cnt, &th);
    }
    __syncwarp();
    alive = alive && hit != 0.f;
    const float3 x = make_float3(o.x + th * v.x, o.y + th * v.y, o.z + th * v.z);
    if (alive) {
      thr *= P.albedo;
      Mask mn = sample_mask(F, P.lod_nee, P.light, P.seed, pix, (uint32_t)s, (uint32_t)b,
                            TAG_NEE_MASK);
      mn.bits &= allow;
      cnt.rays += 1;
      float Tl;
      if constexpr (FF != GF_FLIGHT_DELTA)
        Tl = expf(-closed_tau(F, mn, x, P.light, 0.f, INFINITY, cnt));
      else
        Tl = track<false>(F, mn, x, P.light, 0.f, INFINITY, true, P.seed, pix,
                          stream_word((uint32_t)s, (uint32_t)b, TAG_NEE), env, cnt, nullptr);
      Lsum += thr * P.irradiance * Tl * (0.25f / 3.14159265358979f);
      const uint4 y = rng4(P.seed, 0, kNoPrim, pix, stream_word((uint32_t)s, (uint32_t)b, TAG_SCATTER));
      const float z = 1.0f - 2.0f * u01(y.x);
      const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
      float sn, cs;
      sincosf(2.0f * 3.14159265358979f * u01(y.y), &sn, &cs);
      v = make_float3(rr * cs, rr * sn, z);
      o = x;
    }
    __syncwarp();
    if (!__any_sync(kFull, alive)) break;
  }
  GF_TOC(cnt, 4, ct);
  return Lsum;
}

}  // namespace gf
