// gf_device.cuh -- device-side data structures and helpers of the Gabor-field
// renderer (sm_103a).  Notation follows arXiv 2602.05081: mu, Sigma, omega,
// the per-ray quadratic q(t) = a t^2 + 2 beta t + gamma and phase B t + delta
// of App. A.1, the k-sigma support of Sec. 3.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gf {

constexpr int kMaxCells = 64;
constexpr int kCones = 8;
constexpr uint32_t kNoPrim = 0xFFFFFFFFu;
constexpr unsigned kFull = 0xffffffffu;

enum : uint32_t {
  TAG_CAMERA = 1,
  TAG_MASK = 2,
  TAG_TRACK = 3,
  TAG_NEE = 4,
  TAG_NEE_MASK = 5,
  TAG_SCATTER = 6
};

// ERR_INDEX: a tree index out of its array (the traversals check every node and
// leaf index they follow and skip the access)
enum : int {
  ERR_STACK = 1, ERR_WINDOW = 2, ERR_POINTS = 4, ERR_GUARD = 8, ERR_INPUT = 16, ERR_INDEX = 32
};

// Binary BVH node holding the boxes, children and cell masks of both children
// (one 80-byte fetch tests two boxes).  child >= 0: internal node; child < 0:
// leaf of the sorted primitive ~child.
struct __align__(16) Node {
  float4 a;  // c0.lo.xyz, c0.hi.x
  float4 b;  // c0.hi.yz, c1.lo.xy
  float4 c;  // c1.lo.z, c1.hi.xyz
  int4 d;    // child0, child1, parent (build only), unused
  uint4 e;   // cell mask of child0 (lo, hi), child1 (lo, hi)
};

// Four-wide node of the scattering renderer's BVH, collapsed from the binary
// tree (every even-depth binary node with its children's children).  Child
// boxes are 8-bit codes on a per-node grid: box = lo + code * s per axis,
// floor/ceil rounded on the builder and checked with the decoding formula so
// that each decoded box contains the exact child box.  Unused children have
// an empty code box and a zero cell mask.  child >= 0: four-wide node;
// child < 0: leaf of the sorted primitive ~child.
struct __align__(16) Node4 {
  float4 v0;  // lo.xyz, s.x
  float4 v1;  // s.yz, bits: qlo.x (4 children x u8), qlo.y
  uint4 q;    // qlo.z, qhi.x, qhi.y, qhi.z (4 children x u8 each)
  int4 child;
  uint4 m01;  // cell masks of children 0, 1 (lo, hi)
  uint4 m23;  // cell masks of children 2, 3
};

struct LodDev {
  int freq_policy, max_band, cone_policy;
  float beta;   // power-law shape of the band choice, [0, 1)
  float delta;  // alignment threshold of the cone choice, [0, 1]
};

// Everything a kernel needs to read a packed field; passed by value.
// Coefficients of Weideman's rational expansion of the Faddeeva function
// (J. A. C. Weideman, "Computation of the complex error function", SIAM J.
// Numer. Anal. 31 (1994) 1497-1518): a[n-1] = a_n, n = 1..N, and the scale L.
// N = 20 reaches FP32 rounding over the closed upper half plane.
constexpr int kWeidN = 20;
struct Weideman {
  float a[kWeidN];
  float L;
};

struct DevField {
  const float4* rec;       // FP32 records: 4 x float4 per primitive, BVH order
  const uint4* rec16;      // FP16/BF16 records: 2 x uint4 per primitive, BVH order
  const Node* nodes;
  const Node4* nodes4;     // four-wide collapse of nodes (root 0 when n >= 2)
  int64_t n;
  int64_t n_nodes4;        // four-wide nodes
  int root;                // internal root node, -1 when n == 1
  int precision;           // 0 FP32, 1 FP16, 2 BF16
  float ksig, k2;
  float3 lo, hi;           // scene bounds (union of all ellipsoid boxes)
  unsigned long long occupied;
  float kbar[kMaxCells];   // mean |k_W| per cell
  float band_wmax[8];      // largest world carrier |omega| (rad/unit) per band
  float axes[kCones][3];   // orientation-bin axes
  float env[8];            // exp(-n^2/2), n = 0..7
  const int* orig16;       // reduced-precision records: BVH position -> original index
  float3 qlo, qscale;      // reduced-precision records: mean = qlo + code * qscale
  const float* gl;         // Gauss-Legendre nodes then weights (2 x kGLTotal)
  Weideman wd;             // Faddeeva expansion (closed-form chord integrals)
  const float* ext2;       // reduced-precision records: support radius squared per primitive,
                           // BVH order, -1 = not in the mixture (FP32 records carry their own);
                           // null when every radius is k_sigma (no clamping, no camera selection)
  unsigned long long cells_on;  // cells holding a primitive of the mixture (all ones by default)
  int* err;
  unsigned long long* stats;  // rays, chords, evals, nodes, points
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), written from the published round
// function: 10 rounds, Weyl key bump between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}
__device__ __forceinline__ uint4 rng4(uint64_t seed, uint32_t draw, uint32_t prim, uint32_t ray,
                                      uint32_t word) {
  return philox(make_uint4(draw, prim, ray, word),
                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }
__device__ __forceinline__ uint32_t stream_word(uint32_t sample, uint32_t bounce, uint32_t tag) {
  return (sample << 12) | ((bounce & 15u) << 8) | (tag & 255u);
}

// ---------------------------------------------------------------------------
// fast math: MUFU exp2 and cos
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cosf_fast(float x) { return __cosf(x); }

// phase reduction to [-pi, pi]: x - 2 pi rint(x / 2 pi) with 2 pi split into a
// short head (exact product with small integers) and a tail (Cody-Waite)
__device__ __forceinline__ float reduce_2pi(float x) {
  const float kInv2Pi = 0.15915494309189535f;
  const float kHead = 6.28125f;                 // 2 pi rounded to 7 significant bits
  const float kTail = 1.9353071795864769e-3f;   // 2 pi - kHead
  float k = rintf(x * kInv2Pi);
  float r = fmaf(-k, kHead, x);
  return fmaf(-k, kTail, r);
}

constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------------------
// Faddeeva function w(z) = exp(-z^2) erfc(-iz) for z = x + iy, y >= 0, by
// Weideman's expansion: with Z = (L + iz)/(L - iz), which stays in the unit
// disc for y >= 0,
//   w(z) = 2 sum_{n=1..N} a_n Z^(n-1) / (L - iz)^2 + 1 / (sqrt(pi) (L - iz)).
// Here L - iz = (L + y) - ix, so 1/(L - iz) = ((L + y) + ix)/D and
// Z = ((L^2 - y^2 - x^2) + 2iLx)/D with D = (L + y)^2 + x^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 faddeeva_w(const Weideman& W, float x, float y) {
  const float kRsqrtPi = 0.56418958354775628f;
  const float lp = W.L + y, lm = W.L - y;
  const float iD = 1.0f / fmaf(lp, lp, x * x);
  const float zr = fmaf(lm, lp, -x * x) * iD, zi = 2.0f * W.L * x * iD;
  float pr = W.a[kWeidN - 1], pim = 0.0f;
#pragma unroll
  for (int n = kWeidN - 2; n >= 0; --n) {
    const float t = fmaf(pr, zr, fmaf(-pim, zi, W.a[n]));
    pim = fmaf(pr, zi, pim * zr);
    pr = t;
  }
  const float ir = lp * iD, ii = x * iD;                    // 1/(L - iz)
  const float sr = fmaf(ir, ir, -ii * ii), si = 2.0f * ir * ii;  // 1/(L - iz)^2
  return make_float2(fmaf(2.0f, fmaf(pr, sr, -pim * si), kRsqrtPi * ir),
                     fmaf(2.0f, fmaf(pr, si, pim * sr), kRsqrtPi * ii));
}

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}
__device__ __forceinline__ long long warp_sum_ll(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Neumaier accumulation of x into (s, c)
__device__ __forceinline__ void neumaier_add(float& s, float& c, float x) {
  float t = __fadd_rn(s, x);
  if (fabsf(s) >= fabsf(x))
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, t), x));
  else
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(x, t), s));
  s = t;
}
// compensated warp sum of (s + c) pairs; every lane receives the total
__device__ __forceinline__ float warp_sum_comp(float s, float c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float so = __shfl_xor_sync(kFull, s, o), co = __shfl_xor_sync(kFull, c, o);
    float t, e;
    two_sum(s, so, t, e);
    s = t;
    c = __fadd_rn(__fadd_rn(c, co), e);
  }
  return __fadd_rn(s, c);
}

// ---------------------------------------------------------------------------
// records
// FP32 record (64 B): {mu.xyz, A}, {P00, P01, P02, P11}, {P12, P22, phi, cell},
// {omega.xyz, orig index}, P = Sigma^-1.
// ---------------------------------------------------------------------------
// FP32 record word 15: original index (26 bits) | cell << 26
constexpr uint32_t kOrigMask = (1u << 26) - 1u;

struct Prim {
  float3 mu;
  float A;
  float p00, p01, p02, p11, p12, p22;
  float phi;
  float k2;  // support radius squared: k^2, the adaptive extent, or -1 (not in the mixture)
  uint32_t cell;
  float3 om;
  uint32_t orig;
};

__device__ __forceinline__ Prim load_prim(const DevField& F, int j) {
  Prim P;
  const float4* r = F.rec + 4 * (int64_t)j;
  float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
  P.mu = make_float3(r0.x, r0.y, r0.z);
  P.A = r0.w;
  P.p00 = r1.x; P.p01 = r1.y; P.p02 = r1.z; P.p11 = r1.w;
  P.p12 = r2.x; P.p22 = r2.y; P.phi = r2.z; P.k2 = r2.w;
  P.om = make_float3(r3.x, r3.y, r3.z);
  P.orig = __float_as_uint(r3.w) & kOrigMask;
  P.cell = __float_as_uint(r3.w) >> 26;
  return P;
}

// Per-(ray, primitive) chord in coordinates dt = t - tc around a reference tc
// near the envelope peak.  Along the ray the kernel is
//   A exp(-(a dt^2 + 2 b dt + g)/2) cos(B dt + delta)
// (App. A.1 with the origin moved to tc); the chord is where the quadratic is
// <= k^2, clipped to the ray's [tmin, tmax].
struct Chord {
  float tc;          // reference t (absolute)
  float dtin, dtout; // clipped chord, relative to tc
  float a, b, g;     // quadratic coefficients in dt
  float B, delta;    // phase slope and phase at tc, delta in [-pi, pi]
  float absA;        // |A| (the sign of A is folded into delta)
  float qmin, dts;   // minimum of the quadratic and its position (relative to tc)
  float hw;          // half-width of the unclipped chord
  float3 p;          // o + tc v - mu (compensated)
  uint32_t cell, orig;
};

__device__ __forceinline__ bool chord_setup(const Prim& P, float3 o, float3 v, float tmin,
                                            float tmax, float k2, Chord& c) {
  // u = Sigma^-1 v, a = v^T Sigma^-1 v
  float ux = fmaf(P.p00, v.x, fmaf(P.p01, v.y, P.p02 * v.z));
  float uy = fmaf(P.p01, v.x, fmaf(P.p11, v.y, P.p12 * v.z));
  float uz = fmaf(P.p02, v.x, fmaf(P.p12, v.y, P.p22 * v.z));
  float a = fmaf(v.x, ux, fmaf(v.y, uy, v.z * uz));
  // d0 = o - mu, error-free split; reference tc = -(d0 . u)/a
  float d0x = __fsub_rn(o.x, P.mu.x), d0y = __fsub_rn(o.y, P.mu.y), d0z = __fsub_rn(o.z, P.mu.z);
  const float ia = __frcp_rn(a);
  float tc = -fmaf(d0x, ux, fmaf(d0y, uy, d0z * uz)) * ia;
  // p = (o - mu) + tc v with compensated arithmetic (positions ~1, offsets ~sigma)
  float ex, ey, ez;
  {
    float s, bb;
    s = d0x; bb = __fsub_rn(s, o.x); ex = __fsub_rn(__fsub_rn(o.x, __fsub_rn(s, bb)), __fadd_rn(P.mu.x, bb));
    s = d0y; bb = __fsub_rn(s, o.y); ey = __fsub_rn(__fsub_rn(o.y, __fsub_rn(s, bb)), __fadd_rn(P.mu.y, bb));
    s = d0z; bb = __fsub_rn(s, o.z); ez = __fsub_rn(__fsub_rn(o.z, __fsub_rn(s, bb)), __fadd_rn(P.mu.z, bb));
  }
  float prx = __fmul_rn(tc, v.x), pry = __fmul_rn(tc, v.y), prz = __fmul_rn(tc, v.z);
  float erx = fmaf(tc, v.x, -prx), ery = fmaf(tc, v.y, -pry), erz = fmaf(tc, v.z, -prz);
  float px = __fadd_rn(__fadd_rn(d0x, prx), __fadd_rn(ex, erx));
  float py = __fadd_rn(__fadd_rn(d0y, pry), __fadd_rn(ey, ery));
  float pz = __fadd_rn(__fadd_rn(d0z, prz), __fadd_rn(ez, erz));
  // b = v^T Sigma^-1 p (~0), g = p^T Sigma^-1 p
  float b = fmaf(ux, px, fmaf(uy, py, uz * pz));
  float qx = fmaf(P.p00, px, fmaf(P.p01, py, P.p02 * pz));
  float qy = fmaf(P.p01, px, fmaf(P.p11, py, P.p12 * pz));
  float qz = fmaf(P.p02, px, fmaf(P.p12, py, P.p22 * pz));
  float g = fmaf(px, qx, fmaf(py, qy, pz * qz));
  float dts = -b * ia;
  float qmin = fmaf(b, dts, g);
  float disc = k2 - qmin;
  if (!(disc > 0.0f)) return false;
  float hw = sqrtf(disc * ia);
  float lo = fmaxf(dts - hw, tmin - tc);
  float hi = fminf(dts + hw, tmax - tc);
  if (!(lo < hi)) return false;
  c.tc = tc;
  c.dtin = lo;
  c.dtout = hi;
  c.a = a;
  c.b = b;
  c.g = g;
  c.B = fmaf(P.om.x, v.x, fmaf(P.om.y, v.y, P.om.z * v.z));
  float ph = fmaf(P.om.x, px, fmaf(P.om.y, py, fmaf(P.om.z, pz, P.phi)));
  if (P.A < 0.0f) ph += 3.14159265358979f;
  c.delta = reduce_2pi(ph);
  c.absA = fabsf(P.A);
  c.qmin = qmin;
  c.dts = dts;
  c.hw = hw;
  c.p = make_float3(px, py, pz);
  c.cell = P.cell;
  c.orig = P.orig;
  return true;
}

// ---------------------------------------------------------------------------
// Reduced-precision record (32 B = 2 x uint4), BVH order:
//   x0 = mu.x | mu.y << 16            (u16 fixed point in the means' box)
//   y0 = mu.z | T00 << 16             (T: 6 entries as FP16 or BF16, times 2^-E)
//   z0 = T01  | T02 << 16
//   w0 = T11  | T12 << 16
//   x1 = T22  | kT.x << 16            (kT, A as FP16 or BF16)
//   y1 = kT.y | kT.z << 16
//   z1 = A    | phase << 16           (phase as u16 in [0, 2 pi))
//   w1 = cell | (E + 127) << 8
// T is the upper-triangular whitening factor, T^T T = Sigma^-1 (Sec. 4.4 with
// the whitening matrix taken triangular), and kT the whitened carrier in its
// frame.  Decoded to FP32; the chord is set up in T's frame: u = T v,
// p_T = T (o + tc v - mu), phase kT . p_T + phi.
// ---------------------------------------------------------------------------
// exact integer-to-float conversions by exponent insertion (0x4B000000 is 2^23)
__device__ __forceinline__ float u16_float(uint32_t x) {
  return __int_as_float((int)(0x4B000000u | x)) - 8388608.0f;
}
__device__ __forceinline__ float half_bits_to_float(uint32_t h, int prec) {
  return prec == 2 ? __uint_as_float(h << 16) : __half2float(__ushort_as_half((unsigned short)h));
}

__device__ __forceinline__ bool chord_setup16(const DevField& F, uint4 r0, uint4 r1, int j,
                                              float3 o, float3 v, float tmin, float tmax,
                                              Chord& c) {
  const int prec = F.precision;
  const float3 mu = make_float3(fmaf(u16_float(r0.x & 0xFFFFu), F.qscale.x, F.qlo.x),
                                fmaf(u16_float(r0.x >> 16), F.qscale.y, F.qlo.y),
                                fmaf(u16_float(r0.y & 0xFFFFu), F.qscale.z, F.qlo.z));
  const float sT = __uint_as_float(((r1.w >> 8) & 0xFFu) << 23);  // 2^E
  const float T00 = half_bits_to_float(r0.y >> 16, prec) * sT;
  const float T01 = half_bits_to_float(r0.z & 0xFFFFu, prec) * sT;
  const float T02 = half_bits_to_float(r0.z >> 16, prec) * sT;
  const float T11 = half_bits_to_float(r0.w & 0xFFFFu, prec) * sT;
  const float T12 = half_bits_to_float(r0.w >> 16, prec) * sT;
  const float T22 = half_bits_to_float(r1.x & 0xFFFFu, prec) * sT;
  // whitened direction and offset (T upper triangular)
  const float ux = fmaf(T00, v.x, fmaf(T01, v.y, T02 * v.z));
  const float uy = fmaf(T11, v.y, T12 * v.z);
  const float uz = T22 * v.z;
  const float a = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
  const float d0x = __fsub_rn(o.x, mu.x), d0y = __fsub_rn(o.y, mu.y), d0z = __fsub_rn(o.z, mu.z);
  const float w0x = fmaf(T00, d0x, fmaf(T01, d0y, T02 * d0z));
  const float w0y = fmaf(T11, d0y, T12 * d0z);
  const float w0z = T22 * d0z;
  const float ia = __frcp_rn(a);
  const float tc = -fmaf(ux, w0x, fmaf(uy, w0y, uz * w0z)) * ia;
  // whitened offset at tc, T (o + tc v - mu) = T d0 + tc T v: its FP32 rounding,
  // ~2^-24 |T d0|, stays below the record's own (T's entries round by 2^-11 or
  // 2^-8 of themselves), so no compensated world offset is needed here
  const float pwx = fmaf(tc, ux, w0x), pwy = fmaf(tc, uy, w0y), pwz = fmaf(tc, uz, w0z);
  const float px = fmaf(tc, v.x, d0x), py = fmaf(tc, v.y, d0y), pz = fmaf(tc, v.z, d0z);
  const float b = fmaf(ux, pwx, fmaf(uy, pwy, uz * pwz));
  const float g = fmaf(pwx, pwx, fmaf(pwy, pwy, pwz * pwz));
  const float dts = -b * ia;
  const float qmin = fmaf(b, dts, g);
  const float disc = (F.ext2 ? __ldg(F.ext2 + j) : F.k2) - qmin;
  if (!(disc > 0.0f)) return false;
  const float hw = sqrtf(disc * ia);
  const float lo = fmaxf(dts - hw, tmin - tc);
  const float hi = fminf(dts + hw, tmax - tc);
  if (!(lo < hi)) return false;
  c.tc = tc;
  c.dtin = lo;
  c.dtout = hi;
  c.a = a;
  c.b = b;
  c.g = g;
  const float k0 = half_bits_to_float(r1.x >> 16, prec);
  const float k1 = half_bits_to_float(r1.y & 0xFFFFu, prec);
  const float k2 = half_bits_to_float(r1.y >> 16, prec);
  const float A = half_bits_to_float(r1.z & 0xFFFFu, prec);
  const float phi = u16_float(r1.z >> 16) * (6.28318530717958647692f / 65536.0f);
  c.B = fmaf(k0, ux, fmaf(k1, uy, k2 * uz));
  float ph = fmaf(k0, pwx, fmaf(k1, pwy, fmaf(k2, pwz, phi)));
  if (A < 0.0f) ph += 3.14159265358979f;
  c.delta = reduce_2pi(ph);
  c.absA = fabsf(A);
  c.qmin = qmin;
  c.dts = dts;
  c.hw = hw;
  c.p = make_float3(px, py, pz);
  c.cell = r1.w & 63u;
  c.orig = (uint32_t)__ldg(F.orig16 + j);
  return true;
}

// Chord of BVH primitive j for either record precision; `weight(cell)` is the
// LoD weight of the primitive's cell (no chord when it is 0).
template <class WeightFn>
__device__ __forceinline__ bool prim_chord(const DevField& F, int j, float3 o, float3 v,
                                           float tmin, float tmax, WeightFn weight, float& w,
                                           Chord& ch) {
  if (F.precision == 0) {
    const Prim P = load_prim(F, j);
    w = weight(P.cell & 63u);
    if (!(w > 0.f)) return false;
    return chord_setup(P, o, v, tmin, tmax, P.k2, ch);
  }
  const uint4* r = F.rec16 + 2 * (int64_t)j;
  const uint4 r0 = __ldg(r), r1 = __ldg(r + 1);
  w = weight(r1.w & 63u);
  if (!(w > 0.f)) return false;
  return chord_setup16(F, r0, r1, j, o, v, tmin, tmax, ch);
}

// ray-box slab test over [t0, t1]
__device__ __forceinline__ bool slab(float3 o, float3 inv, float lx, float ly, float lz, float hx,
                                     float hy, float hz, float t0, float t1) {
  float tx0 = (lx - o.x) * inv.x, tx1 = (hx - o.x) * inv.x;
  float ty0 = (ly - o.y) * inv.y, ty1 = (hy - o.y) * inv.y;
  float tz0 = (lz - o.z) * inv.z, tz1 = (hz - o.z) * inv.z;
  float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), t0));
  float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), t1));
  return tn <= tf;
}

// Unit direction of a caller's ray, d / |d| rounded once to FP32 (FP32
// arithmetic only).  The argument is scaled by a power of two (exact), |d|^2
// is formed as an unevaluated sum hi + lo of error-free products and sums,
// r = 1/sqrt(|d|^2) is refined from the FP32 estimate by one Newton step on
// the residual 1 - |d|^2 r^2 (relative error ~1e-14), and each component
// d_i (r + dr) is rounded once.  Results differ from the correctly rounded
// unit vector only where a component lies within ~1e-14 of a rounding tie.
// A zero vector gives NaN.
__device__ __forceinline__ float3 unit_dir(float3 d) {
  const float m = fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z)));
  if (!(m > 0.0f) || !(m < INFINITY)) {
    const float q = __int_as_float(0x7fc00000);
    return make_float3(q, q, q);
  }
  int e;
  (void)frexpf(m, &e);
  const float x = ldexpf(d.x, -e), y = ldexpf(d.y, -e), z = ldexpf(d.z, -e);
  const float px = __fmul_rn(x, x), ex = fmaf(x, x, -px);
  const float py = __fmul_rn(y, y), ey = fmaf(y, y, -py);
  const float pz = __fmul_rn(z, z), ez = fmaf(z, z, -pz);
  float s1, e1, hi, e2;
  two_sum(px, py, s1, e1);
  two_sum(s1, pz, hi, e2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(ex, ey), __fadd_rn(ez, e1)), e2);
  const float r0 = __fdiv_rn(1.0f, __fsqrt_rn(hi));
  // residual 1 - (hi + lo) r0^2: r0^2 = q + eq exactly, hi q = mq + emq exactly,
  // and 1 - mq is exact (Sterbenz: mq is within a few ulp of 1)
  const float q = __fmul_rn(r0, r0), eq = fmaf(r0, r0, -q);
  const float mq = __fmul_rn(hi, q), emq = fmaf(hi, q, -mq);
  const float res = __fsub_rn(__fsub_rn(1.0f, mq),
                              __fadd_rn(emq, __fadd_rn(__fmul_rn(hi, eq), __fmul_rn(lo, q))));
  const float dr = __fmul_rn(__fmul_rn(0.5f, r0), res);
  auto comp = [&](float a) {
    const float p = __fmul_rn(a, r0), err = fmaf(a, r0, -p);
    return __fadd_rn(p, __fadd_rn(err, __fmul_rn(a, dr)));
  };
  return make_float3(comp(x), comp(y), comp(z));
}

__device__ __forceinline__ float3 safe_inv(float3 v) {
  const float tiny = 1e-30f;
  float x = fabsf(v.x) < tiny ? copysignf(tiny, v.x) : v.x;
  float y = fabsf(v.y) < tiny ? copysignf(tiny, v.y) : v.y;
  float z = fabsf(v.z) < tiny ? copysignf(tiny, v.z) : v.z;
  return make_float3(1.0f / x, 1.0f / y, 1.0f / z);
}

// entry/exit of the scene box; returns false if missed
__device__ __forceinline__ bool scene_span(const DevField& F, float3 o, float3 inv, float tmin,
                                           float tmax, float& t0, float& t1) {
  float tx0 = (F.lo.x - o.x) * inv.x, tx1 = (F.hi.x - o.x) * inv.x;
  float ty0 = (F.lo.y - o.y) * inv.y, ty1 = (F.hi.y - o.y) * inv.y;
  float tz0 = (F.lo.z - o.z) * inv.z, tz1 = (F.hi.z - o.z) * inv.z;
  t0 = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
  t1 = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  return t0 <= t1;
}

__device__ __forceinline__ void set_err(const DevField& F, int code) { atomicOr(F.err, code); }

// ---------------------------------------------------------------------------
// Per-thread traversal of one ray under a cell mask: every lane of a warp owns
// its own ray, so a warp advances 32 independent rays per step.  One 80-byte
// fetch gives both child boxes of a node; test(tn, tf) decides whether a child
// whose box spans [tn, tf] along the ray can matter (the test may tighten as
// the traversal proceeds); hit leaves go to leaf(j) at once; the nearer
// internal child is visited first and the other pushed on a per-thread stack
// together with its entry t, re-tested when popped.
// ---------------------------------------------------------------------------
constexpr int kStack = 64;

__device__ __forceinline__ void slab_interval(float3 o, float3 inv, float lx, float ly, float lz,
                                              float hx, float hy, float hz, float& tn, float& tf) {
  float tx0 = (lx - o.x) * inv.x, tx1 = (hx - o.x) * inv.x;
  float ty0 = (ly - o.y) * inv.y, ty1 = (hy - o.y) * inv.y;
  float tz0 = (lz - o.z) * inv.z, tz1 = (hz - o.z) * inv.z;
  tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fminf(tz0, tz1));
  tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
}

// the subtree that lane `sub` of a group of `group` lanes (a power of two)
// walks: log2(group) levels down from the root along the bits of sub, most
// significant first, so the group's lanes cover the tree without overlap.  A
// leaf met on the way belongs to the lane whose remaining bits are all zero.
// Returns an internal node (>= 0), a leaf ~j (< 0), or kNoStart.
constexpr int kNoStart = -2147483647 - 1;
__device__ __forceinline__ int group_start(const DevField& F, int sub, int group) {
  int node = F.root < 0 ? ~0 : F.root;
  for (int l = 31 - __clz(group) - 1; l >= 0; --l) {
    if (node < 0) return (sub & ((2 << l) - 1)) == 0 ? node : kNoStart;
    const int4 d = __ldg(&F.nodes[node].d);
    node = (sub >> l & 1) ? d.y : d.x;
  }
  return node;
}

// traversal of the subtree `start` (group_start's result)
template <class TestFn, class LeafFn>
__device__ __forceinline__ void traverse_from(const DevField& F, int start, float3 o, float3 inv,
                                              unsigned long long mask, TestFn& test, LeafFn& leaf,
                                              unsigned long long& nvis,
                                              unsigned long long& nleaves) {
  if (start == kNoStart) return;
  if (start < 0) {
    if ((int64_t)~start >= F.n) {
      set_err(F, ERR_INDEX);
      return;
    }
    ++nleaves;
    leaf(~start);
    return;
  }
  // lanes that entered together stay together: they reconverge after every
  // traversal burst and leave the loop only when all of them are done
  const unsigned am = __activemask();
  int st_node[kStack];
  float st_tn[kStack];
  int sp = 0;
  int node = start;            // next internal node, -1 once the tree is exhausted
  int pend0 = -1, pend1 = -1;  // queued leaves
  // each internal node is fetched at most once per traversal
  const long long max_steps = F.n + 64;
  long long steps = 0;
  for (;;) {
    // while-while: traverse until a leaf is queued or the tree is exhausted; the
    // lanes then process their leaves together
    while (node >= 0 && pend0 < 0) {
      if (++steps > max_steps) {
        set_err(F, ERR_GUARD);
        node = -1;
        break;
      }
      if ((int64_t)node >= F.n - 1) {  // internal nodes 0 .. n-2
        set_err(F, ERR_INDEX);
        node = -1;
        break;
      }
      const Node* N = F.nodes + node;
      const float4 a = __ldg(&N->a), b = __ldg(&N->b), c = __ldg(&N->c);
      const int4 d = __ldg(&N->d);
      const uint4 e = __ldg(&N->e);
      ++nvis;
      const unsigned long long m0 = (unsigned long long)e.x | ((unsigned long long)e.y << 32);
      const unsigned long long m1 = (unsigned long long)e.z | ((unsigned long long)e.w << 32);
      float tn0, tf0, tn1, tf1;
      slab_interval(o, inv, a.x, a.y, a.z, a.w, b.x, b.y, tn0, tf0);
      slab_interval(o, inv, b.z, b.w, c.x, c.y, c.z, c.w, tn1, tf1);
      bool h0 = (m0 & mask) && test(tn0, tf0);
      bool h1 = (m1 & mask) && test(tn1, tf1);
      int c0 = d.x, c1 = d.y;
      if (c0 < 0 && (int64_t)~c0 >= F.n) {  // a leaf beyond the records
        set_err(F, ERR_INDEX);
        c0 = 0;
        h0 = false;
      }
      if (c1 < 0 && (int64_t)~c1 >= F.n) {
        set_err(F, ERR_INDEX);
        c1 = 0;
        h1 = false;
      }
      if (h0 && c0 < 0) pend0 = ~c0;
      if (h1 && c1 < 0) {
        if (pend0 < 0) pend0 = ~c1;
        else pend1 = ~c1;
      }
      const bool g0 = h0 && c0 >= 0, g1 = h1 && c1 >= 0;
      if (g0 && g1) {
        const bool first0 = tn0 <= tn1;
        if (sp < kStack) {
          st_node[sp] = first0 ? c1 : c0;
          st_tn[sp] = first0 ? tn1 : tn0;
          ++sp;
        } else {
          set_err(F, ERR_STACK);
        }
        node = first0 ? c0 : c1;
      } else if (g0) {
        node = c0;
      } else if (g1) {
        node = c1;
      } else {
        // pop, skipping entries the (possibly tightened) test now rejects
        node = -1;
        while (sp > 0) {
          --sp;
          if (test(st_tn[sp], INFINITY)) {
            node = st_node[sp];
            break;
          }
        }
      }
    }
    __syncwarp(am);
    if (pend0 >= 0) {
      ++nleaves;
      leaf(pend0);
      pend0 = pend1;
      pend1 = -1;
    }
    if (!__any_sync(am, node >= 0 || pend0 >= 0)) return;
  }
}

// traversal of the whole tree
template <class TestFn, class LeafFn>
__device__ __forceinline__ void traverse_ray(const DevField& F, float3 o, float3 inv,
                                             unsigned long long mask, TestFn& test, LeafFn& leaf,
                                             unsigned long long& nvis,
                                             unsigned long long& nleaves) {
  traverse_from(F, F.root < 0 ? ~0 : F.root, o, inv, mask, test, leaf, nvis, nleaves);
}

}  // namespace gf
