// gf_adjoint.cu -- hand-written adjoint of the tomography renderer.
//
// Image I_p = (1/spp) sum_s exp(-tau_s) (Sec. 4.6 tomography), tau_s the
// optical depth of Eq. 2-3 along the jittered camera ray.  Given dL/dI:
//   dL/dtheta_i = sum_{p,s} dL/dI_p (-exp(-tau_s)/spp) dtau_s/dtheta_i,
//   dtau/dtheta = int_chord d(integrand)/dtheta dt
//               + g(t_out) dt_out/dtheta - g(t_in) dt_in/dtheta,
// with the ellipsoid ends moving as dt/dtheta = -(dq/dtheta)/(dq/dt)
// (Leibniz rule for the k-sigma-truncated kernel).  Each ray is traversed
// twice (forward optical depth, then the adjoint pass): nothing is stored
// per path.  Gradients are accumulated with atomics in SoA layout.
#include <cuda_runtime.h>

#include "gf_host.h"
#include "gf_trace.cuh"

namespace gf {

struct BackArgs {
  const float* quat;
  const float* ls;
  const float* om;
  const float* w;
  int frame, wmode;
  int64_t n;
  float* grad;
};

// Derivatives of one kernel g = A exp(-q/2) cos(theta) with respect to its 15
// raw parameters (mu 3, quaternion 4 through qhat = q/|q|, log scale 3, omega 3
// in the input frame, phase, weight), at offsets y = x - mu.
struct PrimDeriv {
  float R[3][3];
  float qh[4], iqn;    // unit quaternion (w, x, y, z) and 1/|q| of the raw one
  float s[3], is2[3], kin[3];
  float A, dAdw;
  float3 om;
  float phi;
  bool local, normalized;

  __device__ void init(const BackArgs& B, const Prim& P, int64_t i) {
    float q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = B.quat[4 * i + k];
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    iqn = 1.f / qn;
#pragma unroll
    for (int k = 0; k < 4; ++k) qh[k] = q[k] * iqn;
    const float qw = qh[0], qx = qh[1], qy = qh[2], qz = qh[3];
    R[0][0] = 1.f - 2.f * (qy * qy + qz * qz); R[0][1] = 2.f * (qx * qy - qw * qz);
    R[0][2] = 2.f * (qx * qz + qw * qy);
    R[1][0] = 2.f * (qx * qy + qw * qz); R[1][1] = 1.f - 2.f * (qx * qx + qz * qz);
    R[1][2] = 2.f * (qy * qz - qw * qx);
    R[2][0] = 2.f * (qx * qz - qw * qy); R[2][1] = 2.f * (qy * qz + qw * qx);
    R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      s[k] = expf(B.ls[3 * i + k]);
      is2[k] = 1.f / (s[k] * s[k]);
      kin[k] = B.om[3 * i + k];
    }
    local = B.frame == GF_OMEGA_LOCAL;
    normalized = B.wmode == GF_WEIGHT_NORMALIZED;
    A = P.A;
    dAdw = normalized ? A / B.w[i] : 1.f;
    om = P.om;
    phi = P.phi;
  }

  // value g at y; d[15] = dg/dparam; dq[10] = dq/dparam (mu, quaternion, log scale)
  __device__ float at(const float y[3], float d[15], float dq[10]) const {
    float z[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) z[k] = R[0][k] * y[0] + R[1][k] * y[1] + R[2][k] * y[2];
    const float qq = z[0] * z[0] * is2[0] + z[1] * z[1] * is2[1] + z[2] * z[2] * is2[2];
    const float env = expf(-0.5f * qq);
    const float th = om.x * y[0] + om.y * y[1] + om.z * y[2] + phi;
    float sn, cs;
    sincosf(th, &sn, &cs);
    float dth[15], dA[15];
#pragma unroll
    for (int r = 0; r < 15; ++r) {
      dth[r] = 0.f;
      dA[r] = 0.f;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
      dq[a] = -2.f * (R[a][0] * z[0] * is2[0] + R[a][1] * z[1] * is2[1] + R[a][2] * z[2] * is2[2]);
    dth[0] = -om.x;
    dth[1] = -om.y;
    dth[2] = -om.z;
    // dz/d(qhat_l) = (dR/d qhat_l)^T y, written out from R(qhat); then through
    // qhat = q/|q|: dz/dq_m = (g_m - qhat_m sum_l qhat_l g_l) / |q|
    const float w = qh[0], x = qh[1], yq = qh[2], zq = qh[3];
    const float y0 = y[0], y1 = y[1], y2 = y[2];
    float g[4][3];
    g[0][0] = 2.f * (zq * y1 - yq * y2);
    g[0][1] = 2.f * (-zq * y0 + x * y2);
    g[0][2] = 2.f * (yq * y0 - x * y1);
    g[1][0] = 2.f * (yq * y1 + zq * y2);
    g[1][1] = 2.f * (yq * y0 - 2.f * x * y1 + w * y2);
    g[1][2] = 2.f * (zq * y0 - w * y1 - 2.f * x * y2);
    g[2][0] = 2.f * (-2.f * yq * y0 + x * y1 - w * y2);
    g[2][1] = 2.f * (x * y0 + zq * y2);
    g[2][2] = 2.f * (w * y0 + zq * y1 - 2.f * yq * y2);
    g[3][0] = 2.f * (-2.f * zq * y0 + w * y1 + x * y2);
    g[3][1] = 2.f * (-w * y0 - 2.f * zq * y1 + yq * y2);
    g[3][2] = 2.f * (x * y0 + yq * y1);
    float sg[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sg[k] = w * g[0][k] + x * g[1][k] + yq * g[2][k] + zq * g[3][k];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float dqm = 0.f, dthm = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float dz = (g[m][k] - qh[m] * sg[k]) * iqn;
        dqm += 2.f * z[k] * dz * is2[k];
        if (local) dthm += kin[k] / s[k] * dz;
      }
      dq[3 + m] = dqm;
      dth[3 + m] = dthm;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dq[7 + k] = -2.f * z[k] * z[k] * is2[k];
      if (local) dth[7 + k] = -kin[k] * z[k] / s[k];
      if (normalized) dA[7 + k] = -A;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) dth[10 + k] = local ? z[k] / s[k] : y[k];
    dth[13] = 1.f;
    dA[14] = dAdw;
#pragma unroll
    for (int r = 0; r < 15; ++r) {
      const float dqr = r < 10 ? dq[r] : 0.f;
      d[r] = A * env * (-0.5f * dqr * cs - sn * dth[r]) + dA[r] * env * cs;
    }
    return A * env * cs;
  }
};

__device__ __forceinline__ void add_grad(const BackArgs& B, int64_t i, const float acc[15],
                                         float scale) {
  const int64_t N = B.n;
  float* g = B.grad;
  for (int k = 0; k < 3; ++k) atomicAdd(g + 3 * i + k, scale * acc[k]);
  for (int k = 0; k < 4; ++k) atomicAdd(g + 3 * N + 4 * i + k, scale * acc[3 + k]);
  for (int k = 0; k < 3; ++k) atomicAdd(g + 7 * N + 3 * i + k, scale * acc[7 + k]);
  for (int k = 0; k < 3; ++k) atomicAdd(g + 10 * N + 3 * i + k, scale * acc[10 + k]);
  atomicAdd(g + 13 * N + i, scale * acc[13]);
  atomicAdd(g + 14 * N + i, scale * acc[14]);
}

struct BackLeaf {
  const DevField* F;
  const BackArgs* B;
  float3 o, v;
  float tmin, tmax;
  float dLdtau;
  const float* glx;
  const float* glw;
  unsigned long long nev = 0;
  __device__ void operator()(int j) {
    Prim P = load_prim(*F, j);
    Chord ch;
    // the support radius is a constant of the differentiation (adaptive extents too)
    if (!chord_setup(P, o, v, tmin, tmax, P.k2, ch)) return;
    const int64_t i = ch.orig;
    PrimDeriv D;
    D.init(*B, P, i);
    float acc[15];
    for (int r = 0; r < 15; ++r) acc[r] = 0.f;
    const float len = ch.dtout - ch.dtin;
    const float m = sqrtf(ch.a) * len + 0.5f * fabsf(ch.B) * len;
    const int rule = gl_rule(m);
    int n = gl_n(0), off = 0;
    for (int r = 0; r <= rule; ++r) {
      n = gl_n(r);
      off = gl_off(r);
    }
    const float mid = 0.5f * (ch.dtin + ch.dtout), hl = 0.5f * len;
    for (int k = 0; k < n; ++k) {
      const float dt = fmaf(hl, glx[off + k], mid), wq = hl * glw[off + k];
      const float y[3] = {fmaf(dt, v.x, ch.p.x), fmaf(dt, v.y, ch.p.y), fmaf(dt, v.z, ch.p.z)};
      float d[15], dq[10];
      D.at(y, d, dq);
      for (int r = 0; r < 15; ++r) acc[r] = fmaf(wq, d[r], acc[r]);
    }
    nev += (unsigned long long)n;
    // Leibniz terms where a chord end lies on the ellipsoid (not on tmin/tmax):
    // the end moves as dt/dtheta = -(dq/dtheta)/(dq/dt)
    const bool on_in = ch.dts - ch.hw > tmin - ch.tc, on_out = ch.dts + ch.hw < tmax - ch.tc;
    for (int e = 0; e < 2; ++e) {
      if (e == 0 ? !on_in : !on_out) continue;
      const float dt = e == 0 ? ch.dtin : ch.dtout, sgn = e == 0 ? -1.f : 1.f;
      const float y[3] = {fmaf(dt, v.x, ch.p.x), fmaf(dt, v.y, ch.p.y), fmaf(dt, v.z, ch.p.z)};
      float d[15], dq[10];
      const float g = D.at(y, d, dq);
      const float dqdt = -(v.x * dq[0] + v.y * dq[1] + v.z * dq[2]);
      if (dqdt != 0.f)
        for (int r = 0; r < 10; ++r) acc[r] += sgn * g * (-dq[r] / dqdt);
    }
    add_grad(*B, i, acc, dLdtau);
  }
};

// The primitives whose chords cross a ray under its mask, gathered by one
// traversal; the replay passes then visit the list instead of the tree.
constexpr int kRayList = 1024;
struct RayList {
  int* idx;    // this thread's first entry; entry k at idx[k * stride] (a warp's
  int stride;  // lanes hold neighbouring words: coalesced)
  int n;       // listed primitives; > kRayList: overflow, traverse instead
  __device__ bool ok() const { return n <= kRayList; }
  __device__ int at(int k) const { return idx[(int64_t)k * stride]; }
};

struct ListLeaf {
  const DevField* F;
  const Mask* M;
  float3 o, v;
  RayList* L;
  __device__ void operator()(int j) {
    const Mask& Mk = *M;
    Chord ch;
    float w;
    if (!prim_chord(*F, j, o, v, 0.f, INFINITY, [&](uint32_t c) { return mask_weight(Mk, c); }, w, ch))
      return;
    if (L->n < kRayList) L->idx[(int64_t)L->n * L->stride] = j;
    ++L->n;
  }
};

__device__ __forceinline__ void gather_list(const DevField& F, const Mask& M, float3 o, float3 v,
                                            RayList& L, Counters& cnt) {
  L.n = 0;
  const float3 inv = safe_inv(v);
  float t0, t1;
  if (M.bits == 0ull || !scene_span(F, o, inv, 0.f, INFINITY, t0, t1)) return;
  ListLeaf leaf{&F, &M, o, v, &L};
  SpanTest test{t0, t1};
  traverse_ray(F, o, inv, M.bits, test, leaf, cnt.nodes, cnt.leaves);
}

// every primitive of the list, or a traversal with `test` when it overflowed
template <class Test, class Leaf>
__device__ __forceinline__ void visit(const DevField& F, const RayList* L, float3 o, float3 inv,
                                      unsigned long long mask, Test& test, Leaf& leaf,
                                      Counters& cnt) {
  if (L && L->ok()) {
    for (int k = 0; k < L->n; ++k) leaf(L->at(k));
    cnt.leaves += (unsigned long long)L->n;
  } else {
    traverse_ray(F, o, inv, mask, test, leaf, cnt.nodes, cnt.leaves);
  }
}

constexpr int kBackBlock = 128;
struct BackSmem {
  float glx[kGLTotal], glw[kGLTotal];
};

// one pixel per lane (8x4 tiles per warp), samples in order
__global__ void __launch_bounds__(kBackBlock)
    k_tomo_backward(const __grid_constant__ DevField F, const PathParams P, const BackArgs Bk,
                    const float* dLdI, int* counter) {
  __shared__ BackSmem sm;
  for (int i = threadIdx.x; i < kGLTotal; i += blockDim.x) {
    sm.glx[i] = F.gl[i];
    sm.glw[i] = F.gl[kGLTotal + i];
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  Mask all;
  all.bits = F.occupied;
#pragma unroll
  for (int b = 0; b < 8; ++b) all.bw[b] = 1.f;
  Counters cnt;
  const int tiles_x = (P.cam.W + 7) / 8, tiles_y = (P.cam.H + 3) / 4;
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = atomicAdd(counter, 1);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= tiles_x * tiles_y) break;
    const int px = (tile % tiles_x) * 8 + (int)(lane % 8);
    const int py = (tile / tiles_x) * 4 + (int)(lane / 8);
    if (px >= P.cam.W || py >= P.cam.H) continue;  // every lane returns to the tile fetch
    const float gI = dLdI[(int64_t)py * P.cam.W + px];
    if (gI == 0.f) continue;
    for (int s = P.s0; s < P.s0 + P.spp; ++s) {
      float3 o, v;
      camera_ray(P.cam, P.seed, px, py, s, o, v);
      cnt.rays += 1;
      const float3 inv = safe_inv(v);
      float t0, t1;
      if (!scene_span(F, o, inv, 0.f, INFINITY, t0, t1)) continue;
      // forward optical depth, then the adjoint pass (two traversals: a primitive
      // list measured slower here, the Gauss-Legendre work dominating)
      const float tau = det_tau(F, all, o, v, 0.f, INFINITY, sm.glx, sm.glw, cnt);
      SpanTest test{t0, t1};
      BackLeaf leaf;
      leaf.F = &F;
      leaf.B = &Bk;
      leaf.o = o;
      leaf.v = v;
      leaf.tmin = 0.f;
      leaf.tmax = INFINITY;
      leaf.dLdtau = -gI * expf(-tau) / (float)P.spp;
      leaf.glx = sm.glx;
      leaf.glw = sm.glw;
      traverse_ray(F, o, inv, F.occupied, test, leaf, cnt.nodes, cnt.leaves);
      cnt.evals += leaf.nev;
    }
  }
  flush_counters(F, cnt, lane);
}


cudaError_t launch_tomo_backward(const Field& F, const PathParams& P, const float* dLdI,
                                 float* grad, cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  cudaError_t e = cudaMemsetAsync(F.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  BackArgs B;
  B.quat = F.p_quat;
  B.ls = F.p_ls;
  B.om = F.p_om;
  B.w = F.p_w;
  B.frame = F.opts.omega_frame;
  B.wmode = F.opts.weight_mode;
  B.n = F.n;
  B.grad = grad;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tomo_backward, kBackBlock, 0) != cudaSuccess)
    (void)cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  const int64_t tiles = (int64_t)((P.cam.W + 7) / 8) * ((P.cam.H + 3) / 4);
  const int64_t need = (tiles + kBackBlock / 32 - 1) / (kBackBlock / 32);
  int64_t g = (int64_t)F.ctx.sm_count * per_sm;
  if (need < g) g = need;
  if (g < 1) g = 1;
  k_tomo_backward<<<(unsigned)g, kBackBlock, 0, s>>>(F.dev, P, B, dLdI, F.counter);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint of the single-scattering radiance.
//
// Per camera sample, the expected-value form of delta tracking over all
// tentative points t_j of the camera ray (Poisson process of rate kappa_bar):
//   I = sum_j W_j G(t_j),   W_j = prod_{i<j} (1 - p_i) p_j,   p = kappa+/kappa_bar,
// has the mean of the delta-tracking estimator (Sec. 3, Eq. 4 majorants; the
// points before t form a Poisson process independent of the point at t).  One
// point js is drawn with probability W_j / sum W by weighted reservoir
// sampling in t order (point j replaces the candidate when u_j S_j < W_j, u_j
// its own second uniform, S_j the running sum), and G(t_js) = albedo E/(4 pi)
// T_light comes from ratio tracking of the NEE ray, so a sample is S G.  The
// derivative holds the points, kappa_bar and the draw probabilities fixed:
//   d/d p_i = S G / (1 - p_i) * (-1)  (i < js),   S G / p_js  (i = js),
//   d/d q_k = -S albedo E/(4 pi) T_light / (1 - q_k)   (NEE points),
// and d p / d theta = 1[kappa > 0] d kappa/d theta / kappa_bar, where
// d kappa/d theta sums the mask-weighted derivatives of the kernels covering
// the point.  Each ray is re-tracked (same Philox streams, same windows) for
// the derivative passes: nothing per path is stored.
// ---------------------------------------------------------------------------

// Windows of kPts tentative points, in t order, with kappa and kappa_bar
// (the windows of track()); win(B, n, kap, kb) returns false to stop.
template <class Win>
__device__ void for_windows(const DevField& F, const Mask& M, float3 o, float3 v, uint64_t seed,
                            uint32_t ray, uint32_t word, const float* env, Counters& cnt,
                            const RayList* L, Win win) {
  const unsigned am = __activemask();
  const float3 inv = safe_inv(v);
  float t0 = 0.f, t1 = 0.f;
  bool more = M.bits != 0ull && scene_span(F, o, inv, 0.f, INFINITY, t0, t1);
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
    CollectLeaf cl;
    cl.F = &F;
    cl.M = &M;
    cl.o = o;
    cl.v = v;
    cl.tmin = 0.f;
    cl.tmax = INFINITY;
    cl.ta = ta;
    cl.first = first;
    cl.bound = t1;
    cl.B = &B;
    cl.seed = seed;
    cl.ray = ray;
    cl.word = word;
    cl.env = env;
    CollectTest ctest{&cl.ta, &cl.bound};
    visit(F, L, o, inv, M.bits, ctest, cl, cnt);
    int n = 0;
#pragma unroll
    for (int i = 0; i < kPts; ++i) n += B.t[i] < INFINITY ? 1 : 0;
    if (n == 0) {
      more = false;
      continue;
    }
    AccumLeaf al;
    al.F = &F;
    al.M = &M;
    al.o = o;
    al.v = v;
    al.tmin = 0.f;
    al.tmax = INFINITY;
    al.B = &B;
    al.n = n;
    al.env = env;
#pragma unroll
    for (int i = 0; i < kPts; ++i) {
      al.kap[i] = 0.f;
      al.kb[i] = 0.f;
    }
    PointTest ptest{&B, n};
    visit(F, L, o, inv, M.bits, ptest, al, cnt);
    cnt.evals += al.nev;
    if (!win(B, n, al.kap, al.kb) || n < kPts) {
      more = false;
      continue;
    }
    ta = B.t[kPts - 1];
    first = false;
  }
}

// coef_i * d kappa(x(t_i)) / d theta, scattered over the kernels at the points
struct RadScatter {
  const DevField* F;
  const BackArgs* B;
  const Mask* M;
  float3 o, v;
  const PointBuf* P;
  const float* coef;
  int n;
  __device__ void operator()(int j) {
    const Prim Pr = load_prim(*F, j);
    Chord ch;
    if (!chord_setup(Pr, o, v, 0.f, INFINITY, Pr.k2, ch)) return;
    const float w = mask_weight(*M, ch.cell);
    if (w == 0.f) return;
    const float tin = ch.tc + ch.dtin, tout = ch.tc + ch.dtout;
    bool any = false;
#pragma unroll
    for (int i = 0; i < kPts; ++i)
      any |= i < n && coef[i] != 0.f && P->t[i] >= tin && P->t[i] <= tout;
    if (!any) return;
    PrimDeriv D;
    D.init(*B, Pr, ch.orig);
    float acc[15];
    for (int r = 0; r < 15; ++r) acc[r] = 0.f;
    for (int i = 0; i < n; ++i) {
      const float t = P->t[i];
      if (coef[i] == 0.f || t < tin || t > tout) continue;
      const float dt = t - ch.tc;
      const float y[3] = {fmaf(dt, v.x, ch.p.x), fmaf(dt, v.y, ch.p.y), fmaf(dt, v.z, ch.p.z)};
      float d[15], dq[10];
      D.at(y, d, dq);
      for (int r = 0; r < 15; ++r) acc[r] = fmaf(coef[i], d[r], acc[r]);
    }
    add_grad(*B, ch.orig, acc, w);
  }
};

__device__ __forceinline__ void scatter_window(const DevField& F, const BackArgs& Bk, const Mask& M,
                                               float3 o, float3 v, const PointBuf& P,
                                               const float* coef, int n, const RayList* L,
                                               Counters& cnt) {
  bool any = false;
#pragma unroll
  for (int i = 0; i < kPts; ++i) any |= i < n && coef[i] != 0.f;
  if (!any) return;
  RadScatter rs{&F, &Bk, &M, o, v, &P, coef, n};
  PointTest ptest{&P, n};
  visit(F, L, o, safe_inv(v), M.bits, ptest, rs, cnt);
}

struct RadSmem {
  float env[8];
};

// ---------------------------------------------------------------------------
// Adjoint of the multiple-scattering radiance (max_bounces >= 2).
//
// The delta-tracking path: segment b accepts its first tentative point js_b
// (probability P_b = prod_{i<js} (1 - p_i) p_js) or escapes; the collision
// x_{b+1} adds C_b = thr_b E0 T_b with thr_b = albedo^(b+1), E0 = E/(4 pi) and
// T_b the ratio-tracked NEE product prod_k (1 - q_k).  C_b depends on the
// segments 0..b and on NEE b, so with the points and majorants held fixed
//   d E[L] = E[ sum_b S_b d log P_b + sum_b C_b d log T_b ],  S_b = sum_{b'>=b} C_b',
//   d log P_b = sum_{i<js} -dp_i / (1 - p_i) + dp_js / p_js,
//   C_b d log T_b = -thr_b E0 sum_k dq_k T_b / (1 - q_k),
// dp = 1[kappa > 0] d kappa / kappa_bar.  Pass 1 follows the path (the
// renderer's streams and decisions) and keeps only T_b per collision; pass 2
// follows it again, scattering each segment's points up to the accepted one
// and each NEE ray's points with those coefficients.  Nothing per tentative
// point or per segment ray is stored.
// ---------------------------------------------------------------------------
constexpr int kMaxSeg = 15;

// one segment of the path from (o, v): delta tracking to the first accepted
// point (returns false on escape, else t); with coefficients (S != 0), the
// points up to the accepted one are scattered, -S/(1 - p) before it, S/p at it
__device__ __forceinline__ bool path_segment(const DevField& F, const PathParams& P,
                                             const BackArgs& Bk, float3 o, float3 v,
                                             uint32_t pix, uint32_t s, int b, float S,
                                             const float* env, Counters& cnt, RayList& L,
                                             float& th) {
  const Mask M = sample_mask_impl<true>(F, P.lod, v, P.seed, pix, s, (uint32_t)b, TAG_MASK);
  const uint32_t wt = stream_word(s, (uint32_t)b, TAG_TRACK);
  gather_list(F, M, o, v, L, cnt);
  bool hit = false;
  for_windows(F, M, o, v, P.seed, pix, wt, env, cnt, &L,
              [&](const PointBuf& B, int n, const float* kap, const float* kb) {
                float coef[kPts];
                int acc = -1;
#pragma unroll
                for (int i = 0; i < kPts; ++i) {
                  coef[i] = 0.f;
                  if (i < n && acc < 0) {
                    const bool take = B.u[i] * kb[i] < fmaxf(kap[i], 0.f);
                    if (S != 0.f && kap[i] > 0.f && kb[i] > 0.f) {
                      const float p = kap[i] / kb[i];
                      coef[i] = (take ? S / p : -S / (1.f - p)) / kb[i];
                    }
                    if (take) acc = i;
                  }
                }
                if (S != 0.f) scatter_window(F, Bk, M, o, v, B, coef, n, &L, cnt);
                if (acc >= 0) {
                  hit = true;
                  th = B.t[acc];
                  return false;
                }
                return true;
              });
  return hit;
}

// NEE ray of collision b from x: returns T = prod (1 - q_k); with cn != 0 the
// points are scattered with cn / (1 - q_k) / kappa_bar_k
__device__ __forceinline__ float path_nee(const DevField& F, const PathParams& P,
                                          const BackArgs& Bk, float3 x, uint32_t pix,
                                          uint32_t s, int b, float cn, const float* env,
                                          Counters& cnt, RayList& L) {
  const Mask Mn = sample_mask_impl<true>(F, P.lod_nee, P.light, P.seed, pix, s, (uint32_t)b,
                                         TAG_NEE_MASK);
  const uint32_t wn = stream_word(s, (uint32_t)b, TAG_NEE);
  gather_list(F, Mn, x, P.light, L, cnt);
  float Tl = 1.f;
  for_windows(F, Mn, x, P.light, P.seed, pix, wn, env, cnt, &L,
              [&](const PointBuf& B, int n, const float* kap, const float* kb) {
                float coef[kPts];
#pragma unroll
                for (int i = 0; i < kPts; ++i) {
                  coef[i] = 0.f;
                  if (i < n && kb[i] > 0.f) {
                    const float q = fmaxf(kap[i], 0.f) / kb[i];
                    Tl *= 1.f - q;
                    if (cn != 0.f && kap[i] > 0.f && 1.f - q > 0.f) coef[i] = cn / (1.f - q) / kb[i];
                  }
                }
                if (cn != 0.f) scatter_window(F, Bk, Mn, x, P.light, B, coef, n, &L, cnt);
                return true;
              });
  return Tl;
}

__device__ __forceinline__ float3 path_scatter_dir(const PathParams& P, uint32_t pix, uint32_t s,
                                                   int b) {
  const uint4 y = rng4(P.seed, 0, kNoPrim, pix, stream_word(s, (uint32_t)b, TAG_SCATTER));
  const float z = 1.0f - 2.0f * u01(y.x);
  const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
  float sn, cs;
  sincosf(2.0f * 3.14159265358979f * u01(y.y), &sn, &cs);
  return make_float3(rr * cs, rr * sn, z);
}

__device__ void path_backward(const DevField& F, const PathParams& P, const BackArgs& Bk,
                              float3 o0, float3 v0, uint32_t pix, uint32_t s, float base,
                              const float* env, Counters& cnt, RayList& Lc, RayList& Ln) {
  const float E0 = P.irradiance * (0.25f / 3.14159265358979f);
  float Tb[kMaxSeg];
  int nseg = 0;
  // pass 1: the path, its NEE products
  {
    float3 o = o0, v = v0;
    for (int b = 0; b < P.max_bounces && b < kMaxSeg; ++b) {
      float th = 0.f;
      cnt.rays += 1;
      if (!path_segment(F, P, Bk, o, v, pix, s, b, 0.f, env, cnt, Lc, th)) break;
      const float3 x = make_float3(fmaf(th, v.x, o.x), fmaf(th, v.y, o.y), fmaf(th, v.z, o.z));
      cnt.rays += 1;
      Tb[nseg++] = path_nee(F, P, Bk, x, pix, s, b, 0.f, env, cnt, Ln);
      o = x;
      v = path_scatter_dir(P, pix, s, b);
    }
  }
  if (nseg == 0) return;
  // S_b = sum_{b' >= b} C_b', C_b = albedo^(b+1) E0 T_b
  float Ssuf = 0.f, thr = 1.f;
  for (int b = 0; b < nseg; ++b) {
    thr *= P.albedo;
    Ssuf += thr * E0 * Tb[b];
  }
  // pass 2: the same path again, scattering the coefficients
  float3 o = o0, v = v0;
  thr = 1.f;
  for (int b = 0; b < nseg; ++b) {
    float th = 0.f;
    if (!path_segment(F, P, Bk, o, v, pix, s, b, base * Ssuf, env, cnt, Lc, th)) break;
    const float3 x = make_float3(fmaf(th, v.x, o.x), fmaf(th, v.y, o.y), fmaf(th, v.z, o.z));
    thr *= P.albedo;
    const float Cb = thr * E0 * Tb[b];
    if (Tb[b] > 0.f) (void)path_nee(F, P, Bk, x, pix, s, b, -base * Cb, env, cnt, Ln);
    Ssuf -= Cb;
    o = x;
    v = path_scatter_dir(P, pix, s, b);
  }
}

// PATH = false: single scattering (the expected-value estimator above);
// PATH = true: multiple scattering (path_backward), each with its own frame
template <bool PATH>
__global__ void __launch_bounds__(kBackBlock)
    k_radiance_backward(const __grid_constant__ DevField F, const PathParams P, const BackArgs Bk,
                        const float* dLdI, int* counter, int* lists) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  RayList Lc{lists + tid, nth, 0}, Ln{lists + (int64_t)kRayList * nth + tid, nth, 0};
  __shared__ RadSmem sm;
  if (threadIdx.x < 8) sm.env[threadIdx.x] = F.env[threadIdx.x];
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  Counters cnt;
  const float E = P.albedo * P.irradiance * (0.25f / 3.14159265358979f);
  const int tiles_x = (P.cam.W + 7) / 8, tiles_y = (P.cam.H + 3) / 4;
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = atomicAdd(counter, 1);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= tiles_x * tiles_y) break;
    const int px = (tile % tiles_x) * 8 + (int)(lane % 8);
    const int py = (tile / tiles_x) * 4 + (int)(lane / 8);
    if (px >= P.cam.W || py >= P.cam.H) continue;  // every lane returns to the tile fetch
    const uint32_t pix = (uint32_t)(py * P.cam.W + px);
    const float gI = dLdI[pix];
    if (gI == 0.f) continue;
    const float base = gI / (float)P.spp;
    for (int s = P.s0; s < P.s0 + P.spp; ++s) {
      float3 o, v;
      camera_ray(P.cam, P.seed, px, py, s, o, v);
      if constexpr (PATH) {
        path_backward(F, P, Bk, o, v, pix, (uint32_t)s, base, sm.env, cnt, Lc, Ln);
        continue;
      }
      cnt.rays += 1;
      const Mask M = sample_mask_impl<true>(F, P.lod, v, P.seed, pix, (uint32_t)s, 0, TAG_MASK);
      const uint32_t wt = stream_word((uint32_t)s, 0, TAG_TRACK);
      gather_list(F, M, o, v, Lc, cnt);
      // pass 1: weights, their sum and the reservoir draw
      float Pr = 1.f, S = 0.f, pjs = 0.f, tjs = 0.f;
      int idx = 0, js = -1;
      for_windows(F, M, o, v, P.seed, pix, wt, sm.env, cnt, &Lc,
                  [&](const PointBuf& B, int n, const float* kap, const float* kb) {
                    for (int i = 0; i < n; ++i) {
                      const float p = kb[i] > 0.f ? fmaxf(kap[i], 0.f) / kb[i] : 0.f;
                      const float W = Pr * p;
                      S += W;
                      if (W > 0.f && B.u[i] * S < W) {
                        js = idx + i;
                        pjs = p;
                        tjs = B.t[i];
                      }
                      Pr *= 1.f - p;
                    }
                    idx += n;
                    return true;
                  });
      if (js < 0 || !(S > 0.f)) continue;
      // NEE from the drawn point by ratio tracking
      const float3 x = make_float3(fmaf(tjs, v.x, o.x), fmaf(tjs, v.y, o.y), fmaf(tjs, v.z, o.z));
      const Mask Mn = sample_mask_impl<true>(F, P.lod_nee, P.light, P.seed, pix, (uint32_t)s, 0, TAG_NEE_MASK);
      const uint32_t wn = stream_word((uint32_t)s, 0, TAG_NEE);
      cnt.rays += 1;
      gather_list(F, Mn, x, P.light, Ln, cnt);
      // ratio tracking of the NEE ray, T = prod (1 - kappa+/kappa_bar)
      float Tl = 1.f;
      for_windows(F, Mn, x, P.light, P.seed, pix, wn, sm.env, cnt, &Ln,
                  [&](const PointBuf& B, int n, const float* kap, const float* kb) {
                    for (int i = 0; i < n; ++i)
                      if (kb[i] > 0.f) Tl *= 1.f - fmaxf(kap[i], 0.f) / kb[i];
                    return true;
                  });
      const float G = E * Tl;
      // pass 2: camera points 0..js
      idx = 0;
      for_windows(F, M, o, v, P.seed, pix, wt, sm.env, cnt, &Lc,
                  [&](const PointBuf& B, int n, const float* kap, const float* kb) {
                    float coef[kPts];
#pragma unroll
                    for (int i = 0; i < kPts; ++i) {
                      coef[i] = 0.f;
                      const int gi = idx + i;
                      if (i < n && gi <= js && kap[i] > 0.f && kb[i] > 0.f) {
                        const float p = kap[i] / kb[i];
                        const float c = gi == js ? S * G / pjs : -S * G / (1.f - p);
                        coef[i] = base * c / kb[i];
                      }
                    }
                    scatter_window(F, Bk, M, o, v, B, coef, n, &Lc, cnt);
                    idx += n;
                    return idx <= js;
                  });
      // pass 3: NEE points
      if (Tl > 0.f) {
        for_windows(F, Mn, x, P.light, P.seed, pix, wn, sm.env, cnt, &Ln,
                    [&](const PointBuf& B, int n, const float* kap, const float* kb) {
                      float coef[kPts];
#pragma unroll
                      for (int i = 0; i < kPts; ++i) {
                        coef[i] = 0.f;
                        if (i < n && kap[i] > 0.f && kb[i] > 0.f) {
                          const float q = kap[i] / kb[i];
                          if (1.f - q > 0.f) coef[i] = -base * S * E * Tl / (1.f - q) / kb[i];
                        }
                      }
                      scatter_window(F, Bk, Mn, x, P.light, B, coef, n, &Ln, cnt);
                      return true;
                    });
      }
    }
  }
  flush_counters(F, cnt, lane);
}

static BackArgs back_args(const Field& F, float* grad) {
  BackArgs B;
  B.quat = F.p_quat;
  B.ls = F.p_ls;
  B.om = F.p_om;
  B.w = F.p_w;
  B.frame = F.opts.omega_frame;
  B.wmode = F.opts.weight_mode;
  B.n = F.n;
  B.grad = grad;
  return B;
}

// per-thread primitive lists of the radiance adjoint (2 per thread of a full
// persistent grid), grown through the field's allocator
cudaError_t ensure_adjoint_lists(const Field& F, cudaStream_t s) {
  int per_sm = 0;
  for (auto k : {k_radiance_backward<false>, k_radiance_backward<true>}) {
    int q = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k, kBackBlock, 0) != cudaSuccess)
      (void)cudaGetLastError();
    per_sm = q > per_sm ? q : per_sm;
  }
  if (per_sm < 1) per_sm = 1;
  const int64_t threads = (int64_t)F.ctx.sm_count * per_sm * kBackBlock;
  return grow(F, (void**)&F.rlist, F.rlist_bytes, (size_t)threads * 2 * kRayList * sizeof(int), s);
}

cudaError_t launch_radiance_backward(const Field& F, const PathParams& P, const float* dLdI,
                                     float* grad, cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  cudaError_t e = cudaMemsetAsync(F.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const BackArgs B = back_args(F, grad);
  auto kernel = P.max_bounces >= 2 ? k_radiance_backward<true> : k_radiance_backward<false>;
  // the kernel's local frame must fit the context's stack limit as it stands
  cudaFuncAttributes fa;
  size_t limit = 0;
  if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetLimit(&limit, cudaLimitStackSize)) != cudaSuccess) return e;
  if (fa.localSizeBytes > limit) return cudaErrorLaunchOutOfResources;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBackBlock, 0) != cudaSuccess)
    (void)cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  const int64_t tiles = (int64_t)((P.cam.W + 7) / 8) * ((P.cam.H + 3) / 4);
  const int64_t need = (tiles + kBackBlock / 32 - 1) / (kBackBlock / 32);
  int64_t g = (int64_t)F.ctx.sm_count * per_sm;
  if (need < g) g = need;
  if (g < 1) g = 1;
  // lists sized for a full grid (allocated ahead by gf_reserve, else here)
  if ((e = ensure_adjoint_lists(F, s)) != cudaSuccess) return e;
  kernel<<<(unsigned)g, kBackBlock, 0, s>>>(F.dev, P, B, dLdI, F.counter, F.rlist);
  return cudaGetLastError();
}

}  // namespace gf
