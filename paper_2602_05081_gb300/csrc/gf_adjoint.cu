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
    if (!chord_setup(P, o, v, tmin, tmax, F->k2, ch)) return;
    const int64_t i = ch.orig;
    // raw parameters of primitive i
    float q[4];
    for (int k = 0; k < 4; ++k) q[k] = B->quat[4 * i + k];
    float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    float qw = q[0] / qn, qx = q[1] / qn, qy = q[2] / qn, qz = q[3] / qn;
    float R[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                     {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                     {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
    // dR/d(qhat_m), m = w, x, y, z
    float dRh[4][3][3] = {
        {{0.f, -2.f * qz, 2.f * qy}, {2.f * qz, 0.f, -2.f * qx}, {-2.f * qy, 2.f * qx, 0.f}},
        {{0.f, 2.f * qy, 2.f * qz}, {2.f * qy, -4.f * qx, -2.f * qw}, {2.f * qz, 2.f * qw, -4.f * qx}},
        {{-4.f * qy, 2.f * qx, 2.f * qw}, {2.f * qx, 0.f, 2.f * qz}, {-2.f * qw, 2.f * qz, -4.f * qy}},
        {{-4.f * qz, -2.f * qw, 2.f * qx}, {2.f * qw, -4.f * qz, 2.f * qy}, {2.f * qx, 2.f * qy, 0.f}}};
    float qh[4] = {qw, qx, qy, qz};
    float s[3], is2[3], kin[3];
    for (int k = 0; k < 3; ++k) {
      s[k] = expf(B->ls[3 * i + k]);
      is2[k] = 1.f / (s[k] * s[k]);
      kin[k] = B->om[3 * i + k];
    }
    const bool local = B->frame == GF_OMEGA_LOCAL;
    const float A = P.A, wgt = B->w[i];
    // dA/dweight
    const float dAdw = B->wmode == GF_WEIGHT_NORMALIZED ? A / wgt : 1.f;
    float acc[15];
    for (int r = 0; r < 15; ++r) acc[r] = 0.f;
    // per-point derivatives at offset y = p + dt v
    auto point = [&](float dt, float wq, bool endpoint, float sgn) {
      float y[3] = {fmaf(dt, v.x, ch.p.x), fmaf(dt, v.y, ch.p.y), fmaf(dt, v.z, ch.p.z)};
      float z[3];
      for (int k = 0; k < 3; ++k) z[k] = R[0][k] * y[0] + R[1][k] * y[1] + R[2][k] * y[2];
      float qq = z[0] * z[0] * is2[0] + z[1] * z[1] * is2[1] + z[2] * z[2] * is2[2];
      float env = expf(-0.5f * qq);
      float th = P.om.x * y[0] + P.om.y * y[1] + P.om.z * y[2] + P.phi;
      float sn, cs;
      sincosf(th, &sn, &cs);
      float dq[10], dth[15], dA[15];
      for (int r = 0; r < 15; ++r) {
        dth[r] = 0.f;
        dA[r] = 0.f;
      }
      // mu
      for (int a = 0; a < 3; ++a) {
        dq[a] = -2.f * (R[a][0] * z[0] * is2[0] + R[a][1] * z[1] * is2[1] + R[a][2] * z[2] * is2[2]);
      }
      dth[0] = -P.om.x;
      dth[1] = -P.om.y;
      dth[2] = -P.om.z;
      // quaternion (through qhat = q/|q|)
      for (int m = 0; m < 4; ++m) {
        float dqm = 0.f, dthm = 0.f;
        for (int k = 0; k < 3; ++k) {
          float dz = 0.f;
          for (int a = 0; a < 3; ++a) {
            float dR = 0.f;
            for (int l = 0; l < 4; ++l) dR += dRh[l][a][k] * ((l == m ? 1.f : 0.f) - qh[l] * qh[m]);
            dz += dR / qn * y[a];
          }
          dqm += 2.f * z[k] * dz * is2[k];
          if (local) dthm += kin[k] / s[k] * dz;
        }
        dq[3 + m] = dqm;
        dth[3 + m] = dthm;
      }
      // log scale
      for (int k = 0; k < 3; ++k) {
        dq[7 + k] = -2.f * z[k] * z[k] * is2[k];
        if (local) dth[7 + k] = -kin[k] * z[k] / s[k];
        if (B->wmode == GF_WEIGHT_NORMALIZED) dA[7 + k] = -A;
      }
      for (int k = 0; k < 3; ++k) dth[10 + k] = local ? z[k] / s[k] : y[k];
      dth[13] = 1.f;
      dA[14] = dAdw;
      if (!endpoint) {
        for (int r = 0; r < 15; ++r) {
          float dqr = r < 10 ? dq[r] : 0.f;
          acc[r] = fmaf(wq, A * env * (-0.5f * dqr * cs - sn * dth[r]) + dA[r] * env * cs, acc[r]);
        }
      } else {
        float g = A * env * cs;
        float dqdt = -(v.x * dq[0] + v.y * dq[1] + v.z * dq[2]);
        if (dqdt != 0.f)
          for (int r = 0; r < 10; ++r) acc[r] += sgn * g * (-dq[r] / dqdt);
      }
    };
    float len = ch.dtout - ch.dtin;
    float m = sqrtf(ch.a) * len + 0.5f * fabsf(ch.B) * len;
    int rule = gl_rule(m);
    int n = gl_n(0), off = 0;
    for (int r = 0; r <= rule; ++r) {
      n = gl_n(r);
      off = gl_off(r);
    }
    float mid = 0.5f * (ch.dtin + ch.dtout), hl = 0.5f * len;
    for (int k = 0; k < n; ++k) point(fmaf(hl, glx[off + k], mid), hl * glw[off + k], false, 0.f);
    nev += (unsigned long long)n;
    // Leibniz terms where a chord end lies on the ellipsoid (not on tmin/tmax)
    if (ch.dts - ch.hw > tmin - ch.tc) point(ch.dtin, 0.f, true, -1.f);
    if (ch.dts + ch.hw < tmax - ch.tc) point(ch.dtout, 0.f, true, 1.f);
    const int64_t N = B->n;
    float* g = B->grad;
    for (int k = 0; k < 3; ++k) atomicAdd(g + 3 * i + k, dLdtau * acc[k]);
    for (int k = 0; k < 4; ++k) atomicAdd(g + 3 * N + 4 * i + k, dLdtau * acc[3 + k]);
    for (int k = 0; k < 3; ++k) atomicAdd(g + 7 * N + 3 * i + k, dLdtau * acc[7 + k]);
    for (int k = 0; k < 3; ++k) atomicAdd(g + 10 * N + 3 * i + k, dLdtau * acc[10 + k]);
    atomicAdd(g + 13 * N + i, dLdtau * acc[13]);
    atomicAdd(g + 14 * N + i, dLdtau * acc[14]);
  }
};

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
    for (int s = 0; s < P.spp; ++s) {
      float3 o, v;
      camera_ray(P.cam, P.seed, px, py, s, o, v);
      cnt.rays += 1;
      const float tau = det_tau(F, all, o, v, 0.f, INFINITY, sm.glx, sm.glw, cnt);
      const float3 inv = safe_inv(v);
      float t0, t1;
      if (!scene_span(F, o, inv, 0.f, INFINITY, t0, t1)) continue;
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
      SpanTest test{t0, t1};
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
  k_tomo_backward<<<(unsigned)(g < 1 ? 1 : g), kBackBlock, 0, s>>>(F.dev, P, B, dLdI, F.counter);
  return cudaGetLastError();
}

}  // namespace gf
