// gf_kernels.cu -- render, transmittance and test kernels of the Gabor-field
// renderer.  Persistent warps pull work tiles from a global counter: 32 rays,
// or an 8x4 block of pixels, per warp, each lane owning one ray or pixel
// (gf_trace.cuh); small transmittance batches take one ray per warp instead,
// the whole warp traversing and integrating it together.
#include <cuda_runtime.h>

#include "gf_host.h"
#include "gf_trace.cuh"

namespace gf {

constexpr int kBlock = 128;
constexpr int kTileW = 8, kTileH = 4;

struct BlockTables {
  float glx[kGLTotal], glw[kGLTotal];
  float env[8];
};

__device__ __forceinline__ void init_tables(BlockTables& sm, const DevField& F) {
  for (int i = threadIdx.x; i < kGLTotal; i += blockDim.x) {
    sm.glx[i] = F.gl[i];
    sm.glw[i] = F.gl[kGLTotal + i];
  }
  if (threadIdx.x < 8) sm.env[threadIdx.x] = F.env[threadIdx.x];
  __syncthreads();
}

__device__ __forceinline__ int next_tile(int* counter, uint32_t lane) {
  int it = 0;
  if (lane == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(kFull, it, 0);
}

// ---------------------------------------------------------------------------
// transmittance: deterministic optical depth (Gauss-Legendre quadrature or
// closed-form chord integrals) or ratio tracking, one ray per lane
// ---------------------------------------------------------------------------
template <int MODE>  // GF_TR_DETERMINISTIC, GF_TR_RATIO_TRACKING or GF_TR_CLOSED_FORM
__global__ void __launch_bounds__(kBlock, 3)  // at most 168 registers: 12 warps per SM
    k_transmittance(const __grid_constant__ DevField F, const TrParams P) {
  constexpr bool TRACK = MODE == GF_TR_RATIO_TRACKING;
  __shared__ BlockTables sm;
  init_tables(sm, F);
  const uint32_t lane = threadIdx.x & 31u;
  Counters cnt;
  const bool det_mask = lod_is_deterministic(P.lod);
  // deterministic modes: G = P.group lanes per ray, each walking its own part of
  // the tree (group_start), 32/G rays per tile
  const int G = TRACK ? 1 : P.group;
  const int rpt = 32 / G;
  const int sub = (int)lane % G;
  for (;;) {
    const int tile = next_tile(P.counter, lane);
    if ((int64_t)tile * rpt >= P.n) break;
    const int64_t r = (int64_t)tile * rpt + (int)lane / G;
    if (!TRACK) {
      float s_acc = 0.f, c_acc = 0.f;
      const int spp = det_mask ? 1 : P.spp;
      if (r < P.n) {
        const float3 o = make_float3(P.o[3 * r], P.o[3 * r + 1], P.o[3 * r + 2]);
        const float3 v = unit_dir(make_float3(P.d[3 * r], P.d[3 * r + 1], P.d[3 * r + 2]));
        const float tmin = P.trange ? P.trange[2 * r] : 0.f;
        const float tmax = P.trange ? P.trange[2 * r + 1] : INFINITY;
        for (int s = 0; s < spp; ++s) {
          const Mask m = sample_mask(F, P.lod, v, P.seed, (uint32_t)r, (uint32_t)s, 0, TAG_MASK);
          if (sub == 0) cnt.rays += 1;
          neumaier_add(s_acc, c_acc,
                       MODE == GF_TR_CLOSED_FORM
                           ? closed_tau(F, m, o, v, tmin, tmax, cnt, sub, G)
                           : det_tau(F, m, o, v, tmin, tmax, sm.glx, sm.glw, cnt, sub, G));
        }
      }
      // compensated sum over the ray's G lanes (fixed butterfly order)
      for (int off = 1; off < G; off <<= 1) {
        const float so = __shfl_xor_sync(kFull, s_acc, off), co = __shfl_xor_sync(kFull, c_acc, off);
        float t, e;
        two_sum(s_acc, so, t, e);
        s_acc = t;
        c_acc = __fadd_rn(__fadd_rn(c_acc, co), e);
      }
      if (r < P.n && sub == 0) {
        const float tau = __fadd_rn(s_acc, c_acc) / (float)spp;
        P.out_T[r] = expf(-tau);
        if (P.out_tau) P.out_tau[r] = tau;
      }
    } else if (r < P.n) {
      const float3 o = make_float3(P.o[3 * r], P.o[3 * r + 1], P.o[3 * r + 2]);
      const float3 v = unit_dir(make_float3(P.d[3 * r], P.d[3 * r + 1], P.d[3 * r + 2]));
      const float tmin = P.trange ? P.trange[2 * r] : 0.f;
      const float tmax = P.trange ? P.trange[2 * r + 1] : INFINITY;
      {
        float acc = 0.f;
        for (int s = 0; s < P.spp; ++s) {
          const Mask m = sample_mask(F, P.lod, v, P.seed, (uint32_t)r, (uint32_t)s, 0, TAG_MASK);
          cnt.rays += 1;
          acc += track<false>(F, m, o, v, tmin, tmax, false, P.seed, (uint32_t)r,
                              stream_word((uint32_t)s, 0, TAG_TRACK), sm.env, cnt, nullptr);
        }
        P.out_T[r] = acc / (float)P.spp;
      }
    }
  }
  flush_counters(F, cnt, lane);
}

// ---------------------------------------------------------------------------
// Deterministic optical depth of small batches, one ray per warp.  The warp
// traverses the ray's tree together (a shared stack of binary nodes, up to 32
// per step) and sets up the chords of the leaves it reaches 32 at a time.
// Gauss-Legendre mode: the nodes of those chords are shared out evenly among
// the lanes (the rule per chord as in det_tau); closed form: each lane
// integrates its own chord.  Every term goes into its lane's compensated sum;
// the lanes' sums are combined in a fixed butterfly order.
// ---------------------------------------------------------------------------
constexpr int kCoopStack = 512;   // node entries per warp
constexpr int kCoopMargin = 128;  // a step pushes <= 64; depth first above kCoopStack - margin
constexpr int kCoopLeafQ = 96;    // <= 31 left + 64 new
struct CoopTrav {
  int stk[kCoopStack];
  int lq[kCoopLeafQ];
};
struct CoopChord {
  float mid, hl, y2, y1, y0, scale, B, delta;
  int off;  // first node of the chord's rule in the tables
};
struct CoopQ {
  CoopTrav t;
  CoopChord ch[32];  // the round's chords, one per lane
  int end[33];       // end[c]: nodes of chords 0..c-1
};

// The tree of one ray, traversed by the whole warp: a shared stack of binary
// nodes (up to 32 popped per step, their hit children pushed), the leaves
// reached queued; every 32 queued leaves (and the last ones) make a round, in
// which round(j) is called by every lane, j the sorted primitive of the lane's
// leaf or -1.
template <class Round>
__device__ void coop_traverse(const DevField& F, CoopTrav& Q, const Mask& M, float3 o, float3 inv,
                              float t0, float t1, uint32_t lane, Counters& cnt, Round&& round) {
  const unsigned lt = (1u << lane) - 1u;
  const SpanTest test{t0, t1};
  int sp = F.root >= 0 ? 1 : 0, lq_n = F.root >= 0 ? 0 : 1;
  if (lane == 0) {
    if (F.root >= 0) Q.stk[0] = F.root;
    else Q.lq[0] = 0;  // a one-primitive field has no internal node
  }
  __syncwarp();
  // every internal node enters the stack at most once
  const long long max_it = F.n + 64;
  for (long long it = 0;; ++it) {
    if (it > max_it) {
      if (lane == 0) set_err(F, ERR_GUARD);
      break;
    }
    int take = sp < 32 ? sp : 32;
    if (sp > kCoopStack - kCoopMargin) take = 1;  // near capacity: depth first
    const int node = (int)lane < take ? Q.stk[sp - take + (int)lane] : -1;
    __syncwarp();
    sp -= take;
    int c0 = 0, c1 = 0;
    bool h0 = false, h1 = false;
    if (node >= 0 && (int64_t)node >= F.n - 1) {  // internal nodes 0 .. n-2
      set_err(F, ERR_INDEX);
    } else if (node >= 0) {
      const Node* N = F.nodes + node;
      const float4 a = __ldg(&N->a), b = __ldg(&N->b), c = __ldg(&N->c);
      const int4 d = __ldg(&N->d);
      const uint4 e = __ldg(&N->e);
      ++cnt.nodes;
      const unsigned long long m0 = (unsigned long long)e.x | ((unsigned long long)e.y << 32);
      const unsigned long long m1 = (unsigned long long)e.z | ((unsigned long long)e.w << 32);
      float tn0, tf0, tn1, tf1;
      slab_interval(o, inv, a.x, a.y, a.z, a.w, b.x, b.y, tn0, tf0);
      slab_interval(o, inv, b.z, b.w, c.x, c.y, c.z, c.w, tn1, tf1);
      c0 = d.x;
      c1 = d.y;
      h0 = (m0 & M.bits) && test(tn0, tf0);
      h1 = (m1 & M.bits) && test(tn1, tf1);
      if (c0 < 0 && (int64_t)~c0 >= F.n) {  // a leaf beyond the records
        set_err(F, ERR_INDEX);
        h0 = false;
      }
      if (c1 < 0 && (int64_t)~c1 >= F.n) {
        set_err(F, ERR_INDEX);
        h1 = false;
      }
    }
    // push internal children, queue leaves (ballots keep the entries contiguous)
    int np = 0, nl = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const bool h = k ? h1 : h0;
      const int ch = k ? c1 : c0;
      const unsigned bp = __ballot_sync(kFull, h && ch >= 0);
      const unsigned bl = __ballot_sync(kFull, h && ch < 0);
      if (h && ch >= 0) {
        const int pos = sp + np + __popc(bp & lt);
        if (pos < kCoopStack) Q.stk[pos] = ch;
      }
      if (h && ch < 0) Q.lq[lq_n + nl + __popc(bl & lt)] = ~ch;
      np += __popc(bp);
      nl += __popc(bl);
    }
    if (sp + np > kCoopStack) {
      if (lane == 0) set_err(F, ERR_STACK);
      np = kCoopStack - sp;
    }
    sp += np;
    lq_n += nl;
    __syncwarp();
    const bool more = sp > 0;
    while (lq_n >= 32 || (!more && lq_n > 0)) {
      const int tk = lq_n < 32 ? lq_n : 32;
      const int j = (int)lane < tk ? Q.lq[lq_n - tk + (int)lane] : -1;
      __syncwarp();
      lq_n -= tk;
      if (j >= 0) ++cnt.leaves;
      round(j);
      __syncwarp();
    }
    if (!more && lq_n == 0) break;
  }
}

// inclusive prefix sum over the warp's lanes
__device__ __forceinline__ int warp_incl_sum(int x, uint32_t lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(kFull, x, d);
    if ((int)lane >= d) x += y;
  }
  return x;
}

template <int MODE>  // GF_TR_DETERMINISTIC or GF_TR_CLOSED_FORM
__device__ void coop_tau(const DevField& F, CoopQ& Q, const Mask& M, float3 o, float3 v,
                         float3 inv, float tmin, float tmax, float t0, float t1, const float* glx,
                         const float* glw, uint32_t lane, float& s_acc, float& c_acc,
                         Counters& cnt) {
  coop_traverse(F, Q.t, M, o, inv, t0, t1, lane, cnt, [&](int j) {
    // chords set up one per lane, then their nodes shared out
    int n = 0;
    Chord ch;
    float w;
    if (j >= 0 &&
        prim_chord(F, j, o, v, tmin, tmax, [&](uint32_t cl) { return mask_weight(M, cl); }, w, ch)) {
      ++cnt.chords;
      if (MODE == GF_TR_CLOSED_FORM) {
        neumaier_add(s_acc, c_acc, w * chord_closed(F.wd, ch));
      } else {
        const float len = ch.dtout - ch.dtin;
        int off;
        gl_pick(gl_rule(sqrtf(ch.a) * len + 0.5f * fabsf(ch.B) * len), n, off);
        CoopChord C;
        C.mid = 0.5f * (ch.dtin + ch.dtout);
        C.hl = 0.5f * len;
        C.y2 = -0.5f * kLog2e * ch.a;
        C.y1 = -kLog2e * ch.b;
        C.y0 = -0.5f * kLog2e * ch.g;
        C.scale = w * ch.absA * C.hl;
        C.B = ch.B;
        C.delta = ch.delta;
        C.off = off;
        Q.ch[lane] = C;
      }
    }
    if (MODE == GF_TR_CLOSED_FORM) return;
    const int incl = warp_incl_sum(n, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    Q.end[lane + 1] = incl;
    if (lane == 0) Q.end[0] = 0;
    __syncwarp();
    for (int f = (int)lane; f < total; f += 32) {
      int c = 0;  // the chord of node f: the largest c with end[c] <= f
#pragma unroll
      for (int wd = 16; wd > 0; wd >>= 1)
        if (Q.end[c + wd] <= f) c += wd;
      const CoopChord& C = Q.ch[c];
      const int k = C.off + (f - Q.end[c]);
      const float dt = fmaf(C.hl, glx[k], C.mid);
      const float y = fmaf(fmaf(C.y2, dt, C.y1), dt, C.y0);
      neumaier_add(s_acc, c_acc, C.scale * glw[k] * ex2f(y) * cosf(fmaf(C.B, dt, C.delta)));
      ++cnt.evals;
    }
  });
}

template <int MODE>
__global__ void __launch_bounds__(kBlock, 3)
    k_transmittance_coop(const __grid_constant__ DevField F, const TrParams P) {
  __shared__ BlockTables sm;
  __shared__ CoopQ qs[kBlock / 32];
  init_tables(sm, F);
  const uint32_t lane = threadIdx.x & 31u;
  CoopQ& Q = qs[threadIdx.x >> 5];
  Counters cnt;
  const int spp = lod_is_deterministic(P.lod) ? 1 : P.spp;
  for (;;) {
    const int64_t r = next_tile(P.counter, lane);  // one ray per warp
    if (r >= P.n) break;
    const float3 o = make_float3(P.o[3 * r], P.o[3 * r + 1], P.o[3 * r + 2]);
    const float3 v = unit_dir(make_float3(P.d[3 * r], P.d[3 * r + 1], P.d[3 * r + 2]));
    const float tmin = P.trange ? P.trange[2 * r] : 0.f;
    const float tmax = P.trange ? P.trange[2 * r + 1] : INFINITY;
    const float3 inv = safe_inv(v);
    float s_acc = 0.f, c_acc = 0.f;
    for (int s = 0; s < spp; ++s) {
      const Mask m = sample_mask(F, P.lod, v, P.seed, (uint32_t)r, (uint32_t)s, 0, TAG_MASK);
      if (lane == 0) cnt.rays += 1;
      float t0, t1;
      if (m.bits == 0ull || !scene_span(F, o, inv, tmin, tmax, t0, t1)) continue;
      if (lane == 0) cnt.windows += 1;
      coop_tau<MODE>(F, Q, m, o, v, inv, tmin, tmax, t0, t1, sm.glx, sm.glw, lane, s_acc, c_acc,
                     cnt);
    }
    // compensated sum over the warp's lanes (fixed butterfly order)
    for (int off = 1; off < 32; off <<= 1) {
      const float so = __shfl_xor_sync(kFull, s_acc, off), co = __shfl_xor_sync(kFull, c_acc, off);
      float t, e;
      two_sum(s_acc, so, t, e);
      s_acc = t;
      c_acc = __fadd_rn(__fadd_rn(c_acc, co), e);
    }
    if (lane == 0) {
      const float tau = __fadd_rn(s_acc, c_acc) / (float)spp;
      P.out_T[r] = expf(-tau);
      if (P.out_tau) P.out_tau[r] = tau;
    }
  }
  flush_counters(F, cnt, lane);
}

// ---------------------------------------------------------------------------
// Ratio tracking of small batches, one ray per warp.  The warp traverses the
// ray's tree together; each round's chords (one per lane) store their
// evaluation records in shared memory and draw all their tentative points in
// [t0, t1] (chord_points: the per-chord streams of the per-thread tracker, so
// the same points), written in lane order after a counting pass.  Then each
// lane takes points i = lane, lane + 32, ..., sums kappa and kappa_bar at them
// over all stored chords in order, and multiplies its factors 1 - kappa /
// kappa_bar; the lanes' products are combined in a fixed butterfly order.  A
// ray with more chords or points than the buffers hold is tracked by the
// per-thread tracker instead (lane 0).
// ---------------------------------------------------------------------------
constexpr int kRtChords = 256;  // chords of one ray held in shared memory
constexpr int kRtPts = 128;     // tentative points of one ray
struct RtQ {
  CoopTrav t;
  float4 rec[kRtChords][2];  // centred on the envelope peak t*: (t*, t_in, t_out, B),
                             // (-a log2(e) / 2, log2 h, phase at t*, sqrt(a))
  float pt[kRtPts], pu[kRtPts];
};

__device__ float rt_coop(const DevField& F, RtQ& Q, const Mask& M, float3 o, float3 v, float3 inv,
                         float tmin, float tmax, float t0, float t1, uint64_t seed, uint32_t ray,
                         uint32_t word, const float* env, uint32_t lane, Counters& cnt) {
  const unsigned lt = (1u << lane) - 1u;
  int nch = 0, npts = 0;  // warp-uniform
  coop_traverse(F, Q.t, M, o, inv, t0, t1, lane, cnt, [&](int j) {
    Chord ch;
    float w, h = 0.f;
    bool ok = false;
    if (j >= 0 &&
        prim_chord(F, j, o, v, tmin, tmax, [&](uint32_t cl) { return mask_weight(M, cl); }, w, ch) &&
        ch.tc + ch.dtin <= t1 && ch.tc + ch.dtout >= t0) {
      ok = true;
      h = w * ch.absA * expf(-0.5f * ch.qmin);
    }
    const unsigned bc = __ballot_sync(kFull, ok);
    if (ok) {
      ++cnt.chords;
      const int k = nch + __popc(bc & lt);
      if (k < kRtChords) {
        Q.rec[k][0] = make_float4(ch.tc + ch.dts, ch.tc + ch.dtin, ch.tc + ch.dtout, ch.B);
        Q.rec[k][1] = make_float4(-0.5f * kLog2e * ch.a, __log2f(h),
                                  reduce_2pi(fmaf(ch.B, ch.dts, ch.delta)), sqrtf(ch.a));
      }
    }
    nch += __popc(bc);
    // the round's points in lane order: count, then write at the prefix offsets
    int m = 0;
    if (ok)
      chord_points(F, ch, h, seed, ray, word, env, [&](float t, float) {
        if (t > t1) return false;
        if (t >= t0) ++m;
        return true;
      });
    const int incl = warp_incl_sum(m, lane);
    if (ok && m > 0) {
      int q = npts + incl - m;
      chord_points(F, ch, h, seed, ray, word, env, [&](float t, float u) {
        if (t > t1) return false;
        if (t >= t0) {
          if (q < kRtPts) {
            Q.pt[q] = t;
            Q.pu[q] = u;
          }
          ++q;
        }
        return true;
      });
    }
    npts += __shfl_sync(kFull, incl, 31);
  });
  if (lane == 0) cnt.points += (unsigned long long)npts;
  __syncwarp();
  if (nch > kRtChords || npts > kRtPts) {  // too many for the buffers: per-thread tracker
    float T = 1.f;
    if (lane == 0) T = track<false>(F, M, o, v, tmin, tmax, false, seed, ray, word, env, cnt, nullptr);
    return __shfl_sync(kFull, T, 0);
  }
  float prod = 1.f;
  for (int i = (int)lane; i < npts; i += 32) {
    const float t = Q.pt[i];
    float kap = 0.f, kb = 0.f;
    for (int c = 0; c < nch; ++c) {
      const float4 a = Q.rec[c][0];
      if (t >= a.y && t <= a.z) {
        const float4 b = Q.rec[c][1];
        const float dt = t - a.x;
        kap = fmaf(ex2f(fmaf(b.x, dt * dt, b.y)), cosf_fast(fmaf(a.w, dt, b.z)), kap);
        int mm = (int)(fabsf(dt) * b.w);
        mm = mm > 7 ? 7 : mm;
        kb = fmaf(ex2f(b.y), env[mm], kb);  // h exp(-m^2/2)
        ++cnt.evals;
      }
    }
    if (kb > 0.f) prod *= 1.f - kap / kb;
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) prod *= __shfl_xor_sync(kFull, prod, off);
  return prod;
}

__global__ void __launch_bounds__(kBlock, 3)
    k_transmittance_rt_coop(const __grid_constant__ DevField F, const TrParams P) {
  __shared__ BlockTables sm;
  __shared__ RtQ qs[kBlock / 32];
  init_tables(sm, F);
  const uint32_t lane = threadIdx.x & 31u;
  RtQ& Q = qs[threadIdx.x >> 5];
  Counters cnt;
  for (;;) {
    const int64_t r = next_tile(P.counter, lane);  // one ray per warp
    if (r >= P.n) break;
    const float3 o = make_float3(P.o[3 * r], P.o[3 * r + 1], P.o[3 * r + 2]);
    const float3 v = unit_dir(make_float3(P.d[3 * r], P.d[3 * r + 1], P.d[3 * r + 2]));
    const float tmin = P.trange ? P.trange[2 * r] : 0.f;
    const float tmax = P.trange ? P.trange[2 * r + 1] : INFINITY;
    const float3 inv = safe_inv(v);
    float acc = 0.f;
    for (int s = 0; s < P.spp; ++s) {
      const Mask m = sample_mask(F, P.lod, v, P.seed, (uint32_t)r, (uint32_t)s, 0, TAG_MASK);
      if (lane == 0) cnt.rays += 1;
      float t0, t1, T = 1.f;
      if (m.bits != 0ull && scene_span(F, o, inv, tmin, tmax, t0, t1)) {
        if (lane == 0) cnt.windows += 1;
        T = rt_coop(F, Q, m, o, v, inv, tmin, tmax, t0, t1, P.seed, (uint32_t)r,
                    stream_word((uint32_t)s, 0, TAG_TRACK), sm.env, lane, cnt);
      }
      acc += T;
    }
    if (lane == 0) P.out_T[r] = acc / (float)P.spp;
  }
  flush_counters(F, cnt, lane);
}

// ---------------------------------------------------------------------------
// render: each lane owns one pixel of an 8x4 tile and runs its samples in
// order (deterministic per pixel); FF: the free flight of scattering
// (GF_FLIGHT_DELTA here means tomography: delta tracking renders in the
// wavefront kernel)
// ---------------------------------------------------------------------------
template <int FF>
__global__ void __launch_bounds__(kBlock)
    k_render(const __grid_constant__ DevField F, const PathParams P, float* out, int* counter) {
  __shared__ BlockTables sm;
  init_tables(sm, F);
  const uint32_t lane = threadIdx.x & 31u;
  Counters cnt;
  const int tiles_x = (P.cam.W + kTileW - 1) / kTileW;
  const int tiles_y = (P.cam.H + kTileH - 1) / kTileH;
  for (;;) {
    const int tile = next_tile(counter, lane);
    if (tile >= tiles_x * tiles_y) break;
    const int px = (tile % tiles_x) * kTileW + (int)(lane % kTileW);
    const int py = (tile / tiles_x) * kTileH + (int)(lane / kTileW);
    const bool active = px < P.cam.W && py < P.cam.H;
    float acc = 0.f;
    for (int s = 0; s < P.spp; ++s)
      acc += path_sample<FF>(F, P, active, px, py, P.s0 + s, sm.glx, sm.glw, sm.env, cnt);
    if (active) out[(int64_t)py * P.cam.W + px] = acc / (float)P.spp;
  }
  flush_counters(F, cnt, lane);
}

__global__ void k_faddeeva(const Weideman W, const float* z, float* w, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = z[2 * i], y = z[2 * i + 1];
  float2 r = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
  if (y >= 0.0f) r = faddeeva_w(W, x, y);
  w[2 * i] = r.x;
  w[2 * i + 1] = r.y;
}

// ---------------------------------------------------------------------------
// chord sets (testing)
// ---------------------------------------------------------------------------
struct ListLeaf {
  const DevField* F;
  const Mask* M;
  float3 o, v;
  float tmin, tmax;
  const ChordParams* P;
  int64_t r;
  int n = 0;
  __device__ __forceinline__ void operator()(int j) {
    const Mask& Mk = *M;
    Chord ch;
    float w;
    if (!prim_chord(*F, j, o, v, tmin, tmax, [&](uint32_t c) { return mask_weight(Mk, c); }, w, ch))
      return;
    if (n < P->cap) {
      const int64_t at = r * P->cap + n;
      P->prims[at] = (int)ch.orig;
      if (P->tin) P->tin[at] = ch.tc + ch.dtin;
      if (P->tout) P->tout[at] = ch.tc + ch.dtout;
    }
    ++n;
  }
};

__global__ void __launch_bounds__(kBlock) k_ray_chords(const __grid_constant__ DevField F,
                                                       const ChordParams P) {
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    const int tile = next_tile(P.counter, lane);
    if ((int64_t)tile * 32 >= P.n) break;
    const int64_t r = (int64_t)tile * 32 + lane;
    if (r >= P.n) continue;  // next_tile below is reached by every lane
    const float3 o = make_float3(P.o[3 * r], P.o[3 * r + 1], P.o[3 * r + 2]);
    const float3 v = unit_dir(make_float3(P.d[3 * r], P.d[3 * r + 1], P.d[3 * r + 2]));
    const float tmin = P.trange ? P.trange[2 * r] : 0.f;
    const float tmax = P.trange ? P.trange[2 * r + 1] : INFINITY;
    const Mask m = sample_mask(F, P.lod, v, 0, (uint32_t)r, 0, 0, TAG_MASK);
    const float3 inv = safe_inv(v);
    float t0, t1;
    int n = 0;
    if (m.bits && scene_span(F, o, inv, tmin, tmax, t0, t1)) {
      ListLeaf leaf;
      leaf.F = &F;
      leaf.M = &m;
      leaf.o = o;
      leaf.v = v;
      leaf.tmin = tmin;
      leaf.tmax = tmax;
      leaf.P = &P;
      leaf.r = r;
      SpanTest test{t0, t1};
      unsigned long long nv = 0, nl = 0;
      traverse_ray(F, o, inv, m.bits, test, leaf, nv, nl);
      n = leaf.n;
    }
    P.counts[r] = n;
  }
}

__global__ void k_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
  const uint4 r = philox(c, k);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

// ---------------------------------------------------------------------------
// launchers: persistent grids of (resident blocks per SM) x SMs
// ---------------------------------------------------------------------------
// every kernel's per-thread stack (its local memory frame, callees included)
// must fit the context's stack limit as it stands at launch (gf_create raises
// it to at least kStackLimit; another component of the process may change it)
template <class K>
static bool stack_fits(K kernel) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, kernel) != cudaSuccess) return false;
  size_t limit = 0;
  if (cudaDeviceGetLimit(&limit, cudaLimitStackSize) != cudaSuccess) return false;
  return a.localSizeBytes <= limit;
}

template <class K>
static int persistent_grid(const Field& F, K kernel, int64_t warps_of_work) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess)
    (void)cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (warps_of_work + kBlock / 32 - 1) / (kBlock / 32);
  int64_t g = (int64_t)F.ctx.sm_count * per_sm;
  if (need < g) g = need;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_transmittance(const Field& F, const TrParams& P, cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (P.mode == GF_TR_DETERMINISTIC || P.mode == GF_TR_CLOSED_FORM) {
    // few rays: several lanes per ray so that enough warps hide the latency
    // (about 16 resident warps of 32 lanes per SM as the target)
    TrParams Q = P;
    const int64_t lanes = (int64_t)F.ctx.sm_count * 16 * 32;
    Q.group = 1;
    while (Q.group < 32 && P.n * Q.group <= lanes) Q.group *= 2;
    const int64_t tiles_g = (P.n + 32 / Q.group - 1) / (32 / Q.group);
    if (Q.group >= 16) {
      // few rays: the whole warp on each ray (k_transmittance_coop)
      if (P.mode == GF_TR_DETERMINISTIC) {
        auto k = k_transmittance_coop<GF_TR_DETERMINISTIC>;
        k<<<persistent_grid(F, k, P.n), kBlock, 0, s>>>(F.dev, Q);
      } else {
        auto k = k_transmittance_coop<GF_TR_CLOSED_FORM>;
        k<<<persistent_grid(F, k, P.n), kBlock, 0, s>>>(F.dev, Q);
      }
    } else if (P.mode == GF_TR_DETERMINISTIC) {
      auto k = k_transmittance<GF_TR_DETERMINISTIC>;
      k<<<persistent_grid(F, k, tiles_g), kBlock, 0, s>>>(F.dev, Q);
    } else {
      auto k = k_transmittance<GF_TR_CLOSED_FORM>;
      k<<<persistent_grid(F, k, tiles_g), kBlock, 0, s>>>(F.dev, Q);
    }
  } else if (P.n * 8 <= (int64_t)F.ctx.sm_count * 16 * 32) {
    // few rays: the whole warp on each ray (k_transmittance_rt_coop)
    auto k = k_transmittance_rt_coop;
    k<<<persistent_grid(F, k, P.n), kBlock, 0, s>>>(F.dev, P);
  } else {
    const int64_t tiles = (P.n + 31) / 32;
    auto k = k_transmittance<GF_TR_RATIO_TRACKING>;
    k<<<persistent_grid(F, k, tiles), kBlock, 0, s>>>(F.dev, P);
  }
  return cudaGetLastError();
}

cudaError_t launch_render(const Field& F, const PathParams& P, float* out, cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  cudaError_t e = cudaMemsetAsync(F.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (P.integrator == GF_INTEG_SCATTER && P.free_flight == GF_FLIGHT_DELTA)
    return launch_render_scatter(F, P, out, s);
  const int64_t tiles = (int64_t)((P.cam.W + kTileW - 1) / kTileW) * ((P.cam.H + kTileH - 1) / kTileH);
  if (P.integrator == GF_INTEG_SCATTER) {
    auto k = P.free_flight == GF_FLIGHT_SEGMENT ? k_render<GF_FLIGHT_SEGMENT> : k_render<GF_FLIGHT_CDF>;
    if (!stack_fits(k)) return cudaErrorLaunchOutOfResources;
    k<<<persistent_grid(F, k, tiles), kBlock, 0, s>>>(F.dev, P, out, F.counter);
  } else {
    auto k = k_render<GF_FLIGHT_DELTA>;
    if (!stack_fits(k)) return cudaErrorLaunchOutOfResources;
    k<<<persistent_grid(F, k, tiles), kBlock, 0, s>>>(F.dev, P, out, F.counter);
  }
  return cudaGetLastError();
}

cudaError_t launch_ray_chords(const Field& F, const ChordParams& P, cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_ray_chords<<<persistent_grid(F, k_ray_chords, (P.n + 31) / 32), kBlock, 0, s>>>(F.dev, P);
  return cudaGetLastError();
}

cudaError_t launch_faddeeva(const Weideman& W, const float* z, float* w, int64_t n,
                           cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_faddeeva<<<(unsigned)blocks, 256, 0, s>>>(W, z, w, n);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                          cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_philox<<<(unsigned)blocks, 256, 0, s>>>(ctr, key, out, n);
  return cudaGetLastError();
}

}  // namespace gf
