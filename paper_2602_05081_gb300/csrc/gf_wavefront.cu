// gf_wavefront.cu -- scattering renderer: lanes traverse, the warp processes.
//
// Every lane of a warp owns one path (one pixel's samples in order).  The
// warp traverses the BVH for all 32 current rays together: one shared stack
// of (node, lane) entries, from which every step pops up to 32 entries, so the
// lanes stay busy while rays of different lengths are in flight.  Leaves that
// are reached go to a per-warp queue in shared memory, and whenever 32 are
// queued the whole warp sets up their chords at once (chord set-up on the
// owning lane's ray).  Each chord that overlaps the owner's window [ta, te)
// is stored (its evaluation record, in a per-warp global store) and queued;
// queued chords are walked 32 at a time, drawing the chord's tentative points
// of Sec. 3's per-segment majorant from its own Philox stream.  Points land in
// the owner's buffer through shared-memory atomics.  kappa and kappa_bar at
// the points are then summed from the stored records (the warp scans each
// lane's list and reduces by shuffles), after which each lane takes its
// delta-tracking or ratio-tracking decision and moves its path on (camera
// ray -> collision -> NEE -> scattering).
//
// The tentative points are a function of the chords and their Philox streams
// only, so results equal a per-ray formulation up to floating-point summation
// order.
#include <cuda_runtime.h>

#include <climits>

#include "gf_host.h"
#include "gf_trace.cuh"

namespace gf {

constexpr int kWWarps = 4;      // warps per block
constexpr int kLeafQ = 96;      // queued leaves per warp (<= 31 left + 64 new)
constexpr int kChordQ = 64;     // queued chords per warp (<= 31 left + 32 new)
constexpr int kPK = 8;          // tentative points per lane and window
constexpr int kSlotCh = 256;    // stored chords per lane and window (global scratch)

// One slot per lane, 89 words: an odd stride keeps same-field accesses of the
// 32 slots in distinct shared-memory banks.
struct LaneRay {
  float o[3], v[3], inv[3];
  float tmin, tmax, ta, te;     // ray range and window [ta, te)
  uint32_t ray, word;
  float bw[8];                  // LoD band weights
  uint32_t mask_lo, mask_hi;    // LoD cell bits
  int npts;                     // points emitted in the window (may exceed kPK)
  int nch;                      // chords stored for the window (may exceed kSlotCh)
  float pt[kPK], pu[kPK], kap[kPK], kb[kPK];
};
static_assert(sizeof(LaneRay) % 8 == 4, "odd word stride");
struct ChordItem {
  float tc, dtin, dtout, h, sa, dts, smax;
  uint32_t orig;
  int owner;
};
constexpr int kWStack = 1024;   // shared (node, slot) stack entries per warp
struct WarpQ {
  LaneRay r[32];
  int stk[kWStack];
  int lq_prim[kLeafQ];
  int lq_own[kLeafQ];
  ChordItem cq[kChordQ];
};

__device__ __forceinline__ int ord_f(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float unord_f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__device__ __forceinline__ unsigned long long slot_mask(const LaneRay& R) {
  return (unsigned long long)R.mask_lo | ((unsigned long long)R.mask_hi << 32);
}
__device__ __forceinline__ float ray_weight(const LaneRay& R, uint32_t cell) {
  if (!(slot_mask(R) >> cell & 1ull)) return 0.f;
  const int b = cell == 0 ? 0 : (int)((cell - 1u) >> 3) + 1;
  return R.bw[b];
}

// chord of sorted primitive j on the ray of slot R
__device__ __forceinline__ bool slot_chord(const DevField& F, const LaneRay& R, int j, Prim& P,
                                           Chord& ch, float& w) {
  P = load_prim(F, j);
  w = ray_weight(R, P.cell & 63u);
  if (!(w > 0.f)) return false;
  return chord_setup(P, make_float3(R.o[0], R.o[1], R.o[2]), make_float3(R.v[0], R.v[1], R.v[2]),
                     R.tmin, R.tmax, F.k2, ch);
}

// walk one queued chord: emit its tentative points in [ta, te) to the owner
__device__ __forceinline__ void walk_chord(const DevField& F, WarpQ& Q, const ChordItem& c,
                                           uint64_t seed, const float* env, unsigned long long& npt) {
  LaneRay& R = Q.r[c.owner];
  const float ta = R.ta, te = R.te;
  const float invs = 1.0f / c.sa;
  int J = (int)ceilf(c.smax) - 1;
  J = J < 0 ? 0 : (J > 6 ? 6 : J);
  float dt = c.dtin;
  int p = 0;
  while (p < 2 * J) {
    const float bp = p < J ? c.dts - (float)(J - p) * invs : c.dts + (float)(p - J + 1) * invs;
    if (bp <= dt) ++p;
    else break;
  }
  for (uint32_t draw = 0; draw < (1u << 16); ++draw) {
    const uint4 x = rng4(seed, draw, c.orig, R.ray, R.word);
    float z = -logf(1.0f - u01(x.x));
    bool emit = false;
    for (int q = 0; q < 2 * J + 2; ++q) {
      const float bp = p < J ? c.dts - (float)(J - p) * invs : c.dts + (float)(p - J + 1) * invs;
      const float end = p < 2 * J ? fminf(bp, c.dtout) : c.dtout;
      const int nn = p < J ? J - p : p - J;
      const float lam = c.h * env[nn];
      const float capz = lam * (end - dt);
      if (z < capz) {
        dt += z / lam;
        emit = true;
        break;
      }
      z -= capz;
      dt = end;
      if (dt >= c.dtout) return;
      ++p;
    }
    if (!emit) return;
    const float t = c.tc + dt;
    if (t >= te) return;
    if (t >= ta) {
      ++npt;
      const int slot = atomicAdd(&R.npts, 1);
      if (slot < kPK) {
        R.pt[slot] = t;
        R.pu[slot] = u01(x.y);
      } else {
        return;  // overflow: the owner halves the window and redoes it
      }
    }
  }
  set_err(F, ERR_GUARD);
}

// One traversal phase for the slots with want = true.  The warp shares one
// stack of (node, slot) entries: every step pops up to 32 entries from the
// frontiers of all its rays, so lanes stay busy while 32 rays are in flight.
// It collects the tentative points of each slot's window and stores the
// window's chords for their evaluation.
__device__ void warp_phase(const DevField& F, WarpQ& Q, bool want, uint32_t lane, uint64_t seed,
                           const float* env, float4* wch, Counters& cnt) {
  const unsigned lt = (1u << lane) - 1u;
  int sp = 0, lq_n = 0, cq_n = 0;  // warp-uniform sizes
  {
    const unsigned bal = __ballot_sync(kFull, want);
    const int idx = __popc(bal & lt);
    if (F.root >= 0) {
      if (want) Q.stk[idx] = (F.root << 5) | (int)lane;
      sp = __popc(bal);
    } else {  // a one-primitive field has no internal node: queue its leaf
      if (want) {
        Q.lq_prim[idx] = 0;
        Q.lq_own[idx] = (int)lane;
      }
      lq_n = __popc(bal);
    }
    __syncwarp();
  }
  const long long max_it = 4 * (F.n + 64) * 32 / 32 + 4096;
  for (long long it = 0;; ++it) {
    if (it > max_it * 32) {
      if (lane == 0) set_err(F, ERR_GUARD);
      break;
    }
    // ---------------- one traversal step: up to 32 (node, slot) entries
    GF_TIC(t_step);
    int take = sp < 32 ? sp : 32;
    if (sp > kWStack - 96) take = 1;  // near capacity: depth first
    int ent = (int)lane < take ? Q.stk[sp - take + (int)lane] : -1;
    __syncwarp();
    sp -= take;
    int c0 = 0, c1 = 0, l0 = -1, l1 = -1, slot = 0;
    bool g0 = false, g1 = false;
    if (ent >= 0) {
      const int node = ent >> 5;
      slot = ent & 31;
      const LaneRay& R = Q.r[slot];
      const float3 o = make_float3(R.o[0], R.o[1], R.o[2]);
      const float3 inv = make_float3(R.inv[0], R.inv[1], R.inv[2]);
      const unsigned long long mask = slot_mask(R);
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
      bool h0 = fmaxf(tn0, R.ta) <= fminf(tf0, R.te);
      bool h1 = fmaxf(tn1, R.ta) <= fminf(tf1, R.te);
      h0 = h0 && (m0 & mask);
      h1 = h1 && (m1 & mask);
      c0 = d.x;
      c1 = d.y;
      if (h0 && c0 < 0) l0 = ~c0;
      if (h1 && c1 < 0) l1 = ~c1;
      g0 = h0 && c0 >= 0;
      g1 = h1 && c1 >= 0;
    }
    // ---------------- push internal children, queue leaves
    {
      const unsigned p0 = __ballot_sync(kFull, g0), p1 = __ballot_sync(kFull, g1);
      const int np0 = __popc(p0), np1 = __popc(p1);
      if (sp + np0 + np1 > kWStack) {
        if (lane == 0) set_err(F, ERR_STACK);
      } else {
        if (g0) Q.stk[sp + __popc(p0 & lt)] = (c0 << 5) | slot;
        if (g1) Q.stk[sp + np0 + __popc(p1 & lt)] = (c1 << 5) | slot;
        sp += np0 + np1;
      }
      const unsigned b0 = __ballot_sync(kFull, l0 >= 0), b1 = __ballot_sync(kFull, l1 >= 0);
      const int n0 = __popc(b0);
      if (l0 >= 0) {
        const int idx = lq_n + __popc(b0 & lt);
        Q.lq_prim[idx] = l0;
        Q.lq_own[idx] = slot;
      }
      if (l1 >= 0) {
        const int idx = lq_n + n0 + __popc(b1 & lt);
        Q.lq_prim[idx] = l1;
        Q.lq_own[idx] = slot;
      }
      lq_n += n0 + __popc(b1);
      __syncwarp();
    }
    const bool any_trav = sp > 0;
    if (lane == 0) GF_TOC(cnt, 0, t_step);
    // ---------------- leaf rounds: 32 leaves of any slots' rays at a time
    while (lq_n >= 32 || (!any_trav && lq_n > 0)) {
      const int tk = lq_n < 32 ? lq_n : 32;
      const bool have = (int)lane < tk;
      int j = 0, own = 0;
      if (have) {
        j = Q.lq_prim[lq_n - tk + (int)lane];
        own = Q.lq_own[lq_n - tk + (int)lane];
      }
      __syncwarp();
      lq_n -= tk;
      cnt.leaves += have ? 1ull : 0ull;
      GF_TIC(t_leaf);
      bool ok = false;
      ChordItem ci;
      if (have) {
        const LaneRay& R = Q.r[own];
        Prim P;
        Chord ch;
        float w;
        if (slot_chord(F, R, j, P, ch, w)) {
          const float tin = ch.tc + ch.dtin, tout = ch.tc + ch.dtout;
          if (tin < R.te && tout >= R.ta) {
            ok = true;
            const float wa = w * ch.absA;
            const float h = wa * expf(-0.5f * ch.qmin), sa = sqrtf(ch.a);
            // evaluation record for the points of this window
            const int k = atomicAdd(&Q.r[own].nch, 1);
            if (k < kSlotCh) {
              float4* dst = wch + ((size_t)own * kSlotCh + k) * 3;
              dst[0] = make_float4(ch.tc, tin, tout, ch.B);
              dst[1] = make_float4(-0.5f * kLog2e * ch.a, -kLog2e * ch.b,
                                   fmaf(-0.5f * kLog2e, ch.g, log2f(wa)), ch.delta);
              dst[2] = make_float4(h, sa, ch.dts, 0.f);
            }
            ci.tc = ch.tc;
            ci.dtin = ch.dtin;
            ci.dtout = ch.dtout;
            ci.h = h;
            ci.sa = sa;
            ci.dts = ch.dts;
            ci.smax = ci.sa * ch.hw;
            ci.orig = ch.orig;
            ci.owner = own;
          }
        }
      }
      const unsigned bc = __ballot_sync(kFull, ok);
      if (ok) Q.cq[cq_n + __popc(bc & lt)] = ci;
      cq_n += __popc(bc);
      cnt.chords += ok ? 1ull : 0ull;
      __syncwarp();
      if (lane == 0) GF_TOC(cnt, 1, t_leaf);
      GF_TIC(t_walk);
      while (cq_n >= 32) {
        const bool hv = true;
        ChordItem cw = Q.cq[cq_n - 32 + (int)lane];
        __syncwarp();
        cq_n -= 32;
        if (hv) walk_chord(F, Q, cw, seed, env, cnt.points);
        __syncwarp();
      }
      if (lane == 0) GF_TOC(cnt, 2, t_walk);
    }
    if (!any_trav && lq_n == 0) {
      // traversal over and no leaf left: walk the remaining chords
      while (cq_n > 0) {
        const int tk = cq_n < 32 ? cq_n : 32;
        const bool hv = (int)lane < tk;
        ChordItem cw;
        if (hv) cw = Q.cq[cq_n - tk + (int)lane];
        __syncwarp();
        cq_n -= tk;
        if (hv) walk_chord(F, Q, cw, seed, env, cnt.points);
        __syncwarp();
      }
    }
    if (!any_trav && lq_n == 0 && cq_n == 0) break;
  }
  __syncwarp();
}

// per-lane path state
struct PathState {
  int pix;        // -1: no pixel
  int s, b;       // sample, bounce
  int kind;       // 0 idle, 1 delta tracking, 2 ratio tracking (NEE)
  float acc, Lsum, thr, T;
  float3 o, v;    // current ray
  float t0, t1;   // scene span of the current ray
  float step;     // window length for delta tracking
};

__device__ __forceinline__ void set_slot(LaneRay& R, float3 o, float3 v, const Mask& m,
                                         uint32_t ray, uint32_t word) {
  R.o[0] = o.x; R.o[1] = o.y; R.o[2] = o.z;
  R.v[0] = v.x; R.v[1] = v.y; R.v[2] = v.z;
  const float3 iv = safe_inv(v);
  R.inv[0] = iv.x; R.inv[1] = iv.y; R.inv[2] = iv.z;
  R.tmin = 0.f;
  R.tmax = INFINITY;
  R.ray = ray;
  R.word = word;
  R.mask_lo = (uint32_t)m.bits;
  R.mask_hi = (uint32_t)(m.bits >> 32);
#pragma unroll
  for (int k = 0; k < 8; ++k) R.bw[k] = m.bw[k];
}

// Start a tracking ray: returns false if it misses the scene (nothing to do).
__device__ __forceinline__ bool start_ray(const DevField& F, LaneRay& R, PathState& S, int kind,
                                          float3 o, float3 v, const Mask& m, uint32_t ray,
                                          uint32_t word) {
  S.kind = kind;
  S.o = o;
  S.v = v;
  set_slot(R, o, v, m, ray, word);
  float t0, t1;
  const bool hit = m.bits != 0ull && scene_span(F, o, safe_inv(v), 0.f, INFINITY, t0, t1);
  S.t0 = t0;
  S.t1 = t1;
  if (!hit) return false;
  S.step = kind == 1 ? fmaxf(0.25f * (t1 - t0), 1e-6f) : (t1 - t0);
  R.ta = t0;
  R.te = kind == 1 ? fminf(t1, t0 + S.step) : t1;
  if (R.te >= t1) R.te = t1 * (1.0f + 1e-7f) + 1e-30f;  // last window includes t1
  return true;
}

// kappa and kappa_bar at the points of every slot, from the chords pass 1
// stored: the warp scans each slot's list (lanes over chords), then reduces.
__device__ void eval_stored(WarpQ& Q, const float4* wch, const float* env, uint32_t lane,
                            Counters& cnt) {
  for (int s = 0; s < 32; ++s) {
    LaneRay& R = Q.r[s];
    const int ns = R.npts;
    if (ns <= 0) continue;  // uniform: every lane reads the same slot
    const int mc = R.nch;
    float pt[kPK], kap[kPK], kb[kPK];
#pragma unroll
    for (int i = 0; i < kPK; ++i) {
      pt[i] = i < ns ? R.pt[i] : INFINITY;
      kap[i] = 0.f;
      kb[i] = 0.f;
    }
    const float4* base = wch + (size_t)s * kSlotCh * 3;
    for (int c = (int)lane; c < mc; c += 32) {
      const float4 a = base[3 * c], b = base[3 * c + 1], e = base[3 * c + 2];
#pragma unroll
      for (int i = 0; i < kPK; ++i) {
        const float t = pt[i];
        if (t >= a.y && t <= a.z) {
          const float dt = t - a.x;
          const float y = fmaf(fmaf(b.x, dt, b.y), dt, b.z);
          kap[i] = fmaf(ex2f(y), cosf_fast(fmaf(a.w, dt, b.w)), kap[i]);
          int m = (int)(fabsf(dt - e.z) * e.y);
          m = m > 7 ? 7 : m;
          kb[i] = fmaf(e.x, env[m], kb[i]);
          ++cnt.evals;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kPK; ++i) {
      if (i < ns) {
        const float k1 = warp_sum(kap[i]), k2 = warp_sum(kb[i]);
        if (lane == 0) {
          R.kap[i] = k1;
          R.kb[i] = k2;
        }
      }
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kWWarps * 32)
    k_render_scatter(const __grid_constant__ DevField F, const PathParams P, float* out,
                     int* counter, float4* chord_store) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* env = reinterpret_cast<float*>(smraw);
  WarpQ* Qs = reinterpret_cast<WarpQ*>(smraw + 64);
  if (threadIdx.x < 8) env[threadIdx.x] = F.env[threadIdx.x];
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  WarpQ& Q = Qs[wid];
  LaneRay& R = Q.r[lane];
  float4* wch = chord_store + ((size_t)blockIdx.x * kWWarps + wid) * 32 * kSlotCh * 3;
  Counters cnt;
  const int npix = P.cam.W * P.cam.H;
  const float inv4pi = 0.25f / 3.14159265358979f;

  PathState S;
  S.pix = -1;
  S.kind = 0;
  S.acc = 0.f;

  // begin the next sample of the lane's pixel (or the next pixel); kind = 0 if none left
  auto begin_sample = [&]() {
    for (;;) {
      if (S.pix < 0) {
        S.pix = atomicAdd(counter, 1);
        if (S.pix >= npix) {
          S.pix = -1;
          S.kind = 0;
          return;
        }
        S.s = 0;
        S.acc = 0.f;
      }
      if (S.s >= P.spp) {
        out[S.pix] = S.acc / (float)P.spp;
        S.pix = -1;
        continue;
      }
      const int px = S.pix % P.cam.W, py = S.pix / P.cam.W;
      float3 o, v;
      camera_ray(P.cam, P.seed, px, py, S.s, o, v);
      S.b = 0;
      S.thr = 1.f;
      S.Lsum = 0.f;
      const Mask m = sample_mask(F, P.lod, v, P.seed, (uint32_t)S.pix, (uint32_t)S.s, 0, TAG_MASK);
      cnt.rays += 1;
      if (start_ray(F, R, S, 1, o, v, m, (uint32_t)S.pix,
                    stream_word((uint32_t)S.s, 0, TAG_TRACK)))
        return;
      // the camera ray misses the field: the sample is 0
      S.s += 1;
    }
  };
  // the lane's current ray is finished: move the path on
  auto finish_ray = [&](bool hit, float th) {
    for (;;) {
      if (S.kind == 1) {
        if (!hit) {
          S.acc += S.Lsum;
          S.s += 1;
          begin_sample();
          return;
        }
        const float3 x = make_float3(S.o.x + th * S.v.x, S.o.y + th * S.v.y, S.o.z + th * S.v.z);
        S.thr *= P.albedo;
        S.T = 1.f;
        const Mask mn = sample_mask(F, P.lod_nee, P.light, P.seed, (uint32_t)S.pix, (uint32_t)S.s,
                                    (uint32_t)S.b, TAG_NEE_MASK);
        cnt.rays += 1;
        if (start_ray(F, R, S, 2, x, P.light, mn, (uint32_t)S.pix,
                      stream_word((uint32_t)S.s, (uint32_t)S.b, TAG_NEE)))
          return;
        // NEE ray misses every primitive: T = 1
        S.o = x;
      }
      // S.kind == 2: NEE finished with transmittance S.T
      S.Lsum += S.thr * P.irradiance * S.T * inv4pi;
      const uint4 y = rng4(P.seed, 0, kNoPrim, (uint32_t)S.pix,
                           stream_word((uint32_t)S.s, (uint32_t)S.b, TAG_SCATTER));
      const float z = 1.0f - 2.0f * u01(y.x);
      const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
      float sn, cs;
      sincosf(2.0f * 3.14159265358979f * u01(y.y), &sn, &cs);
      const float3 nv = make_float3(rr * cs, rr * sn, z);
      S.b += 1;
      if (S.b >= P.max_bounces) {
        S.acc += S.Lsum;
        S.s += 1;
        begin_sample();
        return;
      }
      const float3 xo = S.o;
      const Mask m = sample_mask(F, P.lod, nv, P.seed, (uint32_t)S.pix, (uint32_t)S.s,
                                 (uint32_t)S.b, TAG_MASK);
      cnt.rays += 1;
      if (start_ray(F, R, S, 1, xo, nv, m, (uint32_t)S.pix,
                    stream_word((uint32_t)S.s, (uint32_t)S.b, TAG_TRACK)))
        return;
      S.kind = 1;
      hit = false;  // the scattered ray leaves the field at once
    }
  };

  begin_sample();
  for (int guard = 0; guard < (1 << 30); ++guard) {
    const bool want = S.kind != 0;
    if (!__any_sync(kFull, want)) break;
    // ---- pass 1: tentative points of the window
    R.npts = 0;
    R.nch = 0;
    __syncwarp();
    warp_phase(F, Q, want, lane, P.seed, env, wch, cnt);
    // owner: a window whose points overflowed the slots is halved and redone;
    // otherwise its points are sorted by t for the decisions
    int n = 0;
    bool ovf = false;
    if (want) {
      ovf = R.npts > kPK || R.nch > kSlotCh;
      n = ovf ? 0 : R.npts;
      for (int k = 1; k < n; ++k) {
        const float t = R.pt[k], u = R.pu[k];
        int q = k;
        while (q > 0 && R.pt[q - 1] > t) {
          R.pt[q] = R.pt[q - 1];
          R.pu[q] = R.pu[q - 1];
          --q;
        }
        R.pt[q] = t;
        R.pu[q] = u;
      }
      R.npts = n;
      for (int i = 0; i < n; ++i) {
        R.kap[i] = 0.f;
        R.kb[i] = 0.f;
      }
    }
    cnt.windows += want ? 1ull : 0ull;
    __syncwarp();
    // ---- kappa and kappa_bar at the points, from the stored chords
    if (__any_sync(kFull, want && n > 0)) eval_stored(Q, wch, env, lane, cnt);
    // ---- decisions
    GF_TIC(t_dec);
    if (want) {
      const bool last = R.te >= S.t1;
      if (ovf) {
        const float w = R.te - R.ta;
        if (w <= 1e-6f * (1.0f + fabsf(R.ta))) {
          // more than kPK points at one t: give up on this ray
          set_err(F, ERR_POINTS);
          finish_ray(false, 0.f);
        } else {
          R.te = R.ta + 0.5f * w;
          S.step = 0.5f * w;
        }
      } else if (S.kind == 1) {
        float th = 0.f;
        bool acc = false;
        for (int i = 0; i < n && !acc; ++i) {
          if (R.pu[i] * R.kb[i] < fmaxf(R.kap[i], 0.f)) {
            acc = true;
            th = R.pt[i];
          }
        }
        if (acc) {
          finish_ray(true, th);
        } else if (!last) {
          R.ta = R.te;
          R.te = fminf(S.t1, R.ta + S.step);
          if (R.te >= S.t1) R.te = S.t1 * (1.0f + 1e-7f) + 1e-30f;
        } else {
          finish_ray(false, 0.f);
        }
      } else {
        for (int i = 0; i < n; ++i)
          if (R.kb[i] > 0.f) S.T *= 1.f - fmaxf(R.kap[i], 0.f) / R.kb[i];
        if (!last) {
          S.step *= 2.0f;
          R.ta = R.te;
          R.te = fminf(S.t1, R.ta + S.step);
          if (R.te >= S.t1) R.te = S.t1 * (1.0f + 1e-7f) + 1e-30f;
        } else {
          finish_ray(false, 0.f);
        }
      }
    }
    __syncwarp();
    if (lane == 0) GF_TOC(cnt, 4, t_dec);
  }
  flush_counters(F, cnt, lane);
}

size_t scatter_smem_bytes() { return 64 + sizeof(WarpQ) * kWWarps; }

cudaError_t launch_render_scatter(const Field& F, const PathParams& P, float* out, cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  cudaError_t e = cudaMemsetAsync(F.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t smem = scatter_smem_bytes();
  e = cudaFuncSetAttribute(k_render_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_scatter, kWWarps * 32, smem) != cudaSuccess)
    (void)cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  const int64_t npix = (int64_t)P.cam.W * P.cam.H;
  const int64_t need = (npix + kWWarps * 32 - 1) / (kWWarps * 32);
  int64_t g = (int64_t)F.ctx.sm_count * per_sm;
  if (need < g) g = need;
  if (g < 1) g = 1;
  // per-warp chord store: 32 slots x kSlotCh records of 3 float4
  const size_t store = (size_t)g * kWWarps * 32 * kSlotCh * 3 * sizeof(float4);
  if (F.wscratch_bytes < store) {
    if (F.wscratch) cudaFree(F.wscratch);
    F.wscratch = nullptr;
    F.wscratch_bytes = 0;
    e = cudaMalloc((void**)&F.wscratch, store);
    if (e != cudaSuccess) return e;
    F.wscratch_bytes = store;
  }
  k_render_scatter<<<(unsigned)g, kWWarps * 32, smem, s>>>(F.dev, P, out, F.counter, F.wscratch);
  return cudaGetLastError();
}

}  // namespace gf
