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
// queued chords are walked 32 at a time, one draw per chord and round, each
// drawing the chord's next tentative point of Sec. 3's per-segment majorant
// from its own Philox stream (chords that may hold more points go back to the
// queue, so the lanes stay busy).  Points land in
// the owner's buffer through shared-memory atomics.  kappa and kappa_bar at
// the points are then summed from the stored records (the lanes share out the
// (slot, chord) pairs of all slots and add into per-point sums in shared
// memory), after which each lane takes its delta-tracking or
// ratio-tracking decision and moves its path on (camera ray -> collision ->
// NEE -> scattering).
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
constexpr int kBlocksPerSM = 4; // resident blocks per SM the kernels are built for
constexpr int kLeafQ = 160;     // queued leaves per warp (<= 31 left + 128 new)
constexpr int kChordQ = 64;     // queued chords per warp (<= 31 left + 32 new)
constexpr int kPK = 8;          // tentative points per lane and window
constexpr int kSlotCh = 256;    // stored chords per lane and window (global scratch)
constexpr int kRecF4 = 2;       // float4s per stored chord record

// One slot per lane, 47 words: an odd stride keeps same-field accesses of the
// 32 slots in distinct shared-memory banks.
struct LaneRay {
  float o[3], v[3], inv[3];
  float ta, te;                 // window [ta, te) of the ray (which spans t >= 0)
  uint32_t ray, word;
  uint32_t seed_lo, seed_hi;    // Philox key of the path's render
  int asset;                    // field of the path
  float bw[8];                  // LoD band weights
  uint32_t cx[2];               // per band: one cone with an extra weight factor (Mask::cx)
  uint32_t mask_lo, mask_hi;    // LoD cell bits
  int npts;                     // points emitted in the window (may exceed kPK)
  int nch;                      // chords stored for the window (may exceed kSlotCh)
  int hmax;                     // bits of the largest chord peak h of the window (h >= 0)
  float pt[kPK], pu[kPK];       // the window's tentative points (t, acceptance uniform)
};
static_assert(sizeof(LaneRay) % 8 == 4, "odd word stride");
struct ChordItem {
  float tc;
  float dt;           // where the walk stands (relative to tc): the chord's entry, then
                      // the last point drawn
  float dtout, h, sa, dts;
  uint32_t jd;        // majorant pieces per side J (3 bits) | next draw << 3
  uint32_t orig_own;  // original primitive index | owning slot << 26
};
static_assert(sizeof(ChordItem) == 32, "chord items of 32 bytes");
// Shared (node, slot) stack entries per warp.  A step pushes at most 128
// entries (32 four-wide nodes); above kWStack - kStackMargin the warp goes
// depth first (one entry per step, net growth <= 3 per tree level), so the
// stack holds a full step plus 40 levels of descent.
constexpr int kWStack = 640;
constexpr int kStackMargin = 248;
struct TravQ {
  int stk[kWStack];   // (node << 5) | slot
  int lq[kLeafQ];     // (sorted primitive << 5) | slot
  ChordItem cq[kChordQ];
};
// The point evaluation that follows a traversal phase reuses the queues' space:
// 64-bit fixed-point sums of kappa and kappa_bar per (slot, point), and the
// running ends of the slots' chord lists.
struct EvalQ {
  unsigned long long kap[32 * kPK], kb[32 * kPK];
  int end[33];  // chords of slots 0..s-1 to evaluate: end[s]
};
struct WarpQ {
  LaneRay r[32];
  union {
    TravQ t;  // traversal phase
    EvalQ e;  // point evaluation
  };
};

__device__ __forceinline__ unsigned long long slot_mask(const LaneRay& R) {
  return (unsigned long long)R.mask_lo | ((unsigned long long)R.mask_hi << 32);
}
__device__ __forceinline__ float ray_weight(const LaneRay& R, uint32_t cell) {
  if (!(slot_mask(R) >> cell & 1ull)) return 0.f;
  const int b = cell == 0 ? 0 : (int)((cell - 1u) >> 3) + 1;
  if (b == 0 || (R.cx[0] | R.cx[1]) == 0u) return R.bw[b];
  return R.bw[b] * cone_factor(R.cx, cell, b);
}

// byte k of x as a float, exactly: 0x4B0000xx is 2^23 + xx
__device__ __forceinline__ float byte_float(uint32_t x, int k) {
  return __int_as_float((int)__byte_perm(x, 0x4Bu, (uint32_t)k | 0x4550u)) - 8388608.0f;
}

__device__ __forceinline__ uint64_t slot_seed(const LaneRay& R) {
  return (uint64_t)R.seed_lo | ((uint64_t)R.seed_hi << 32);
}

// chord of sorted primitive j on the ray of slot R
__device__ __forceinline__ bool slot_chord(const DevField& F, const LaneRay& R, int j, Chord& ch,
                                           float& w) {
  return prim_chord(F, j, make_float3(R.o[0], R.o[1], R.o[2]), make_float3(R.v[0], R.v[1], R.v[2]),
                    0.f, INFINITY, [&](uint32_t c) { return ray_weight(R, c); }, w, ch);
}

// One draw of a queued chord's walk: the next tentative point of its majorant
// (Sec. 3) from the chord's own Philox stream, recorded for the owner when it
// falls in the window [ta, te).  Returns true when the chord may hold further
// points (c then stands at the point drawn, with the next draw index); false
// when the walk left the chord or the window, or the owner's point buffer is
// full (the owner then halves the window and redoes it).
__device__ __forceinline__ bool walk_step(const DevField& F, WarpQ& Q, ChordItem& c,
                                          const float* env, unsigned long long& npt) {
  LaneRay& R = Q.r[c.orig_own >> 26];
  const uint32_t draw = c.jd >> 3;
  if (draw >= (1u << 16)) {
    set_err(F, ERR_GUARD);
    return false;
  }
  const float invs = 1.0f / c.sa;
  const int J = (int)(c.jd & 7u);
  float dt = c.dt;
  int p = 0;  // the majorant piece holding dt
  while (p < 2 * J) {
    const float bp = p < J ? c.dts - (float)(J - p) * invs : c.dts + (float)(p - J + 1) * invs;
    if (bp <= dt) ++p;
    else break;
  }
  const uint4 x = rng4(slot_seed(R), draw, c.orig_own & kOrigMask, R.ray, R.word);
  float z = -__logf(1.0f - u01(x.x));
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
    if (dt >= c.dtout) return false;
    ++p;
  }
  if (!emit) return false;
  const float t = c.tc + dt;
  if (t >= R.te) return false;
  if (t >= R.ta) {
    ++npt;
    const int slot = atomicAdd(&R.npts, 1);
    if (slot >= kPK) return false;  // overflow: the owner halves the window and redoes it
    R.pt[slot] = t;
    R.pu[slot] = u01(x.y);
  }
  c.dt = dt;
  c.jd += 8u;
  return true;
}

// One traversal phase for the slots with want = true.  The warp shares one
// stack of (node, slot) entries: every step pops up to 32 entries from the
// frontiers of all its rays, so lanes stay busy while 32 rays are in flight.
// It collects the tentative points of each slot's window and stores the
// window's chords for their evaluation.
template <class Work>
__device__ void warp_phase(const Work& Wk, WarpQ& Q, bool want, uint32_t lane, const float* env,
                           float4* wch, Counters& cnt) {
  const unsigned lt = (1u << lane) - 1u;
  int sp = 0, lq_n = 0, cq_n = 0;  // warp-uniform sizes
  {
    // a one-primitive field has no internal node: its leaf is queued instead
    const int root = want ? Wk.field(Q.r[lane].asset).root : -1;
    const unsigned bs = __ballot_sync(kFull, want && root >= 0);
    const unsigned bl = __ballot_sync(kFull, want && root < 0);
    if (want && root >= 0) Q.t.stk[__popc(bs & lt)] = (root << 5) | (int)lane;
    if (want && root < 0) Q.t.lq[__popc(bl & lt)] = (0 << 5) | (int)lane;
    sp = __popc(bs);
    lq_n = __popc(bl);
    __syncwarp();
  }
  const long long max_it = 4 * (Wk.max_n() + 64) + 4096;
  for (long long it = 0;; ++it) {
    if (it > max_it * 32) {
      if (lane == 0) set_err(Wk.err_field(), ERR_GUARD);
      break;
    }
    // ---------------- one traversal step: up to 32 (four-wide node, slot) entries
    GF_TIC(t_step);
    int take = sp < 32 ? sp : 32;
    if (sp > kWStack - kStackMargin) take = 1;  // near capacity: depth first
    const int ent = (int)lane < take ? Q.t.stk[sp - take + (int)lane] : -1;
    __syncwarp();
    sp -= take;
    if (lane == 0) ++cnt.steps;
    int slot = 0;
    int ch[4] = {0, 0, 0, 0};
    unsigned hit = 0u;  // bit k: child k overlaps the window and the ray's cells
    if (ent >= 0 && (int64_t)(ent >> 5) >= Wk.field(Q.r[ent & 31].asset).n_nodes4) {
      set_err(Wk.err_field(), ERR_INDEX);  // a node beyond the tree: skipped
    } else if (ent >= 0) {
      const int node = ent >> 5;
      slot = ent & 31;
      const LaneRay& R = Q.r[slot];
      const float3 o = make_float3(R.o[0], R.o[1], R.o[2]);
      const float3 inv = make_float3(R.inv[0], R.inv[1], R.inv[2]);
      const unsigned long long mask = slot_mask(R);
      const Node4* N = Wk.field(R.asset).nodes4 + node;
      const float4 v0 = __ldg(&N->v0), v1 = __ldg(&N->v1);
      const uint4 q = __ldg(&N->q);
      const int4 c4 = __ldg(&N->child);
      const uint4 m01 = __ldg(&N->m01), m23 = __ldg(&N->m23);
      ++cnt.nodes;
      const uint32_t qlx = __float_as_uint(v1.z), qly = __float_as_uint(v1.w);
      // slab distances straight from the codes: t = (lo + c s - o) inv = c (s inv) + (lo - o) inv
      const float ax = v0.w * inv.x, ay = v1.x * inv.y, az = v1.y * inv.z;
      const float bx = (v0.x - o.x) * inv.x, by = (v0.y - o.y) * inv.y, bz = (v0.z - o.z) * inv.z;
      const unsigned long long mk[4] = {
          (unsigned long long)m01.x | ((unsigned long long)m01.y << 32),
          (unsigned long long)m01.z | ((unsigned long long)m01.w << 32),
          (unsigned long long)m23.x | ((unsigned long long)m23.y << 32),
          (unsigned long long)m23.z | ((unsigned long long)m23.w << 32)};
      ch[0] = c4.x;
      ch[1] = c4.y;
      ch[2] = c4.z;
      ch[3] = c4.w;
      // near and far planes by the ray's direction signs, chosen once per node
      const uint32_t nx = inv.x >= 0.f ? qlx : q.y, fx = inv.x >= 0.f ? q.y : qlx;
      const uint32_t ny = inv.y >= 0.f ? qly : q.z, fy = inv.y >= 0.f ? q.z : qly;
      const uint32_t nz = inv.z >= 0.f ? q.x : q.w, fz = inv.z >= 0.f ? q.w : q.x;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float txn = fmaf(byte_float(nx, k), ax, bx), txf = fmaf(byte_float(fx, k), ax, bx);
        const float tyn = fmaf(byte_float(ny, k), ay, by), tyf = fmaf(byte_float(fy, k), ay, by);
        const float tzn = fmaf(byte_float(nz, k), az, bz), tzf = fmaf(byte_float(fz, k), az, bz);
        const float tn = fmaxf(fmaxf(txn, tyn), fmaxf(tzn, R.ta));
        const float tf = fminf(fminf(txf, tyf), fminf(tzf, R.te));
        if ((mk[k] & mask) && tn <= tf) hit |= 1u << k;
      }
    }
    // ---------------- push internal children, queue leaves: per child slot k a
    // ballot places the lanes' entries contiguously (no bank conflicts)
    {
      int np = 0, nl = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool h = (hit >> k & 1u) != 0u;
        const unsigned bp = __ballot_sync(kFull, h && ch[k] >= 0);
        const unsigned bl = __ballot_sync(kFull, h && ch[k] < 0);
        if (h && ch[k] >= 0) {
          const int pos = sp + np + __popc(bp & lt);
          if (pos < kWStack) Q.t.stk[pos] = (ch[k] << 5) | slot;
        }
        if (h && ch[k] < 0) Q.t.lq[lq_n + nl + __popc(bl & lt)] = (~ch[k] << 5) | slot;
        np += __popc(bp);
        nl += __popc(bl);
      }
      if (sp + np > kWStack) {
        if (lane == 0) set_err(Wk.err_field(), ERR_STACK);
        np = kWStack - sp;
      }
      sp += np;
      lq_n += nl;
      __syncwarp();
    }
    const bool any_trav = sp > 0;
    if (lane == 0) GF_TOC(cnt, 0, t_step);
    // ---------------- leaf rounds: 32 leaves of any slots' rays at a time; once
    // the traversal is over, the last leaves and then the last chords (one
    // walk site, for the instruction cache)
    while (lq_n >= 32 || (!any_trav && (lq_n > 0 || cq_n > 0))) {
      const int tk = lq_n < 32 ? lq_n : 32;
      bool have = (int)lane < tk;
      int j = 0, own = 0;
      if (have) {
        const int e = Q.t.lq[lq_n - tk + (int)lane];
        j = e >> 5;
        own = e & 31;
        if ((int64_t)j >= Wk.field(Q.r[own].asset).n) {  // a leaf beyond the records
          set_err(Wk.err_field(), ERR_INDEX);
          have = false;
        }
      }
      __syncwarp();
      lq_n -= tk;
      cnt.leaves += have ? 1ull : 0ull;
      GF_TIC(t_leaf);
      bool ok = false;
      ChordItem ci;
      if (have) {
        const LaneRay& R = Q.r[own];
        Chord ch;
        float w;
        if (slot_chord(Wk.field(R.asset), R, j, ch, w)) {
          const float tin = ch.tc + ch.dtin, tout = ch.tc + ch.dtout;
          if (tin < R.te && tout >= R.ta) {
            ok = true;
            const float wa = w * ch.absA;
            const float h = wa * expf(-0.5f * ch.qmin), sa = sqrtf(ch.a);
            // evaluation record for the points of this window
            atomicMax(&Q.r[own].hmax, __float_as_int(h));
            const int k = atomicAdd(&Q.r[own].nch, 1);
            if (k < kSlotCh) {
              // centred on the envelope peak t* = tc + dts: exponent y2 dt^2 + log2 h,
              // phase B dt + delta*, majorant piece floor(|dt| sqrt(a))
              float4* dst = wch + ((size_t)own * kSlotCh + k) * kRecF4;
              dst[0] = make_float4(ch.tc + ch.dts, tin, tout, ch.B);
              dst[1] = make_float4(-0.5f * kLog2e * ch.a, __log2f(h),
                                   reduce_2pi(fmaf(ch.B, ch.dts, ch.delta)), sa);
            }
            ci.tc = ch.tc;
            ci.dt = ch.dtin;
            ci.dtout = ch.dtout;
            ci.h = h;
            ci.sa = sa;
            ci.dts = ch.dts;
            // majorant pieces per side: whitened half-length sa hw rounded up, less one
            int J = (int)ceilf(sa * ch.hw) - 1;
            J = J < 0 ? 0 : (J > 6 ? 6 : J);
            ci.jd = (uint32_t)J;
            ci.orig_own = ch.orig | ((uint32_t)own << 26);
          }
        }
      }
      const unsigned bc = __ballot_sync(kFull, ok);
      if (ok) Q.t.cq[cq_n + __popc(bc & lt)] = ci;
      cq_n += __popc(bc);
      cnt.chords += ok ? 1ull : 0ull;
      __syncwarp();
      if (lane == 0) GF_TOC(cnt, 1, t_leaf);
      GF_TIC(t_walk);
      const bool drain = !any_trav && lq_n == 0;
      while (cq_n >= 32 || (drain && cq_n > 0)) {
        const int tw = cq_n < 32 ? cq_n : 32;
        const bool hv = (int)lane < tw;
        ChordItem cw;
        if (hv) cw = Q.t.cq[cq_n - tw + (int)lane];
        __syncwarp();
        cq_n -= tw;
        // one draw per chord and round; chords that may hold more points go back
        // to the queue, so every round keeps the lanes busy
        const bool again = hv && walk_step(Wk.err_field(), Q, cw, env, cnt.points);
        const unsigned ba = __ballot_sync(kFull, again);
        if (again) Q.t.cq[cq_n + __popc(ba & lt)] = cw;
        cq_n += __popc(ba);
        __syncwarp();
      }
      if (lane == 0) GF_TOC(cnt, 2, t_walk);
    }
    if (!any_trav && lq_n == 0 && cq_n == 0) break;
  }
  __syncwarp();
}

// per-lane path state
struct PathState {
  int rq;         // request of the pixel (0 for a single render)
  int pix;        // -1: no pixel
  int s, b;       // sample, bounce
  int s_end;      // end of the lane's sample range of the pixel
  int kind;       // 0 idle, 1 delta tracking, 2 ratio tracking (NEE)
  long long acc;  // sum of the range's samples in fixed point (2^-32 units)
  float Lsum, thr, T;
  float3 o, v;    // current ray
  float t0, t1;   // scene span of the current ray
  float step;     // window length for delta tracking
  unsigned long long allow;  // cells the foveation keeps for the sample's path
};

__device__ __forceinline__ void set_slot(LaneRay& R, float3 o, float3 v, const Mask& m,
                                         uint32_t ray, uint32_t word) {
  R.o[0] = o.x; R.o[1] = o.y; R.o[2] = o.z;
  R.v[0] = v.x; R.v[1] = v.y; R.v[2] = v.z;
  const float3 iv = safe_inv(v);
  R.inv[0] = iv.x; R.inv[1] = iv.y; R.inv[2] = iv.z;
  R.ray = ray;
  R.word = word;
  R.mask_lo = (uint32_t)m.bits;
  R.mask_hi = (uint32_t)(m.bits >> 32);
#pragma unroll
  for (int k = 0; k < 8; ++k) R.bw[k] = m.bw[k];
  R.cx[0] = m.cx[0];
  R.cx[1] = m.cx[1];
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
// stored.  The lanes share out the (slot, chord) pairs of all slots evenly, so
// no lane waits on one slot's short list; each pair tests the chord against
// the slot's points and adds its terms to the slot's sums in shared memory.
// The sums are exact in 64-bit fixed point: a term is at most the peak h of
// its chord, so with H the largest peak of the slot's window and at most
// kSlotCh = 2^8 chords, scaling by 2^(54 - e) (H < 2^e) keeps every partial
// sum below 2^62.  Each term is rounded once (to 2^(e-54), far below FP32
// resolution) and integer addition does not depend on order, so a path's
// decisions do not depend on which other rays shared its warp or on the order
// in which its chords were stored or evaluated.
__device__ __forceinline__ int slot_exp(const LaneRay& R) {
  const int ex = ((R.hmax >> 23) & 0xFF) - 126;  // H < 2^ex
  return ex < -70 ? -70 : ex;
}
__device__ void eval_stored(WarpQ& Q, const float4* wch, const float* env, uint32_t lane,
                            Counters& cnt) {
  LaneRay& Rl = Q.r[lane];
  const int ns_l = Rl.npts;  // 0: no points (or an overflowed window)
  const int m = ns_l > 0 ? Rl.nch : 0;
  int incl = m;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if ((int)lane >= o) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  EvalQ& E = Q.e;
  E.end[lane + 1] = incl;
  if (lane == 0) E.end[0] = 0;
#pragma unroll
  for (int i = 0; i < kPK; ++i) {
    E.kap[i * 32 + lane] = 0ull;
    E.kb[i * 32 + lane] = 0ull;
  }
  __syncwarp();
  // lane l takes the pairs [l per, (l + 1) per): a lane stays within one slot
  // for most of its pairs, and lanes of a long list sit in different slots at
  // any moment, so the atomics below rarely meet on one address.  Each pair's
  // record is loaded one pair ahead, so that its latency overlaps the work on
  // the pair before.
  const int per = (total + 31) >> 5;
  int f = (int)lane * per;
  const int fe = min(f + per, total);
  int s = 0;  // the slot of pair f: the number of slot ends at or below f
  float4 an = make_float4(0.f, 0.f, 0.f, 0.f), bn = an;
  if (f < fe) {
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
      if (E.end[s + w] <= f) s += w;
    const float4* rec = wch + ((size_t)s * kSlotCh + (f - E.end[s])) * kRecF4;
    an = rec[0];
    bn = rec[1];
  }
  for (; f < fe; ++f) {
    const float4 a = an, b = bn;
    const int sc = s;
    if (f + 1 < fe) {
      while (E.end[s + 1] <= f + 1) ++s;  // the next slot with chords (f + 1 < end[32])
      const float4* rec = wch + ((size_t)s * kSlotCh + (f + 1 - E.end[s])) * kRecF4;
      an = rec[0];
      bn = rec[1];
    }
    const LaneRay& R = Q.r[sc];
    const int ex = slot_exp(R);
    const float S = __int_as_float((127 + 54 - ex) << 23);  // 2^(54 - ex)
    const int ns = R.npts;
    for (int i = 0; i < ns; ++i) {
      const float t = R.pt[i];
      if (t > a.z) break;  // the points are sorted by t
      if (t >= a.y) {
        const float dt = t - a.x;
        const long long k1 =
            __float2ll_rn(ex2f(fmaf(b.x, dt * dt, b.y)) * cosf_fast(fmaf(a.w, dt, b.z)) * S);
        int mm = (int)(fabsf(dt) * b.w);
        mm = mm > 7 ? 7 : mm;
        const long long k2 = __float2ll_rn(ex2f(b.y + env[8 + mm]) * S);  // h exp(-m^2/2)
        atomicAdd(&E.kap[i * 32 + sc], (unsigned long long)k1);
        atomicAdd(&E.kb[i * 32 + sc], (unsigned long long)k2);
        ++cnt.evals;
      }
    }
  }
  __syncwarp();
}
// kappa (k = 0) or kappa_bar (k = 1) at point i of the calling lane's slot,
// from the sums eval_stored left
__device__ __forceinline__ float slot_sum(const WarpQ& Q, uint32_t lane, int i, int k) {
  const unsigned long long v = (k ? Q.e.kb : Q.e.kap)[i * 32 + lane];
  return __ll2float_rn((long long)v) * __int_as_float((127 - 54 + slot_exp(Q.r[lane])) << 23);
}

// ---------------------------------------------------------------------------
// Work sources.  A lane takes pixels one at a time; a pixel belongs to a
// request (its camera, LoD descriptors, seed and framebuffer) and a request to
// a field.  A single render is one request on one field; the render server
// hands the kernel a batch of items from many requests on several fields.
// ---------------------------------------------------------------------------
// Radiance samples are summed in 64-bit fixed point (2^-32 units): a pixel's
// value then does not depend on how its samples were split between lanes or
// in which order the partial sums arrived.
constexpr float kFixScale = 4294967296.0f;  // 2^32
__device__ __forceinline__ long long fix_sample(float L) { return __float2ll_rn(L * kFixScale); }
__device__ __forceinline__ float fix_mean(long long sum, int spp) {
  return __ll2float_rn(sum) * (1.0f / kFixScale) / (float)spp;
}

// A single render: units of `chunk` consecutive samples of one pixel, so the
// lanes stay busy to the end of the launch; partial sums meet in acc64.
struct ImageWork {
  const DevField* F;
  const PathParams* P;
  unsigned long long* acc64;
  int* counter;
  int npix, chunk, nchunk;
  __device__ const DevField& field(int) const { return *F; }
  __device__ const DevField& err_field() const { return *F; }
  __device__ int64_t max_n() const { return F->n; }
  __device__ const PathParams& params(int) const { return *P; }
  __device__ int asset(int) const { return 0; }
  __device__ bool next(int& rq, int& pix, int& s0, int& s1) const {
    const int u = atomicAdd(counter, 1);
    rq = 0;
    if (u >= npix * nchunk) return false;
    pix = u / nchunk;
    s0 = P->s0 + (u - pix * nchunk) * chunk;
    s1 = min(s0 + chunk, P->s0 + P->spp);
    return true;
  }
  __device__ void finish(int, int pix, long long acc) const {
    atomicAdd(acc64 + pix, (unsigned long long)acc);
  }
};

struct ServerWork {
  const ServerLaunch* L;
  __device__ const DevField& field(int a) const { return L->fields[a]; }
  __device__ const DevField& err_field() const { return L->fields[0]; }
  __device__ int64_t max_n() const { return L->max_n; }
  __device__ const PathParams& params(int rq) const { return L->reqs[rq].P; }
  __device__ int asset(int rq) const { return L->reqs[rq].asset; }
  // the batch's units (chunk consecutive samples of one pixel) are numbered
  // 0..total-1 item after item; a lane takes the next number and finds its
  // item by binary search over the item bases
  __device__ bool next(int& rq, int& pix, int& s0, int& s1) const {
    const int f = atomicAdd(L->counter, 1);
    if (f >= L->total) return false;
    int lo = 0, hi = L->n_items - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (L->items[mid].base <= f) lo = mid;
      else hi = mid - 1;
    }
    const ServerItem it = L->items[lo];
    rq = it.req;
    const ServerReqDev& R = L->reqs[rq];
    const int u = f - it.base, q = u / R.nchunk;
    pix = it.pix0 + q;
    s0 = R.P.s0 + (u - q * R.nchunk) * R.chunk;
    s1 = min(s0 + R.chunk, R.P.s0 + R.P.spp);
    return true;
  }
  // partial sums of a pixel's samples meet in the request's fixed-point sums
  __device__ void finish(int rq, int pix, long long acc) const {
    atomicAdd(L->reqs[rq].acc + pix, (unsigned long long)acc);
  }
};

// The paths of one warp: each lane runs its pixels' samples in order (camera
// ray -> delta tracking -> NEE by ratio tracking -> isotropic scattering), the
// tracking windows of all 32 lanes advancing together through warp_phase.
template <class Work>
__device__ __forceinline__ void render_paths(const Work& Wk, const float* env, WarpQ& Q,
                                             float4* wch) {
  const uint32_t lane = threadIdx.x & 31u;
  LaneRay& R = Q.r[lane];
  Counters cnt;
  const float inv4pi = 0.25f / 3.14159265358979f;

  PathState S;
  S.rq = 0;
  S.pix = -1;
  S.kind = 0;
  S.acc = 0;
  S.allow = ~0ull;

  // Move the lane's path on from its finished ray (hit: a collision at th on a
  // tracking ray; kind 0: the lane has no path yet) until a new ray starts or
  // no work is left: collision -> NEE, NEE -> isotropic scattering, escape or
  // the last bounce -> the next sample (or pixel).  Every kind of ray is
  // started from one site, which keeps the loop small for the instruction cache.
  auto advance = [&](bool hit, float th) {
    for (int guard = 0; guard < (1 << 20); ++guard) {
      int kind = 0;  // the ray to start: 1 tracking (camera or bounce), 2 NEE
      float3 ro = S.o, rv = S.v;
      bool nee = false;
      if (S.kind == 1 && hit) {
        // collision: next-event estimation towards the light
        const PathParams& P = Wk.params(S.rq);
        ro = make_float3(S.o.x + th * S.v.x, S.o.y + th * S.v.y, S.o.z + th * S.v.z);
        rv = P.light;
        S.thr *= P.albedo;
        S.T = 1.f;
        kind = 2;
        nee = true;
      } else if (S.kind == 2) {
        // NEE finished with transmittance S.T: add it, then scatter isotropically
        const PathParams& P = Wk.params(S.rq);
        S.Lsum += S.thr * P.irradiance * S.T * inv4pi;
        const uint4 y = rng4(P.seed, 0, kNoPrim, (uint32_t)S.pix,
                             stream_word((uint32_t)S.s, (uint32_t)S.b, TAG_SCATTER));
        const float z = 1.0f - 2.0f * u01(y.x);
        const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
        float sn, cs;
        sincosf(2.0f * 3.14159265358979f * u01(y.y), &sn, &cs);
        S.b += 1;
        if (S.b < P.max_bounces) {
          rv = make_float3(rr * cs, rr * sn, z);
          kind = 1;
        }
      }
      if (kind == 0) {
        // the sample is over (escape or last bounce): the next sample, or pixel
        if (S.kind != 0) {
          S.acc += fix_sample(S.Lsum);
          S.s += 1;
        }
        for (;;) {
          if (S.pix < 0) {
            int rq = 0, pix = -1, s0 = 0, s1 = 0;
            if (!Wk.next(rq, pix, s0, s1)) {
              S.pix = -1;
              S.kind = 0;
              return;
            }
            const PathParams& P = Wk.params(rq);
            S.rq = rq;
            S.pix = pix;
            S.s = s0;
            S.s_end = s1;
            S.acc = 0;
            R.asset = Wk.asset(rq);
            R.seed_lo = (uint32_t)P.seed;
            R.seed_hi = (uint32_t)(P.seed >> 32);
          }
          if (S.s < S.s_end) break;
          Wk.finish(S.rq, S.pix, S.acc);
          S.pix = -1;
        }
        const PathParams& P = Wk.params(S.rq);
        camera_ray(P.cam, P.seed, S.pix % P.cam.W, S.pix / P.cam.W, S.s, ro, rv);
        S.b = 0;
        S.thr = 1.f;
        S.Lsum = 0.f;
        S.allow = fov_cells(Wk.field(R.asset), P, rv, (uint32_t)S.pix, (uint32_t)S.s);
        kind = 1;
      }
      const PathParams& P = Wk.params(S.rq);
      const DevField& F = Wk.field(R.asset);
      Mask m = sample_mask(F, nee ? P.lod_nee : P.lod, rv, P.seed, (uint32_t)S.pix, (uint32_t)S.s,
                           (uint32_t)S.b, nee ? TAG_NEE_MASK : TAG_MASK);
      m.bits &= S.allow;
      cnt.rays += 1;
      if (start_ray(F, R, S, kind, ro, rv, m, (uint32_t)S.pix,
                    stream_word((uint32_t)S.s, (uint32_t)S.b, nee ? TAG_NEE : TAG_TRACK)))
        return;
      // the ray misses every primitive: it is over at once (no collision; T = 1 for NEE)
      hit = false;
    }
    set_err(Wk.err_field(), ERR_GUARD);
    S.kind = 0;
  };

  // the first pass takes each lane's first work; every later pass is one window
  bool first = true;
  for (int guard = 0; guard < (1 << 30); ++guard) {
    bool fin = first, fhit = false;
    float fth = 0.f;
    const bool want = S.kind != 0;
    if (!first && !__any_sync(kFull, want)) break;
    if (!first) {
      // ---- pass 1: tentative points of the window
      R.npts = 0;
      R.nch = 0;
      R.hmax = 0;
      __syncwarp();
      warp_phase(Wk, Q, want, lane, env, wch, cnt);
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
      }
      cnt.windows += want ? 1ull : 0ull;
      __syncwarp();
      // ---- kappa and kappa_bar at the points, from the stored chords
      GF_TIC(t_eval);
      if (__any_sync(kFull, want && n > 0)) eval_stored(Q, wch, env, lane, cnt);
      if (lane == 0) GF_TOC(cnt, 3, t_eval);
      // ---- decisions: the window either continues the ray or finishes it
      GF_TIC(t_dec);
      if (want) {
        const bool last = R.te >= S.t1;
        bool next_window = false;
        if (ovf) {
          const float w = R.te - R.ta;
          if (w <= 1e-6f * (1.0f + fabsf(R.ta))) {
            // more than kPK points at one t: give up on this ray
            set_err(Wk.err_field(), ERR_POINTS);
            fin = true;
          } else {
            R.te = R.ta + 0.5f * w;
            S.step = 0.5f * w;
          }
        } else if (S.kind == 1) {
          for (int i = 0; i < n && !fhit; ++i) {
            if (R.pu[i] * slot_sum(Q, lane, i, 1) < fmaxf(slot_sum(Q, lane, i, 0), 0.f)) {
              fhit = true;
              fth = R.pt[i];
            }
          }
          fin = fhit || last;
          next_window = !fin;
        } else {
          for (int i = 0; i < n; ++i) {
            const float kb = slot_sum(Q, lane, i, 1);
            if (kb > 0.f) S.T *= 1.f - fmaxf(slot_sum(Q, lane, i, 0), 0.f) / kb;
          }
          if (!last) S.step *= 2.0f;
          fin = last;
          next_window = !last;
        }
        if (next_window) {
          R.ta = R.te;
          R.te = fminf(S.t1, R.ta + S.step);
          if (R.te >= S.t1) R.te = S.t1 * (1.0f + 1e-7f) + 1e-30f;
        }
      }
      if (lane == 0) GF_TOC(cnt, 4, t_dec);
    }
    first = false;
    if (fin) advance(fhit, fth);
    __syncwarp();
  }
  flush_counters(Wk.err_field(), cnt, lane);
}

__device__ __forceinline__ WarpQ& setup_block(unsigned char* smraw, const float* env_src) {
  // env[0..7] = exp(-n^2/2), env[8..15] = its log2 (-n^2 log2(e) / 2)
  float* env = reinterpret_cast<float*>(smraw);
  WarpQ* Qs = reinterpret_cast<WarpQ*>(smraw + 64);
  if (threadIdx.x < 8) {
    env[threadIdx.x] = env_src[threadIdx.x];
    env[8 + threadIdx.x] = -0.5f * kLog2e * (float)(threadIdx.x * threadIdx.x);
  }
  __syncthreads();
  return Qs[threadIdx.x >> 5];
}

__device__ __forceinline__ float4* warp_store(float4* chord_store) {
  return chord_store + ((size_t)blockIdx.x * kWWarps + (threadIdx.x >> 5)) * 32 * kSlotCh * kRecF4;
}

__global__ void __launch_bounds__(kWWarps * 32, kBlocksPerSM)
    k_render_scatter(const __grid_constant__ DevField F, const __grid_constant__ PathParams P,
                     unsigned long long* acc64, int* counter, int chunk, float4* chord_store) {
  extern __shared__ __align__(16) unsigned char smraw[];
  WarpQ& Q = setup_block(smraw, F.env);
  const ImageWork Wk{&F, &P, acc64, counter, P.cam.W * P.cam.H, chunk, (P.spp + chunk - 1) / chunk};
  render_paths(Wk, reinterpret_cast<const float*>(smraw), Q, warp_store(chord_store));
}

__global__ void k_fix_to_image(const unsigned long long* acc64, int64_t npix, int spp, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npix) out[i] = fix_mean((long long)acc64[i], spp);
}

__global__ void __launch_bounds__(kWWarps * 32, kBlocksPerSM)
    k_render_server(const __grid_constant__ ServerLaunch L, float4* chord_store) {
  extern __shared__ __align__(16) unsigned char smraw[];
  WarpQ& Q = setup_block(smraw, L.fields[0].env);
  const ServerWork Wk{&L};
  render_paths(Wk, reinterpret_cast<const float*>(smraw), Q, warp_store(chord_store));
}

size_t scatter_smem_bytes() { return 64 + sizeof(WarpQ) * kWWarps; }
// 228 KB of shared memory per SM, 1 KB of it reserved per resident block
static_assert((64 + sizeof(WarpQ) * kWWarps + 1024) * kBlocksPerSM <= 233472,
              "kBlocksPerSM blocks fit one SM's shared memory");

size_t scatter_store_bytes(int64_t grid) {
  return (size_t)grid * kWWarps * 32 * kSlotCh * kRecF4 * sizeof(float4);
}

// persistent grid of the scattering kernels: every SM filled, never more
// warps than work (4 warps x 32 lanes per block)
template <class K>
static cudaError_t scatter_grid(K kernel, int sm_count, int64_t pixels, int64_t& g) {
  const size_t smem = scatter_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWWarps * 32, smem) != cudaSuccess)
    (void)cudaGetLastError();
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (pixels + kWWarps * 32 - 1) / (kWWarps * 32);
  g = (int64_t)sm_count * per_sm;
  if (need < g) g = need;
  if (g < 1) g = 1;
  return cudaSuccess;
}

// pixel sums (8 bytes per pixel) and the per-warp chord store of a full
// persistent grid, grown through the field's allocator
cudaError_t ensure_render_scratch(const Field& F, int64_t npix, cudaStream_t s) {
  int64_t g = 1;
  cudaError_t e = scatter_grid(k_render_scatter, F.ctx.sm_count, (int64_t)1 << 40, g);
  if (e != cudaSuccess) return e;
  if ((e = grow(F, (void**)&F.acc64, F.acc_bytes, (size_t)npix * 8, s)) != cudaSuccess) return e;
  return grow(F, (void**)&F.wscratch, F.wscratch_bytes, scatter_store_bytes(g), s);
}

cudaError_t launch_render_scatter(const Field& F, const PathParams& P, float* out, cudaStream_t s) {
  (void)cudaGetLastError();  // a stale error of an unrelated call is not ours
  cudaError_t e = cudaMemsetAsync(F.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int64_t npix = (int64_t)P.cam.W * P.cam.H;
  int64_t g = 1;
  if ((e = scatter_grid(k_render_scatter, F.ctx.sm_count, npix * P.spp, g)) != cudaSuccess) return e;
  // about 16 units per lane: chunk = ceil(npix spp / (16 lanes)), in [1, spp]
  const int64_t lanes = g * kWWarps * 32;
  int64_t chunk = (npix * P.spp + 16 * lanes - 1) / (16 * lanes);
  chunk = chunk < 1 ? 1 : (chunk > P.spp ? P.spp : chunk);
  const int64_t nchunk = (P.spp + chunk - 1) / chunk;
  if (npix * nchunk >= (int64_t)INT_MAX) return cudaErrorInvalidValue;
  // fixed-point pixel sums and the chord store (allocated ahead by gf_reserve, else here)
  if ((e = ensure_render_scratch(F, npix, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(F.acc64, 0, (size_t)npix * 8, s)) != cudaSuccess) return e;
  k_render_scatter<<<(unsigned)g, kWWarps * 32, scatter_smem_bytes(), s>>>(
      F.dev, P, F.acc64, F.counter, (int)chunk, F.wscratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_fix_to_image<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(F.acc64, npix, P.spp, out);
  return cudaGetLastError();
}

cudaError_t server_grid(int sm_count, int64_t& g) {
  (void)cudaGetLastError();
  return scatter_grid(k_render_server, sm_count, (int64_t)1 << 40, g);
}

cudaError_t launch_fix_to_image(const unsigned long long* acc, int64_t npix, int spp, float* out,
                                cudaStream_t s) {
  k_fix_to_image<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(acc, npix, spp, out);
  return cudaGetLastError();
}

cudaError_t launch_render_server(const ServerLaunch& L, int64_t grid, float4* chord_store,
                                 cudaStream_t s) {
  (void)cudaGetLastError();
  k_render_server<<<(unsigned)grid, kWWarps * 32, scatter_smem_bytes(), s>>>(L, chord_store);
  return cudaGetLastError();
}

}  // namespace gf
