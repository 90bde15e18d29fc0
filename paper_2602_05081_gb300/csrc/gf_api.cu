// gf_api.cu -- the C ABI of include/gf.h: argument checks, memory ownership,
// host-buffer staging and error mapping around the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gf_host.h"
#include "gf_trace.cuh"

using namespace gf;

namespace {

thread_local std::string g_err;

gf_status fail(gf_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
gf_status cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}
#define GF_CUDA(call, where)                   \
  do {                                         \
    cudaError_t _e = (call);                   \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on the
// three-term Legendre recurrence (double precision)
void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void cone_axes(float axes[kCones][3]) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < kCones; ++k) {
    double z = 1.0 - (k + 0.5) / kCones;
    double r = std::sqrt(1.0 - z * z);
    double ph = k * pi * (3.0 - std::sqrt(5.0));
    axes[k][0] = (float)(r * std::cos(ph));
    axes[k][1] = (float)(r * std::sin(ph));
    axes[k][2] = (float)z;
  }
}

struct Staging {
  std::vector<std::pair<void*, const void*>> back;  // device -> host copies
};

// device view of a caller buffer: the pointer itself, or a slice of the
// field's staging area (copied in when `in`)
gf_status stage(Field& F, const void* p, size_t bytes, bool in, cudaStream_t s, size_t& off,
                void** out) {
  if (!p || is_device_ptr(p)) {
    *out = const_cast<void*>(p);
    return GF_OK;
  }
  size_t need = off + ((bytes + 255) & ~size_t(255));
  if (need > F.stage_bytes) return fail(GF_ESTATE, "staging area too small");
  void* d = (char*)F.stage + off;
  off = need;
  if (in) GF_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s), "stage in");
  *out = d;
  return GF_OK;
}

// Host buffers of the context-free test helpers (gf_philox, gf_faddeeva) pass
// through this fixed device array in chunks, so those calls allocate nothing;
// a mutex serialises them.
constexpr size_t kHelperBytes = 1u << 20;
static __device__ __align__(256) unsigned char g_helper[kHelperBytes];
std::mutex g_helper_mu;
void* g_helper_dev[64] = {nullptr};

gf_status helper_area(void** out) {
  int dev = 0;
  GF_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(GF_EINVAL, "device index beyond 63");
  if (!g_helper_dev[dev]) GF_CUDA(cudaGetSymbolAddress(&g_helper_dev[dev], g_helper), "helper area");
  *out = g_helper_dev[dev];
  return GF_OK;
}

gf_status ensure_stage(Field& F, size_t bytes, cudaStream_t s) {
  GF_CUDA(grow(F, &F.stage, F.stage_bytes, bytes, s), "staging alloc");
  return GF_OK;
}

}  // namespace

namespace gf {
cudaError_t dev_alloc(const Ctx& c, void** p, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (!c.alloc.alloc) return cudaMalloc(p, bytes);
  void* q = c.alloc.alloc(c.alloc.user, bytes, (gf_stream)s);
  if (!q) return cudaErrorMemoryAllocation;
  *p = q;
  return cudaSuccess;
}

void dev_free(const Ctx& c, void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (!c.alloc.free) {
    cudaFree(p);
    return;
  }
  c.alloc.free(c.alloc.user, p, bytes, (gf_stream)s);
}

cudaError_t grow(const Field& F, void** p, size_t& have, size_t bytes, cudaStream_t s) {
  if (bytes <= have && *p) return cudaSuccess;
  if (*p) {
    // earlier calls (on any stream) may still read the old buffer
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    F.mem.release(*p, s);
    *p = nullptr;
    have = 0;
  }
  const cudaError_t e = F.mem.alloc(p, bytes, s);
  if (e == cudaSuccess) have = bytes;
  return e;
}

// The field's device error word, read after the stream has been synchronised
// (host-buffer paths): mapped to a status and cleared, as gf_sync does.
gf_status take_device_error(Field& F) {
  int err = 0;
  GF_CUDA(cudaMemcpy(&err, F.err, 4, cudaMemcpyDeviceToHost), "read error word");
  if (!err) return GF_OK;
  GF_CUDA(cudaMemset(F.err, 0, 4), "clear error word");
  if (err & (ERR_STACK | ERR_WINDOW | ERR_POINTS))
    return fail(GF_EOVERFLOW, "device buffer overflow (code " + std::to_string(err) + ")");
  if (err & ERR_GUARD) return fail(GF_ETIMEOUT, "bounded device loop gave up");
  if (err & ERR_INDEX) return fail(GF_ECUDA, "a tree index left its array (access skipped)");
  return fail(GF_EINVAL, "device-side input error (code " + std::to_string(err) + ")");
}

bool lod_ok(const gf_lod_desc* l) {
  return l && l->freq_policy >= 0 && l->freq_policy <= 6 && l->cone_policy >= 0 &&
         l->cone_policy <= 4 && l->max_band >= 0 && l->max_band <= 7 && l->beta >= 0.f &&
         l->beta < 1.f && l->delta >= 0.f && l->delta <= 1.f;
}

LodDev lod_dev(const gf_lod_desc& l) {
  return LodDev{l.freq_policy, l.max_band, l.cone_policy, l.beta, l.delta};
}

gf_status camera_params(const gf_camera* c, const gf_render_opts* o, uint64_t seed,
                        const Field& F, PathParams& P) {
  if (!c || !o) return fail(GF_EINVAL, "camera/opts null");
  if (c->width < 1 || c->height < 1 || (int64_t)c->width * c->height > (1ll << 31) - 1)
    return fail(GF_EINVAL, "bad image size");
  if (o->spp < 1 || o->spp > (1 << 20)) return fail(GF_EINVAL, "spp must be in [1, 2^20]");
  if (o->max_bounces < 0 || o->max_bounces > 15) return fail(GF_EINVAL, "max_bounces in [0, 15]");
  if (o->integrator != GF_INTEG_TOMO && o->integrator != GF_INTEG_SCATTER)
    return fail(GF_EINVAL, "bad integrator");
  if (!(c->vfov_deg > 0.f && c->vfov_deg < 180.f)) return fail(GF_EINVAL, "vfov in (0,180)");
  double e[3] = {c->eye[0], c->eye[1], c->eye[2]};
  double f[3] = {c->look_at[0] - e[0], c->look_at[1] - e[1], c->look_at[2] - e[2]};
  double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(fn > 0)) return fail(GF_EINVAL, "eye == look_at");
  for (double& x : f) x /= fn;
  double u[3] = {c->up[0], c->up[1], c->up[2]};
  double r[3] = {u[1] * f[2] - u[2] * f[1], u[2] * f[0] - u[0] * f[2], u[0] * f[1] - u[1] * f[0]};
  double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(rn > 0)) return fail(GF_EINVAL, "up parallel to view direction");
  for (double& x : r) x /= rn;
  double uv[3] = {f[1] * r[2] - f[2] * r[1], f[2] * r[0] - f[0] * r[2], f[0] * r[1] - f[1] * r[0]};
  P.cam.eye = make_float3((float)e[0], (float)e[1], (float)e[2]);
  P.cam.fw = make_float3((float)f[0], (float)f[1], (float)f[2]);
  P.cam.rt = make_float3((float)r[0], (float)r[1], (float)r[2]);
  P.cam.up = make_float3((float)uv[0], (float)uv[1], (float)uv[2]);
  P.cam.tanh = (float)std::tan(0.5 * (double)c->vfov_deg * 3.14159265358979323846 / 180.0);
  P.cam.aspect = (float)((double)c->width / (double)c->height);
  P.cam.W = c->width;
  P.cam.H = c->height;
  P.fov = 0;
  P.gaze = make_float3(0.f, 0.f, 1.f);
  P.fov_f0 = P.fov_slope = P.fov_smooth = 0.f;
  if (o->foveation == 1) {
    // the ray through the gaze point (continuous pixel coordinates), as camera_ray forms it
    const double sx = (2.0 * (double)o->gaze[0] / c->width - 1.0) * (double)P.cam.tanh * P.cam.aspect;
    const double sy = (1.0 - 2.0 * (double)o->gaze[1] / c->height) * (double)P.cam.tanh;
    double g[3] = {f[0] + sx * r[0] + sy * uv[0], f[1] + sx * r[1] + sy * uv[1],
                   f[2] + sx * r[2] + sy * uv[2]};
    const double gn = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    P.fov = 1;
    P.gaze = make_float3((float)(g[0] / gn), (float)(g[1] / gn), (float)(g[2] / gn));
    P.fov_f0 = o->fov_f0;
    P.fov_slope = o->fov_slope;
    P.fov_smooth = o->fov_smooth;
  }
  if (o->free_flight != GF_FLIGHT_DELTA && o->free_flight != GF_FLIGHT_CDF &&
      o->free_flight != GF_FLIGHT_SEGMENT)
    return fail(GF_EINVAL, "bad free_flight");
  if (o->first_sample < 0 || (int64_t)o->first_sample + o->spp > (1 << 20))
    return fail(GF_EINVAL, "first_sample must be >= 0 with first_sample + spp <= 2^20");
  if (o->foveation != 0 && o->foveation != 1) return fail(GF_EINVAL, "foveation must be 0 or 1");
  if (o->foveation &&
      !(o->fov_f0 >= 0.f && o->fov_f0 < INFINITY && o->fov_slope >= 0.f && o->fov_slope < INFINITY &&
        o->fov_smooth >= 0.f && o->fov_smooth < 1.f && std::isfinite(o->gaze[0]) &&
        std::isfinite(o->gaze[1])))
    return fail(GF_EINVAL, "foveation needs fov_f0, fov_slope >= 0, fov_smooth in [0,1), a finite gaze");
  P.integrator = o->integrator;
  P.free_flight = o->free_flight;
  P.spp = o->spp;
  P.s0 = o->first_sample;
  P.max_bounces = o->max_bounces;
  P.albedo = o->albedo;
  P.irradiance = o->light_irradiance;
  double l[3] = {o->light_dir[0], o->light_dir[1], o->light_dir[2]};
  double ln = std::sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
  if (o->integrator == GF_INTEG_SCATTER && !(ln > 0)) return fail(GF_EINVAL, "light_dir zero");
  if (!(ln > 0)) ln = 1.0;
  P.light = make_float3((float)(l[0] / ln), (float)(l[1] / ln), (float)(l[2] / ln));
  P.seed = seed;
  P.lod = F.lod;
  P.lod_nee = F.lod_nee;
  return GF_OK;
}


// Weideman's coefficients a_n, n = 1..N, of the Faddeeva expansion: the
// Fourier cosine coefficients of f(theta) = (L^2 + t^2) exp(-t^2),
// t = L tan(theta/2), by the trapezoidal rule on theta_k = k pi / M,
// |k| < M = 2N (f vanishes at theta = pi), with L = sqrt(N / sqrt(2))
// (SIAM J. Numer. Anal. 31 (1994) 1497-1518).
void weideman_coefficients(Weideman& W) {
  const double pi = 3.14159265358979323846;
  const int N = kWeidN, M = 2 * N;
  const double L = std::sqrt(N / std::sqrt(2.0));
  for (int n = 1; n <= N; ++n) {
    double acc = 0.0;
    for (int k = -M + 1; k < M; ++k) {
      const double th = k * pi / M, t = L * std::tan(0.5 * th);
      acc += (L * L + t * t) * std::exp(-t * t) * std::cos(n * th);
    }
    W.a[n - 1] = (float)(acc / (2.0 * M));
  }
  W.L = (float)L;
}

}  // namespace gf

namespace {

// every buffer of the field goes back to its allocator once no work uses it
void free_field(Field& F) {
  cudaDeviceSynchronize();
  F.mem.release_all();
}

}  // namespace

namespace gf {
gf_status report(gf_status s, const std::string& msg) { return fail(s, msg); }
}  // namespace gf

extern "C" {

const char* gf_last_error(void) { return g_err.c_str(); }

gf_status gf_create(int device, gf_ctx** out) { return gf_create_ex(device, nullptr, out); }

gf_status gf_create_ex(int device, const gf_allocator* allocator, gf_ctx** out) {
  if (!out) return fail(GF_EINVAL, "out null");
  *out = nullptr;
  if (allocator && (!allocator->alloc || !allocator->free))
    return fail(GF_EINVAL, "allocator with a null alloc or free");
  Ctx base;
  if (allocator) base.alloc = *allocator;
  int ndev = 0;
  GF_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(GF_EINVAL, "no such device");
  GF_CUDA(cudaSetDevice(device), "cudaSetDevice");
  cudaDeviceProp prop;
  GF_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(GF_ECUDA, "libgf is built for sm_103a (GB300); device is sm_" +
                              std::to_string(prop.major) + std::to_string(prop.minor));
  // the per-thread stack of this context (a limit of the process, not of the GPU):
  // raised to kStackLimit when below it, never lowered (another library may have
  // set a larger one); the launchers compare each kernel's frame with the limit
  // in force at launch time
  size_t stack = 0;
  GF_CUDA(cudaDeviceGetLimit(&stack, cudaLimitStackSize), "cudaDeviceGetLimit");
  if (stack < (size_t)kStackLimit)
    GF_CUDA(cudaDeviceSetLimit(cudaLimitStackSize, kStackLimit), "cudaDeviceSetLimit");
  std::vector<float> x(kGLTotal), w(kGLTotal);
  for (int r = 0; r < kNumRules; ++r) {
    int n = gl_n(r), off = gl_off(r);
    std::vector<double> xd(n), wd(n);
    gauss_legendre(n, xd.data(), wd.data());
    for (int k = 0; k < n; ++k) {
      x[off + k] = (float)xd[k];
      w[off + k] = (float)wd[k];
    }
  }
  float* gl = nullptr;
  GF_CUDA(dev_alloc(base, (void**)&gl, 2 * kGLTotal * sizeof(float), nullptr), "alloc GL tables");
  cudaError_t e = cudaMemcpy(gl, x.data(), kGLTotal * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(gl + kGLTotal, w.data(), kGLTotal * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    dev_free(base, gl, 2 * kGLTotal * sizeof(float), nullptr);
    return cuda_fail(e, "GL tables");
  }
  gf_ctx* c = new gf_ctx;
  c->c = base;
  c->c.gl = gl;
  c->c.device = device;
  c->c.sm_count = prop.multiProcessorCount;
  c->c.cc_major = prop.major;
  c->c.cc_minor = prop.minor;
  *out = c;
  return GF_OK;
}

gf_status gf_destroy(gf_ctx* ctx) {
  if (ctx) {
    cudaSetDevice(ctx->c.device);
    cudaDeviceSynchronize();
    dev_free(ctx->c, ctx->c.gl, 2 * kGLTotal * sizeof(float), nullptr);
  }
  delete ctx;
  return GF_OK;
}

gf_status gf_load_field(gf_ctx* ctx, const gf_params* p, const gf_field_opts* opts,
                        gf_stream stream, gf_field** out) {
  if (!ctx || !p || !opts || !out) return fail(GF_EINVAL, "null argument");
  *out = nullptr;
  // node and primitive indices share a 32-bit word with a 5-bit lane index
  if (p->n < 1 || p->n >= (1ll << 26)) return fail(GF_EINVAL, "n must be in [1, 2^26)");
  if (!p->mu || !p->quat || !p->log_scale || !p->omega || !p->phase || !p->weight)
    return fail(GF_EINVAL, "parameter array null");
  if (!(opts->k_sigma > 0.f && opts->k_sigma <= 6.f)) return fail(GF_EINVAL, "k_sigma in (0,6]");
  if (opts->precision < 0 || opts->precision > 2) return fail(GF_EINVAL, "bad precision");
  if (opts->weight_mode < 0 || opts->weight_mode > 1) return fail(GF_EINVAL, "bad weight_mode");
  if (opts->omega_frame < 0 || opts->omega_frame > 1) return fail(GF_EINVAL, "bad omega_frame");
  if (!(opts->clamp_eps >= 0.f && opts->clamp_eps < INFINITY))
    return fail(GF_EINVAL, "clamp_eps must be finite and >= 0");
  GF_CUDA(cudaSetDevice(ctx->c.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  gf_field* h = new gf_field;
  Field& F = h->f;
  F.ctx = ctx->c;
  F.mem.ctx = ctx->c;
  F.n = p->n;
  F.opts = *opts;
  const int64_t n = p->n;
  auto A = [&](void** q, size_t bytes) { return F.mem.alloc(q, bytes, s); };
  cudaError_t e = cudaSuccess;
  void* band_dev = nullptr;
  do {
    if ((e = A((void**)&F.p_mu, 3 * n * 4)) || (e = A((void**)&F.p_quat, 4 * n * 4)) ||
        (e = A((void**)&F.p_ls, 3 * n * 4)) || (e = A((void**)&F.p_om, 3 * n * 4)) ||
        (e = A((void**)&F.p_ph, n * 4)) || (e = A((void**)&F.p_w, n * 4)) ||
        (e = A((void**)&F.rec_orig, 64 * n)) || (e = A((void**)&F.box_orig, 24 * n)) ||
        (e = A((void**)&F.kw_orig, 4 * n)) || (e = A((void**)&F.labels, 3 * n)) ||
        (e = A((void**)&F.err, 4)) || (e = A((void**)&F.stats, 8 * kNumStats)) ||
        (e = A((void**)&F.counter, 16)) || (e = A((void**)&F.cell_acc, sizeof(CellAcc))) ||
        (e = A((void**)&F.gl, 2 * kGLTotal * sizeof(float))))
      break;
    if ((e = A((void**)&F.ext2_orig, 4 * n)) || (e = A((void**)&F.ext2, 4 * n))) break;
    if ((e = cudaMemcpyAsync(F.gl, ctx->c.gl, 2 * kGLTotal * sizeof(float),
                             cudaMemcpyDeviceToDevice, s)))
      break;
    if (p->band && (e = A(&band_dev, n))) break;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    };
    if ((e = cp(F.p_mu, p->mu, 3 * n * 4)) || (e = cp(F.p_quat, p->quat, 4 * n * 4)) ||
        (e = cp(F.p_ls, p->log_scale, 3 * n * 4)) || (e = cp(F.p_om, p->omega, 3 * n * 4)) ||
        (e = cp(F.p_ph, p->phase, n * 4)) || (e = cp(F.p_w, p->weight, n * 4)))
      break;
    if (p->band && (e = cp(band_dev, p->band, n))) break;
    if ((e = cudaMemsetAsync(F.err, 0, 4, s)) || (e = cudaMemsetAsync(F.stats, 0, 8 * kNumStats, s)) ||
        (e = cudaMemsetAsync(F.cell_acc, 0, sizeof(CellAcc), s)))
      break;
  } while (0);
  if (e != cudaSuccess) {
    free_field(F);  // band_dev included
    delete h;
    return cuda_fail(e, "gf_load_field alloc/copy");
  }
  cone_axes(F.dev.axes);
  gf_params dp = *p;
  dp.mu = F.p_mu;
  dp.quat = F.p_quat;
  dp.log_scale = F.p_ls;
  dp.omega = F.p_om;
  dp.phase = F.p_ph;
  dp.weight = F.p_w;
  dp.band = (const uint8_t*)band_dev;
  e = launch_pack(F, dp, s);
  int herr = 0;
  CellAcc acc;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, F.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, F.cell_acc, sizeof(CellAcc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) F.mem.release(band_dev, s);
  if (e != cudaSuccess) {
    free_field(F);
    delete h;
    return cuda_fail(e, "gf_load_field pack");
  }
  if (herr) {
    free_field(F);
    delete h;
    return fail(GF_EINVAL, "non-finite parameter, zero quaternion or band label > 7");
  }
  F.dev.n = n;
  F.dev.precision = opts->precision;
  F.dev.ksig = opts->k_sigma;
  F.dev.k2 = opts->k_sigma * opts->k_sigma;
  F.dev.occupied = 0;
  for (int c = 0; c < kMaxCells; ++c) {
    const unsigned long long cnt = acc.count[c];
    if (cnt > 0) F.dev.occupied |= 1ull << c;
    F.dev.kbar[c] = cnt > 0 ? (float)((double)acc.kw_fix[c] *
                                      std::ldexp(1.0, cell_fix_exp(acc.kw_max) - 36) / (double)cnt)
                            : 0.f;
  }
  for (int k = 0; k < 8; ++k) F.dev.env[k] = (float)std::exp(-0.5 * k * k);
  for (int b = 0; b < 8; ++b) {  // 0 for an empty band
    float w;
    std::memcpy(&w, &acc.band_wmax[b], 4);
    F.dev.band_wmax[b] = w;
  }
  F.dev.err = F.err;
  F.dev.stats = F.stats;
  F.dev.gl = F.gl;
  weideman_coefficients(F.dev.wd);
  F.dev.cells_on = ~0ull;
  F.dev.root = -1;
  *out = h;
  return GF_OK;
}

gf_status gf_field_free(gf_field* h) {
  if (!h) return GF_OK;
  cudaSetDevice(h->f.ctx.device);
  free_field(h->f);
  delete h;
  return GF_OK;
}

gf_status gf_build_bvh(gf_field* h, gf_stream stream) {
  if (!h) return fail(GF_EINVAL, "field null");
  Field& F = h->f;
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  if (F.built) return GF_OK;
  const int64_t n = F.n;
  cudaStream_t s = (cudaStream_t)stream;
  GF_CUDA(F.mem.get(&F.rec, 64 * n, s), "alloc records");
  GF_CUDA(F.mem.get(&F.nodes, n > 1 ? (n - 1) * sizeof(Node) : 16, s), "alloc nodes");
  GF_CUDA(F.mem.get(&F.sorted_orig, 4 * n, s), "alloc order");
  GF_CUDA(F.mem.get(&F.muw, 16 * n, s), "alloc means");
  GF_CUDA(build_bvh(F, s), "build_bvh");
  if (F.depth > kStack)
    return fail(GF_EOVERFLOW, "the tree is " + std::to_string(F.depth) +
                                  " levels deep, beyond the per-thread traversal stack of " +
                                  std::to_string(kStack) + " entries");
  GF_CUDA(cudaStreamSynchronize(s), "sync");  // the build has read the original-order data
  F.mem.release(F.rec_orig, s);
  F.rec_orig = nullptr;
  F.mem.release(F.box_orig, s);
  F.box_orig = nullptr;
  F.mem.release(F.ext2_orig, s);
  F.ext2_orig = nullptr;
  if (F.opts.precision != GF_PREC_FP32) {
    // 32-byte records replace the 64-byte ones on the rendering path
    GF_CUDA(F.mem.get(&F.rec16, 32 * n, s), "alloc reduced records");
    int herr = 0;
    GF_CUDA(launch_pack16(F, s), "pack reduced records");
    GF_CUDA(cudaMemcpyAsync(&herr, F.err, 4, cudaMemcpyDeviceToHost, s), "read error word");
    GF_CUDA(cudaStreamSynchronize(s), "sync");
    if (herr) {
      cudaMemset(F.err, 0, 4);
      return fail(GF_EINVAL, "amplitude or whitened carrier outside the FP16 range (use BF16 records), or scales beyond 2^126");
    }
    F.dev.rec16 = F.rec16;
    F.dev.orig16 = F.sorted_orig;
    F.mem.release(F.rec, s);  // the 64-byte records are not read again (stream synchronised)
    F.rec = nullptr;
    F.dev.rec = nullptr;
  }
  F.built = true;
  return GF_OK;
}

gf_status gf_set_lod_camera(gf_field* h, const gf_camera* cam, gf_stream stream) {
  if (!h) return fail(GF_EINVAL, "field null");
  Field& F = h->f;
  if (!F.built) return fail(GF_ESTATE, "gf_build_bvh has not run");
  if (cam && (cam->width < 1 || cam->height < 1 || !(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f)))
    return fail(GF_EINVAL, "bad camera");
  if (F.server_refs > 0) return fail(GF_ESTATE, "a render server holds this field");
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const bool reduced = F.opts.precision != GF_PREC_FP32;
  if (!F.cells_dev) GF_CUDA(F.mem.get(&F.cells_dev, sizeof(unsigned long long), s), "alloc");
  if (reduced && !F.keff2) GF_CUDA(F.mem.get(&F.keff2, 4 * F.n, s), "alloc");
  // the finest resolved carrier at distance d is c / d (pixel pitch 2 d tan(phi/2) / H)
  const double pi = 3.14159265358979323846;
  float3 eye = make_float3(0.f, 0.f, 0.f);
  float c = INFINITY;
  if (cam) {
    const double th = std::tan(0.5 * (double)cam->vfov_deg * pi / 180.0);
    c = (float)(pi * (double)cam->height / (2.0 * th));
    eye = make_float3(cam->eye[0], cam->eye[1], cam->eye[2]);
  }
  GF_CUDA(launch_camera_lod(F, eye, c, s), "camera lod launch");
  unsigned long long cells = 0;
  GF_CUDA(cudaMemcpyAsync(&cells, F.cells_dev, sizeof(cells), cudaMemcpyDeviceToHost, s), "cells");
  GF_CUDA(cudaStreamSynchronize(s), "sync");
  F.dev.cells_on = cam ? cells : ~0ull;
  F.camera_lod = cam != nullptr;
  if (reduced) F.dev.ext2 = cam ? F.keff2 : (F.opts.clamp_eps > 0.f ? F.ext2 : nullptr);
  return GF_OK;
}

gf_status gf_reserve(gf_field* h, const gf_reserve_opts* o, gf_stream stream) {
  if (!h || !o) return fail(GF_EINVAL, "null argument");
  Field& F = h->f;
  if (!F.built) return fail(GF_ESTATE, "gf_build_bvh has not run");
  if (o->max_rays < 0 || o->max_rays > (1ll << 31) - 1 || o->max_chords < 0 || o->max_pixels < 0 ||
      o->max_pixels > (1ll << 31) - 1)
    return fail(GF_EINVAL, "reserve sizes out of range");
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)o->max_rays, nc = n * (size_t)o->max_chords;
  const size_t npix = (size_t)o->max_pixels;
  // the largest staging any call within these sizes asks for
  size_t stage = 0;
  if (n) stage = std::max(256 * 6 + n * 4 * 10, 256 * 8 + n * 4 * 9 + nc * 12);
  if (npix) stage = std::max(stage, npix * 4 + 256);
  if (npix && o->adjoint) stage = std::max(stage, npix * 4 + (size_t)F.n * 60 + 512);
  gf_status st;
  if (stage && (st = ensure_stage(F, stage, s))) return st;
  if (o->render && npix) GF_CUDA(ensure_render_scratch(F, (int64_t)npix, s), "render scratch");
  if (o->adjoint) GF_CUDA(ensure_adjoint_lists(F, s), "adjoint lists");
  return GF_OK;
}

gf_status gf_set_lod_mask(gf_field* h, const gf_lod_desc* primary, const gf_lod_desc* nee) {
  if (!h || !lod_ok(primary) || (nee && !lod_ok(nee))) return fail(GF_EINVAL, "bad lod descriptor");
  h->f.lod = lod_dev(*primary);
  const gf_lod_desc* n2 = nee ? nee : primary;
  h->f.lod_nee = lod_dev(*n2);
  return GF_OK;
}

gf_status gf_transmittance(gf_field* h, const float* o, const float* d, const float* trange,
                           int64_t n_rays, int mode, int spp, uint64_t seed, float* out_T,
                           float* out_tau, gf_stream stream) {
  if (!h || !o || !d || !out_T) return fail(GF_EINVAL, "null argument");
  Field& F = h->f;
  if (!F.built) return fail(GF_ESTATE, "gf_build_bvh has not run");
  if (n_rays < 0 || n_rays > (1ll << 31) - 1) return fail(GF_EINVAL, "n_rays out of range");
  if (mode != GF_TR_DETERMINISTIC && mode != GF_TR_RATIO_TRACKING && mode != GF_TR_CLOSED_FORM)
    return fail(GF_EINVAL, "bad mode");
  if (spp < 1 || spp > (1 << 20)) return fail(GF_EINVAL, "spp in [1, 2^20]");
  if (n_rays == 0) return GF_OK;
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  size_t n = (size_t)n_rays;
  gf_status st = ensure_stage(F, 256 * 6 + n * 4 * (3 + 3 + 2 + 1 + 1), s);
  if (st) return st;
  size_t off = 0;
  void *od, *dd, *td, *Td, *taud;
  if ((st = stage(F, o, 12 * n, true, s, off, &od)) || (st = stage(F, d, 12 * n, true, s, off, &dd)) ||
      (st = stage(F, trange, 8 * n, true, s, off, &td)) ||
      (st = stage(F, out_T, 4 * n, false, s, off, &Td)) ||
      (st = stage(F, mode != GF_TR_RATIO_TRACKING ? out_tau : nullptr, 4 * n, false, s, off, &taud)))
    return st;
  TrParams P;
  P.o = (const float*)od;
  P.d = (const float*)dd;
  P.trange = (const float*)td;
  P.n = n_rays;
  P.mode = mode;
  P.spp = spp;
  P.seed = seed;
  P.lod = F.lod;
  P.out_T = (float*)Td;
  P.out_tau = (float*)taud;
  P.counter = F.counter;
  GF_CUDA(launch_transmittance(F, P, s), "transmittance launch");
  bool sync = false;
  if (Td != out_T) {
    GF_CUDA(cudaMemcpyAsync(out_T, Td, 4 * n, cudaMemcpyDeviceToHost, s), "copy T");
    sync = true;
  }
  if (out_tau && taud && taud != out_tau) {
    GF_CUDA(cudaMemcpyAsync(out_tau, taud, 4 * n, cudaMemcpyDeviceToHost, s), "copy tau");
    sync = true;
  }
  if (sync) {
    GF_CUDA(cudaStreamSynchronize(s), "sync");
    return take_device_error(F);
  }
  return GF_OK;
}

gf_status gf_render(gf_field* h, const gf_camera* camera, const gf_render_opts* opts,
                    uint64_t seed, float* out_image, gf_stream stream) {
  if (!h || !out_image) return fail(GF_EINVAL, "null argument");
  Field& F = h->f;
  if (!F.built) return fail(GF_ESTATE, "gf_build_bvh has not run");
  PathParams P;
  gf_status st = camera_params(camera, opts, seed, F, P);
  if (st) return st;
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  size_t bytes = (size_t)P.cam.W * P.cam.H * 4;
  void* od = out_image;
  if (!is_device_ptr(out_image)) {
    if ((st = ensure_stage(F, bytes + 256, s))) return st;
    od = F.stage;
  }
  GF_CUDA(launch_render(F, P, (float*)od, s), "render launch");
  if (od != out_image) {
    GF_CUDA(cudaMemcpyAsync(out_image, od, bytes, cudaMemcpyDeviceToHost, s), "copy image");
    GF_CUDA(cudaStreamSynchronize(s), "sync");
    return take_device_error(F);
  }
  return GF_OK;
}

gf_status gf_render_backward(gf_field* h, const gf_camera* camera, const gf_render_opts* opts,
                             uint64_t seed, const float* dL_dimage, float* grad,
                             gf_stream stream) {
  if (!h || !dL_dimage || !grad) return fail(GF_EINVAL, "null argument");
  Field& F = h->f;
  if (!F.built) return fail(GF_ESTATE, "gf_build_bvh has not run");
  PathParams P;
  gf_status st = camera_params(camera, opts, seed, F, P);
  if (st) return st;
  if (P.free_flight != GF_FLIGHT_DELTA) return fail(GF_EINVAL, "the adjoint differentiates GF_FLIGHT_DELTA");
  if (P.fov) return fail(GF_EINVAL, "the adjoint renders without foveation");
  if (opts->integrator == GF_INTEG_SCATTER && opts->max_bounces < 1)
    return fail(GF_EINVAL, "the radiance adjoint needs max_bounces >= 1");
  if (F.opts.precision != GF_PREC_FP32)
    return fail(GF_EINVAL, "the adjoint needs FP32 records");
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  size_t npix = (size_t)P.cam.W * P.cam.H;
  size_t gbytes = (size_t)F.n * 15 * 4;
  if ((st = ensure_stage(F, npix * 4 + gbytes + 512, s))) return st;
  size_t off = 0;
  void *dl, *gd;
  if ((st = stage(F, dL_dimage, npix * 4, true, s, off, &dl)) ||
      (st = stage(F, grad, gbytes, false, s, off, &gd)))
    return st;
  GF_CUDA(cudaMemsetAsync(gd, 0, gbytes, s), "zero grad");
  if (opts->integrator == GF_INTEG_TOMO)
    GF_CUDA(launch_tomo_backward(F, P, (const float*)dl, (float*)gd, s), "backward launch");
  else
    GF_CUDA(launch_radiance_backward(F, P, (const float*)dl, (float*)gd, s), "backward launch");
  if (gd != grad) {
    GF_CUDA(cudaMemcpyAsync(grad, gd, gbytes, cudaMemcpyDeviceToHost, s), "copy grad");
    GF_CUDA(cudaStreamSynchronize(s), "sync");
    return take_device_error(F);
  }
  return GF_OK;
}

gf_status gf_field_labels(gf_field* h, uint8_t* band, uint8_t* cone, uint8_t* cell,
                          gf_stream stream) {
  if (!h) return fail(GF_EINVAL, "field null");
  Field& F = h->f;
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  size_t n = (size_t)F.n;
  if (band) GF_CUDA(cudaMemcpyAsync(band, F.labels, n, cudaMemcpyDefault, s), "labels");
  if (cone) GF_CUDA(cudaMemcpyAsync(cone, F.labels + n, n, cudaMemcpyDefault, s), "labels");
  if (cell) GF_CUDA(cudaMemcpyAsync(cell, F.labels + 2 * n, n, cudaMemcpyDefault, s), "labels");
  GF_CUDA(cudaStreamSynchronize(s), "sync");
  return GF_OK;
}

gf_status gf_ray_chords(gf_field* h, const float* o, const float* d, const float* trange,
                        int64_t n_rays, int cap, int32_t* counts, int32_t* prims, float* t_in,
                        float* t_out, gf_stream stream) {
  if (!h || !o || !d || !counts || !prims || cap < 1) return fail(GF_EINVAL, "bad argument");
  Field& F = h->f;
  if (!F.built) return fail(GF_ESTATE, "gf_build_bvh has not run");
  if (!lod_is_deterministic(F.lod)) return fail(GF_EINVAL, "chord lists need a deterministic mask");
  if (n_rays <= 0) return GF_OK;
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  size_t n = (size_t)n_rays, nc = n * (size_t)cap;
  gf_status st = ensure_stage(F, 256 * 8 + n * 4 * 9 + nc * 12, s);
  if (st) return st;
  size_t off = 0;
  void *od, *dd, *td, *cd, *pd, *tid, *tod;
  if ((st = stage(F, o, 12 * n, true, s, off, &od)) || (st = stage(F, d, 12 * n, true, s, off, &dd)) ||
      (st = stage(F, trange, 8 * n, true, s, off, &td)) ||
      (st = stage(F, counts, 4 * n, false, s, off, &cd)) ||
      (st = stage(F, prims, 4 * nc, false, s, off, &pd)) ||
      (st = stage(F, t_in, 4 * nc, false, s, off, &tid)) ||
      (st = stage(F, t_out, 4 * nc, false, s, off, &tod)))
    return st;
  ChordParams P;
  P.o = (const float*)od;
  P.d = (const float*)dd;
  P.trange = (const float*)td;
  P.n = n_rays;
  P.cap = cap;
  P.lod = F.lod;
  P.counts = (int*)cd;
  P.prims = (int*)pd;
  P.tin = (float*)tid;
  P.tout = (float*)tod;
  P.counter = F.counter;
  GF_CUDA(launch_ray_chords(F, P, s), "chords launch");
  if (cd != counts) GF_CUDA(cudaMemcpyAsync(counts, cd, 4 * n, cudaMemcpyDeviceToHost, s), "copy");
  if (pd != prims) GF_CUDA(cudaMemcpyAsync(prims, pd, 4 * nc, cudaMemcpyDeviceToHost, s), "copy");
  if (t_in && tid != t_in) GF_CUDA(cudaMemcpyAsync(t_in, tid, 4 * nc, cudaMemcpyDeviceToHost, s), "copy");
  if (t_out && tod != t_out) GF_CUDA(cudaMemcpyAsync(t_out, tod, 4 * nc, cudaMemcpyDeviceToHost, s), "copy");
  GF_CUDA(cudaStreamSynchronize(s), "sync");
  return take_device_error(F);
}

gf_status gf_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                    gf_stream stream) {
  if (!ctr || !key || !out || n < 0) return fail(GF_EINVAL, "bad argument");
  if (n == 0) return GF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  bool host = !is_device_ptr(ctr) || !is_device_ptr(key) || !is_device_ptr(out);
  if (!host) {
    GF_CUDA(launch_philox(ctr, key, out, n, s), "philox launch");
    return GF_OK;
  }
  std::lock_guard<std::mutex> lock(g_helper_mu);
  void* area = nullptr;
  gf_status st = helper_area(&area);
  if (st) return st;
  const int64_t chunk = kHelperBytes / 40;  // counter 16 B + key 8 B + block 16 B
  uint32_t* c = (uint32_t*)area;
  uint32_t* k = c + 4 * chunk;
  uint32_t* r = k + 2 * chunk;
  cudaError_t e = cudaSuccess;
  for (int64_t i = 0; i < n && !e; i += chunk) {
    const int64_t m = n - i < chunk ? n - i : chunk;
    e = cudaMemcpyAsync(c, ctr + 4 * i, 16 * m, cudaMemcpyDefault, s);
    if (!e) e = cudaMemcpyAsync(k, key + 2 * i, 8 * m, cudaMemcpyDefault, s);
    if (!e) e = launch_philox(c, k, r, m, s);
    if (!e) e = cudaMemcpyAsync(out + 4 * i, r, 16 * m, cudaMemcpyDefault, s);
    if (!e) e = cudaStreamSynchronize(s);
  }
  if (e) return cuda_fail(e, "gf_philox");
  return GF_OK;
}

gf_status gf_faddeeva(const float* z, float* w, int64_t n, gf_stream stream) {
  if (!z || !w || n < 0) return fail(GF_EINVAL, "bad argument");
  if (n == 0) return GF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Weideman W;
  weideman_coefficients(W);
  if (is_device_ptr(z) && is_device_ptr(w)) {
    GF_CUDA(launch_faddeeva(W, z, w, n, s), "faddeeva launch");
    return GF_OK;
  }
  std::lock_guard<std::mutex> lock(g_helper_mu);
  void* area = nullptr;
  gf_status st = helper_area(&area);
  if (st) return st;
  const int64_t chunk = kHelperBytes / 16;  // z 8 B + w 8 B
  float* zd = (float*)area;
  float* wd = zd + 2 * chunk;
  cudaError_t e = cudaSuccess;
  for (int64_t i = 0; i < n && !e; i += chunk) {
    const int64_t m = n - i < chunk ? n - i : chunk;
    e = cudaMemcpyAsync(zd, z + 2 * i, 8 * m, cudaMemcpyDefault, s);
    if (!e) e = launch_faddeeva(W, zd, wd, m, s);
    if (!e) e = cudaMemcpyAsync(w + 2 * i, wd, 8 * m, cudaMemcpyDefault, s);
    if (!e) e = cudaStreamSynchronize(s);
  }
  if (e) return cuda_fail(e, "gf_faddeeva");
  return GF_OK;
}

gf_status gf_get_stats(gf_field* h, gf_stats* out, int reset) {
  if (!h || !out) return fail(GF_EINVAL, "null argument");
  Field& F = h->f;
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  unsigned long long v[kNumStats];
  GF_CUDA(cudaDeviceSynchronize(), "sync");
  GF_CUDA(cudaMemcpy(v, F.stats, sizeof(v), cudaMemcpyDeviceToHost), "stats");
  out->rays = v[ST_RAYS];
  out->chords = v[ST_CHORDS];
  out->evals = v[ST_EVALS];
  out->nodes = v[ST_NODES];
  out->points = v[ST_POINTS];
  out->windows = v[ST_WINDOWS];
  out->steps = v[ST_STEPS];
  out->leaves = v[ST_LEAVES];
  for (int k = 0; k < 5; ++k) out->cycles[k] = v[ST_CYC_TRAV + k];
  if (reset) GF_CUDA(cudaMemset(F.stats, 0, sizeof(v)), "reset stats");
  return GF_OK;
}

gf_status gf_sync(gf_field* h, gf_stream stream) {
  if (!h) return fail(GF_EINVAL, "field null");
  Field& F = h->f;
  GF_CUDA(cudaSetDevice(F.ctx.device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  GF_CUDA(cudaStreamSynchronize(s), "stream sync");
  return take_device_error(F);
}

gf_status gf_field_info(gf_field* h, int64_t* n, int* precision, uint64_t* occupied) {
  if (!h) return fail(GF_EINVAL, "field null");
  if (n) *n = h->f.n;
  if (precision) *precision = h->f.opts.precision;
  if (occupied) *occupied = h->f.dev.occupied;
  return GF_OK;
}

}  // extern "C"
