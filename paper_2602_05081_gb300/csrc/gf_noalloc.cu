// gf_noalloc.cu -- transmittance for callers that cannot allocate device memory.
//
// gf_transmittance stages host buffers through memory it allocates with
// cudaMalloc (and its kernel's work counter lives in memory allocated when the
// field was loaded).  Some callers cannot allocate at call time: code running
// under an external memory manager that forbids allocation, hosts that have
// exhausted or pinned their device allocation budget, or integrations that
// only hand the library host arrays.  gf_transmittance_static serves them: it
// computes exactly what gf_transmittance computes, but its scratch -- the
// kernel's work-queue counter and the device copies of host inputs and
// outputs -- lives in one file-scope device array of fixed size, so the call
// allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gf_host.h"

namespace {

// Scratch shared by every call: 8 MiB, loaded with the library on every GPU
// that loads it and held until the process exits.
constexpr size_t kStaticScratchBytes = 8u << 20;
// per ray: o (12 B) + d (12 B) + trange (8 B) + T (4 B) + tau (4 B) = 40 B,
// plus 256-byte alignment slack per region and the counter's 256-byte slot
constexpr int64_t kStaticMaxRays = 200000;
static_assert(256 + 5 * 255 + 40 * kStaticMaxRays <= kStaticScratchBytes,
              "the largest call's counter slot and five staged buffers fit the array");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_dev[64] = {nullptr};  // device address of the array, per device

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" gf_status gf_transmittance_static(gf_field* h, const float* o, const float* d,
                                             const float* trange, int64_t n_rays, int mode,
                                             int spp, uint64_t seed, float* out_T,
                                             float* out_tau, gf_stream stream) {
  using gf::report;
  if (!h || !o || !d || !out_T) return report(GF_EINVAL, "null argument");
  gf::Field& F = h->f;
  if (!F.built) return report(GF_ESTATE, "gf_build_bvh has not run");
  if (n_rays < 0) return report(GF_EINVAL, "n_rays out of range");
  if (n_rays > kStaticMaxRays)
    return report(GF_EINVAL, "n_rays exceeds the static scratch capacity of " +
                                 std::to_string(kStaticMaxRays) + " rays; split the call");
  if (mode != GF_TR_DETERMINISTIC && mode != GF_TR_RATIO_TRACKING && mode != GF_TR_CLOSED_FORM)
    return report(GF_EINVAL, "bad mode");
  if (spp < 1 || spp > (1 << 20)) return report(GF_EINVAL, "spp in [1, 2^20]");
  if (n_rays == 0) return GF_OK;
  const int dev = F.ctx.device;
  if (dev < 0 || dev >= 64) return report(GF_EINVAL, "device index beyond 63");
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return report(GF_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  // first call on this device: look up the array's device address with the
  // device current (a host-side name of a __device__ array is not an address)
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p)
        return report(GF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_dev[dev] = p;
    }
    base = g_scratch_dev[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)n_rays;
  char* cur = (char*)base;
  int* counter = (int*)cur;
  cur += 256;
  // device view of each buffer: the caller's device pointer, or a scratch slice
  auto view = [&](const void* p, size_t bytes, bool in, void** out) -> cudaError_t {
    if (!p || is_device_pointer(p)) {
      *out = const_cast<void*>(p);
      return cudaSuccess;
    }
    *out = cur;
    cur += align256(bytes);
    return in ? cudaMemcpyAsync(*out, p, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  float* tau_arg = mode != GF_TR_RATIO_TRACKING ? out_tau : nullptr;
  void *od, *dd, *td, *Td, *taud;
  if ((e = view(o, 12 * n, true, &od)) || (e = view(d, 12 * n, true, &dd)) ||
      (e = view(trange, 8 * n, true, &td)) || (e = view(out_T, 4 * n, false, &Td)) ||
      (e = view(tau_arg, 4 * n, false, &taud)))
    return report(GF_ECUDA, std::string("staging: ") + cudaGetErrorString(e));
  gf::TrParams P;
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
  P.counter = counter;  // cleared by the launcher before the kernel
  if ((e = gf::launch_transmittance(F, P, s)) != cudaSuccess)
    return report(GF_ECUDA, std::string("transmittance launch: ") + cudaGetErrorString(e));
  bool sync = false;
  if (Td != out_T) {
    if ((e = cudaMemcpyAsync(out_T, Td, 4 * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return report(GF_ECUDA, std::string("copy T: ") + cudaGetErrorString(e));
    sync = true;
  }
  if (tau_arg && taud != tau_arg) {
    if ((e = cudaMemcpyAsync(tau_arg, taud, 4 * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return report(GF_ECUDA, std::string("copy tau: ") + cudaGetErrorString(e));
    sync = true;
  }
  if (sync) {
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
      return report(GF_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
    return gf::take_device_error(F);
  }
  return GF_OK;
}
