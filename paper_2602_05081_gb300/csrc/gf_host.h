// gf_host.h -- host-side structures shared by the translation units of libgf.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <unordered_map>

#include "../../include/gf.h"
#include "gf_device.cuh"
#include "gf_trace.cuh"

namespace gf {

struct Ctx {
  int device = 0;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  float* gl = nullptr;  // device Gauss-Legendre tables
  gf_allocator alloc{nullptr, nullptr, nullptr};  // null alloc: cudaMalloc / cudaFree
};

// Device memory through the context's allocator (bytes == 0 allocates 16)
cudaError_t dev_alloc(const Ctx& c, void** p, size_t bytes, cudaStream_t s);
// Return memory that no pending work uses any more (callers synchronise first)
void dev_free(const Ctx& c, void* p, size_t bytes, cudaStream_t s);

// The device buffers of one owner (a field, a render server), each returned to
// the allocator with the size it was asked for.
struct DevMem {
  Ctx ctx;
  std::unordered_map<void*, size_t> sizes;
  cudaError_t alloc(void** p, size_t bytes, cudaStream_t s) {
    void* q = nullptr;
    const cudaError_t e = dev_alloc(ctx, &q, bytes, s);
    if (e != cudaSuccess) return e;
    sizes[q] = bytes;
    *p = q;
    return cudaSuccess;
  }
  template <class T>
  cudaError_t get(T** p, size_t bytes, cudaStream_t s) {
    return alloc(reinterpret_cast<void**>(p), bytes, s);
  }
  // p == nullptr is allowed; the caller has synchronised the work that used p
  void release(void* p, cudaStream_t s) {
    if (!p) return;
    auto it = sizes.find(p);
    if (it == sizes.end()) return;
    dev_free(ctx, p, it->second, s);
    sizes.erase(it);
  }
  void release_all() {
    for (auto& kv : sizes) dev_free(ctx, kv.first, kv.second, nullptr);
    sizes.clear();
  }
};

struct TrParams {
  const float* o;
  const float* d;
  const float* trange;
  int64_t n;
  int mode, spp;
  uint64_t seed;
  LodDev lod;
  float* out_T;
  float* out_tau;
  int* counter;
  int group = 1;  // lanes per ray of the deterministic mode (1, 2, ..., 32)
};

struct ChordParams {
  const float* o;
  const float* d;
  const float* trange;
  int64_t n;
  int cap;
  LodDev lod;
  int* counts;
  int* prims;
  float* tin;
  float* tout;
  int* counter;
};

// Label statistics of a field, gathered at load time with integer atomics only,
// so that they (and every render that uses them) do not depend on the order in
// which threads arrive: per cell the sum of |k_W| in fixed point (units of
// 2^(e - 36), 2^e above the largest |k_W|; at most 2^36 per kernel and 2^26
// kernels) and the member count; per band the largest world carrier |omega|;
// and the largest |k_W| (non-negative floats order as their bits).
struct CellAcc {
  unsigned long long kw_fix[64];
  unsigned long long count[64];
  unsigned int band_wmax[8];
  unsigned int kw_max;
};
// exponent e of the fixed-point unit: 2^e > the largest |k_W| (bits mb), clamped
// so that 2^(36 - e) is a normal float
inline __host__ __device__ int cell_fix_exp(unsigned int mb) {
  int e = (int)((mb >> 23) & 0xFFu) - 126;
  return e < -60 ? -60 : (e > 100 ? 100 : e);
}
struct Field {
  Ctx ctx;                     // copy: a field outlives the gf_ctx it came from
  mutable DevMem mem;          // every device buffer of the field, through ctx.alloc
  float* gl = nullptr;         // the field's own Gauss-Legendre tables
  int64_t n = 0;
  gf_field_opts opts{};
  // raw parameters (device copies, original order) for the adjoint
  float* p_mu = nullptr;
  float* p_quat = nullptr;
  float* p_ls = nullptr;
  float* p_om = nullptr;
  float* p_ph = nullptr;
  float* p_w = nullptr;
  // packed data
  float4* rec_orig = nullptr;   // FP32 records in original order (until the build)
  float* box_orig = nullptr;    // 6 floats per primitive
  float* kw_orig = nullptr;     // |k_W| per primitive
  float* ext2_orig = nullptr;   // own support radius squared per primitive (until the build)
  float* ext2 = nullptr;        // own support radius squared, BVH order (k^2 or adaptive)
  float* keff2 = nullptr;       // reduced precision + camera LoD: effective k_i^2, BVH order
  float4* muw = nullptr;        // BVH order: mean and |omega| (camera LoD selection)
  unsigned long long* cells_dev = nullptr;  // camera LoD selection: cells still occupied
  float4* rec = nullptr;        // FP32 records in BVH order
  uint4* rec16 = nullptr;       // reduced-precision records in BVH order
  Node* nodes = nullptr;
  Node4* nodes4 = nullptr;      // four-wide collapse (built by gf_build_bvh)
  int* sorted_orig = nullptr;   // BVH position -> original index
  uint8_t* labels = nullptr;    // band, cone, cell per primitive (3N, original order)
  int* err = nullptr;
  unsigned long long* stats = nullptr;
  int* counter = nullptr;
  CellAcc* cell_acc = nullptr;  // label statistics of the load (exact, order-free)
  int depth = 0;                // levels of internal nodes of the binary tree
  int64_t n_nodes4 = 0;         // four-wide nodes
  bool built = false;
  bool camera_lod = false;  // a camera LoD selection is active
  int server_refs = 0;      // render servers holding this field
  float mu_lo[3] = {0, 0, 0}, mu_hi[3] = {0, 0, 0};  // box of the means (from the build)
  DevField dev{};
  LodDev lod{0, 7, 0, 0.f, 0.f}, lod_nee{0, 7, 0, 0.f, 0.f};
  // staging for host buffers
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // per-warp chord store of the scattering renderer (grows on demand)
  mutable float4* wscratch = nullptr;
  mutable size_t wscratch_bytes = 0;
  // fixed-point pixel sums of the scattering renderer (grows on demand)
  mutable unsigned long long* acc64 = nullptr;
  mutable size_t acc_bytes = 0;
  // per-thread primitive lists of the radiance adjoint (grows on demand)
  mutable int* rlist = nullptr;
  mutable size_t rlist_bytes = 0;
};

// Render server batch (one launch of k_render_server): items of many requests
// on several fields.  Item i covers pixels [pix0, pix0 + npix) of request
// req, every pixel split into nchunk units of chunk consecutive samples, and
// the batch's flat unit numbers [base, base + npix * nchunk); bases ascend.
struct ServerItem {
  int req, pix0, npix, base;
};
struct ServerReqDev {
  PathParams P;
  unsigned long long* acc;  // fixed-point sample sums of the request (W x H, 2^-32 units)
  int asset;                // index into ServerLaunch::fields
  int chunk, nchunk;        // samples per unit, units per pixel
  int pad_;
};
struct ServerLaunch {
  const DevField* fields;  // device array, one per asset (err/stats point at the server's)
  int64_t max_n;           // largest primitive count over the assets
  const ServerItem* items;
  int n_items;
  const ServerReqDev* reqs;
  int* counter;            // zero at launch
  int total;               // units in the batch
};

// launchers (return cudaError_t of the launch)
// per-thread stack limit set on every context (bytes); kernels above it are not launched
constexpr int kStackLimit = 2048;

cudaError_t launch_transmittance(const Field& F, const TrParams& P, cudaStream_t s);
cudaError_t launch_render(const Field& F, const PathParams& P, float* out, cudaStream_t s);
cudaError_t launch_render_scatter(const Field& F, const PathParams& P, float* out, cudaStream_t s);
cudaError_t launch_ray_chords(const Field& F, const ChordParams& P, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                          cudaStream_t s);
cudaError_t launch_faddeeva(const Weideman& W, const float* z, float* w, int64_t n,
                           cudaStream_t s);
cudaError_t launch_camera_lod(Field& F, float3 eye, float c, cudaStream_t s);
void weideman_coefficients(Weideman& W);
cudaError_t launch_pack(Field& F, const gf_params& P, cudaStream_t s);
cudaError_t build_bvh(Field& F, cudaStream_t s);
cudaError_t launch_pack16(Field& F, cudaStream_t s);
size_t scatter_store_bytes(int64_t grid);
cudaError_t server_grid(int sm_count, int64_t& grid);
cudaError_t launch_render_server(const ServerLaunch& L, int64_t grid, float4* chord_store,
                                 cudaStream_t s);
// image = fixed-point sums / spp
cudaError_t launch_fix_to_image(const unsigned long long* acc, int64_t npix, int spp, float* out,
                                cudaStream_t s);
// scratch of the compute calls, grown through the field's allocator: the pixel sums and
// chord store of the scattering renderer, the radiance adjoint's primitive lists
cudaError_t ensure_render_scratch(const Field& F, int64_t npix, cudaStream_t s);
cudaError_t ensure_adjoint_lists(const Field& F, cudaStream_t s);
// grow a field-owned buffer to at least `bytes` (synchronises the device before
// returning the old one)
cudaError_t grow(const Field& F, void** p, size_t& have, size_t bytes, cudaStream_t s);
cudaError_t launch_radiance_backward(const Field& F, const PathParams& P, const float* dLdI,
                                     float* grad, cudaStream_t s);
cudaError_t launch_tomo_backward(const Field& F, const PathParams& P, const float* dLdI,
                                 float* grad, cudaStream_t s);

// sets the thread-local message returned by gf_last_error and returns s
gf_status report(gf_status s, const std::string& msg);
// after a stream synchronisation: the field's device error word as a status (cleared)
gf_status take_device_error(Field& F);
// camera and integrator options -> kernel parameters (LoD from the field)
gf_status camera_params(const gf_camera* c, const gf_render_opts* o, uint64_t seed, const Field& F,
                        PathParams& P);
bool lod_ok(const gf_lod_desc* l);
LodDev lod_dev(const gf_lod_desc& l);

}  // namespace gf

// opaque handles of include/gf.h
struct gf_ctx {
  gf::Ctx c;
};
struct gf_field {
  gf::Field f;
};
