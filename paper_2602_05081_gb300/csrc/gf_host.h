// gf_host.h -- host-side structures shared by the translation units of libgf.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/gf.h"
#include "gf_device.cuh"
#include "gf_trace.cuh"

namespace gf {

struct Ctx {
  int device = 0;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  float* gl = nullptr;  // device Gauss-Legendre tables
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

struct Field {
  Ctx ctx;                     // copy: a field outlives the gf_ctx it came from
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
  float* cell_acc = nullptr;    // per-cell |k_W| sums (64) and counts (64)
  int depth = 0;                // levels of internal nodes of the binary tree
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
// req and the batch's flat pixel numbers [base, base + npix); bases ascend.
struct ServerItem {
  int req, pix0, npix, base;
};
struct ServerReqDev {
  PathParams P;
  float* fb;   // device framebuffer of the request (W x H floats)
  int asset;   // index into ServerLaunch::fields
  int pad_;
};
struct ServerLaunch {
  const DevField* fields;  // device array, one per asset (err/stats point at the server's)
  int64_t max_n;           // largest primitive count over the assets
  const ServerItem* items;
  int n_items;
  int total;               // pixels in the batch
  const ServerReqDev* reqs;
  int* counter;            // zero at launch
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
