"""ctypes binding of libgf.so (include/gf.h), one Python function per C entry point.

Argument marshalling only: every step of the rendering path runs in the CUDA
kernels behind the C ABI.  Pointer arguments accept torch tensors (device or
host), numpy arrays or None; streams are torch.cuda.Stream objects, raw
cudaStream_t integers or None (legacy default stream).  A non-zero status
raises GfError with the library's message.  There is no CPU fallback: if the
library is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GF_LIB selects an alternative build of the same sources (e.g. with phase timers)
LIB_PATH = os.environ.get("GF_LIB") or os.path.join(HERE, "_build", "libgf.so")

GF_OK, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_EOVERFLOW, GF_ETIMEOUT, GF_ESTATE = range(7)
STATUS_NAMES = {0: "GF_OK", 1: "GF_EINVAL", 2: "GF_ENOMEM", 3: "GF_ECUDA", 4: "GF_EOVERFLOW",
                5: "GF_ETIMEOUT", 6: "GF_ESTATE"}
GF_PREC_FP32, GF_PREC_FP16, GF_PREC_BF16 = 0, 1, 2
GF_WEIGHT_PEAK, GF_WEIGHT_NORMALIZED = 0, 1
GF_OMEGA_WORLD, GF_OMEGA_LOCAL = 0, 1
(GF_FREQ_ALL, GF_FREQ_CUTOFF, GF_FREQ_UNIF_CV, GF_FREQ_UNIFORM, GF_FREQ_POWER, GF_FREQ_POW_CV,
 GF_FREQ_POW_CV_ACC) = range(7)
GF_CONE_ALL, GF_CONE_IS, GF_CONE_UNIFORM, GF_CONE_THRESH, GF_CONE_THRESH_UNIFORM = range(5)
GF_TR_DETERMINISTIC, GF_TR_RATIO_TRACKING, GF_TR_CLOSED_FORM = 0, 1, 2
GF_FLIGHT_DELTA, GF_FLIGHT_CDF = 0, 1
GF_INTEG_TOMO, GF_INTEG_SCATTER = 0, 1


class GfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class gf_params(C.Structure):
    _fields_ = [("n", C.c_int64), ("mu", C.c_void_p), ("quat", C.c_void_p),
                ("log_scale", C.c_void_p), ("omega", C.c_void_p), ("phase", C.c_void_p),
                ("weight", C.c_void_p), ("band", C.c_void_p)]


class gf_field_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("weight_mode", C.c_int), ("omega_frame", C.c_int),
                ("k_sigma", C.c_float), ("clamp_eps", C.c_float)]


class gf_lod_desc(C.Structure):
    _fields_ = [("freq_policy", C.c_int), ("max_band", C.c_int), ("cone_policy", C.c_int),
                ("beta", C.c_float), ("delta", C.c_float)]


class gf_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int), ("height", C.c_int)]


class gf_render_opts(C.Structure):
    _fields_ = [("integrator", C.c_int), ("spp", C.c_int), ("max_bounces", C.c_int),
                ("albedo", C.c_float), ("light_dir", C.c_float * 3),
                ("light_irradiance", C.c_float), ("free_flight", C.c_int),
                ("first_sample", C.c_int), ("foveation", C.c_int), ("gaze", C.c_float * 2),
                ("fov_f0", C.c_float), ("fov_slope", C.c_float), ("fov_smooth", C.c_float)]


class gf_stats(C.Structure):
    _fields_ = [("rays", C.c_uint64), ("chords", C.c_uint64), ("evals", C.c_uint64),
                ("nodes", C.c_uint64), ("points", C.c_uint64), ("windows", C.c_uint64),
                ("steps", C.c_uint64), ("leaves", C.c_uint64), ("cycles", C.c_uint64 * 5)]


# device allocator callbacks (include/gf.h gf_allocator)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class gf_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class gf_reserve_opts(C.Structure):
    _fields_ = [("max_rays", C.c_int64), ("max_chords", C.c_int), ("max_pixels", C.c_int64),
                ("render", C.c_int), ("adjoint", C.c_int)]


GF_REQ_QUEUED, GF_REQ_RUNNING, GF_REQ_DONE, GF_REQ_FAILED = range(4)


class gf_server_opts(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("max_inflight", C.c_int), ("max_queue", C.c_int),
                ("batch_samples", C.c_int64)]


class gf_request(C.Structure):
    _fields_ = [("asset", C.c_int), ("camera", gf_camera), ("opts", gf_render_opts),
                ("lod", gf_lod_desc), ("lod_nee", gf_lod_desc), ("seed", C.c_uint64),
                ("out", C.c_void_p)]


class gf_result(C.Structure):
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("t_submit_ms", C.c_double),
                ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double), ("launches", C.c_int64)]


class gf_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("launches", C.c_int64), ("items", C.c_int64), ("max_inflight_seen", C.c_int),
                ("max_bytes_seen", C.c_int64), ("busy_ms", C.c_double), ("work", gf_stats)]


if not os.path.exists(LIB_PATH):
    raise ImportError("libgf.so is not built (%s); run paper_2602_05081_gb300.build.build()"
                      % LIB_PATH)
lib = C.CDLL(LIB_PATH)

_vp, _i64, _u64, _int = C.c_void_p, C.c_int64, C.c_uint64, C.c_int
_SIGS = {
    "gf_create": [_int, C.POINTER(_vp)],
    "gf_create_ex": [_int, C.POINTER(gf_allocator), C.POINTER(_vp)],
    "gf_reserve": [_vp, C.POINTER(gf_reserve_opts), _vp],
    "gf_destroy": [_vp],
    "gf_load_field": [_vp, C.POINTER(gf_params), C.POINTER(gf_field_opts), _vp, C.POINTER(_vp)],
    "gf_field_free": [_vp],
    "gf_build_bvh": [_vp, _vp],
    "gf_set_lod_mask": [_vp, C.POINTER(gf_lod_desc), C.POINTER(gf_lod_desc)],
    "gf_set_lod_camera": [_vp, C.POINTER(gf_camera), _vp],
    "gf_transmittance": [_vp, _vp, _vp, _vp, _i64, _int, _int, _u64, _vp, _vp, _vp],
    "gf_transmittance_static": [_vp, _vp, _vp, _vp, _i64, _int, _int, _u64, _vp, _vp, _vp],
    "gf_render": [_vp, C.POINTER(gf_camera), C.POINTER(gf_render_opts), _u64, _vp, _vp],
    "gf_render_backward": [_vp, C.POINTER(gf_camera), C.POINTER(gf_render_opts), _u64, _vp, _vp,
                           _vp],
    "gf_field_labels": [_vp, _vp, _vp, _vp, _vp],
    "gf_ray_chords": [_vp, _vp, _vp, _vp, _i64, _int, _vp, _vp, _vp, _vp, _vp],
    "gf_philox": [_vp, _vp, _vp, _i64, _vp],
    "gf_faddeeva": [_vp, _vp, _i64, _vp],
    "gf_get_stats": [_vp, C.POINTER(gf_stats), _int],
    "gf_sync": [_vp, _vp],
    "gf_field_info": [_vp, C.POINTER(_i64), C.POINTER(_int), C.POINTER(_u64)],
    "gf_server_create": [_vp, C.POINTER(_vp), _int, C.POINTER(gf_server_opts), C.POINTER(_vp)],
    "gf_server_submit": [_vp, C.POINTER(gf_request), C.POINTER(_u64)],
    "gf_server_poll": [_vp, _u64, C.POINTER(gf_result)],
    "gf_server_wait": [_vp, _u64, C.c_double, C.POINTER(gf_result)],
    "gf_server_get_stats": [_vp, C.POINTER(gf_server_stats)],
    "gf_server_destroy": [_vp],
    "gf_measure_peaks": [_int, C.POINTER(C.c_double), C.POINTER(C.c_double)],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
lib.gf_last_error.restype = C.c_char_p
lib.gf_last_error.argtypes = []


def gf_last_error() -> str:
    return lib.gf_last_error().decode()


def _check(status):
    if status != GF_OK:
        raise GfError(status, gf_last_error())


def ptr(x):
    """Raw address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError("unsupported buffer type %r" % type(x))


def stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- entry points
def gf_create(device: int = 0):
    h = _vp()
    _check(lib.gf_create(int(device), C.byref(h)))
    return h


def gf_create_ex(device: int, allocator: "gf_allocator | None"):
    """Context whose device memory comes from `allocator` (None: cudaMalloc/cudaFree);
    the caller keeps the allocator and its callbacks alive as long as the context."""
    h = _vp()
    _check(lib.gf_create_ex(int(device), None if allocator is None else C.byref(allocator),
                            C.byref(h)))
    return h


def gf_reserve(field, max_rays=0, max_chords=0, max_pixels=0, render=False, adjoint=False,
               stream=None):
    o = gf_reserve_opts(int(max_rays), int(max_chords), int(max_pixels), int(bool(render)),
                        int(bool(adjoint)))
    _check(lib.gf_reserve(field, C.byref(o), stream_handle(stream)))


def gf_destroy(ctx):
    _check(lib.gf_destroy(ctx))


def gf_load_field(ctx, params: gf_params, opts: gf_field_opts, stream=None):
    h = _vp()
    _check(lib.gf_load_field(ctx, C.byref(params), C.byref(opts), stream_handle(stream), C.byref(h)))
    return h


def gf_field_free(field):
    _check(lib.gf_field_free(field))


def gf_build_bvh(field, stream=None):
    _check(lib.gf_build_bvh(field, stream_handle(stream)))


def gf_set_lod_mask(field, primary: gf_lod_desc, nee: gf_lod_desc | None = None):
    _check(lib.gf_set_lod_mask(field, C.byref(primary), None if nee is None else C.byref(nee)))


def gf_set_lod_camera(field, camera: "gf_camera | None", stream=None):
    _check(lib.gf_set_lod_camera(field, None if camera is None else C.byref(camera),
                                 stream_handle(stream)))


def gf_transmittance(field, o, d, trange, n_rays, mode, spp, seed, out_T, out_tau=None,
                     stream=None):
    _check(lib.gf_transmittance(field, ptr(o), ptr(d), ptr(trange), int(n_rays), int(mode),
                                int(spp), int(seed), ptr(out_T), ptr(out_tau),
                                stream_handle(stream)))


def gf_transmittance_static(field, o, d, trange, n_rays, mode, spp, seed, out_T, out_tau=None,
                            stream=None):
    _check(lib.gf_transmittance_static(field, ptr(o), ptr(d), ptr(trange), int(n_rays),
                                       int(mode), int(spp), int(seed), ptr(out_T), ptr(out_tau),
                                       stream_handle(stream)))


def gf_render(field, camera: gf_camera, opts: gf_render_opts, seed, out_image, stream=None):
    _check(lib.gf_render(field, C.byref(camera), C.byref(opts), int(seed), ptr(out_image),
                         stream_handle(stream)))


def gf_render_backward(field, camera: gf_camera, opts: gf_render_opts, seed, dL_dimage, grad,
                       stream=None):
    _check(lib.gf_render_backward(field, C.byref(camera), C.byref(opts), int(seed),
                                  ptr(dL_dimage), ptr(grad), stream_handle(stream)))


def gf_field_labels(field, band=None, cone=None, cell=None, stream=None):
    _check(lib.gf_field_labels(field, ptr(band), ptr(cone), ptr(cell), stream_handle(stream)))


def gf_ray_chords(field, o, d, trange, n_rays, cap, counts, prims, t_in=None, t_out=None,
                  stream=None):
    _check(lib.gf_ray_chords(field, ptr(o), ptr(d), ptr(trange), int(n_rays), int(cap),
                             ptr(counts), ptr(prims), ptr(t_in), ptr(t_out),
                             stream_handle(stream)))


def gf_philox(ctr, key, out, n, stream=None):
    _check(lib.gf_philox(ptr(ctr), ptr(key), ptr(out), int(n), stream_handle(stream)))


def gf_faddeeva(z, w, n, stream=None):
    _check(lib.gf_faddeeva(ptr(z), ptr(w), int(n), stream_handle(stream)))


def gf_get_stats(field, reset=False) -> dict:
    s = gf_stats()
    _check(lib.gf_get_stats(field, C.byref(s), int(bool(reset))))
    out = {k: int(getattr(s, k)) for k, _ in gf_stats._fields_ if k != "cycles"}
    out["cycles"] = [int(x) for x in s.cycles]
    return out


def gf_sync(field, stream=None):
    _check(lib.gf_sync(field, stream_handle(stream)))


def gf_field_info(field):
    n = _i64(); p = _int(); occ = _u64()
    _check(lib.gf_field_info(field, C.byref(n), C.byref(p), C.byref(occ)))
    return int(n.value), int(p.value), int(occ.value)


def _result(r: gf_result) -> dict:
    return {k: (float(getattr(r, k)) if k.startswith("t_") else int(getattr(r, k)))
            for k, _ in gf_result._fields_}


def gf_server_create(ctx, fields, opts: gf_server_opts):
    arr = (_vp * len(fields))(*[f.value if isinstance(f, _vp) else f for f in fields])
    h = _vp()
    _check(lib.gf_server_create(ctx, arr, len(fields), C.byref(opts), C.byref(h)))
    return h


def gf_server_submit(server, request: gf_request) -> int:
    t = _u64()
    _check(lib.gf_server_submit(server, C.byref(request), C.byref(t)))
    return int(t.value)


def gf_server_poll(server, ticket) -> dict:
    r = gf_result()
    _check(lib.gf_server_poll(server, int(ticket), C.byref(r)))
    return _result(r)


def gf_server_wait(server, ticket, timeout_ms=60000.0) -> dict:
    r = gf_result()
    _check(lib.gf_server_wait(server, int(ticket), float(timeout_ms), C.byref(r)))
    return _result(r)


def gf_server_get_stats(server) -> dict:
    s = gf_server_stats()
    _check(lib.gf_server_get_stats(server, C.byref(s)))
    out = {k: (float(getattr(s, k)) if k == "busy_ms" else int(getattr(s, k)))
           for k, _ in gf_server_stats._fields_ if k != "work"}
    out["work"] = {k: int(getattr(s.work, k)) for k, _ in gf_stats._fields_ if k != "cycles"}
    return out


def gf_server_destroy(server):
    _check(lib.gf_server_destroy(server))


def gf_measure_peaks(device: int = 0):
    """(ex2, cos) pairs per second and FP32 FMAs per second, measured on the device."""
    sfu, fma = C.c_double(), C.c_double()
    _check(lib.gf_measure_peaks(int(device), C.byref(sfu), C.byref(fma)))
    return sfu.value, fma.value


EXPORTED = tuple(_SIGS) + ("gf_last_error",)
