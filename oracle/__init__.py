"""FP64 CPU oracle for the Gabor-field rendering path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2602_05081_gb300``) and never imports it.

The arithmetic lives in ``gf_oracle.c`` (plain C, FP64, OpenMP over rays);
this module compiles it with gcc on first use and marshals numpy arrays.
Every function states the passage of arXiv 2602.05081 it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_HDR = os.path.join(_HERE, "gf_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgf_oracle.so")
_lock = threading.Lock()
_lib = None

TAG_CAMERA, TAG_MASK, TAG_TRACK, TAG_NEE, TAG_NEE_MASK, TAG_SCATTER = 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class FieldDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("mu", C.c_void_p), ("quat", C.c_void_p),
                ("log_scale", C.c_void_p), ("omega", C.c_void_p), ("phase", C.c_void_p),
                ("weight", C.c_void_p), ("band", C.c_void_p), ("weight_mode", C.c_int),
                ("omega_frame", C.c_int), ("k_sigma", C.c_double), ("clamp_eps", C.c_double)]


class Lod(C.Structure):
    _fields_ = [("freq_policy", C.c_int), ("max_band", C.c_int), ("cone_policy", C.c_int),
                ("beta", C.c_float), ("delta", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int), ("height", C.c_int)]


class RenderOpts(C.Structure):
    _fields_ = [("integrator", C.c_int), ("spp", C.c_int), ("max_bounces", C.c_int),
                ("albedo", C.c_float), ("light_dir", C.c_float * 3),
                ("light_irradiance", C.c_float), ("free_flight", C.c_int),
                ("foveation", C.c_int), ("gaze", C.c_float * 2), ("fov_f0", C.c_float),
                ("fov_slope", C.c_float), ("fov_smooth", C.c_float)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp, i64, u64, u32, dbl, i32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.c_double, C.c_int
        lib.or_field_create.restype = vp
        lib.or_field_create.argtypes = [C.POINTER(FieldDesc)]
        lib.or_field_free.argtypes = [vp]
        lib.or_field_labels.argtypes = [vp, vp, vp, vp]
        lib.or_field_cells.argtypes = [vp, vp, vp]
        lib.or_field_prim.argtypes = [vp, i64, vp, vp, vp]
        lib.or_field_extent.restype = dbl
        lib.or_field_extent.argtypes = [vp, i64]
        lib.or_field_set_camera_lod.argtypes = [vp, vp]
        lib.or_philox4x32_10.argtypes = [vp, vp, vp]
        lib.or_sample_mask.argtypes = [vp, C.POINTER(Lod), vp, u64, u32, u32, u32, u32, vp, vp]
        lib.or_density.restype = dbl
        lib.or_density.argtypes = [vp, vp, u64, vp]
        lib.or_chord.restype = i32
        lib.or_chord.argtypes = [vp, i64, vp, vp, dbl, dbl, vp, vp]
        lib.or_chord_integral.restype = dbl
        lib.or_chord_integral.argtypes = [vp, i64, vp, vp, dbl, dbl]
        lib.or_chord_points.restype = i32
        lib.or_chord_points.argtypes = [vp, i64, vp, vp, dbl, dbl, dbl, u64, u32, u32, vp, vp, i32]
        lib.or_majorant.restype = dbl
        lib.or_majorant.argtypes = [vp, vp, vp, dbl, dbl, dbl, u64, vp]
        lib.or_transmittance.argtypes = [vp, C.POINTER(Lod), vp, vp, vp, i64, i32, i32, u64, vp,
                                         vp, i32]
        lib.or_cdf_flight.restype = i32
        lib.or_cdf_flight.argtypes = [vp, vp, vp, dbl, dbl, u64, vp, u64, u32, u32, vp]
        lib.or_segment_flight.restype = i32
        lib.or_segment_flight.argtypes = [vp, vp, vp, dbl, dbl, u64, vp, u64, u32, u32, vp]
        lib.or_delta_track.restype = i32
        lib.or_delta_track.argtypes = [vp, vp, vp, dbl, dbl, u64, vp, u64, u32, u32, vp]
        lib.or_render.argtypes = [vp, C.POINTER(Lod), C.POINTER(Lod), C.POINTER(Camera),
                                  C.POINTER(RenderOpts), u64, i32, i32, i32, i32, vp, i32]
        lib.or_render_samples.argtypes = lib.or_render.argtypes
        lib.or_camera_ray.argtypes = [C.POINTER(Camera), u64, i32, i32, i32, vp, vp]
        lib.or_tomo_loss_grad.restype = dbl
        lib.or_tomo_loss_grad.argtypes = [C.POINTER(FieldDesc), C.POINTER(Camera), i32, u64, vp,
                                          vp, i32]
        lib.or_tomo_image.argtypes = [C.POINTER(FieldDesc), C.POINTER(Camera), i32, u64, vp, i32]
        lib.or_radiance_grad_rays.argtypes = [C.POINTER(FieldDesc), C.POINTER(Lod), C.POINTER(Lod),
                                              C.POINTER(RenderOpts), vp, vp, i64, i32, u64, vp,
                                              vp, vp, i32]
        lib.or_radiance_grad_image.argtypes = [C.POINTER(FieldDesc), C.POINTER(Lod), C.POINTER(Lod),
                                               C.POINTER(Camera), C.POINTER(RenderOpts), u64, vp,
                                               vp, vp, i32]
        lib.or_rays_traced.restype = C.c_longlong
        lib.or_rays_traced.argtypes = [i32]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


WEIGHT_MODES = {"peak": 0, "normalized": 1}
OMEGA_FRAMES = {"world": 0, "local": 1}


class Field:
    """Primitive set held by the oracle (Sec. 3 Eq. 1 mixture, Sec. 4.2 kernels).

    ``params`` is a dict of numpy arrays: mu (N,3), quat (N,4) as (w,x,y,z),
    log_scale (N,3), omega (N,3), phase (N,), weight (N,), optional band (N,) u8.
    """

    def __init__(self, params, weight_mode="peak", omega_frame="world", k_sigma=3.0, clamp_eps=0.0):
        self.lib = _load()
        self._arrs = {k: _f32(params[k]).reshape(-1) for k in
                      ("mu", "quat", "log_scale", "omega", "phase", "weight")}
        band = params.get("band")
        self._band = None if band is None else np.ascontiguousarray(np.asarray(band, np.uint8))
        self.n = int(self._arrs["phase"].shape[0])
        self.desc = FieldDesc(self.n, _ptr(self._arrs["mu"]), _ptr(self._arrs["quat"]),
                              _ptr(self._arrs["log_scale"]), _ptr(self._arrs["omega"]),
                              _ptr(self._arrs["phase"]), _ptr(self._arrs["weight"]),
                              _ptr(self._band), WEIGHT_MODES[weight_mode],
                              OMEGA_FRAMES[omega_frame], float(k_sigma), float(clamp_eps))
        self.h = self.lib.or_field_create(C.byref(self.desc))
        self.k_sigma = float(k_sigma)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.or_field_free(self.h)
                self.h = None
        except Exception:
            pass

    def labels(self):
        b = np.zeros(self.n, np.uint8); c = np.zeros(self.n, np.uint8); e = np.zeros(self.n, np.uint8)
        self.lib.or_field_labels(self.h, _ptr(b), _ptr(c), _ptr(e))
        return b, c, e

    def cells(self):
        occ = np.zeros(1, np.uint64); kb = np.zeros(64, np.float64)
        self.lib.or_field_cells(self.h, _ptr(occ), _ptr(kb))
        return int(occ[0]), kb

    def extents(self):
        """Support radius of every primitive in sigma units (Sec. 4.4 adaptive
        clamping when clamp_eps > 0; 0 = dropped)."""
        return np.array([self.lib.or_field_extent(self.h, i) for i in range(self.n)])

    def set_camera_lod(self, cam):
        """Camera-Nyquist LoD selection (Supp. A) for ``cam`` (None: every kernel)."""
        self._lod_cam = cam
        self.lib.or_field_set_camera_lod(self.h, None if cam is None else C.byref(cam))

    def prim(self, i):
        s = np.zeros(9); w = np.zeros(3); a = np.zeros(1)
        self.lib.or_field_prim(self.h, int(i), _ptr(s), _ptr(w), _ptr(a))
        return s.reshape(3, 3), w, float(a[0])

    def sample_mask(self, lod, v, seed, ray, sample, bounce, tag):
        m = np.zeros(1, np.uint64); w = np.zeros(64)
        self.lib.or_sample_mask(self.h, C.byref(lod), _ptr(_f64(v)), int(seed), int(ray),
                                int(sample), int(bounce), int(tag), _ptr(m), _ptr(w))
        return int(m[0]), w

    def density(self, x, mask=(1 << 64) - 1, w64=None):
        return self.lib.or_density(self.h, _ptr(_f64(x)), int(mask),
                                   None if w64 is None else _ptr(_f64(w64)))

    def chord(self, i, o, v, tmin=0.0, tmax=np.inf):
        lo = np.zeros(1); hi = np.zeros(1)
        r = self.lib.or_chord(self.h, int(i), _ptr(_f64(o)), _ptr(_f64(v)), float(tmin),
                              float(tmax), _ptr(lo), _ptr(hi))
        return bool(r), float(lo[0]), float(hi[0])

    def chord_integral(self, i, o, v, tmin=0.0, tmax=np.inf):
        return self.lib.or_chord_integral(self.h, int(i), _ptr(_f64(o)), _ptr(_f64(v)),
                                          float(tmin), float(tmax))

    def chord_points(self, i, o, v, seed, ray, word, weight=1.0, tmin=0.0, tmax=np.inf, cap=4096):
        t = np.zeros(cap); u = np.zeros(cap)
        n = self.lib.or_chord_points(self.h, int(i), _ptr(_f64(o)), _ptr(_f64(v)), float(tmin),
                                     float(tmax), float(weight), int(seed), int(ray), int(word),
                                     _ptr(t), _ptr(u), int(cap))
        n = min(n, cap)
        return t[:n].copy(), u[:n].copy()

    def majorant(self, o, v, t, tmin=0.0, tmax=np.inf, mask=(1 << 64) - 1, w64=None):
        return self.lib.or_majorant(self.h, _ptr(_f64(o)), _ptr(_f64(v)), float(tmin),
                                    float(tmax), float(t), int(mask),
                                    None if w64 is None else _ptr(_f64(w64)))

    def transmittance(self, o, d, trange=None, mode="det", spp=1, seed=0, lod=None, threads=0):
        o = _f32(o).reshape(-1); d = _f32(d).reshape(-1)
        n = o.shape[0] // 3
        tr = None if trange is None else _f32(trange).reshape(-1)
        T = np.zeros(n); tau = np.zeros(n)
        lod = lod if lod is not None else Lod(0, 7, 0)
        self.lib.or_transmittance(self.h, C.byref(lod), _ptr(o), _ptr(d), _ptr(tr), n,
                                  0 if mode == "det" else 1, int(spp), int(seed), _ptr(T), _ptr(tau),
                                  int(threads))
        return T, tau

    def cdf_flight(self, o, v, seed, ray, word, tmin=0.0, tmax=np.inf, mask=(1 << 64) - 1,
                   w64=None):
        """Free flight by inversion of the optical-depth CDF (bisection)."""
        t = np.zeros(1)
        hit = self.lib.or_cdf_flight(self.h, _ptr(_f64(o)), _ptr(_f64(v)), float(tmin), float(tmax),
                                     int(mask), None if w64 is None else _ptr(_f64(w64)),
                                     int(seed), int(ray), int(word), _ptr(t))
        return bool(hit), float(t[0])

    def segment_flight(self, o, v, seed, ray, word, tmin=0.0, tmax=np.inf, mask=(1 << 64) - 1,
                       w64=None):
        """Free flight by uniform sampling within the crossing segment."""
        t = np.zeros(1)
        hit = self.lib.or_segment_flight(self.h, _ptr(_f64(o)), _ptr(_f64(v)), float(tmin),
                                         float(tmax), int(mask),
                                         None if w64 is None else _ptr(_f64(w64)), int(seed),
                                         int(ray), int(word), _ptr(t))
        return bool(hit), float(t[0])

    def delta_track(self, o, v, seed, ray, word, tmin=0.0, tmax=np.inf, mask=(1 << 64) - 1,
                    w64=None):
        t = np.zeros(1)
        hit = self.lib.or_delta_track(self.h, _ptr(_f64(o)), _ptr(_f64(v)), float(tmin),
                                      float(tmax), int(mask),
                                      None if w64 is None else _ptr(_f64(w64)), int(seed),
                                      int(ray), int(word), _ptr(t))
        return bool(hit), float(t[0])

    def render(self, cam, ropts, seed, lod=None, lod_nee=None, crop=None, threads=0,
               samples=False):
        lod = lod if lod is not None else Lod(0, 7, 0)
        lod_nee = lod_nee if lod_nee is not None else lod
        x0, y0, w, h = crop if crop is not None else (0, 0, cam.width, cam.height)
        if samples:
            out = np.zeros(w * h * ropts.spp)
            self.lib.or_render_samples(self.h, C.byref(lod), C.byref(lod_nee), C.byref(cam),
                                       C.byref(ropts), int(seed), x0, y0, w, h, _ptr(out),
                                       int(threads))
            return out.reshape(h, w, ropts.spp)
        out = np.zeros(w * h)
        self.lib.or_render(self.h, C.byref(lod), C.byref(lod_nee), C.byref(cam), C.byref(ropts),
                           int(seed), x0, y0, w, h, _ptr(out), int(threads))
        return out.reshape(h, w)

    def tomo_loss_grad(self, cam, spp, seed, target, threads=0):
        tgt = _f32(target).reshape(-1)
        g = np.zeros(15 * self.n)
        L = self.lib.or_tomo_loss_grad(C.byref(self.desc), C.byref(cam), int(spp), int(seed),
                                       _ptr(tgt), _ptr(g), int(threads))
        return L, g

    def radiance_grad_rays(self, o, v, ropts, spp, seed, dLdI=None, lod=None, lod_nee=None,
                           threads=0):
        """Single-scattering radiance estimator and its adjoint along fixed rays:
        returns (value per ray, gradient (15 N, SoA)); gradient is None without dLdI."""
        o = _f64(o).reshape(-1)
        v = _f64(v).reshape(-1)
        n = o.size // 3
        val = np.zeros(n)
        g = np.zeros(15 * self.n) if dLdI is not None else None
        lod = lod if lod is not None else Lod(0, 7, 0)
        lod_nee = lod_nee if lod_nee is not None else lod
        self.lib.or_radiance_grad_rays(C.byref(self.desc), C.byref(lod), C.byref(lod_nee),
                                       C.byref(ropts), _ptr(o), _ptr(v), n, int(spp), int(seed),
                                       _ptr(None if dLdI is None else _f64(dLdI).reshape(-1)),
                                       _ptr(val), _ptr(g), int(threads))
        return val, g

    def radiance_grad(self, cam, ropts, seed, dLdI=None, lod=None, lod_nee=None, threads=0):
        """Image version (jittered camera rays, spp from ropts): (image, gradient)."""
        img = np.zeros(cam.width * cam.height)
        g = np.zeros(15 * self.n) if dLdI is not None else None
        lod = lod if lod is not None else Lod(0, 7, 0)
        lod_nee = lod_nee if lod_nee is not None else lod
        self.lib.or_radiance_grad_image(C.byref(self.desc), C.byref(lod), C.byref(lod_nee),
                                        C.byref(cam), C.byref(ropts), int(seed),
                                        _ptr(None if dLdI is None else _f64(dLdI).reshape(-1)),
                                        _ptr(img), _ptr(g), int(threads))
        return img.reshape(cam.height, cam.width), g

    def tomo_image(self, cam, spp, seed, threads=0):
        img = np.zeros(cam.width * cam.height)
        self.lib.or_tomo_image(C.byref(self.desc), C.byref(cam), int(spp), int(seed), _ptr(img),
                               int(threads))
        return img.reshape(cam.height, cam.width)


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, np.uint32)); k = np.ascontiguousarray(np.asarray(key, np.uint32))
    out = np.zeros(4, np.uint32)
    lib.or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def camera(eye, look_at, up, vfov_deg, width, height):
    return Camera((C.c_float * 3)(*eye), (C.c_float * 3)(*look_at), (C.c_float * 3)(*up),
                  float(vfov_deg), int(width), int(height))


def camera_ray(cam, seed, px, py, s):
    lib = _load()
    o = np.zeros(3); v = np.zeros(3)
    lib.or_camera_ray(C.byref(cam), int(seed), int(px), int(py), int(s), _ptr(o), _ptr(v))
    return o, v


def render_opts(integrator="scatter", spp=1, max_bounces=1, albedo=0.8,
                light_dir=(1.0, 1.0, -1.0), light_irradiance=1.0, free_flight="delta",
                foveation=None):
    fv = foveation or {}
    return RenderOpts(0 if integrator == "tomo" else 1, int(spp), int(max_bounces), float(albedo),
                      (C.c_float * 3)(*light_dir), float(light_irradiance),
                      {"delta": 0, "cdf": 1, "segment": 2}[free_flight], 1 if foveation else 0,
                      (C.c_float * 2)(*fv.get("gaze", (0.0, 0.0))), float(fv.get("f0", 0.0)),
                      float(fv.get("slope", 0.0)), float(fv.get("smooth", 0.0)))


def rays_traced(reset=False):
    """Rays (camera, bounce and NEE segments) traced by the render calls since the last reset."""
    return int(_load().or_rays_traced(int(bool(reset))))


def stream_word(sample, bounce, tag):
    return (int(sample) << 12) | ((int(bounce) & 15) << 8) | (int(tag) & 255)
