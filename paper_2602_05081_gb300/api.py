"""Conveniences over the C ABI (marshalling only; the work runs in libgf.so).

``Field`` packs a primitive set on the GPU (gf_load_field + gf_build_bvh) and
forwards the rendering calls; ``TomoRender`` is a torch.autograd.Function whose
backward is the hand-written adjoint kernel (gf_render_backward); ``Server``
wraps the continuous-batching render server (gf_server_*).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi as A

_KEYS = ("mu", "quat", "log_scale", "omega", "phase", "weight")
_FRAMES = {"world": A.GF_OMEGA_WORLD, "local": A.GF_OMEGA_LOCAL}
_WMODES = {"peak": A.GF_WEIGHT_PEAK, "normalized": A.GF_WEIGHT_NORMALIZED}
_PRECS = {"fp32": A.GF_PREC_FP32, "fp16": A.GF_PREC_FP16, "bf16": A.GF_PREC_BF16}


class TorchAllocator:
    """Device memory of the library from PyTorch's caching allocator
    (gf_create_ex): the library's records, trees and scratch show up in
    torch.cuda.memory_reserved and are reused by torch once the library returns
    them.  Counts the calls, so a caller can check that a stretch of work
    allocated nothing."""

    def __init__(self, device: int):
        self.device = int(device)
        self.calls_alloc = 0
        self.calls_free = 0
        self.live_bytes = 0
        self._sizes = {}
        self._alloc = A.ALLOC_FN(self._on_alloc)
        self._free = A.FREE_FN(self._on_free)
        self.c = A.gf_allocator(self._alloc, self._free, None)

    def _on_alloc(self, user, nbytes, stream):
        try:
            p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
        except Exception:  # reported to the library as a failed allocation
            return None
        self.calls_alloc += 1
        self.live_bytes += int(nbytes)
        self._sizes[int(p)] = int(nbytes)
        return int(p)

    def _on_free(self, user, ptr, nbytes, stream):
        self.calls_free += 1
        self.live_bytes -= self._sizes.pop(int(ptr), int(nbytes))
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:  # interpreter shutdown: the process releases the memory
            pass


class Context:
    """A gf context on one GPU.  allocator: "torch" (default; PyTorch's caching
    allocator holds every device buffer of the library), None (cudaMalloc and
    cudaFree inside the library) or a TorchAllocator."""

    def __init__(self, device: int = 0, allocator="torch"):
        self.device = int(device)
        if allocator == "torch":
            allocator = TorchAllocator(self.device)
        self.allocator = allocator
        self.h = A.gf_create_ex(self.device, None if allocator is None else allocator.c)

    def close(self):
        if getattr(self, "h", None):
            A.gf_destroy(self.h)
            self.h = None


def _as_tensor(x, device, dtype=torch.float32):
    if isinstance(x, torch.Tensor):
        return x.detach().to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device).contiguous()


def lod(freq="all", max_band=7, cone="all", beta=0.0, delta=0.5):
    """LoD mask descriptor (strategy tables of App. B): freq in all, cutoff,
    unif_cv, uniform, power, pow_cv, pow_cv_acc; cone in all, is, uniform,
    thresh, thresh_uniform; beta the power-law shape, delta the alignment
    threshold."""
    f = {"all": A.GF_FREQ_ALL, "cutoff": A.GF_FREQ_CUTOFF, "unif_cv": A.GF_FREQ_UNIF_CV,
         "uniform": A.GF_FREQ_UNIFORM, "power": A.GF_FREQ_POWER, "pow_cv": A.GF_FREQ_POW_CV,
         "pow_cv_acc": A.GF_FREQ_POW_CV_ACC}[freq]
    c = {"all": A.GF_CONE_ALL, "is": A.GF_CONE_IS, "uniform": A.GF_CONE_UNIFORM,
         "thresh": A.GF_CONE_THRESH, "thresh_uniform": A.GF_CONE_THRESH_UNIFORM}[cone]
    return A.gf_lod_desc(f, int(max_band), c, float(beta), float(delta))


def camera(eye, look_at, up, vfov_deg, width, height):
    return A.gf_camera((C.c_float * 3)(*eye), (C.c_float * 3)(*look_at), (C.c_float * 3)(*up),
                       float(vfov_deg), int(width), int(height))


def render_opts(integrator="scatter", spp=1, max_bounces=1, albedo=0.8,
                light_dir=(1.0, 1.0, -1.0), light_irradiance=1.0, free_flight="delta",
                first_sample=0, foveation=None):
    """free_flight: "delta" (delta tracking), "cdf" (inversion of the optical-depth CDF) or
    "segment" (uniform within the crossing segment); samples first_sample ..
    first_sample + spp - 1 of each pixel are averaged; foveation: None or a dict with
    gaze (pixel coordinates), f0 (rad/unit at the gaze), slope (rad/unit per radian of
    eccentricity) and smooth (stochastic smoothing, [0, 1))."""
    fv = foveation or {}
    return A.gf_render_opts(A.GF_INTEG_TOMO if integrator == "tomo" else A.GF_INTEG_SCATTER,
                            int(spp), int(max_bounces), float(albedo),
                            (C.c_float * 3)(*light_dir), float(light_irradiance),
                            {"delta": 0, "cdf": 1, "segment": 2}[free_flight], int(first_sample),
                            1 if foveation else 0, (C.c_float * 2)(*fv.get("gaze", (0.0, 0.0))),
                            float(fv.get("f0", 0.0)), float(fv.get("slope", 0.0)),
                            float(fv.get("smooth", 0.0)))


class Field:
    """A packed primitive set with its BVH on one GPU.

    precision: "fp32", "fp16" or "bf16" records (FP32 math either way);
    k_sigma: support radius in sigma units; clamp_eps > 0 turns on adaptive
    clamping of each kernel's support (gf_field_opts.clamp_eps);
    transmittance modes: "det" (Gauss-Legendre), "closed" (closed form),
    "rt" (ratio tracking); set_lod / set_lod_camera choose the LoD masks.
    """

    def __init__(self, ctx: Context, params: dict, precision="fp32", weight_mode=None,
                 omega_frame=None, k_sigma=3.0, stream=None, device_inputs=True, clamp_eps=0.0):
        self.ctx = ctx
        dev = torch.device("cuda", ctx.device) if device_inputs else torch.device("cpu")
        self._keep = {k: _as_tensor(params[k], dev) for k in _KEYS}
        band = params.get("band")
        self._keep["band"] = None if band is None else _as_tensor(band, dev, torch.uint8)
        self.n = int(self._keep["phase"].numel())
        p = A.gf_params(self.n, *(A.ptr(self._keep[k]) for k in _KEYS),
                        A.ptr(self._keep["band"]))
        wm = weight_mode or params.get("weight_mode", "peak")
        fr = omega_frame or params.get("omega_frame", "world")
        opts = A.gf_field_opts(_PRECS[precision], _WMODES[wm], _FRAMES[fr], float(k_sigma),
                               float(clamp_eps))
        self.h = A.gf_load_field(ctx.h, p, opts, stream)
        A.gf_build_bvh(self.h, stream)
        if not device_inputs:
            self._keep = None

    def reserve(self, max_rays=0, max_chords=0, max_pixels=0, render=False, adjoint=False,
                stream=None):
        """Allocate the compute calls' scratch ahead (gf_reserve), so that calls within
        these sizes allocate nothing."""
        A.gf_reserve(self.h, max_rays, max_chords, max_pixels, render, adjoint, stream)

    def free(self):
        if getattr(self, "h", None):
            A.gf_field_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def set_lod(self, primary=None, nee=None):
        A.gf_set_lod_mask(self.h, primary if primary is not None else lod(), nee)

    def set_lod_camera(self, cam=None, stream=None):
        """Camera-Nyquist LoD selection (Supp. A) for ``cam``; None restores all kernels."""
        A.gf_set_lod_camera(self.h, cam, stream)

    def transmittance(self, o, d, trange=None, mode="det", spp=1, seed=0, out_T=None,
                      out_tau=None, stream=None):
        n = int(o.shape[0])
        if out_T is None:
            dev = o.device if isinstance(o, torch.Tensor) else torch.device("cpu")
            out_T = torch.empty(n, dtype=torch.float32, device=dev)
            if mode != "rt" and out_tau is None:
                out_tau = torch.empty(n, dtype=torch.float32, device=dev)
        m = {"det": A.GF_TR_DETERMINISTIC, "rt": A.GF_TR_RATIO_TRACKING,
             "closed": A.GF_TR_CLOSED_FORM}[mode]
        A.gf_transmittance(self.h, o, d, trange, n, m, spp, seed, out_T, out_tau, stream)
        return out_T, out_tau

    def render(self, cam, opts, seed=0, out=None, stream=None):
        if out is None:
            out = torch.empty(cam.height, cam.width, dtype=torch.float32,
                              device=torch.device("cuda", self.ctx.device))
        A.gf_render(self.h, cam, opts, seed, out, stream)
        return out

    def render_backward(self, cam, opts, seed, dL_dimage, grad=None, stream=None):
        if grad is None:
            grad = torch.empty(15 * self.n, dtype=torch.float32, device=dL_dimage.device)
        A.gf_render_backward(self.h, cam, opts, seed, dL_dimage, grad, stream)
        return grad

    def labels(self):
        b = np.zeros(self.n, np.uint8); c = np.zeros(self.n, np.uint8); e = np.zeros(self.n, np.uint8)
        A.gf_field_labels(self.h, b, c, e)
        return b, c, e

    def chords(self, o, d, trange=None, cap=512):
        n = int(o.shape[0])
        counts = np.zeros(n, np.int32)
        prims = np.zeros(n * cap, np.int32)
        tin = np.zeros(n * cap, np.float32)
        tout = np.zeros(n * cap, np.float32)
        A.gf_ray_chords(self.h, o, d, trange, n, cap, counts, prims, tin, tout)
        return counts, prims.reshape(n, cap), tin.reshape(n, cap), tout.reshape(n, cap)

    def stats(self, reset=False):
        return A.gf_get_stats(self.h, reset)

    def sync(self, stream=None):
        A.gf_sync(self.h, stream)

    def info(self):
        return A.gf_field_info(self.h)


def split_grad(g: torch.Tensor, n: int) -> dict:
    """SoA gradient (15 N floats) -> per-parameter tensors shaped like the inputs."""
    return {"mu": g[0:3 * n].view(n, 3), "quat": g[3 * n:7 * n].view(n, 4),
            "log_scale": g[7 * n:10 * n].view(n, 3), "omega": g[10 * n:13 * n].view(n, 3),
            "phase": g[13 * n:14 * n], "weight": g[14 * n:15 * n]}


class TomoRender(torch.autograd.Function):
    """I = tomography image of the field given by the parameter tensors.

    Forward packs the field and renders (GF_INTEG_TOMO, all cells); backward
    runs the adjoint kernel with per-ray recomputation.
    """

    @staticmethod
    def forward(ctx_, mu, quat, log_scale, omega, phase, weight, gctx, cam, spp, seed,
                omega_frame, weight_mode, k_sigma):
        params = {"mu": mu, "quat": quat, "log_scale": log_scale, "omega": omega,
                  "phase": phase, "weight": weight}
        f = Field(gctx, params, omega_frame=omega_frame, weight_mode=weight_mode,
                  k_sigma=k_sigma)
        opts = render_opts("tomo", spp=spp)
        img = f.render(cam, opts, seed)
        ctx_.field = f
        ctx_.cam, ctx_.opts, ctx_.seed = cam, opts, seed
        return img

    @staticmethod
    def backward(ctx_, g_img):
        f = ctx_.field
        g = f.render_backward(ctx_.cam, ctx_.opts, ctx_.seed, g_img.contiguous())
        parts = split_grad(g, f.n)
        f.free()
        return (parts["mu"], parts["quat"], parts["log_scale"], parts["omega"], parts["phase"],
                parts["weight"], None, None, None, None, None, None, None)


class RadianceRender(torch.autograd.Function):
    """I = scattering image (max_bounces collisions per path, 1 = single
    scattering) of the field given by the parameter tensors.

    Forward packs the field and renders with delta tracking (seed); backward runs
    the radiance adjoint kernel with its own seed (grad_seed), so the image and
    the gradient estimate are independent Monte Carlo estimates.
    """

    @staticmethod
    def forward(ctx_, mu, quat, log_scale, omega, phase, weight, gctx, cam, spp, seed, grad_seed,
                lod_primary, lod_nee, omega_frame, weight_mode, k_sigma, albedo=0.8,
                light_dir=(1.0, 1.0, -1.0), max_bounces=1):
        params = {"mu": mu, "quat": quat, "log_scale": log_scale, "omega": omega, "phase": phase,
                  "weight": weight}
        f = Field(gctx, params, omega_frame=omega_frame, weight_mode=weight_mode, k_sigma=k_sigma)
        f.set_lod(lod_primary, lod_nee)
        opts = render_opts("scatter", spp=spp, max_bounces=max_bounces, albedo=albedo,
                           light_dir=light_dir)
        img = f.render(cam, opts, seed)
        ctx_.field = f
        ctx_.cam, ctx_.opts, ctx_.grad_seed = cam, opts, grad_seed
        return img

    @staticmethod
    def backward(ctx_, g_img):
        f = ctx_.field
        g = f.render_backward(ctx_.cam, ctx_.opts, ctx_.grad_seed, g_img.contiguous())
        parts = split_grad(g, f.n)
        f.free()
        return (parts["mu"], parts["quat"], parts["log_scale"], parts["omega"], parts["phase"],
                parts["weight"]) + (None,) * 13


class Server:
    """Continuous-batching render server over resident fields (gf_server_*)."""

    def __init__(self, ctx: Context, fields, mem_budget=256 << 20, max_inflight=32,
                 max_queue=4096, batch_samples=0):
        self.ctx = ctx
        self.fields = list(fields)  # the fields must outlive the server
        opts = A.gf_server_opts(int(mem_budget), int(max_inflight), int(max_queue),
                                int(batch_samples))
        self.h = A.gf_server_create(ctx.h, [f.h for f in self.fields], opts)
        self._outs = {}

    def submit(self, asset, cam, opts, lod_primary=None, lod_nee=None, seed=0, out=None):
        """Queue a render; returns (ticket, out).  out defaults to a pinned host tensor."""
        if out is None:
            out = torch.empty(cam.height, cam.width, dtype=torch.float32).pin_memory()
        lp = lod_primary if lod_primary is not None else lod()
        ln = lod_nee if lod_nee is not None else lp
        rq = A.gf_request(int(asset), cam, opts, lp, ln, int(seed), A.ptr(out))
        t = A.gf_server_submit(self.h, rq)
        self._outs[t] = out  # keep the buffer alive until the request finishes
        return t, out

    def poll(self, ticket):
        return A.gf_server_poll(self.h, ticket)

    def wait(self, ticket, timeout_ms=600000.0):
        r = A.gf_server_wait(self.h, ticket, timeout_ms)
        return r

    def stats(self):
        return A.gf_server_get_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            A.gf_server_destroy(self.h)
            self.h = None
            self._outs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
